// Internal declarations shared by the host topology and the CUDA kernels.
#pragma once
#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/sem.h"

namespace sem {

constexpr int kMaxN = 6;
constexpr int kFields = 5;

// ---------------------------------------------------------------------------
// error reporting
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
#define SEM_CUDA_TRY(expr)                                                       \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess)                                                       \
      return ::sem::fail(SEM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------
// One-time set-up per device.  __constant__ tables and kernel attributes
// belong to a device: each device ordinal a process uses must get its own
// upload.  DeviceOnce records, per ordinal, that the set-up has succeeded;
// device_once runs `init` for the current device at most once (a failed init
// runs again on the next call), and is safe when several host threads make
// their first call at the same time.
constexpr int kMaxDevices = 64;
struct DeviceOnce {
  std::atomic<unsigned long long> done{0};
  std::mutex mu;
};
template <class F>
int device_once_on(DeviceOnce& o, int dev, F&& init) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SEM_ERR_ARG, "device ordinal out of range");
  const unsigned long long bit = 1ull << dev;
  if (o.done.load(std::memory_order_acquire) & bit) return SEM_OK;
  std::lock_guard<std::mutex> lk(o.mu);
  if (o.done.load(std::memory_order_relaxed) & bit) return SEM_OK;
  const int rc = init();
  if (rc == SEM_OK) o.done.fetch_or(bit, std::memory_order_release);
  return rc;
}
template <class F>
int device_once(DeviceOnce& o, F&& init) {
  int dev = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  return device_once_on(o, dev, init);
}

// ---------------------------------------------------------------------------
// 1-D LGL basis (host, float64)
struct Basis1D {
  int N = 0;
  std::vector<double> xi, w;         // N+1
  std::vector<double> D;             // [i][j] = h_j'(xi_i)
  std::vector<double> P[2];          // child interpolation [i][j] = h_j((xi_i+2c-1)/2)
  std::vector<double> Mex;           // exact mass matrix [i][j]
};
const Basis1D& basis(int N);
double lagrange(const std::vector<double>& xi, int j, double x);

// ---------------------------------------------------------------------------
// Leaf column of the horizontal quadtree forest
struct Leaf {
  int l, i, j;
};

// How a column of an adapted mesh was obtained from the previous mesh.
struct Origin {
  int kind;      // 0 same, 1 refined child, 2 coarsened parent
  int src[4];    // same: src[0]; refined: src[0] = parent; coarsened: 4 children (a + 2b)
  int a, b;      // child position for kind 1
};

struct DeviceTables;

// ---------------------------------------------------------------------------
// Host mesh: topology and numbering; device tables created lazily.
struct Mesh {
  // description
  double Lx = 0, Ly = 0, Lz = 0;
  int nx = 0, ny = 0, nz = 0, N = 0;
  bool px = true, py = true;
  int lvl_max = 0;
  std::vector<Leaf> leaves;          // Morton order
  int Lf = 0;                        // finest level present
  // numbering
  int Nq = 0;                        // (N+1)^2 horizontal local nodes per column
  int P = 0;                         // (N+1)^3
  int NZ = 0;
  long long NH = 0, NG = 0;
  std::vector<int> hmap;             // [Ncol][Nq]
  std::vector<int> hang_h;           // [Nhang][N+1]
  std::vector<double> hang_w;        // [Nhang][N+1]
  std::vector<int> qt_ptr;           // [NH+1]
  std::vector<int> qt_src;           // column*Nq + ab
  std::vector<double> qt_w;
  std::vector<double> Mh, Mz;        // lumped mass factors, M(h,kz) = Mh[h] Mz[kz]
  std::vector<double> xh, yh, zk;    // coordinates of horizontal nodes / levels
  long long n_nonconf_sides = 0;
  // adaptation provenance (set by sem_transfer_plan)
  std::vector<Origin> origin;
  long long parent_serial = -1;
  long long serial = 0;
  // element-kernel launch variant chosen by the autotuner (-1: default)
  int pencil_variant = -1;
  int nc_variant = -1;      // the same for the paper's equation set
  // device
  DeviceTables* dev = nullptr;
  int dev_id = -1;

  long long Ncol() const { return (long long)leaves.size(); }
  long long Ne() const { return Ncol() * nz; }
  double hx(int l) const { return Lx / (double)((long long)nx << l); }
  double hy(int l) const { return Ly / (double)((long long)ny << l); }
  std::vector<double> zf;            // [nz + 1] layer faces
  double hz(int k) const { return zf[k + 1] - zf[k]; }
  // warped layers (warp.cpp): amplitude (m) and wave numbers; A = 0: boxes
  double warp_A = 0.0;
  int warp_kx = 1, warp_ky = 1;
  bool warped() const { return warp_A != 0.0; }
  std::vector<double> zG;            // [NG] node heights
  std::vector<double> zH;            // [Nhang][NZ] heights of the hanging lines' nodes
  std::vector<double> metric;        // [Ncol][Nq][nz][N+1][3] z_xi, z_eta, z_zeta
  std::vector<double> Mg;            // [NG] lumped mass per global node
  int NZr() const { return (NZ + 3) & ~3; }  // level stride of the column residual scratch
};

int build_mesh(Mesh& m);                       // numbering from leaves (host)
int build_warp(Mesh& m);                       // warped-layer geometry (warp.cpp)
double warp_height(const Mesh& m, double x, double y, double zeta);
int check_leaves(const Mesh& m);               // tiling + balance
int adapt_leaves(const Mesh& old, const int8_t* flags, std::vector<Leaf>& out,
                 std::vector<Origin>& origin);

// ---------------------------------------------------------------------------
// Device tables of a mesh
struct DeviceTables {
  int* hmap = nullptr;
  int* hang_h = nullptr;
  double* hang_w = nullptr;
  int* qt_ptr = nullptr;
  int* qt_src = nullptr;
  double* qt_w = nullptr;
  double* Minv_h = nullptr;
  double* Minv_z = nullptr;
  float* Minv_h32 = nullptr;    // float32 copies for the mixed form
  float* Minv_z32 = nullptr;
  float* qt_w32 = nullptr;
  int* qt_rec_src = nullptr;    // [NH][4]: Q_h^T sources of h when it has at most 4 (-1: unused), else -2 (use the CSR lists)
  float* qt_rec_w = nullptr;    // [NH][4]: their float32 weights
  int* qt_rec_unit = nullptr;   // [NH][4]: the sources of h when it has at most 4 and all their
                                // weights are exactly 1 (-1: unused), else -2 (use the CSR lists)
  float* hang_w32 = nullptr;
  float* mirror = nullptr;      // float32 state mirror scratch [5][NG]
  double* Mh = nullptr;
  double* Mz = nullptr;
  double* ref = nullptr;        // [NZ][kRef] float64 reference state
  float* ref32 = nullptr;       // [NZ][kRef] float32 copy, then [NZ][4] packed rows (p0, rho0, (rho theta)0, 1/(rho theta)0)
  int* col_level = nullptr;     // [Ncol]
  double* col_x0 = nullptr;     // [Ncol] lower-left corner of each column (x, y)
  double* col_y0 = nullptr;
  double* xh = nullptr;         // [NH]
  double* yh = nullptr;
  double* zk = nullptr;         // [NZ]
  double* hzk = nullptr;        // [nz] layer thicknesses, float64 and float32
  float* hzk32 = nullptr;
  void* scratch = nullptr;      // column residuals
  size_t scratch_bytes = 0;
  int* status = nullptr;        // device status word
  // transfer
  int* org = nullptr;           // [Ncol][6] kind, src0..3, a+2b
  // adapt and diagnostics
  double* elem_cmax = nullptr;
  int8_t* elem_flags = nullptr;
  double* diag_buf = nullptr;   // [NZ][4]
  // continuous projection of the transfer (coupled coarse-face nodes)
  int n_comp = 0, max_comp = 0;
  int* tr_comp_ptr = nullptr;   // [n_comp+1] into tr_nodes
  int* tr_nodes = nullptr;      // horizontal node ids, grouped by component
  int* tr_A_ptr = nullptr;      // CSR of A_h restricted to each component
  int* tr_A_col = nullptr;      // component-local column
  double* tr_A_val = nullptr;
  int* tr_coupled = nullptr;    // [NH] 1 when the node is solved for
  // the params the ref tables were built with
  double ref_key[8] = {0};
  bool ref_valid = false;
  // warped layers: per-node tables (null on box meshes)
  double* zG = nullptr;         // [NG] node heights
  double* zH = nullptr;         // [Nhang][NZ] heights of the hanging lines' nodes
  double* metric = nullptr;     // [Ncol][Nq][nz][N+1][3] z_xi, z_eta, z_zeta
  float* metric32 = nullptr;
  double* Minv_g = nullptr;     // [NG] inverse lumped mass per node
  float* Minv_g32 = nullptr;
  double* refG = nullptr;       // [NG][kRef] reference state at each node's height
  double* refH = nullptr;       // [Nhang][NZ][kRef] ... at each hanging-line node's height
  float* refG32 = nullptr;      // float32 copies
  float* refH32 = nullptr;
  float* ref4G = nullptr;       // [NG][4] packed p0, rho0, (rho theta)0, 1/(rho theta)0
  float* ref4H = nullptr;       // [Nhang][NZ][4]
  // absorbing-layer rate R(z) per level (float64 and float32) and its key
  double* spg = nullptr;
  float* spg32 = nullptr;
  double spg_key[2] = {-1.0, -1.0};
};
constexpr int kRef = 8;  // theta0, pi0, p0, rho0, rhotheta0, dtheta0/dz, 1/(rho theta)0, z

int ensure_device(Mesh& m);
// reference tables for p (uploaded synchronously when p's reference-state
// parameters differ from those the tables were made with)
int ensure_reference(Mesh& m, const sem_params& p);
// true when ensure_reference(m, p) would upload
bool reference_stale(const Mesh& m, const sem_params& p);
// validates every field of p (SEM_ERR_ARG with a message)
int check_params(const sem_params* p);
void free_device(Mesh& m);

// kernel launchers (k_*.cu)
struct StageArgs {
  const double* qn;
  const double* qs;
  double* out;
  const float* qs32;  // mixed form: float32 mirror of qs (null: made internally)
  float* out32;       // mixed form: float32 mirror of out to write (may be null)
  double a, b, cdt;   // out = a qn + b qs + cdt * tendency; rhs mode: a=b=0, cdt=1
  int rhs_only;
  void* scratch;      // column-residual scratch; null: the mesh's own
  double time = 0.0;  // time at which the tendency is evaluated (heating source)
};
int launch_rhs_stage(Mesh& m, const sem_params& p, const StageArgs& s, cudaStream_t st);
int launch_adapt(Mesh& m, const sem_params& p, const double* q, int8_t* flags, double* cmax,
                 cudaStream_t st, const int8_t* elem_level = nullptr, int level_all = -1);
int launch_merge_flags(const int8_t* crit, const int8_t* pred, const int8_t* level, int lvl_max, long long n,
                       int8_t* out, cudaStream_t st);
int launch_diag(Mesh& m, const sem_params& p, const double* q, double half_width,
                sem_diag_out* out, cudaStream_t st);
int launch_transfer(Mesh& oldm, Mesh& newm, const double* qold, double* qnew, cudaStream_t st);
int launch_coords(Mesh& m, double* xyz, cudaStream_t st);
int launch_mirror(const double* q, float* q32, long long n, cudaStream_t st);
int batch_create(Mesh* const* meshes, int n, void** out);
void batch_destroy(void* b);
int batch_step_mixed(void* b, const sem_params& p, double* const* q, float* const* q32,
                     float* const* work32, const double* dt, int use_graph, cudaStream_t st);
int batch_status(void* b, int* status, cudaStream_t st);
int mlp_create(unsigned long long seed, int max_rows, void** out);
void mlp_destroy(void* m);
int mlp_params(void* m, float* host, int set, int which);
int mlp_param_count();
int mlp_forward_api(void* m, const float* X, int n, float* prob, int8_t* flags, cudaStream_t st);
int mlp_backward_api(void* m, const float* X, const int8_t* y, const float* cw, int n, double* loss_host,
                     cudaStream_t st);
int mlp_adam_api(void* m, float lr, cudaStream_t st);
int mlp_select_forward(void* m, int tc);
int mlp_status(void* m, int* status, cudaStream_t st);
int mlp_features_api(Mesh& mesh, const double* q, const float* scales, float* F, cudaStream_t st);
int autotune_pencil(Mesh& m, const sem_params& p, const float* q32, int reps, sem_tune_out* out,
                    cudaStream_t st);
int select_pencil(Mesh& m, int eqset, int row);
int launch_step_mixed(Mesh& m, const sem_params& p, double* q, float* q32, float* work32, double dt,
                      cudaStream_t st);
// terms of the paper's runs (k_physics.cu): adds the Smagorinsky stress and the
// absorbing layer to the column residuals in `scratch` (null: the mesh's own)
inline bool physics_on(const sem_params& p) {
  return p.smag_cs > 0.0 || p.sponge_gamma > 0.0 || p.heat_q0 > 0.0;
}
// sponge_done, smag_done: the element kernel has added the absorbing layer,
// the Smagorinsky stress already
int launch_physics(Mesh& m, const sem_params& p, const void* q, bool mixed, void* scratch,
                   double time, cudaStream_t st, bool sponge_done = false, bool smag_done = false);
// absorbing-layer rate tables D.spg / D.spg32 for p's gamma and depth
int ensure_sponge(Mesh& m, const sem_params& p);

// per-kernel event timing (profile.cpp); -1 when profiling is off
int prof_begin_kernel(const char* name, cudaStream_t st);
void prof_end_kernel(int rec, cudaStream_t st);
struct ProfScope {
  int rec;
  cudaStream_t st;
  ProfScope(const char* name, cudaStream_t s) : rec(prof_begin_kernel(name, s)), st(s) {}
  ~ProfScope() { prof_end_kernel(rec, st); }
};

}  // namespace sem

struct sem_mesh {
  sem::Mesh m;
};

struct sem_mlp {
  void* impl = nullptr;
  int max_rows = 0;
};

struct sem_batch {
  void* impl = nullptr;
  int n = 0;
  int dev = -1;
};
