/*
 * sem.h - C ABI of the GB300 spectral-element tropical-cyclone hot path.
 *
 * The library evaluates the right-hand side of the split dry compressible
 * Euler equations (Eqs. mass_split, mom_split, ent_split of arXiv 2410.21607,
 * Sec. 2, here with an f-plane Coriolis term) on a hexahedral mesh of
 * tensor-product Lagrange elements of order N on Legendre-Gauss-Lobatto points
 * (Sec. 3), with 2:1 non-conforming faces handled by the modified direct
 * stiffness summation of Sec. 3.1; it advances the state with the stages of an
 * explicit third-order Runge-Kutta scheme (Sec. 4, "Time integration"); it
 * evaluates the threshold refinement criterion (Sec. 3.1) and moves the
 * solution to the refined/coarsened mesh (Sec. 3.2, Algorithm 3).
 *
 * Conventions (every function):
 *   - returns SEM_OK (0) or a SEM_ERR_* code; sem_last_error() gives a
 *     thread-local message for the last failure on the calling thread;
 *   - sem_mesh handles are owned by the library and freed by sem_mesh_destroy;
 *   - field arrays are owned by the caller.  "dev" pointers are CUDA device
 *     memory, "host" pointers are host memory;
 *   - a global field is laid out structure-of-arrays as [5][NH][NZ] float64:
 *     field f, horizontal global node h, vertical level kz at offset
 *     (f * NH + h) * NZ + kz, i.e. [5][NG] with NG = NH * NZ;
 *   - calls taking a cudaStream_t only enqueue work on that stream (0 = the
 *     legacy default stream) and return without synchronising, unless the
 *     description says that the call returns host data;
 *   - no call allocates or frees caller memory.  The library allocates its own
 *     device tables and scratch for a mesh on the first device call for that
 *     mesh (on the current device) and frees them in sem_mesh_destroy.
 */
#ifndef SEM_H
#define SEM_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEM_OK 0
#define SEM_ERR_ARG 1        /* invalid argument (null pointer, bad size)   */
#define SEM_ERR_CUDA 2       /* a CUDA runtime call failed                  */
#define SEM_ERR_TOPOLOGY 3   /* leaves do not tile the domain, 2:1 balance  */
                             /* violated, or a constraint chain was found   */
#define SEM_ERR_NUMERIC 4    /* non-finite value detected on the device     */
#define SEM_ERR_TIMEOUT 5    /* a bounded device wait ran out               */
#define SEM_ERR_IO 6         /* checkpoint read/write failed                */
#define SEM_ERR_UNSUPPORTED 7/* order N or option not compiled in           */

#define SEM_EQ_CONSERVATIVE 0     /* (rho', rho u, rho v, rho w, (rho theta)') */
#define SEM_EQ_NONCONSERVATIVE 1  /* (rho', u, v, w, theta')  Eqs. mass_split..ent_split */

#define SEM_PREC_FP64 0   /* every operation in float64                          */
#define SEM_PREC_MIXED 1  /* float32 perturbation arithmetic in the element and  */
                          /* face work; float64 reference state, metric terms    */
                          /* and stage accumulation of the state                 */

#define SEM_MAX_THRESHOLDS 8

/* Criterion variables (Sec. 3.1: the variable C^l may change with the level;
 * the paper's runs use the speed at every level, and it names vorticity and
 * potential vorticity as candidates).  Element maxima over the nodes. */
#define SEM_CRIT_SPEED 0      /* |u|, 3-D velocity magnitude                       */
#define SEM_CRIT_VORTICITY 1  /* |dv/dx - du/dy|, vertical relative vorticity      */
#define SEM_CRIT_PV 2         /* |(curl u + f e_z) . grad theta| / rho, dry Ertel PV */

/* Mesh description (host).  Domain [-Lx/2, Lx/2] x [-Ly/2, Ly/2] x [0, Lz],
 * base grid nx x ny columns of nz hexahedra of order N (Sec. 3).  Refinement
 * is horizontal and by whole columns (Sec. 3.1): a leaf column is
 * (level, i, j) on the 2^level-times finer horizontal grid.  leaves == NULL
 * (n_leaves == 0) gives the uniform level-0 mesh.  The leaves must tile the
 * domain exactly once and be 2:1 balanced across faces and corners,
 * otherwise SEM_ERR_TOPOLOGY. */
typedef struct {
  double Lx, Ly, Lz;
  int nx, ny, nz;
  int N;                  /* polynomial order, 2..6 */
  int periodic_x, periodic_y;
  int lvl_max;            /* largest level the criterion may request */
  int n_leaves;
  const int* leaves;      /* host, [n_leaves][3] = (level, i, j) */
  const double* z_faces;  /* host, [nz + 1] layer faces 0 = z_0 < z_1 < ... < z_nz = Lz
                             (a stretched vertical grid; every element stays an
                             axis-aligned box), or NULL for nz equal layers */
  /* Warped layers (non-affine elements; 0 = none): every node moves vertically
   * to z = zeta + warp_amplitude sin(2 pi warp_kx (x + Lx/2) / Lx)
   * sin(2 pi warp_ky (y + Ly/2) / Ly) sin(pi zeta / Lz) (zeta its height on the
   * box mesh): curved layer surfaces, flat lids, periodic.  Each element is the
   * isoparametric image of the reference cube through its nodal coordinates
   * (Sec. 3's LGL basis), with float64 metric terms and Jacobian per node and
   * the lumped mass per node; hanging nodes take the coarse face's
   * interpolated height (Sec. 3.1), so the mesh stays watertight.  A
   * non-positive Jacobian gives SEM_ERR_ARG.  On warped meshes the right-hand
   * side, the stages and steps (float64 and mixed forms), the terms of the
   * paper's runs (the horizontal Smagorinsky stress with gradients at constant
   * height, the absorbing layer and the heating at each node's height), the
   * criteria (speed; vorticity and potential vorticity with derivatives at
   * constant height), coordinates, diagnostics and checkpoints are available;
   * adaptation (sem_transfer_plan) and batching give SEM_ERR_UNSUPPORTED, and
   * the mixed conservative form uses the line-exchange element kernels
   * only. */
  double warp_amplitude;
  int warp_kx, warp_ky;
} sem_mesh_desc;

typedef struct sem_mesh sem_mesh;

typedef struct {
  long long Ne;           /* elements                                   */
  long long NL;           /* local nodes, Ne * (N+1)^3                  */
  long long NG;           /* global (non-hanging) nodes, NH * NZ        */
  long long NH;           /* horizontal global nodes                    */
  long long NZ;           /* vertical levels, nz * N + 1                */
  long long Ncol;         /* leaf columns                               */
  long long n_hanging_h;  /* hanging horizontal local nodes (per column layer) */
  long long n_nonconforming_faces; /* coarse sides with finer neighbours, per layer */
  int N, nz, max_level;
  long long level_hist[16]; /* columns per level */
} sem_mesh_info;

/* Physical and scheme parameters (Sec. 2; constants the paper leaves unstated
 * take the defaults of sem_params_default). */
typedef struct {
  double g;           /* 9.81 m s^-2 (Sec. 2)                       */
  double f;           /* Coriolis parameter (f-plane), s^-1         */
  double R_d, c_p;    /* gas constant and heat capacity of dry air  */
  double p00;         /* reference surface pressure, Pa             */
  double theta_s;     /* reference theta at z = 0, K                */
  double N_bv;        /* buoyancy frequency of the reference state  */
  int eqset;          /* SEM_EQ_*                                    */
  int precision;      /* SEM_PREC_*                                  */
  int n_thresholds;   /* criterion thresholds, one per level (Sec. 3.1) */
  int lvl_max;
  double thresholds[SEM_MAX_THRESHOLDS];
  /* Terms of the paper's runs (Sec. 4), off at 0.  smag_cs: Smagorinsky
   * coefficient C_s of the horizontal Smagorinsky-Lilly stress (the paper's
   * 0.21), filter width (hx + hy) / (2N) of each element.  sponge_gamma,
   * sponge_depth: rate gamma (1/s) and depth z_d (m) of the Rayleigh layer
   * at the top of the domain, R(z) = min(1, gamma sin^2(pi/2 (1 - (Lz - z)/z_d)))
   * for z >= Lz - z_d, 0 below, acting as -R(z) q' on every equation (the
   * paper's gamma 1.0, z_d 4 km).  Both enter the element residual (the
   * stress in weak form, the layer as a collocated source).  Not in the
   * batched step. */
  double smag_cs;
  double sponge_gamma;
  double sponge_depth;
  /* criterion[l]: the SEM_CRIT_* variable compared with thresholds[l], i.e.
   * threshold(l+1) of Sec. 3.1 (default SEM_CRIT_SPEED everywhere).  The
   * derivatives are element-local derivatives of the element polynomials. */
  int criterion[SEM_MAX_THRESHOLDS];
  /* Synthetic latent heating (a stand-in for the paper's observed heating,
   * Sec. 4), off at heat_q0 = 0: a theta source
   *   Q = heat_q0 tanh(t / heat_ramp) exp(-((r - heat_r0) / heat_width)^2) sin(pi z / heat_ztop)
   * (K/s) for r <= heat_rmax and z <= heat_ztop, r from the domain centre,
   * entering (rho theta)' as rho Q (or theta' as Q) as a collocated source.
   * time: the time of the state.  sem_rhs evaluates the source at `time`;
   * the stage calls take `time` as the time of qn and evaluate stages 0, 1, 2
   * at time, time + dt, time + dt/2 (SSP-RK3); they do not advance it. */
  double heat_q0, heat_r0, heat_width, heat_rmax, heat_ztop, heat_ramp;
  double time;
} sem_params;

typedef struct {
  double max_wind;        /* max sqrt(u^2+v^2) over |x|,|y| <= half_width (Sec. 4.2) */
  double max_mean_wind;   /* max over heights of the mass-weighted horizontal mean   */
} sem_diag_out;

const char* sem_last_error(void);

/* Defaults: g 9.81, f 5e-5, R_d 287, c_p 1004, p00 1e5, theta_s 300,
 * N_bv 0.01, conservative set, FP64, thresholds [7.5, 15, 22.5] (Sec. 4.1),
 * no Smagorinsky stress, no absorbing layer (sponge_depth 4000). */
int sem_params_default(sem_params* p);

/* Host only.  Builds the leaf columns (Morton order), the global node
 * numbering, the hanging-node interpolation rows (Sec. 3.1) and the lumped
 * mass.  No device work. */
int sem_mesh_create(const sem_mesh_desc* d, sem_mesh** out);
void sem_mesh_destroy(sem_mesh* m);
int sem_mesh_get_info(const sem_mesh* m, sem_mesh_info* out);

/* Host exports (no device work).  coords: [3][NG] (x, y, z of every global
 * node, x and y wrapped into [-L/2, L/2)).  leaves: [Ncol][3].
 * hmap: [Ncol][(N+1)^2] horizontal map of each column's local node
 * (a, b) (a along x, fastest): value h >= 0 is the horizontal global node,
 * value -1-k means hanging row k.  hang_h / hang_w: [n_hanging_h][N+1] the
 * horizontal global nodes and weights of hanging row k.  mass: [NG] lumped
 * mass M = Q^T (w J). */
int sem_mesh_coords_host(const sem_mesh* m, double* coords_host);
int sem_mesh_leaves_host(const sem_mesh* m, int* leaves_host);
int sem_mesh_hmap_host(const sem_mesh* m, int* hmap_host, int* hang_h_host, double* hang_w_host);
int sem_mesh_mass_host(const sem_mesh* m, double* mass_host);

/* Device copy of the coordinates, [3][NG]. */
int sem_mesh_coords(sem_mesh* m, double* coords_dev, cudaStream_t stream);

/* Tendency dq/dt = M^-1 Q^T r(q) of the semi-discrete system (Sec. 3, 3.1),
 * with the rigid-lid condition (zero vertical-momentum tendency at z = 0 and
 * z = Lz).  q_dev, rhs_dev: [5][NG] float64 device arrays, distinct. */
int sem_rhs(sem_mesh* m, const sem_params* p, const double* q_dev, double* rhs_dev,
            cudaStream_t stream);

/* sem_rhs without any device allocation in the call.
 *
 * For callers that must not allocate device memory when they evaluate the
 * right-hand side: code that runs while another allocator (a framework's
 * caching allocator or a memory pool) holds all free device memory, so that a
 * new cudaMalloc would fail, and real-time or certified code whose rules
 * forbid device allocation after start-up.  The paper has no counterpart; it
 * is an interface addition of this library.
 *
 * Same inputs, outputs and result as sem_rhs.  Instead of the mesh's own
 * residual scratch it uses one fixed device array of 16 MiB built into the
 * library (every GPU that loads the library holds it until the process
 * exits), so it serves meshes with Ncol * (N+1)^2 * 5 * NZ4 * 8 <= 16 MiB
 * (NZ4 = NZ rounded up to a multiple of 4)
 * (about 1,000 columns of 16 layers at N = 4); larger meshes get SEM_ERR_ARG
 * before any device work.  The call performs no allocation itself, but it
 * does not save memory: the mesh must already have its device tables, made
 * by any earlier device call on it (for example sem_mesh_coords), else
 * SEM_ERR_ARG, and those tables include the mesh's own residual scratch,
 * which stays allocated.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, kept per device; the CUDA driver may load
 * the library's device code then); make that first call before any stream
 * capture.  A call whose reference-state parameters (g, R_d, c_p, p00,
 * theta_s, N_bv) differ from those of the mesh's previous call uploads the
 * reference tables with a synchronous copy; under stream capture that case
 * is refused with SEM_ERR_ARG, so make one call with new parameters before
 * capturing.  The parameters are validated as in sem_rhs.  All calls share
 * the one array and every element of it that a call reads is first written
 * by the same call, so nothing needs clearing between calls; calls that
 * overlap on the GPU (on different streams, or from several threads) race on
 * the array and must be serialised by the caller.  The optional terms
 * (smag_cs, sponge_gamma, heat_q0) keep tables allocated on first use and
 * are refused here (SEM_ERR_UNSUPPORTED). */
int sem_rhs_noalloc(sem_mesh* m, const sem_params* p, const double* q_dev, double* rhs_dev,
                    cudaStream_t stream);

/* One stage of the SSP-RK3 scheme (Sec. 4, time integration):
 *   q_out = a[stage] qn + b[stage] qs + c[stage] dt rhs(qs)
 * with (a, b, c) = (0, 1, 1), (3/4, 1/4, 1/4), (1/3, 2/3, 2/3).
 * qn, qs, q_out: [5][NG] float64 device arrays; q_out may alias neither. */
int sem_rk_stage(sem_mesh* m, const sem_params* p, int stage, const double* qn_dev,
                 const double* qs_dev, double* qout_dev, double dt, cudaStream_t stream);

/* Mixed form with caller-owned float32 mirrors.  qs32_dev must hold the
 * float32 mirror of qs_dev ([5][NG], as written by sem_mirror or by a previous
 * call of this function into its qout32); the stage writes q_out (float64)
 * and its float32 mirror qout32.  The element and face arithmetic reads the
 * mirror, the float64 stage accumulation reads qn and qs.  Needs
 * p->precision == SEM_PREC_MIXED.  (sem_rk_stage in the mixed form makes the
 * mirror itself, in library scratch, at the cost of one more pass.) */
int sem_rk_stage_mixed(sem_mesh* m, const sem_params* p, int stage, const double* qn_dev,
                       const double* qs_dev, const float* qs32_dev, double* qout_dev,
                       float* qout32_dev, double dt, cudaStream_t stream);

/* A whole SSP-RK3 step of the mixed form, either equation set (the
 * conservative set through the autotuned element kernel, the paper's set
 * through the column element kernel), in increment form: with d_s = q_s - q_n,
 *   d_1 = dt L(q_n), d_2 = (d_1 + dt L(q_1)) / 4, d_3 = 2 (d_2 + dt L(q_2)) / 3,
 *   q_{n+1} = q_n + d_3,
 * which is the Shu-Osher SSP-RK3 step rewritten exactly.  The increments d_s
 * are float32, the state q (float64, [5][NG]) is updated in place with one
 * float64 addition per value, and q32 (its float32 mirror, [5][NG], from
 * sem_mirror or the previous step) is updated with it.  work32_dev is
 * caller-owned float32 scratch of 2 * 5 * NG values. */
int sem_step_mixed(sem_mesh* m, const sem_params* p, double* q_dev, float* q32_dev,
                   float* work32_dev, double dt, cudaStream_t stream);

/* Batched mixed-form steps over many independent meshes (uneven sizes,
 * orders N = 2..6, any refinement levels).  Per stage, one persistent element
 * kernel walks all columns of all meshes from a work queue (costliest columns
 * first) and one gather/increment kernel covers the concatenated global nodes;
 * a step is the increment form of sem_step_mixed for every instance, in
 * p->eqset's equation set (either set; p->precision must be SEM_PREC_MIXED,
 * else SEM_ERR_ARG; box meshes only, and no Smagorinsky stress or absorbing
 * layer: SEM_ERR_UNSUPPORTED).  The meshes must outlive the batch.
 * sem_batch_step_mixed takes per-instance arrays (q[k] float64 [5][NG_k],
 * q32[k] its float32 mirror, work32[k] float32 2 x [5][NG_k]) and time steps
 * dt[k]; with use_graph != 0 the step's launches are captured once into a CUDA
 * graph and replayed (re-captured when an array pointer, a dt, a physical
 * parameter or the equation set changes).  sem_batch_status reads and clears
 * the batch's non-finite flag (synchronises). */
typedef struct sem_batch sem_batch;
int sem_batch_create(sem_mesh* const* meshes, int n, sem_batch** out);
void sem_batch_destroy(sem_batch* b);
int sem_batch_step_mixed(sem_batch* b, const sem_params* p, double* const* q_dev,
                         float* const* q32_dev, float* const* work32_dev, const double* dt,
                         int use_graph, cudaStream_t stream);
int sem_batch_status(sem_batch* b, int* status_host, cudaStream_t stream);

/* Learned refinement flags.  The paper notes (Sec. 5) that its velocity
 * criterion only fires once intensification has begun; this per-element
 * network predicts the criterion's flags (Sec. 3.1) some steps ahead so that
 * adaptation can run less often, with the criterion kept as fallback.
 *
 * Features (sem_mlp_features): for element e (order of sem_mesh_leaves_host,
 * column * nz + layer), the five state fields at the 27 points {-1, 0, 1}^3 of
 * the element (its polynomial evaluated there, hanging nodes interpolated),
 * field f divided by scales[f], stored at feats[e * 136 + f * 27 + a + 3 b +
 * 9 c], and the element's level at feats[e * 136 + 135]; float32, device.
 * Network: Linear(136,128)-ReLU-Linear(128,128)-ReLU-Linear(128,3), softmax
 * over (coarsen, keep, refine) = flags (-1, 0, +1).  Products run on bfloat16
 * tensor cores with float32 accumulation (inputs, weights and hidden
 * activations rounded to bfloat16); the backward pass is float32 on the same
 * rounded values; master weights and Adam moments are float32.  Parameters
 * (sem_mlp_param_count() floats): W1 [136][128] (input-major), b1 [128],
 * W2 [128][128], b2 [128], W3 [128][3], b3 [3].  sem_mlp_create draws the
 * initial weights uniform in +-1/sqrt(fan_in) from splitmix64(seed, index),
 * zero biases; max_rows bounds n for sem_mlp_backward (work arrays).
 * sem_mlp_backward: labels are classes 0..2 (= flag + 1), the loss is the
 * class-weighted mean cross-entropy sum w_y (-log p_y) / sum w_y; it leaves
 * the gradient in the handle (sem_mlp_get_grads) and, if loss_host is not
 * NULL, synchronises and returns the loss.  sem_mlp_adam applies one Adam
 * step (beta 0.9, 0.999, eps 1e-8, bias-corrected) with those gradients. */
typedef struct sem_mlp sem_mlp;
int sem_mlp_create(unsigned long long seed, int max_rows, sem_mlp** out);
void sem_mlp_destroy(sem_mlp* m);
int sem_mlp_param_count(void);
int sem_mlp_get_params(sem_mlp* m, float* params_host);
int sem_mlp_set_params(sem_mlp* m, const float* params_host);
int sem_mlp_get_grads(sem_mlp* m, float* grads_host);
int sem_mlp_features(sem_mesh* mesh, const double* q_dev, const float* scales_host,
                     float* feats_dev, cudaStream_t stream);
int sem_mlp_forward(sem_mlp* m, const float* feats_dev, int n, float* prob_dev, cudaStream_t stream);
int sem_mlp_predict_flags(sem_mlp* m, const float* feats_dev, int n, int8_t* flags_dev,
                          cudaStream_t stream);
int sem_mlp_backward(sem_mlp* m, const float* feats_dev, const int8_t* labels_dev,
                     const float* class_w_host, int n, double* loss_host, cudaStream_t stream);
int sem_mlp_adam(sem_mlp* m, float lr, cudaStream_t stream);
/* The forward pass (sem_mlp_forward, sem_mlp_predict_flags and the forward of
 * sem_mlp_backward) runs on the fifth-generation tensor cores by default
 * (tcgen05.mma kind::f16, bfloat16 operands in shared memory, float32
 * accumulators in tensor memory, 128 rows per CTA); tc = 0 selects the
 * warp-level mma.sync forward instead (same precision contract; kept for
 * comparison).  sem_mlp_status reads and clears the handle's device status
 * word (synchronises the stream): SEM_ERR_TIMEOUT if a bounded wait of the
 * tensor-core forward ran out (its outputs are then not written). */
int sem_mlp_select_forward(sem_mlp* m, int tc);
int sem_mlp_status(sem_mlp* m, int* status_host, cudaStream_t stream);

/* q32 = float32 mirror of q ([5][NG]; significand truncated to 24 bits). */
int sem_mirror(sem_mesh* m, const double* q_dev, float* q32_dev, cudaStream_t stream);

/* A whole SSP-RK3 step in place on q_dev, using two caller-owned work arrays
 * w1_dev, w2_dev of [5][NG] float64. */
int sem_step(sem_mesh* m, const sem_params* p, double* q_dev, double* w1_dev,
             double* w2_dev, double dt, cudaStream_t stream);

/* Sec. 3.1 criterion on the velocity magnitude at every local node:
 * flags[e] = +1 / -1 / 0 (refine / coarsen / keep).  Element e = column *
 * nz + layer in the order of sem_mesh_leaves_host.  The _host variant copies
 * the Ne flags to host memory and synchronises the stream; cmax (optional,
 * may be NULL) receives the per-element maximum speed. */
int sem_adapt_flags(sem_mesh* m, const sem_params* p, const double* q_dev,
                    int8_t* flags_dev, double* cmax_dev, cudaStream_t stream);
int sem_adapt_flags_host(sem_mesh* m, const sem_params* p, const double* q_dev,
                         int8_t* flags_host, cudaStream_t stream);

/* The same rule (Sec. 3.1) evaluated for other levels than the mesh's own:
 * level_dev ([Ne] int8 device array, element order as above) gives each
 * element's level; with level_dev NULL every element is taken at level_all
 * (0..lvl_max, else SEM_ERR_ARG).  The geometry (element sizes for the
 * derivatives of the vorticity and potential-vorticity criteria) stays the
 * mesh's own.  Used to schedule adaptation on levels a caller tracks itself
 * (the flag at the element's level: +1 is a refinement the criterion wants),
 * and for the labels of a flag predictor (the flag each level would get). */
int sem_adapt_flags_levels(sem_mesh* m, const sem_params* p, const double* q_dev,
                           const int8_t* level_dev, int level_all, int8_t* flags_dev,
                           double* cmax_dev, cudaStream_t stream);

/* Merges the criterion's flags with a predictor's (a learned schedule that
 * keeps the criterion as its fallback): out = +1 where either asks for
 * refinement, -1 where both ask for coarsening, else 0; a request the
 * element's level cannot take (+1 at lvl_max, -1 at level 0) counts as 0.
 * crit_dev, pred_dev, level_dev, out_dev: [n] int8 device arrays (out may
 * alias crit or pred).  The paper has no predictor; the merge is this
 * library's reading of "the criterion stays the fallback". */
int sem_merge_flags(const int8_t* crit_dev, const int8_t* pred_dev, const int8_t* level_dev,
                    int lvl_max, long long n, int8_t* out_dev, cudaStream_t stream);

/* Host only: the mesh after one adaptation pass driven by element flags
 * (Sec. 3.1: whole-column horizontal refinement, four-sibling coarsening,
 * one level per pass, 2:1 balance).  The new mesh remembers where each new
 * column comes from, for sem_transfer. */
int sem_transfer_plan(const sem_mesh* old_mesh, const int8_t* flags_host,
                      sem_mesh** new_out);

/* Solution transfer old -> new (new from sem_transfer_plan(old, ...)):
 * interpolation into refined columns, exact L2 projection into coarsened
 * ones, then projection onto the continuous constrained space.
 * q_old_dev [5][NG_old], q_new_dev [5][NG_new] float64 device arrays. */
int sem_transfer(sem_mesh* old_mesh, sem_mesh* new_mesh, const double* q_old_dev,
                 double* q_new_dev, cudaStream_t stream);

/* Wind diagnostics of Sec. 4.2 over |x|, |y| <= half_width; returns host
 * data and synchronises the stream. */
int sem_diag(sem_mesh* m, const sem_params* p, const double* q_dev, double half_width,
             sem_diag_out* out_host, cudaStream_t stream);

/* Reads and clears the device status word that the stage kernels set when
 * they write a non-finite value; synchronises the stream.  *status_host is 0
 * (clean) or SEM_ERR_NUMERIC. */
int sem_status(sem_mesh* m, int* status_host, cudaStream_t stream);

/* Arithmetic-rate probe: the float32 (precision = SEM_PREC_MIXED) or float64
 * (SEM_PREC_FP64) FMA rate of the current GPU in TFLOP/s (2 flop per FMA),
 * from independent FMA chains in 8 blocks of 256 threads per SM; best of
 * three timed launches after a warm-up (CUDA events on `stream`).  The
 * denominators of the element kernels' ALU rooflines.  Allocates and frees
 * a small output buffer (stream-ordered); synchronises the stream.  The
 * paper has no counterpart. */
int sem_peak_probe(int precision, double* tflops_host, cudaStream_t stream);

/* Host-only check of the library's one-time set-up per device (no GPU
 * needed).  The library uploads its constant tables and sets its kernel
 * attributes once per device ordinal, on the first call that needs them on
 * that device.  This call drives that mechanism for the simulated ordinals
 * 0..n_devices-1 from n_threads host threads at once (each thread asks for
 * every ordinal three times, in a different order) and writes to
 * init_calls_host[d] how many times the set-up ran for ordinal d (1 when the
 * mechanism is correct).  n_devices in 1..64, n_threads in 1..64, else
 * SEM_ERR_ARG; an ordinal outside 0..63 is refused by the mechanism itself,
 * which this call also checks (SEM_ERR_ARG from the call if it were not). */
int sem_selftest_device_once(int n_devices, int n_threads, int* init_calls_host);

/* Autotuner of the mixed-form element kernel.  Times every launch variant
 * compiled for the mesh's order and p->eqset's equation set (layers of a
 * column per CTA, and the number of CTAs per SM the register budget is sized
 * for) on the float32 state mirror q32_dev, `reps` launches each after two
 * warm-up launches, keeps the fastest for this mesh and that set (used by
 * sem_rk_stage, sem_rk_stage_mixed and sem_step_mixed afterwards; the two
 * sets' choices are kept apart) and reports all timings.  Warped layers: the
 * line-exchange rows only.  Synchronises the stream; overwrites the mesh's
 * residual scratch. */
#define SEM_TUNE_MAX 16
typedef struct {
  int n_variants;
  int chosen;                          /* index into the arrays below */
  int layers_per_cta[SEM_TUNE_MAX];
  int min_ctas_per_sm[SEM_TUNE_MAX];
  int kind[SEM_TUNE_MAX];              /* 0: z-pencil kernel, 1: line-exchange kernel,
                                          2: line exchange with the x, y contractions on tensor cores,
                                          4: line exchange with the state staged by bulk copies (TMA),
                                          5: line exchange for the paper's equation set */
  double ms[SEM_TUNE_MAX];             /* mean event time per launch */
} sem_tune_out;
int sem_autotune(sem_mesh* m, const sem_params* p, const float* q32_dev, int reps,
                 sem_tune_out* out_host, cudaStream_t stream);
/* Selects row `row` of the table sem_autotune reports for this mesh's order
 * and equation set `eqset` (SEM_EQ_*; 0 <= row < n_variants) as the mesh's
 * element-kernel variant for that set, or the untuned default for row = -1;
 * no timing and no device work.  For tests that run every variant, and for
 * callers that cache a tuning result.  The paper has no counterpart (launch
 * configuration only).  SEM_ERR_ARG for a row outside the table or an
 * unknown set. */
int sem_autotune_select(sem_mesh* m, int eqset, int row);

/* Checkpoint / resume.  sem_checkpoint_write copies the float64 state to the
 * host (synchronises the stream) and writes the mesh description, its leaf
 * columns, its layer faces, its warped-layer parameters, the state, `time`
 * and `step`, and a checksum (format SEMCKPT3; files of the earlier SEMCKPT2
 * format give SEM_ERR_IO), through a temporary
 * file renamed into place.  sem_checkpoint_read_mesh rebuilds the mesh (host
 * only; same leaves, hence the same node numbering) and returns time and step;
 * sem_checkpoint_read_state copies the state into q_dev ([5][NG]) after
 * checking that the file was written for that mesh.  A missing, truncated or
 * corrupted file gives SEM_ERR_IO before any device work. */
int sem_checkpoint_write(sem_mesh* m, const double* q_dev, double time, long long step,
                         const char* path, cudaStream_t stream);
int sem_checkpoint_read_mesh(const char* path, sem_mesh** mesh_out, double* time_out,
                             long long* step_out);
int sem_checkpoint_read_state(const char* path, sem_mesh* m, double* q_dev, cudaStream_t stream);

/* Kernel timing.  Between sem_profile_begin and sem_profile_end every kernel
 * the library launches is bracketed by CUDA events recorded on the stream it
 * is launched on.  sem_profile_end synchronises those streams and returns, per
 * kernel name, the number of launches and the summed event time in
 * milliseconds.  At most SEM_PROFILE_MAX kernel names and 1 << 16 launches
 * are recorded per session; later launches are not timed.  Not thread-safe. */
#define SEM_PROFILE_MAX 16
typedef struct {
  int n_kernels;
  char name[SEM_PROFILE_MAX][48];
  long long launches[SEM_PROFILE_MAX];
  double ms_total[SEM_PROFILE_MAX];
} sem_profile_out;
int sem_profile_begin(void);
int sem_profile_end(sem_profile_out* out_host);

#ifdef __cplusplus
}
#endif
#endif /* SEM_H */
