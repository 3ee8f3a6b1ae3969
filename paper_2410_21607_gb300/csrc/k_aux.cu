// Criterion, diagnostics and coordinate kernels.
//
//   adapt_column<N, EQ>: Sec. 3.1 threshold criterion.  One CTA per leaf
//     column; per element the criterion variables at every local node
//     (hanging nodes interpolated as in the modified DSS), their element
//     maxima, and the flag
//       +1 if max C^(lvl+1) > threshold(lvl+1) and lvl < lvl_max,
//       -1 if max C^lvl <= threshold(lvl) and lvl > 0, else 0,
//     with C^l the variable chosen for level l (speed by default; vertical
//     vorticity or dry Ertel potential vorticity from element-local
//     derivatives).  The speed is evaluated with explicitly rounded float64
//     operations (sqrt(U U + V V + W W) / rho in that order, no contraction
//     into FMA) so that the decision is taken in float64 exactly as written.
//   diag_level: Sec. 4.2 diagnostics, one CTA per vertical level: maximum
//     horizontal speed and the mass-weighted mean speed over the horizontal
//     sub-domain |x|, |y| <= half_width, reduced in a fixed order.
#include <algorithm>

#include "sem_internal.h"

namespace sem {

__constant__ double a_D[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];  // [i][m] = h_m'(xi_i)

static int upload_aux_constants_now() {
  double D[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)] = {};
  for (int N = 2; N <= kMaxN; ++N) {
    const Basis1D& B = basis(N);
    for (int k = 0; k < (N + 1) * (N + 1); ++k) D[N][k] = B.D[k];
  }
  SEM_CUDA_TRY(cudaMemcpyToSymbol(a_D, D, sizeof(D)));
  return SEM_OK;
}

// the tables of the current device (uploaded on its first use)
static int upload_aux_constants() {
  static DeviceOnce once;
  return device_once(once, upload_aux_constants_now);
}

struct AdaptArgs {
  const double* q;
  const int* hmap;
  const int* hang_h;
  const double* hang_w;
  const int* col_level;
  const double* ref;
  const double* refG;             // warped layers: reference rows per node and hanging line, else null
  const double* refH;
  int8_t* flags;
  double* cmax;
  int nz, NZ;
  long long NG;
  int lvl_max;
  int need_grad;                  // 1: vorticity, 2: also potential vorticity
  double f;
  double thr[SEM_MAX_THRESHOLDS];
  int var[SEM_MAX_THRESHOLDS];    // SEM_CRIT_* per threshold
  double gx[16], gy[16];          // 2 / h per level
  const double* hzk;              // [nz] layer thicknesses
  // level the rule is evaluated for: per element (elem_level, [Ne]), or one
  // level for every element (level_all >= 0), else the column's own level;
  // the geometry always uses the column's level
  const int8_t* elem_level;
  int level_all;
  // warped layers: z_xi, z_eta, z_zeta per node of each column line
  // ([Ncol][Nq][nz][N+1][3]), else null
  const double* metric;
};

template <int N, int EQ>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
adapt_column(const AdaptArgs A) {
  constexpr int n1 = N + 1, Nq = n1 * n1, P = n1 * n1 * n1;
  constexpr int NW = (P + 31) / 32;
  __shared__ double red[3][NW];
  __shared__ double sQ[4][P];     // u, v, w, theta at the element's nodes
  const int col = blockIdx.x, t = threadIdx.x;
  const bool act = t < P;
  const int i = t % n1, j = (t / n1) % n1, c = t / Nq;
  const int ab = i + n1 * j;
  const int hm = act ? A.hmap[(long long)col * Nq + ab] : 0;
  const int geo_lev = A.col_level[col];
  for (int k = 0; k < A.nz; ++k) {
    double s = 0.0, zeta = 0.0, pv = 0.0, rho = 1.0;
    if (act) {
      const int kz = k * N + c;
      double v[kFields] = {0, 0, 0, 0, 0};
      if (hm >= 0) {
        const double* p = A.q + (long long)hm * A.NZ + kz;
        for (int f = 0; f < kFields; ++f) v[f] = p[(long long)f * A.NG];
      } else {
        const int h = -1 - hm;
        for (int m = 0; m <= N; ++m) {
          const double w = A.hang_w[h * n1 + m];
          const double* p = A.q + (long long)A.hang_h[h * n1 + m] * A.NZ + kz;
          for (int f = 0; f < kFields; ++f) v[f] = __dadd_rn(v[f], __dmul_rn(w, p[(long long)f * A.NG]));
        }
      }
      double ss = __dadd_rn(__dadd_rn(__dmul_rn(v[1], v[1]), __dmul_rn(v[2], v[2])), __dmul_rn(v[3], v[3]));
      s = __dsqrt_rn(ss);
      const double* rf = !A.refG ? A.ref + (long long)kz * kRef
                         : (hm >= 0 ? A.refG + ((long long)hm * A.NZ + kz) * kRef
                                    : A.refH + ((long long)(-1 - hm) * A.NZ + kz) * kRef);
      rho = rf[3] + v[0];
      if (EQ == 0) s = __ddiv_rn(s, __dadd_rn(rf[3], v[0]));
      if (A.need_grad) {
        if (EQ == 0) {
          sQ[0][t] = v[1] / rho;
          sQ[1][t] = v[2] / rho;
          sQ[2][t] = v[3] / rho;
          sQ[3][t] = (rf[4] + v[4]) / rho;
        } else {
          sQ[0][t] = v[1];
          sQ[1][t] = v[2];
          sQ[2][t] = v[3];
          sQ[3][t] = rf[0] + v[4];
        }
      }
    }
    if (A.need_grad) {
      __syncthreads();
      if (act) {
        // element-local derivatives d/dx (along i), d/dy (along j), d/dz (along c)
        double d[4][3] = {};
        for (int m = 0; m < n1; ++m) {
          const double Di = a_D[N][i * n1 + m], Dj = a_D[N][j * n1 + m], Dc = a_D[N][c * n1 + m];
          const int lx = m + n1 * j + Nq * c, ly = i + n1 * m + Nq * c, lz = i + n1 * j + Nq * m;
          for (int qv = 0; qv < 4; ++qv) {
            d[qv][0] += Di * sQ[qv][lx];
            d[qv][1] += Dj * sQ[qv][ly];
            d[qv][2] += Dc * sQ[qv][lz];
          }
        }
        const double gx = A.gx[geo_lev], gy = A.gy[geo_lev];
        if (A.metric) {
          // warped layers: derivatives at constant height through the node's
          // metric, d/dx = (2/hx) (d/dxi - (z_xi / z_zeta) d/dzeta), d/dz = d/dzeta / z_zeta
          const double* mt = A.metric + ((((long long)col * Nq + ab) * A.nz + k) * n1 + c) * 3;
          const double zx = mt[0], zy = mt[1], zz = mt[2];
          for (int qv = 0; qv < 4; ++qv) {
            const double dz = d[qv][2] / zz;
            d[qv][0] = gx * (d[qv][0] - zx * dz);
            d[qv][1] = gy * (d[qv][1] - zy * dz);
            d[qv][2] = dz;
          }
        } else {
          const double gz = 2.0 / A.hzk[k];
          for (int qv = 0; qv < 4; ++qv) {
            d[qv][0] *= gx;
            d[qv][1] *= gy;
            d[qv][2] *= gz;
          }
        }
        const double wz = d[1][0] - d[0][1];
        zeta = fabs(wz);
        if (A.need_grad > 1) {
          const double wx = d[2][1] - d[1][2], wy = d[0][2] - d[2][0];
          pv = fabs(wx * d[3][0] + wy * d[3][1] + (wz + A.f) * d[3][2]) / rho;
        }
      }
    }
    // block maxima over the element's nodes
    double mv[3] = {s, zeta, pv};
    for (int cv = 0; cv < 3; ++cv) {
      double x = mv[cv];
      for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
      if ((t & 31) == 0) red[cv][t >> 5] = x;
    }
    __syncthreads();
    if (t == 0) {
      double mx[3];
      for (int cv = 0; cv < 3; ++cv) {
        mx[cv] = red[cv][0];
        for (int w = 1; w < NW; ++w) mx[cv] = fmax(mx[cv], red[cv][w]);
      }
      const long long e = (long long)col * A.nz + k;
      const int lev = A.elem_level ? (int)A.elem_level[e] : (A.level_all >= 0 ? A.level_all : geo_lev);
      int flag = 0;
      if (lev < A.lvl_max && mx[A.var[lev]] > A.thr[lev]) flag = 1;
      else if (lev > 0 && mx[A.var[lev - 1]] <= A.thr[lev - 1]) flag = -1;
      A.flags[e] = (int8_t)flag;
      if (A.cmax) {
        const int test = lev < A.lvl_max ? lev : lev - 1;
        A.cmax[e] = mx[(test >= 0 && test < SEM_MAX_THRESHOLDS) ? A.var[test] : A.var[0]];
      }
    }
    __syncthreads();
  }
}

template <int N>
static void launch_adapt_n(const AdaptArgs& A, int ncol, int eq, cudaStream_t st) {
  constexpr int P = (N + 1) * (N + 1) * (N + 1);
  constexpr int nt = (P + 31) / 32 * 32;
  if (eq == 0)
    adapt_column<N, 0><<<ncol, nt, 0, st>>>(A);
  else
    adapt_column<N, 1><<<ncol, nt, 0, st>>>(A);
}

int launch_adapt(Mesh& m, const sem_params& p, const double* q, int8_t* flags, double* cmax,
                 cudaStream_t st, const int8_t* elem_level, int level_all) {
  DeviceTables& D = *m.dev;
  AdaptArgs A;
  A.elem_level = elem_level;
  A.level_all = level_all;
  A.q = q;
  A.hmap = D.hmap;
  A.hang_h = D.hang_h;
  A.hang_w = D.hang_w;
  A.col_level = D.col_level;
  A.ref = D.ref;
  A.refG = m.warped() ? D.refG : nullptr;
  A.refH = m.warped() ? D.refH : nullptr;
  A.flags = flags;
  A.cmax = cmax;
  A.nz = m.nz;
  A.NZ = m.NZ;
  A.NG = m.NG;
  A.lvl_max = p.lvl_max;
  A.need_grad = 0;
  for (int k = 0; k < SEM_MAX_THRESHOLDS; ++k) {
    A.thr[k] = p.thresholds[k];
    A.var[k] = p.criterion[k];
    // only the thresholds the levels use decide whether derivatives are needed
    if (k < p.n_thresholds && k < std::max(p.lvl_max, 1))
      A.need_grad = std::max(A.need_grad, p.criterion[k] == SEM_CRIT_PV ? 2 : (p.criterion[k] == SEM_CRIT_VORTICITY ? 1 : 0));
  }
  A.f = p.f;
  for (int l = 0; l < 16; ++l) {
    A.gx[l] = 2.0 / m.hx(l);
    A.gy[l] = 2.0 / m.hy(l);
  }
  A.hzk = D.hzk;
  A.metric = m.warped() ? D.metric : nullptr;
  if (A.need_grad) {
    int rc = upload_aux_constants();
    if (rc) return rc;
  }
  const int nc = (int)m.Ncol();
  switch (m.N) {
    case 2: launch_adapt_n<2>(A, nc, p.eqset, st); break;
    case 3: launch_adapt_n<3>(A, nc, p.eqset, st); break;
    case 4: launch_adapt_n<4>(A, nc, p.eqset, st); break;
    case 5: launch_adapt_n<5>(A, nc, p.eqset, st); break;
    case 6: launch_adapt_n<6>(A, nc, p.eqset, st); break;
    default: return fail(SEM_ERR_UNSUPPORTED, "order N not compiled");
  }
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
diag_level(const double* q, const double* xh, const double* yh, const double* Mh,
           const double* ref, long long NH, int NZ, long long NG, double hw, int eq,
           const double* refG, const double* Minv_g, double* out /*[NZ][4]*/) {
  __shared__ double s_max[256], s_num[256], s_den[256];
  const int kz = blockIdx.x;
  const double rho0 = ref[(long long)kz * kRef + 3];
  double mx = 0.0, num = 0.0, den = 0.0;
  for (long long h = threadIdx.x; h < NH; h += blockDim.x) {
    if (!(fabs(xh[h]) <= hw + 1e-6 && fabs(yh[h]) <= hw + 1e-6)) continue;
    const long long g = h * NZ + kz;
    const double U = q[NG + g], V = q[2 * NG + g];
    double s = sqrt(U * U + V * V);
    // warped layers: the node's own reference density and lumped mass (the
    // level means are then over a grid level, not a height)
    if (eq == 0) s = s / ((refG ? refG[g * kRef + 3] : rho0) + q[g]);
    const double wm = Minv_g ? 1.0 / Minv_g[g] : Mh[h];
    mx = fmax(mx, s);
    num += wm * s;
    den += wm;
  }
  s_max[threadIdx.x] = mx;
  s_num[threadIdx.x] = num;
  s_den[threadIdx.x] = den;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
      s_num[threadIdx.x] += s_num[threadIdx.x + o];
      s_den[threadIdx.x] += s_den[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[kz * 4 + 0] = s_max[0];
    out[kz * 4 + 1] = s_num[0];
    out[kz * 4 + 2] = s_den[0];
    out[kz * 4 + 3] = 0.0;
  }
}

int launch_diag(Mesh& m, const sem_params& p, const double* q, double hw, sem_diag_out* out,
                cudaStream_t st) {
  DeviceTables& D = *m.dev;
  diag_level<<<m.NZ, 256, 0, st>>>(q, D.xh, D.yh, D.Mh, D.ref, m.NH, m.NZ, m.NG, hw, p.eqset,
                                    m.warped() ? D.refG : nullptr, m.warped() ? D.Minv_g : nullptr,
                                    D.diag_buf);
  SEM_CUDA_TRY(cudaGetLastError());
  std::vector<double> buf((size_t)m.NZ * 4);
  SEM_CUDA_TRY(cudaMemcpyAsync(buf.data(), D.diag_buf, buf.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, st));
  SEM_CUDA_TRY(cudaStreamSynchronize(st));
  double mx = 0.0, mm = -1.0;
  for (int k = 0; k < m.NZ; ++k) {
    mx = std::max(mx, buf[k * 4]);
    if (buf[k * 4 + 2] > 0) mm = std::max(mm, buf[k * 4 + 1] / buf[k * 4 + 2]);
  }
  if (mm < 0) return fail(SEM_ERR_ARG, "no node inside the diagnostic sub-domain");
  out->max_wind = mx;
  out->max_mean_wind = mm;
  return SEM_OK;
}

// ---------------------------------------------------------------------------
// Criterion flags merged with a predictor's flags (the learned schedule, the
// criterion kept as the fallback): refine when either asks, coarsen only when
// both do, keep otherwise; a request the element's level cannot take (refine
// at lvl_max, coarsen at level 0) counts as keep.
__global__ void merge_flags_kernel(const int8_t* crit, const int8_t* pred, const int8_t* level, int lvl_max,
                                   long long n, int8_t* out) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int L = level[e];
    int c = crit[e], p = pred[e];
    if (L >= lvl_max) { c = c > 0 ? 0 : c; p = p > 0 ? 0 : p; }
    if (L <= 0) { c = c < 0 ? 0 : c; p = p < 0 ? 0 : p; }
    out[e] = (int8_t)((c > 0 || p > 0) ? 1 : ((c < 0 && p < 0) ? -1 : 0));
  }
}

int launch_merge_flags(const int8_t* crit, const int8_t* pred, const int8_t* level, int lvl_max, long long n,
                       int8_t* out, cudaStream_t st) {
  const long long blocks = std::max<long long>(1, std::min<long long>((n + 255) / 256, 152 * 8));
  merge_flags_kernel<<<(int)blocks, 256, 0, st>>>(crit, pred, level, lvl_max, n, out);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

// ---------------------------------------------------------------------------
__global__ void coords_kernel(const double* xh, const double* yh, const double* zk, long long NH,
                              int NZ, const double* zG, double* xyz) {
  const long long NG = NH * NZ;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < NG;
       g += (long long)gridDim.x * blockDim.x) {
    const long long h = g / NZ;
    const int k = (int)(g - h * NZ);
    xyz[g] = xh[h];
    xyz[NG + g] = yh[h];
    xyz[2 * NG + g] = zG ? zG[g] : zk[k];
  }
}

int launch_coords(Mesh& m, double* xyz, cudaStream_t st) {
  DeviceTables& D = *m.dev;
  long long blocks = std::min<long long>((m.NG + 255) / 256, 152 * 16);
  coords_kernel<<<(int)blocks, 256, 0, st>>>(D.xh, D.yh, D.zk, m.NH, m.NZ, m.warped() ? D.zG : nullptr, xyz);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
