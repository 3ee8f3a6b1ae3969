// Right-hand side and Runge-Kutta stage kernels.
//
//   volume_column<N, EQ, R>: one CTA per leaf column marches up its nz
//     layers.  Per element it gathers the state through the column's
//     horizontal map (hanging rows interpolated, Sec. 3.1), forms the
//     pointwise fluxes and sources of the split equations (Sec. 2), contracts
//     them with the weak-form derivative matrix (Sec. 3, sum factorisation),
//     adds the face shared with the layer below (vertical DSS inside the
//     CTA) and writes the column residual r_C[column][ab][field][kz].
//   dss_stage<R>: one thread per global node gathers the horizontal
//     contributions through Q_h^T (Sec. 3.1, modified DSS), divides by the
//     lumped mass, applies the rigid-lid condition and fuses the RK stage
//     update  q_out = a qn + b qs + c dt R / M.
//
// R is the arithmetic type of the element work: double for the FP64 form,
// float for the mixed form (perturbation arithmetic in float32; reference
// state and metric terms from float64 tables; stage accumulation in float64).
#include <cstdio>

#include "sem_internal.h"

namespace sem {

__constant__ double c_xi[kMaxN + 1][kMaxN + 1];
__constant__ double c_w[kMaxN + 1][kMaxN + 1];
__constant__ double c_Dw[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];  // [i][m] = w_m D[m][i]
__constant__ double c_D[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];   // [i][m] = h_m'(xi_i)

int upload_basis_constants() {
  static bool done = false;
  if (done) return SEM_OK;
  double xi[kMaxN + 1][kMaxN + 1] = {}, w[kMaxN + 1][kMaxN + 1] = {};
  double Dw[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)] = {};
  double D[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)] = {};
  for (int N = 2; N <= kMaxN; ++N) {
    const Basis1D& B = basis(N);
    const int n = N + 1;
    for (int i = 0; i < n; ++i) {
      xi[N][i] = B.xi[i];
      w[N][i] = B.w[i];
      for (int m = 0; m < n; ++m) {
        Dw[N][i * n + m] = B.w[m] * B.D[m * n + i];
        D[N][i * n + m] = B.D[i * n + m];
      }
    }
  }
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_xi, xi, sizeof(xi)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_w, w, sizeof(w)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_Dw, Dw, sizeof(Dw)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_D, D, sizeof(D)));
  done = true;
  return SEM_OK;
}

struct VolArgs {
  const double* q;
  void* rc;
  const int* hmap;
  const int* hang_h;
  const double* hang_w;
  const int* col_level;
  const double* ref;
  int Ncol, nz, NZ;
  long long NH, NG;
  double Lx, Ly, Lz;
  int nx, ny;
  double g, f, gamma;
};

template <typename R> __device__ __forceinline__ R r_log1p(R x);
template <> __device__ __forceinline__ double r_log1p<double>(double x) { return log1p(x); }
template <> __device__ __forceinline__ float r_log1p<float>(float x) { return log1pf(x); }
template <typename R> __device__ __forceinline__ R r_expm1(R x);
template <> __device__ __forceinline__ double r_expm1<double>(double x) { return expm1(x); }
template <> __device__ __forceinline__ float r_expm1<float>(float x) { return expm1f(x); }

// Gather the 5 fields of local node (ab, kz) of a column (Q row, Sec. 3.1).
template <int N>
__device__ __forceinline__ void gather_node(const VolArgs& A, int hm, int kz, double v[kFields]) {
  if (hm >= 0) {
    const double* p = A.q + (long long)hm * A.NZ + kz;
#pragma unroll
    for (int f = 0; f < kFields; ++f) v[f] = __ldg(p + (long long)f * A.NG);
  } else {
    const int k = -1 - hm;
#pragma unroll
    for (int f = 0; f < kFields; ++f) v[f] = 0.0;
#pragma unroll
    for (int m = 0; m <= N; ++m) {
      const double wm = __ldg(A.hang_w + k * (N + 1) + m);
      const double* p = A.q + (long long)__ldg(A.hang_h + k * (N + 1) + m) * A.NZ + kz;
#pragma unroll
      for (int f = 0; f < kFields; ++f) v[f] += wm * __ldg(p + (long long)f * A.NG);
    }
  }
}

template <int N, int EQ, typename R>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
volume_column(const VolArgs A) {
  constexpr int n1 = N + 1, Nq = n1 * n1, P = n1 * n1 * n1;
  // EQ 0: 15 weak flux components.  EQ 1: 3 weak mass-flux components plus
  // 5 pointwise quantities (u, v, w, p', theta') for strong derivatives.
  constexpr int NS = EQ == 0 ? 15 : 8;
  __shared__ R sF[NS][P];
  __shared__ R sC[2][kFields][Nq];
  const int col = blockIdx.x;
  const int t = threadIdx.x;
  const bool act = t < P;
  const int i = t % n1, j = (t / n1) % n1, c = t / Nq;
  const int ab = i + n1 * j;
  const int lev = A.col_level[col];
  const double hx = A.Lx / (double)((long long)A.nx << lev);
  const double hy = A.Ly / (double)((long long)A.ny << lev);
  const double hz = A.Lz / A.nz;
  const double J = hx * hy * hz * 0.125;
  int hm = 0;
  R Dwi[n1], Dwj[n1], Dwc[n1];
  R wi = 0, wj = 0, wc = 0;
  if (act) {
    hm = A.hmap[(long long)col * Nq + ab];
#pragma unroll
    for (int m = 0; m < n1; ++m) {
      if (EQ == 0) {
        Dwi[m] = (R)c_Dw[N][i * n1 + m];
        Dwj[m] = (R)c_Dw[N][j * n1 + m];
        Dwc[m] = (R)c_Dw[N][c * n1 + m];
      } else {
        Dwi[m] = (R)c_D[N][i * n1 + m];
        Dwj[m] = (R)c_D[N][j * n1 + m];
        Dwc[m] = (R)c_D[N][c * n1 + m];
      }
    }
    wi = (R)c_w[N][i];
    wj = (R)c_w[N][j];
    wc = (R)c_w[N][c];
  }
  // weak-form factors: J dxi/dx = hy hz / 4 etc.
  const R sx = (R)(hy * hz * 0.25), sy = (R)(hx * hz * 0.25), sz = (R)(hx * hy * 0.25);
  const R wJ = (R)((double)c_w[N][i] * c_w[N][j] * c_w[N][c] * J);
  const R gx = (R)(2.0 / hx), gy = (R)(2.0 / hy), gz = (R)(2.0 / hz);
  const R g = (R)A.g, fc = (R)A.f, gam = (R)A.gamma;
  R* rc = (R*)A.rc;

  for (int k = 0; k < A.nz; ++k) {
    const int kz = k * N + c;
    R S[kFields] = {0, 0, 0, 0, 0};
    R pw[5] = {0, 0, 0, 0, 0};  // EQ 1: u, v, w, rho, rho' kept for the strong terms
    R th0dz = 0;
    if (act) {
      double v[kFields];
      gather_node<N>(A, hm, kz, v);
      const double* rf = A.ref + (long long)kz * kRef;
      const R p0 = (R)rf[2], rho0 = (R)rf[3], rt0 = (R)rf[4], inv_rt0 = (R)rf[6];
      const R rp = (R)v[0];
      const R rho = rho0 + rp;
      const R inv = (R)1 / rho;
      if (EQ == 0) {
        const R U = (R)v[1], V = (R)v[2], W = (R)v[3], Tp = (R)v[4];
        const R u = U * inv, vv = V * inv, w = W * inv;
        const R pp = p0 * r_expm1<R>(gam * r_log1p<R>(Tp * inv_rt0));
        const R rt = rt0 + Tp;
        const R ax = wj * wc * sx, ay = wi * wc * sy, az = wi * wj * sz;
        sF[0][t] = U * ax;            sF[1][t] = V * ay;            sF[2][t] = W * az;
        sF[3][t] = (U * u + pp) * ax; sF[4][t] = U * vv * ay;       sF[5][t] = U * w * az;
        sF[6][t] = V * u * ax;        sF[7][t] = (V * vv + pp) * ay; sF[8][t] = V * w * az;
        sF[9][t] = W * u * ax;        sF[10][t] = W * vv * ay;      sF[11][t] = (W * w + pp) * az;
        sF[12][t] = rt * u * ax;      sF[13][t] = rt * vv * ay;     sF[14][t] = rt * w * az;
        S[1] = wJ * (fc * V);
        S[2] = wJ * (-fc * U);
        S[3] = wJ * (-rp * g);
      } else {
        const R u = (R)v[1], vv = (R)v[2], w = (R)v[3], thp = (R)v[4];
        const R th0 = (R)rf[0];
        const R rtp = rho0 * thp + rp * (th0 + thp);
        const R pp = p0 * r_expm1<R>(gam * r_log1p<R>(rtp * inv_rt0));
        const R ax = wj * wc * sx, ay = wi * wc * sy, az = wi * wj * sz;
        sF[0][t] = rho * u * ax;
        sF[1][t] = rho * vv * ay;
        sF[2][t] = rho * w * az;
        sF[3][t] = u;
        sF[4][t] = vv;
        sF[5][t] = w;
        sF[6][t] = pp;
        sF[7][t] = thp;
        pw[0] = u; pw[1] = vv; pw[2] = w; pw[3] = inv; pw[4] = rp;
        th0dz = (R)rf[5];
      }
    }
    __syncthreads();
    R r[kFields];
    if (act) {
      if (EQ == 0) {
#pragma unroll
        for (int fl = 0; fl < kFields; ++fl) {
          R acc = S[fl];
#pragma unroll
          for (int m = 0; m < n1; ++m) {
            acc += Dwi[m] * sF[3 * fl + 0][m + n1 * j + Nq * c];
            acc += Dwj[m] * sF[3 * fl + 1][i + n1 * m + Nq * c];
            acc += Dwc[m] * sF[3 * fl + 2][i + n1 * j + Nq * m];
          }
          r[fl] = acc;
        }
      } else {
        // weak mass flux needs w_m D[m][i]; Dwi holds D[i][m] here
        R acc = 0;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          acc += (R)c_Dw[N][i * n1 + m] * sF[0][m + n1 * j + Nq * c];
          acc += (R)c_Dw[N][j * n1 + m] * sF[1][i + n1 * m + Nq * c];
          acc += (R)c_Dw[N][c * n1 + m] * sF[2][i + n1 * j + Nq * m];
        }
        r[0] = acc;
        R dq[5][3];
#pragma unroll
        for (int qv = 0; qv < 5; ++qv) {
          R ax_ = 0, ay_ = 0, az_ = 0;
#pragma unroll
          for (int m = 0; m < n1; ++m) {
            ax_ += Dwi[m] * sF[3 + qv][m + n1 * j + Nq * c];
            ay_ += Dwj[m] * sF[3 + qv][i + n1 * m + Nq * c];
            az_ += Dwc[m] * sF[3 + qv][i + n1 * j + Nq * m];
          }
          dq[qv][0] = ax_ * gx;
          dq[qv][1] = ay_ * gy;
          dq[qv][2] = az_ * gz;
        }
        const R u = pw[0], vv = pw[1], w = pw[2], inv = pw[3], rp = pw[4];
        auto adv = [&](int qv) { return u * dq[qv][0] + vv * dq[qv][1] + w * dq[qv][2]; };
        r[1] = wJ * (-adv(0) - dq[3][0] * inv + fc * vv);
        r[2] = wJ * (-adv(1) - dq[3][1] * inv - fc * u);
        r[3] = wJ * (-adv(2) - dq[3][2] * inv - rp * inv * g);
        r[4] = wJ * (-w * th0dz - adv(4));
      }
      // vertical direct stiffness summation inside the column
      if (c == 0 && k > 0) {
#pragma unroll
        for (int fl = 0; fl < kFields; ++fl) r[fl] += sC[(k - 1) & 1][fl][ab];
      }
      if (c == N && k < A.nz - 1) {
#pragma unroll
        for (int fl = 0; fl < kFields; ++fl) sC[k & 1][fl][ab] = r[fl];
      } else {
        R* dst = rc + ((long long)((long long)col * Nq + ab) * kFields) * A.NZ + kz;
#pragma unroll
        for (int fl = 0; fl < kFields; ++fl) dst[(long long)fl * A.NZ] = r[fl];
      }
    }
    __syncthreads();
  }
}

struct DssArgs {
  const void* rc;
  const int* qt_ptr;
  const int* qt_src;
  const double* qt_w;
  const double* Minv_h;
  const double* Minv_z;
  const double* qn;
  const double* qs;
  double* out;
  double a, b, cdt;
  int rhs_only;
  long long NH, NG;
  int NZ;
  int* status;
};

template <typename R>
__global__ void __launch_bounds__(256) dss_stage(const DssArgs A) {
  const R* rc = (const R*)A.rc;
  int bad = 0;
  for (long long gidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; gidx < A.NG;
       gidx += (long long)gridDim.x * blockDim.x) {
    const long long h = gidx / A.NZ;
    const int kz = (int)(gidx - h * A.NZ);
    const int beg = __ldg(A.qt_ptr + h), end = __ldg(A.qt_ptr + h + 1);
    const double minv = __ldg(A.Minv_h + h) * __ldg(A.Minv_z + kz);
    const bool lid = (kz == 0) || (kz == A.NZ - 1);
    // FP64 form: float64 sums; mixed form: float32 sums of the float32
    // element residuals, converted once for the float64 stage update.
    R acc[kFields] = {0, 0, 0, 0, 0};
    for (int e = beg; e < end; ++e) {
      const R w = (R)__ldg(A.qt_w + e);
      const R* p = rc + (long long)__ldg(A.qt_src + e) * kFields * A.NZ + kz;
#pragma unroll
      for (int fl = 0; fl < kFields; ++fl) acc[fl] += w * p[(long long)fl * A.NZ];
    }
#pragma unroll
    for (int fl = 0; fl < kFields; ++fl) {
      double T = (double)acc[fl] * minv;
      if (fl == 3 && lid) T = 0.0;
      const long long o = (long long)fl * A.NG + gidx;
      double val;
      if (A.rhs_only) {
        val = T;
      } else {
        val = A.b * __ldg(A.qs + o) + A.cdt * T;
        if (A.a != 0.0) val += A.a * __ldg(A.qn + o);
      }
      A.out[o] = val;
      bad |= !isfinite(val);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(A.status, 1);
}

template <int N, int EQ, typename R>
static void launch_volume(const VolArgs& A, cudaStream_t st) {
  constexpr int P = (N + 1) * (N + 1) * (N + 1);
  constexpr int nt = (P + 31) / 32 * 32;
  ProfScope ps(sizeof(R) == 8 ? "volume_fp64" : "volume_mixed", st);
  volume_column<N, EQ, R><<<A.Ncol, nt, 0, st>>>(A);
}

template <int N>
static void launch_volume_n(const VolArgs& A, int eq, bool mixed, cudaStream_t st) {
  if (eq == 0) {
    if (mixed) launch_volume<N, 0, float>(A, st); else launch_volume<N, 0, double>(A, st);
  } else {
    if (mixed) launch_volume<N, 1, float>(A, st); else launch_volume<N, 1, double>(A, st);
  }
}

int launch_rhs_stage(Mesh& m, const sem_params& p, const StageArgs& s, cudaStream_t st) {
  int rc = upload_basis_constants();
  if (rc) return rc;
  DeviceTables& D = *m.dev;
  const bool mixed = p.precision == SEM_PREC_MIXED;
  VolArgs A;
  A.q = s.qs;
  A.rc = D.scratch;
  A.hmap = D.hmap;
  A.hang_h = D.hang_h;
  A.hang_w = D.hang_w;
  A.col_level = D.col_level;
  A.ref = D.ref;
  A.Ncol = (int)m.Ncol();
  A.nz = m.nz;
  A.NZ = m.NZ;
  A.NH = m.NH;
  A.NG = m.NG;
  A.Lx = m.Lx;
  A.Ly = m.Ly;
  A.Lz = m.Lz;
  A.nx = m.nx;
  A.ny = m.ny;
  A.g = p.g;
  A.f = p.f;
  A.gamma = p.c_p / (p.c_p - p.R_d);
  const int eq = p.eqset;
  switch (m.N) {
    case 2: launch_volume_n<2>(A, eq, mixed, st); break;
    case 3: launch_volume_n<3>(A, eq, mixed, st); break;
    case 4: launch_volume_n<4>(A, eq, mixed, st); break;
    case 5: launch_volume_n<5>(A, eq, mixed, st); break;
    case 6: launch_volume_n<6>(A, eq, mixed, st); break;
    default: return fail(SEM_ERR_UNSUPPORTED, "order N not compiled");
  }
  SEM_CUDA_TRY(cudaGetLastError());
  DssArgs B;
  B.rc = D.scratch;
  B.qt_ptr = D.qt_ptr;
  B.qt_src = D.qt_src;
  B.qt_w = D.qt_w;
  B.Minv_h = D.Minv_h;
  B.Minv_z = D.Minv_z;
  B.qn = s.qn;
  B.qs = s.qs;
  B.out = s.out;
  B.a = s.a;
  B.b = s.b;
  B.cdt = s.cdt;
  B.rhs_only = s.rhs_only;
  B.NH = m.NH;
  B.NG = m.NG;
  B.NZ = m.NZ;
  B.status = D.status;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (m.NG + 255) / 256;
  long long cap = (long long)nsm * 8;
  if (blocks > cap) blocks = cap;
  {
    ProfScope ps(mixed ? "dss_rk_mixed" : "dss_rk_fp64", st);
    if (mixed)
      dss_stage<float><<<(int)blocks, 256, 0, st>>>(B);
    else
      dss_stage<double><<<(int)blocks, 256, 0, st>>>(B);
  }
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
