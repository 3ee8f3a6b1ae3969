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
#include <mutex>

#include "sem_internal.h"

namespace sem {

__constant__ double c_xi[kMaxN + 1][kMaxN + 1];
__constant__ double c_w[kMaxN + 1][kMaxN + 1];
__constant__ double c_Dw[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];  // [i][m] = w_m D[m][i]
__constant__ double c_D[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];   // [i][m] = h_m'(xi_i)
__constant__ float c_wf[kMaxN + 1][kMaxN + 1];
__constant__ float c_Dwf[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];
__constant__ float c_Df[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];

template <typename R> struct Tab;
template <> struct Tab<double> {
  __device__ static double w(int N, int i) { return c_w[N][i]; }
  __device__ static double Dw(int N, int k) { return c_Dw[N][k]; }
  __device__ static double D(int N, int k) { return c_D[N][k]; }
};
template <> struct Tab<float> {
  __device__ static float w(int N, int i) { return c_wf[N][i]; }
  __device__ static float Dw(int N, int k) { return c_Dwf[N][k]; }
  __device__ static float D(int N, int k) { return c_Df[N][k]; }
};

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
  float wf[kMaxN + 1][kMaxN + 1] = {};
  float Dwf[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)] = {};
  float Df[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)] = {};
  for (int N = 0; N <= kMaxN; ++N)
    for (int k = 0; k < (kMaxN + 1) * (kMaxN + 1); ++k) {
      if (k <= kMaxN) wf[N][k] = (float)w[N][k];
      Dwf[N][k] = (float)Dw[N][k];
      Df[N][k] = (float)D[N][k];
    }
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_wf, wf, sizeof(wf)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_Dwf, Dwf, sizeof(Dwf)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_Df, Df, sizeof(Df)));
  done = true;
  return SEM_OK;
}

// per-level geometry: hx, hy, hz, J, sx = hy hz/4, sy = hx hz/4, sz = hx hy/4, unused
constexpr int kLev = 16;
struct VolArgs {
  const void* q;      // double [5][NG] (FP64 form) or float mirror [5][NG] (mixed form)
  void* rc;
  const int* hmap;
  const int* hang_h;
  const void* hang_w;   // double (FP64 form) or float (mixed form) weights
  const int* col_level;
  const double* ref;
  int Ncol, nz, NZ;
  long long NH, NG;
  double Lx, Ly, Lz;
  int nx, ny;
  double g, f, gamma;
  float gf, ff, gammaf;
  double geo[kLev][8];
  float geof[kLev][8];
  const float* ref32;
};

template <typename R> __device__ __forceinline__ const R* geo_of(const VolArgs& A, int l);
template <> __device__ __forceinline__ const double* geo_of<double>(const VolArgs& A, int l) { return A.geo[l]; }
template <> __device__ __forceinline__ const float* geo_of<float>(const VolArgs& A, int l) { return A.geof[l]; }
template <typename R> __device__ __forceinline__ const R* ref_of(const VolArgs& A);
template <> __device__ __forceinline__ const double* ref_of<double>(const VolArgs& A) { return A.ref; }
template <> __device__ __forceinline__ const float* ref_of<float>(const VolArgs& A) { return A.ref32; }
template <typename R> __device__ __forceinline__ R par_g(const VolArgs& A);
template <> __device__ __forceinline__ double par_g<double>(const VolArgs& A) { return A.g; }
template <> __device__ __forceinline__ float par_g<float>(const VolArgs& A) { return A.gf; }
template <typename R> __device__ __forceinline__ R par_f(const VolArgs& A);
template <> __device__ __forceinline__ double par_f<double>(const VolArgs& A) { return A.f; }
template <> __device__ __forceinline__ float par_f<float>(const VolArgs& A) { return A.ff; }
template <typename R> __device__ __forceinline__ R par_gam(const VolArgs& A);
template <> __device__ __forceinline__ double par_gam<double>(const VolArgs& A) { return A.gamma; }
template <> __device__ __forceinline__ float par_gam<float>(const VolArgs& A) { return A.gammaf; }

template <typename R> __device__ __forceinline__ R r_log1p(R x);
template <> __device__ __forceinline__ double r_log1p<double>(double x) { return log1p(x); }
template <> __device__ __forceinline__ float r_log1p<float>(float x) { return log1pf(x); }
template <typename R> __device__ __forceinline__ R r_expm1(R x);
template <> __device__ __forceinline__ double r_expm1<double>(double x) { return expm1(x); }
template <> __device__ __forceinline__ float r_expm1<float>(float x) { return expm1f(x); }

// Gather the 5 fields of local node (ab, kz) of a column (Q row, Sec. 3.1).
template <int N, typename R>
__device__ __forceinline__ void gather_node(const VolArgs& A, int hm, int kz, R v[kFields]) {
  const R* q = (const R*)A.q;
  if (hm >= 0) {
    const R* p = q + (long long)hm * A.NZ + kz;
#pragma unroll
    for (int f = 0; f < kFields; ++f) v[f] = __ldg(p + (long long)f * A.NG);
  } else {
    const int k = -1 - hm;
    const R* hw = (const R*)A.hang_w;
#pragma unroll
    for (int f = 0; f < kFields; ++f) v[f] = (R)0;
#pragma unroll
    for (int m = 0; m <= N; ++m) {
      const R wm = __ldg(hw + k * (N + 1) + m);
      const R* p = q + (long long)__ldg(A.hang_h + k * (N + 1) + m) * A.NZ + kz;
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
  const R* geo = geo_of<R>(A, lev);
  int hm = 0;
  R Dwi[n1], Dwj[n1], Dwc[n1];
  R wi = 0, wj = 0, wc = 0;
  if (act) {
    hm = A.hmap[(long long)col * Nq + ab];
#pragma unroll
    for (int m = 0; m < n1; ++m) {
      if (EQ == 0) {
        Dwi[m] = Tab<R>::Dw(N, i * n1 + m);
        Dwj[m] = Tab<R>::Dw(N, j * n1 + m);
        Dwc[m] = Tab<R>::Dw(N, c * n1 + m);
      } else {
        Dwi[m] = Tab<R>::D(N, i * n1 + m);
        Dwj[m] = Tab<R>::D(N, j * n1 + m);
        Dwc[m] = Tab<R>::D(N, c * n1 + m);
      }
    }
    wi = Tab<R>::w(N, i);
    wj = Tab<R>::w(N, j);
    wc = Tab<R>::w(N, c);
  }
  // weak-form factors: J dxi/dx = hy hz / 4 etc.
  const R sx = geo[4], sy = geo[5], sz = geo[6];
  const R wJ = wi * wj * wc * geo[3];
  const R two = (R)2;
  const R gx = two / geo[0], gy = two / geo[1], gz = two / geo[2];
  const R g = par_g<R>(A), fc = par_f<R>(A), gam = par_gam<R>(A);
  const R* refR = ref_of<R>(A);
  R* rc = (R*)A.rc;

  for (int k = 0; k < A.nz; ++k) {
    const int kz = k * N + c;
    R S[kFields] = {0, 0, 0, 0, 0};
    R pw[5] = {0, 0, 0, 0, 0};  // EQ 1: u, v, w, rho, rho' kept for the strong terms
    R th0dz = 0;
    if (act) {
      R v[kFields];
      gather_node<N, R>(A, hm, kz, v);
      const R* rf = refR + (long long)kz * kRef;
      const R p0 = rf[2], rho0 = rf[3], rt0 = rf[4], inv_rt0 = rf[6];
      const R rp = v[0];
      const R rho = rho0 + rp;
      const R inv = (R)1 / rho;
      if (EQ == 0) {
        const R U = v[1], V = v[2], W = v[3], Tp = v[4];
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
        const R u = v[1], vv = v[2], w = v[3], thp = v[4];
        const R th0 = rf[0];
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
        th0dz = rf[5];
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
          acc += Tab<R>::Dw(N, i * n1 + m) * sF[0][m + n1 * j + Nq * c];
          acc += Tab<R>::Dw(N, j * n1 + m) * sF[1][i + n1 * m + Nq * c];
          acc += Tab<R>::Dw(N, c * n1 + m) * sF[2][i + n1 * j + Nq * m];
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

// float32 <-> float64 conversions with integer operations.  On GB300 a
// hardware F2F conversion issues on the (narrow) float64 pipe; these keep the
// conversions on the integer ALU.  Denormal floats are flushed to zero (they
// are below 1.2e-38 and never matter here); the double -> float direction
// truncates the significand (relative error below 2^-23).
__device__ __forceinline__ double f2d_bits(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned sgn = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  unsigned hi, lo;
  if (e == 0u) {
    hi = sgn;
    lo = 0u;
  } else {
    const unsigned e64 = (e == 0xFFu) ? 0x7FFu : e + 896u;
    hi = sgn | (e64 << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sgn = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 896;
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  unsigned b;
  if (e <= 0) b = sgn;
  else if (e >= 255) b = sgn | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u);
  else b = sgn | ((unsigned)e << 23) | m;
  return __uint_as_float(b);
}
__device__ __forceinline__ bool nonfinite_bits(double x) {
  return (((unsigned)__double2hiint(x) >> 20) & 0x7FFu) == 0x7FFu;
}

struct DssArgs {
  const void* rc;
  const int* qt_ptr;
  const int* qt_src;
  const void* qt_w;       // double (FP64 form) or float (mixed form)
  const void* Minv_h;     // double or float
  const void* Minv_z;
  const double* qn;
  const double* qs;
  double* out;
  float* out32;           // mixed form: float32 mirror of out (may be null)
  double a, b, cdt;
  int rhs_only;
  long long NH, NG;
  int NZ;
  int* status;
};

// FP64 form: float64 throughout.
__global__ void __launch_bounds__(256) dss_stage_fp64(const DssArgs A) {
  const double* rc = (const double*)A.rc;
  const double* qtw = (const double*)A.qt_w;
  const double* mh = (const double*)A.Minv_h;
  const double* mz = (const double*)A.Minv_z;
  int bad = 0;
  for (long long gidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; gidx < A.NG;
       gidx += (long long)gridDim.x * blockDim.x) {
    const long long h = gidx / A.NZ;
    const int kz = (int)(gidx - h * A.NZ);
    const int beg = __ldg(A.qt_ptr + h), end = __ldg(A.qt_ptr + h + 1);
    const double s = A.cdt * (__ldg(mh + h) * __ldg(mz + kz));
    const bool lid = (kz == 0) || (kz == A.NZ - 1);
    double acc[kFields] = {0, 0, 0, 0, 0};
    for (int e = beg; e < end; ++e) {
      const double w = __ldg(qtw + e);
      const double* p = rc + (long long)__ldg(A.qt_src + e) * kFields * A.NZ + kz;
#pragma unroll
      for (int fl = 0; fl < kFields; ++fl) acc[fl] = fma(w, p[(long long)fl * A.NZ], acc[fl]);
    }
#pragma unroll
    for (int fl = 0; fl < kFields; ++fl) {
      const long long o = (long long)fl * A.NG + gidx;
      const double T = (fl == 3 && lid) ? 0.0 : acc[fl];
      double val;
      if (A.rhs_only) {
        val = T * s;
      } else {
        val = A.b * __ldg(A.qs + o);
        if (A.a != 0.0) val = fma(A.a, __ldg(A.qn + o), val);
        val = fma(s, T, val);
      }
      A.out[o] = val;
      bad |= nonfinite_bits(val);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(A.status, 1);
}

// Mixed form: float32 gather sums and increment c dt R / M, then the float64
// stage accumulation q_out = a qn + b qs + increment (one or two DFMA per
// value), and the float32 mirror of q_out for the next stage's element work.
__global__ void __launch_bounds__(256) dss_stage_mixed(const DssArgs A) {
  const float* rc = (const float*)A.rc;
  const float* qtw = (const float*)A.qt_w;
  const float* mh = (const float*)A.Minv_h;
  const float* mz = (const float*)A.Minv_z;
  const float cdt = (float)A.cdt;
  int bad = 0;
  for (long long gidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; gidx < A.NG;
       gidx += (long long)gridDim.x * blockDim.x) {
    const long long h = gidx / A.NZ;
    const int kz = (int)(gidx - h * A.NZ);
    const int beg = __ldg(A.qt_ptr + h), end = __ldg(A.qt_ptr + h + 1);
    const float s = cdt * (__ldg(mh + h) * __ldg(mz + kz));
    const bool lid = (kz == 0) || (kz == A.NZ - 1);
    float acc[kFields] = {0, 0, 0, 0, 0};
    for (int e = beg; e < end; ++e) {
      const float w = __ldg(qtw + e);
      const float* p = rc + (long long)__ldg(A.qt_src + e) * kFields * A.NZ + kz;
#pragma unroll
      for (int fl = 0; fl < kFields; ++fl) acc[fl] = fmaf(w, p[(long long)fl * A.NZ], acc[fl]);
    }
#pragma unroll
    for (int fl = 0; fl < kFields; ++fl) {
      const long long o = (long long)fl * A.NG + gidx;
      const float inc = (fl == 3 && lid) ? 0.f : acc[fl] * s;
      const double incd = f2d_bits(inc);
      double val;
      if (A.rhs_only) {
        val = incd;
      } else if (A.a == 0.0) {
        val = (A.b == 1.0) ? __ldg(A.qs + o) + incd : fma(A.b, __ldg(A.qs + o), incd);
      } else {
        val = fma(A.a, __ldg(A.qn + o), fma(A.b, __ldg(A.qs + o), incd));
      }
      A.out[o] = val;
      if (A.out32) A.out32[o] = d2f_bits(val);
      bad |= nonfinite_bits(val);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(A.status, 1);
}

__global__ void __launch_bounds__(256) mirror_kernel(const double* q, float* q32, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    q32[i] = d2f_bits(q[i]);
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

static int grid_cap(long long work) {
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (work + 255) / 256;
  long long cap = (long long)nsm * 8;
  return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

int launch_mirror(const double* q, float* q32, long long n, cudaStream_t st) {
  ProfScope ps("mirror", st);
  mirror_kernel<<<grid_cap(n), 256, 0, st>>>(q, q32, n);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

int launch_rhs_stage(Mesh& m, const sem_params& p, const StageArgs& s, cudaStream_t st) {
  int rc = upload_basis_constants();
  if (rc) return rc;
  DeviceTables& D = *m.dev;
  const bool mixed = p.precision == SEM_PREC_MIXED;
  const float* qs32 = s.qs32;
  if (mixed && !qs32) {
    // no caller mirror: make one in the mesh scratch
    if ((rc = launch_mirror(s.qs, D.mirror, (long long)kFields * m.NG, st))) return rc;
    qs32 = D.mirror;
  }
  VolArgs A;
  A.q = mixed ? (const void*)qs32 : (const void*)s.qs;
  A.rc = s.scratch ? s.scratch : D.scratch;
  A.hmap = D.hmap;
  A.hang_h = D.hang_h;
  A.hang_w = mixed ? (const void*)D.hang_w32 : (const void*)D.hang_w;
  A.col_level = D.col_level;
  A.ref = D.ref;
  A.ref32 = D.ref32;
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
  A.gf = (float)A.g;
  A.ff = (float)A.f;
  A.gammaf = (float)A.gamma;
  for (int l = 0; l < kLev; ++l) {
    const double hx = m.hx(l), hy = m.hy(l), hz = m.hz();
    const double g[8] = {hx, hy, hz, hx * hy * hz * 0.125, hy * hz * 0.25, hx * hz * 0.25,
                         hx * hy * 0.25, 0.0};
    for (int k = 0; k < 8; ++k) {
      A.geo[l][k] = g[k];
      A.geof[l][k] = (float)g[k];
    }
  }
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
  B.rc = s.scratch ? s.scratch : D.scratch;
  B.qt_ptr = D.qt_ptr;
  B.qt_src = D.qt_src;
  B.qt_w = mixed ? (const void*)D.qt_w32 : (const void*)D.qt_w;
  B.Minv_h = mixed ? (const void*)D.Minv_h32 : (const void*)D.Minv_h;
  B.Minv_z = mixed ? (const void*)D.Minv_z32 : (const void*)D.Minv_z;
  B.qn = s.qn;
  B.qs = s.qs;
  B.out = s.out;
  B.out32 = s.out32;
  B.a = s.a;
  B.b = s.b;
  B.cdt = s.cdt;
  B.rhs_only = s.rhs_only;
  B.NH = m.NH;
  B.NG = m.NG;
  B.NZ = m.NZ;
  B.status = D.status;
  {
    ProfScope ps(mixed ? "dss_rk_mixed" : "dss_rk_fp64", st);
    if (mixed)
      dss_stage_mixed<<<grid_cap(m.NG), 256, 0, st>>>(B);
    else
      dss_stage_fp64<<<grid_cap(m.NG), 256, 0, st>>>(B);
  }
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem

// ---------------------------------------------------------------------------
// Allocation-free right-hand side (sem_rhs_noalloc).
//
// Its column-residual scratch is this file-scope device array instead of
// memory the library allocates per mesh.  Every GPU that loads the library
// holds the array until the process exits.  Host code cannot use the array's
// name as a device address (on the host it names a stand-in object), so the
// device address is looked up once per device with cudaGetSymbolAddress, with
// that device current, and passed to the kernels.
namespace sem {
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];
constexpr int kNoAllocMaxDevices = 64;
static void* g_noalloc_addr[kNoAllocMaxDevices] = {};
static std::mutex g_noalloc_mu;

static int noalloc_scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SEM_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(SEM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return SEM_OK;
}
}  // namespace sem

extern "C" int sem_rhs_noalloc(sem_mesh* mh, const sem_params* p, const double* q, double* rhs,
                               cudaStream_t st) {
  using namespace sem;
  if (!mh || !p || !q || !rhs || q == rhs) return fail(SEM_ERR_ARG, "NULL or aliased argument");
  if ((p->eqset != SEM_EQ_CONSERVATIVE && p->eqset != SEM_EQ_NONCONSERVATIVE) ||
      (p->precision != SEM_PREC_FP64 && p->precision != SEM_PREC_MIXED))
    return fail(SEM_ERR_ARG, "unknown equation set or precision");
  Mesh& m = mh->m;
  const size_t need = (size_t)m.Ncol() * m.Nq * kFields * m.NZ * sizeof(double);
  if (need > kNoAllocScratchBytes)
    return fail(SEM_ERR_ARG, "mesh too large for sem_rhs_noalloc: needs " + std::to_string(need) +
                                 " bytes of scratch, the fixed maximum is " +
                                 std::to_string(kNoAllocScratchBytes));
  int dev = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  if (!m.dev)
    return fail(SEM_ERR_ARG, "the mesh has no device tables yet: make another device call on it "
                             "first (for example sem_mesh_coords)");
  if (m.dev_id != dev) return fail(SEM_ERR_ARG, "mesh tables live on another device");
  int rc = ensure_reference(m, *p);
  if (rc) return rc;
  void* scratch = nullptr;
  if ((rc = noalloc_scratch_address(dev, &scratch))) return rc;
  StageArgs s{nullptr, q, rhs, nullptr, nullptr, 0.0, 0.0, 1.0, 1, scratch};
  return launch_rhs_stage(m, *p, s, st);
}
