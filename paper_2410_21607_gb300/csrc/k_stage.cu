// Right-hand side and Runge-Kutta stage kernels.
//
//   volume_column<N, EQ, R> (the float64 form): one CTA per leaf column marches up its nz
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
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "sem_internal.h"
#include "tcgen05.cuh"

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

static int upload_basis_constants_now() {
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
  return SEM_OK;
}

// the basis tables of the current device (uploaded on its first use)
int upload_basis_constants() {
  static DeviceOnce once;
  return device_once(once, upload_basis_constants_now);
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
  int NZr;              // level stride of the column residuals (NZ rounded up to 4)
  long long NH, NG;
  double Lx, Ly, Lz;
  int nx, ny;
  double g, f, gamma;
  float gf, ff, gammaf;
  float bin[8];         // binomial-series coefficients C(gamma, k), k = 1..7
  double geo[kLev][8];
  float geof[kLev][8];
  const float* ref32;
  const double* hzk;    // [nz] layer thicknesses (geo holds the values for unit thickness)
  const float* hzk32;
  const float4* ref4;   // [NZ] packed p0, rho0, (rho theta)0, 1/(rho theta)0 (float32)
  const float* spg32;   // [NZ] absorbing-layer rate R(z): the line-exchange kernel adds
                        // -R q' (weak form, collocated) when set; null: not added here
  int* status;          // device status word (bit 4: a bounded device wait ran out)
  // warped layers: per-node metric z_xi, z_eta, z_zeta [Ncol][Nq][nz][N+1][3] and the
  // reference state at every node's height (global nodes [NG], hanging lines [Nhang][NZ])
  const double* metric;
  const float* metric32;
  const double* refG;
  const double* refH;
  const float* refG32;
  const float* refH32;
  const float4* ref4G;
  const float4* ref4H;
  float smag[kLev][3];  // per level (C_s Delta)^2, 2/hx, 2/hy: the horizontal
                        // Smagorinsky stress, for the kernels that add it
};

template <typename R> __device__ __forceinline__ const R* geo_of(const VolArgs& A, int l);
template <> __device__ __forceinline__ const double* geo_of<double>(const VolArgs& A, int l) { return A.geo[l]; }
template <> __device__ __forceinline__ const float* geo_of<float>(const VolArgs& A, int l) { return A.geof[l]; }
template <typename R> __device__ __forceinline__ const R* hz_of(const VolArgs& A);
template <> __device__ __forceinline__ const double* hz_of<double>(const VolArgs& A) { return A.hzk; }
template <> __device__ __forceinline__ const float* hz_of<float>(const VolArgs& A) { return A.hzk32; }
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

template <typename R> __device__ __forceinline__ const R* refG_of(const VolArgs& A);
template <> __device__ __forceinline__ const double* refG_of<double>(const VolArgs& A) { return A.refG; }
template <> __device__ __forceinline__ const float* refG_of<float>(const VolArgs& A) { return A.refG32; }
template <typename R> __device__ __forceinline__ const R* refH_of(const VolArgs& A);
template <> __device__ __forceinline__ const double* refH_of<double>(const VolArgs& A) { return A.refH; }
template <> __device__ __forceinline__ const float* refH_of<float>(const VolArgs& A) { return A.refH32; }
template <typename R> __device__ __forceinline__ const R* metric_of(const VolArgs& A);
template <> __device__ __forceinline__ const double* metric_of<double>(const VolArgs& A) { return A.metric; }
template <> __device__ __forceinline__ const float* metric_of<float>(const VolArgs& A) { return A.metric32; }

// Reference-state row of node (column line hm, level kz): per level on box
// meshes, at the node's own height on warped ones.
template <typename R, bool WARP>
__device__ __forceinline__ const R* ref_row(const VolArgs& A, int hm, int kz) {
  if (!WARP) return ref_of<R>(A) + (long long)kz * kRef;
  if (hm >= 0) return refG_of<R>(A) + ((long long)hm * A.NZ + kz) * kRef;
  return refH_of<R>(A) + ((long long)(-1 - hm) * A.NZ + kz) * kRef;
}

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

// W: warped layers.  The weak fluxes are then the contravariant ones,
// J grad xi_i . F, with (per node, hx, hy of the column and z_xi, z_eta,
// z_zeta from the metric table)
//   J grad xi = (hy/2 z_zeta, 0, 0), J grad eta = (0, hx/2 z_zeta, 0),
//   J grad zeta = (-hy/2 z_xi, -hx/2 z_eta, hx hy/4), J = hx hy z_zeta / 4,
// and the strong derivatives of the paper's set d/dx = 2/hx (d/dxi - z_xi/z_zeta d/dzeta),
// d/dy = 2/hy (d/deta - z_eta/z_zeta d/dzeta), d/dz = 1/z_zeta d/dzeta.
template <int N, int EQ, typename R, bool WARP = false>
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
  // per unit layer thickness; scaled by the layer's thickness below
  const R sx1 = geo[4], sy1 = geo[5], sz = geo[6];
  const R wJ1 = wi * wj * wc * geo[3];
  const R two = (R)2;
  const R gx = two / geo[0], gy = two / geo[1];
  const R g = par_g<R>(A), fc = par_f<R>(A), gam = par_gam<R>(A);
  const R* refR = ref_of<R>(A);
  R* rc = (R*)A.rc;

  for (int k = 0; k < A.nz; ++k) {
    const R hk = hz_of<R>(A)[k];
    R sx = sx1 * hk, sy = sy1 * hk, wJ = wJ1 * hk, gz = two / hk;
    const int kz = k * N + c;
    R S[kFields] = {0, 0, 0, 0, 0};
    R pw[5] = {0, 0, 0, 0, 0};  // EQ 1: u, v, w, rho, rho' kept for the strong terms
    R th0dz = 0;
    R cxw = 0, cyw = 0;         // W: z-direction weights of the x and y fluxes
    R rzx = 0, rzy = 0;         // W: z_xi / z_zeta, z_eta / z_zeta
    if (WARP && act) {
      const R* mt = metric_of<R>(A) + ((((long long)col * Nq + ab) * A.nz + k) * n1 + c) * 3;
      const R zx = mt[0], zy = mt[1], zz = mt[2];
      const R hx = geo[0], hy = geo[1];
      sx = (R)0.5 * hy * zz;               // J grad xi . e_x
      sy = (R)0.5 * hx * zz;               // J grad eta . e_y
      cxw = -(R)0.5 * hy * zx * wi * wj;   // weighted J grad zeta . e_x
      cyw = -(R)0.5 * hx * zy * wi * wj;   // weighted J grad zeta . e_y
      wJ = wi * wj * wc * geo[6] * zz;     // w J, geo[6] = hx hy / 4
      gz = (R)1 / zz;
      rzx = zx / zz;
      rzy = zy / zz;
    }
    if (act) {
      R v[kFields];
      gather_node<N, R>(A, hm, kz, v);
      const R* rf = ref_row<R, WARP>(A, hm, kz);
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
        if (!WARP) {
          sF[0][t] = U * ax;            sF[1][t] = V * ay;            sF[2][t] = W * az;
          sF[3][t] = (U * u + pp) * ax; sF[4][t] = U * vv * ay;       sF[5][t] = U * w * az;
          sF[6][t] = V * u * ax;        sF[7][t] = (V * vv + pp) * ay; sF[8][t] = V * w * az;
          sF[9][t] = W * u * ax;        sF[10][t] = W * vv * ay;      sF[11][t] = (W * w + pp) * az;
          sF[12][t] = rt * u * ax;      sF[13][t] = rt * vv * ay;     sF[14][t] = rt * w * az;
        } else {
          const R Fx[kFields] = {U, U * u + pp, V * u, W * u, rt * u};
          const R Fy[kFields] = {V, U * vv, V * vv + pp, W * vv, rt * vv};
          const R Fz[kFields] = {W, U * w, V * w, W * w + pp, rt * w};
#pragma unroll
          for (int fl = 0; fl < kFields; ++fl) {
            sF[3 * fl + 0][t] = Fx[fl] * ax;
            sF[3 * fl + 1][t] = Fy[fl] * ay;
            sF[3 * fl + 2][t] = Fz[fl] * az + Fx[fl] * cxw + Fy[fl] * cyw;
          }
        }
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
        if (WARP) sF[2][t] += rho * u * cxw + rho * vv * cyw;
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
          if (WARP) {
            dq[qv][0] = (ax_ - rzx * az_) * gx;
            dq[qv][1] = (ay_ - rzy * az_) * gy;
          } else {
            dq[qv][0] = ax_ * gx;
            dq[qv][1] = ay_ * gy;
          }
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
        R* dst = rc + ((long long)((long long)col * Nq + ab) * kFields) * A.NZr + kz;
#pragma unroll
        for (int fl = 0; fl < kFields; ++fl) dst[(long long)fl * A.NZr] = r[fl];
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
  const int4* qt_rec_unit;  // FP64 form: unit-weight Q_h^T records
  const int4* qt_rec_src;   // mixed form: compact Q_h^T records (sources, -2: use the lists)
  const float4* qt_rec_w;   //   and their float32 weights
  const void* Minv_g;       // warped layers: inverse lumped mass per node (double or float), else null
  const double* qn;
  const double* qs;
  double* out;
  float* out32;           // mixed form: float32 mirror of out (may be null)
  double a, b, cdt;
  int rhs_only;
  long long NH, NG;
  int NZ, NZr;
  int* status;
};

// FP64 form: float64 throughout.  The float64 pipe of this part is narrow
// (1/64 of the float32 rate), so the kernel issues float64 instructions only
// for the arithmetic itself: node indices are 32-bit (an unsigned division by
// NZ runs on the integer pipe), c dt / M_z(kz) comes from a table the block
// fills once, a horizontal node whose Q_h^T weights are all exactly 1 (every
// node away from 2:1 faces) adds its sources with plain additions (the first
// one is a load), and the stage update is specialised:
//   MODE 0  out = s T                         (right-hand side only)
//   MODE 1  out = qs + s T                    (a = 0, b = 1: the first SSP-RK3 stage)
//   MODE 2  out = a qn + b qs + s T           (any a, b)
//   MODE 3  out = 3/4 qn + qs / 4 + s T       (the second SSP-RK3 stage)
// with s = c dt / M.  MODE 3 forms qs / 4 on the integer pipe (quarter_bits:
// exact, like the product by 0.25 it replaces), so the float64 pipe does two
// fused multiply-adds per value instead of a product and two.  Every sum of
// the gather is formed in the order of the CSR lists.  The block's table
// needs NZ doubles of dynamic shared memory.
//
// x / 4 from the bits of x: the biased binary exponent lowered by 2.  Exact
// for normal x whose quarter is normal (biased exponent above 2); zero and
// values below 2^-1020 in magnitude give a zero of their sign (their quarter
// is below 2^-1022), infinities and NaN pass unchanged.  Integer operations
// only.
__device__ __forceinline__ double quarter_bits(double x) {
  const int hi = __double2hiint(x), lo = __double2loint(x);
  const int e = (hi >> 20) & 0x7ff;
  int rhi = hi - (2 << 20), rlo = lo;
  if (e <= 2) {
    rhi = hi & (int)0x80000000;
    rlo = 0;
  }
  if (e == 0x7ff) {
    rhi = hi;
    rlo = lo;
  }
  return __hiloint2double(rhi, rlo);
}

template <int MODE>
__global__ void __launch_bounds__(256) dss_stage_fp64(const DssArgs A) {
  extern __shared__ double s_cmz[];   // [NZ]: c dt / M_z(kz)
  const double* rc = (const double*)A.rc;
  const double* qtw = (const double*)A.qt_w;
  const double* mh = (const double*)A.Minv_h;
  const double* mz = (const double*)A.Minv_z;
  const unsigned NZ = (unsigned)A.NZ, NG = (unsigned)A.NG;
  const long long NGl = A.NG;
  const int NZr = A.NZr;
  const double cdt = A.cdt;
  for (int k = threadIdx.x; k < (int)NZ; k += blockDim.x) s_cmz[k] = cdt * __ldg(mz + k);
  __syncthreads();
  int bad = 0;
  for (unsigned gidx = blockIdx.x * blockDim.x + threadIdx.x; gidx < NG; gidx += gridDim.x * blockDim.x) {
    const unsigned h = gidx / NZ;
    const int kz = (int)(gidx - h * NZ);
    // the stage state first, so that its latency overlaps the gather's
    double qsv[kFields];
#pragma unroll
    for (int fl = 0; fl < kFields; ++fl)
      if (MODE >= 1) qsv[fl] = __ldg(A.qs + fl * NGl + gidx);
    const double s = A.Minv_g ? cdt * __ldg((const double*)A.Minv_g + gidx) : __ldg(mh + h) * s_cmz[kz];
    const bool lid = (kz == 0) || (kz == (int)NZ - 1);
    double acc[kFields];
    const int4 r = __ldg(A.qt_rec_unit + h);
    if (r.x >= 0) {
      const double* p = rc + (size_t)r.x * kFields * NZr + kz;
#pragma unroll
      for (int fl = 0; fl < kFields; ++fl) acc[fl] = __ldg(p + fl * NZr);
      auto add = [&](int src) {
        const double* pe = rc + (size_t)src * kFields * NZr + kz;
#pragma unroll
        for (int fl = 0; fl < kFields; ++fl) acc[fl] += __ldg(pe + fl * NZr);
      };
      if (r.y >= 0) {
        add(r.y);
        if (r.z >= 0) {
          add(r.z);
          if (r.w >= 0) add(r.w);
        }
      }
    } else {
#pragma unroll
      for (int fl = 0; fl < kFields; ++fl) acc[fl] = 0.0;
      const int beg = __ldg(A.qt_ptr + h), end = __ldg(A.qt_ptr + h + 1);
      for (int e = beg; e < end; ++e) {
        const double w = __ldg(qtw + e);
        const double* p = rc + (size_t)__ldg(A.qt_src + e) * kFields * NZr + kz;
#pragma unroll
        for (int fl = 0; fl < kFields; ++fl) acc[fl] = fma(w, __ldg(p + fl * NZr), acc[fl]);
      }
    }
#pragma unroll
    for (int fl = 0; fl < kFields; ++fl) {
      const double T = (fl == 3 && lid) ? 0.0 : acc[fl];
      double val;
      if (MODE == 0) val = T * s;
      else if (MODE == 1) val = fma(s, T, qsv[fl]);
      else if (MODE == 3) val = fma(s, T, fma(0.75, __ldg(A.qn + fl * NGl + gidx), quarter_bits(qsv[fl])));
      else val = fma(s, T, fma(A.a, __ldg(A.qn + fl * NGl + gidx), A.b * qsv[fl]));
      A.out[fl * NGl + gidx] = val;
      bad |= nonfinite_bits(val);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(A.status, 1);
}

// Mixed form: float32 gather sums and increment c dt R / M, then the float64
// stage accumulation q_out = a qn + b qs + increment (one or two DFMA per
// value), and the float32 mirror of q_out for the next stage's element work.
template <bool WARP = false>
__global__ void __launch_bounds__(256) dss_stage_mixed(const DssArgs A) {
  const float* rc = (const float*)A.rc;
  const float* qtw = (const float*)A.qt_w;
  const float* mh = (const float*)A.Minv_h;
  const float* mz = (const float*)A.Minv_z;
  const float cdt = (float)A.cdt;
  // 32-bit node indices (the caller checks 5 NG < 2^31): the division by NZ
  // runs on the integer pipe
  const unsigned NZ = (unsigned)A.NZ, NG = (unsigned)A.NG;
  const long long NGl = A.NG;
  const int NZr = A.NZr;
  int bad = 0;
  for (unsigned gidx = blockIdx.x * blockDim.x + threadIdx.x; gidx < NG; gidx += gridDim.x * blockDim.x) {
    const unsigned h = gidx / NZ;
    const int kz = (int)(gidx - h * NZ);
    const float s = WARP ? cdt * __ldg((const float*)A.Minv_g + gidx) : cdt * (__ldg(mh + h) * __ldg(mz + kz));
    const bool lid = (kz == 0) || (kz == (int)NZ - 1);
    // Q_h^T gather in the order of the CSR lists: from the compact record
    // (sources and weights after one load each), else from the lists
    float acc[kFields] = {0, 0, 0, 0, 0};
    const int4 s4 = __ldg(A.qt_rec_src + h);
    if (s4.x >= 0) {
      const float4 w4 = __ldg(A.qt_rec_w + h);
      const int src[4] = {s4.x, s4.y, s4.z, s4.w};
      const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (src[e] < 0) break;
        const float* p = rc + (size_t)src[e] * kFields * NZr + kz;
#pragma unroll
        for (int fl = 0; fl < kFields; ++fl) acc[fl] = fmaf(ww[e], __ldg(p + fl * NZr), acc[fl]);
      }
    } else {
      const int beg = __ldg(A.qt_ptr + h), end = __ldg(A.qt_ptr + h + 1);
      for (int e = beg; e < end; ++e) {
        const float w = __ldg(qtw + e);
        const float* p = rc + (size_t)__ldg(A.qt_src + e) * kFields * NZr + kz;
#pragma unroll
        for (int fl = 0; fl < kFields; ++fl) acc[fl] = fmaf(w, __ldg(p + fl * NZr), acc[fl]);
      }
    }
#pragma unroll
    for (int fl = 0; fl < kFields; ++fl) {
      const long long o = (long long)fl * NGl + gidx;
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

// The float64 form's element kernel (both sets, box or warped layers); the
// mixed form runs the line-exchange kernels of the variant table instead.
template <int N, int EQ>
static void launch_volume(const VolArgs& A, cudaStream_t st) {
  constexpr int P = (N + 1) * (N + 1) * (N + 1);
  constexpr int nt = (P + 31) / 32 * 32;
  ProfScope ps("volume_fp64", st);
  if (A.metric)
    volume_column<N, EQ, double, true><<<A.Ncol, nt, 0, st>>>(A);
  else
    volume_column<N, EQ, double><<<A.Ncol, nt, 0, st>>>(A);
}

template <int N>
static void launch_volume_fp64(const VolArgs& A, int eq, cudaStream_t st) {
  if (eq == 0) launch_volume<N, 0>(A, st); else launch_volume<N, 1>(A, st);
}

// ---------------------------------------------------------------------------
// Mixed form, conservative set: z-pencil element kernel.
//
// One CTA per leaf column; thread (ab, kk) owns the N+1 nodes of the vertical
// line (a, b) of layer k = chunk * KL + kk, so consecutive threads walk up a
// column's z-lines and their loads and stores are contiguous.  The z-direction
// contraction runs on the thread's own registers; the x and y flux components
// go to shared memory with the nodes of a z-line side by side, so that one
// 64-bit shared load feeds a packed float32x2 FMA for two nodes.  The face
// shared by consecutive layers is summed inside the CTA (vertical DSS), as in
// volume_column.  Arithmetic: float32; geometry and reference state come from
// tables computed in float64.
__host__ __device__ constexpr int pencil_sk(int N) {
  // n1 * n1 * CW words rounded up to the next value = 2 (mod 32)
  return ((N + 1) * (N + 1) * (2 * ((N + 2) / 2)) + 29) / 32 * 32 + 2;
}

// (1 + x)^gamma - 1 in float32.  For |x| <= 1/8 the binomial series
// sum_{k=1..7} C(gamma, k) x^k (Horner form, no cancellation); its first
// dropped term is below 3e-9 of the result there, under float32 rounding.
// Larger |x| take expm1(gamma log1p(x)).
__device__ __forceinline__ float pow1p_m1(float x, const float* bin, float gam) {
  if (fabsf(x) <= 0.125f) {
    float s = bin[6];
#pragma unroll
    for (int k = 5; k >= 0; --k) s = fmaf(s, x, bin[k]);
    return s * x;
  }
  return expm1f(gam * log1pf(x));
}

// State perturbation v = (rho', rho u, rho v, rho w, (rho theta)') of one node
// of column line `hm` at level kz: a direct load, or for a hanging line the
// interpolation from the coarse neighbour's lines (Sec. 3.1).
template <int N>
__device__ __forceinline__ void load_node(const VolArgs& A, const int hm, const int kz, float (&v)[kFields]) {
  const float* q = (const float*)A.q;
  if (hm >= 0) {
    const float* pq = q + (long long)hm * A.NZ + kz;
#pragma unroll
    for (int f = 0; f < kFields; ++f) v[f] = __ldg(pq + (long long)f * A.NG);
  } else {
    const int hk = -1 - hm;
    const float* hw = (const float*)A.hang_w;
#pragma unroll
    for (int f = 0; f < kFields; ++f) v[f] = 0.f;
#pragma unroll
    for (int m = 0; m < N + 1; ++m) {
      const float wm = __ldg(hw + hk * (N + 1) + m);
      const float* pq = q + (long long)__ldg(A.hang_h + hk * (N + 1) + m) * A.NZ + kz;
#pragma unroll
      for (int f = 0; f < kFields; ++f) v[f] = fmaf(wm, __ldg(pq + (long long)f * A.NG), v[f]);
    }
  }
}

// Pointwise part of the conservative set at one node (Sec. 2, eqs.
// mass_split..ent_split, plus the f-plane Coriolis term): the weighted flux
// components ax F^x, ay F^y, az F^z of the five equations and the weighted
// momentum sources wJ S (Coriolis on rho u and rho v, buoyancy on rho w).
// The reference state of the level is one packed 16-byte row.
struct NodeTerms {
  float fx[kFields], fy[kFields], fz[kFields];
  float su, sv, sw;
};
__device__ __forceinline__ void node_terms(const VolArgs& A, const float (&v)[kFields], const int kz,
                                           const float ax, const float ay, const float az, const float wJ,
                                           NodeTerms& o) {
  const float4 ra = __ldg(A.ref4 + kz);
  const float p0 = ra.x, rho0 = ra.y, rt0 = ra.z, inv_rt0 = ra.w;
  const float rp = v[0], U = v[1], V = v[2], W = v[3], Tp = v[4];
  const float inv = __frcp_rn(rho0 + rp);
  const float u = U * inv, vv = V * inv, w = W * inv;
  const float pp = p0 * pow1p_m1(Tp * inv_rt0, A.bin, A.gammaf);
  const float rt = rt0 + Tp;
  o.fx[0] = U * ax;
  o.fx[1] = (U * u + pp) * ax;
  o.fx[2] = V * u * ax;
  o.fx[3] = W * u * ax;
  o.fx[4] = rt * u * ax;
  o.fy[0] = V * ay;
  o.fy[1] = U * vv * ay;
  o.fy[2] = (V * vv + pp) * ay;
  o.fy[3] = W * vv * ay;
  o.fy[4] = rt * vv * ay;
  o.fz[0] = W * az;
  o.fz[1] = U * w * az;
  o.fz[2] = V * w * az;
  o.fz[3] = (W * w + pp) * az;
  o.fz[4] = rt * w * az;
  o.su = wJ * (A.ff * V);
  o.sv = wJ * (-A.ff * U);
  o.sw = wJ * (-rp * A.gf);
}

// The same on warped layers: the reference row comes with the node (its own
// height), and the weak fluxes are the contravariant ones (the z-direction
// flux takes the x and y fluxes with the weights cx, cy of J grad zeta).
__device__ __forceinline__ void node_terms_w(const VolArgs& A, const float (&v)[kFields], const float4 ra,
                                             const float ax, const float ay, const float az, const float cx,
                                             const float cy, const float wJ, NodeTerms& o) {
  const float p0 = ra.x, rho0 = ra.y, rt0 = ra.z, inv_rt0 = ra.w;
  const float rp = v[0], U = v[1], V = v[2], W = v[3], Tp = v[4];
  const float inv = __frcp_rn(rho0 + rp);
  const float u = U * inv, vv = V * inv, w = W * inv;
  const float pp = p0 * pow1p_m1(Tp * inv_rt0, A.bin, A.gammaf);
  const float rt = rt0 + Tp;
  const float Fx[kFields] = {U, U * u + pp, V * u, W * u, rt * u};
  const float Fy[kFields] = {V, U * vv, V * vv + pp, W * vv, rt * vv};
  const float Fz[kFields] = {W, U * w, V * w, W * w + pp, rt * w};
#pragma unroll
  for (int f = 0; f < kFields; ++f) {
    o.fx[f] = Fx[f] * ax;
    o.fy[f] = Fy[f] * ay;
    o.fz[f] = fmaf(Fy[f], cy, fmaf(Fx[f], cx, Fz[f] * az));
  }
  o.su = wJ * (A.ff * V);
  o.sv = wJ * (-A.ff * U);
  o.sw = wJ * (-rp * A.gf);
}

// Body shared by the single-mesh kernel (one CTA per column) and the batched
// persistent kernel (CTAs pull columns of many meshes from a queue).  Threads
// t >= KL (N+1)^2 of a larger CTA take part in the barriers only.
template <int N, int KL>
__device__ __forceinline__ void pencil_body(const VolArgs& A, const int col, float* smem, const int t) {
  constexpr int n1 = N + 1, Nq = n1 * n1, CP = (n1 + 1) / 2, CW = 2 * CP;
  // words per layer block, padded to 2 (mod 32) so that the 16 layers a
  // half-warp reads (64-bit loads of one z-line's rows) fall on 16 distinct
  // bank pairs
  constexpr int SK = pencil_sk(N);
  constexpr int SXY = kFields * KL * SK;  // floats per flux direction
  const bool part = t < KL * Nq;
  float* sX = smem;                    // [f][kk][j][m][c]
  float* sY = sX + SXY;                // [f][kk][i][m][c]
  float* sT = sY + SXY;                // [f][kk][ab]: top-face residual
  float* sP = sT + kFields * KL * Nq;  // [f][ab]: carry between chunks
  const int kk = t % KL, ab = part ? t / KL : 0;
  const int i = ab % n1, j = ab / n1;
  const int lev = A.col_level[col];
  const float* geo = A.geof[lev];
  const float sx = geo[4], sy = geo[5], sz = geo[6], J = geo[3];
  const int hm = part ? A.hmap[(long long)col * Nq + ab] : 0;
  float Dwi[n1], Dwj[n1];
#pragma unroll
  for (int m = 0; m < n1; ++m) {
    Dwi[m] = c_Dwf[N][i * n1 + m];
    Dwj[m] = c_Dwf[N][j * n1 + m];
  }
  const float wi = c_wf[N][i], wj = c_wf[N][j];
  float* rc = (float*)A.rc;
  const int nchunk = (A.nz + KL - 1) / KL;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int k = ch * KL + kk;
    const bool act = part && k < A.nz;
    const int kz0 = k * N;
    const float hk = act ? __ldg(A.hzk32 + k) : 0.f;   // layer thickness
    float2 r[kFields][CP];
#pragma unroll
    for (int f = 0; f < kFields; ++f)
#pragma unroll
      for (int p = 0; p < CP; ++p) r[f][p] = make_float2(0.f, 0.f);
    float* myX = sX + kk * SK + j * n1 * CW + i * CW;  // + f * FS + c
    float* myY = sY + kk * SK + i * n1 * CW + j * CW;
    constexpr int FS = KL * SK;                         // field stride
    if (act) {
#pragma unroll
      for (int c = 0; c < n1; ++c) {
        float v[kFields];
        const int kz = kz0 + c;
        load_node<N>(A, hm, kz, v);
        const float wc = c_wf[N][c];
        NodeTerms T;
        node_terms(A, v, kz, wj * wc * sx * hk, wi * wc * sy * hk, wi * wj * sz, wi * wj * wc * J * hk, T);
#pragma unroll
        for (int f = 0; f < kFields; ++f) {
          myX[f * FS + c] = T.fx[f];
          myY[f * FS + c] = T.fy[f];
        }
        // z contraction on registers as a rank-1 update per node:
        // r[c'] += Dw[c'][c] Fz[c] for every node c' of the z-line (scalar
        // FMAs: the coefficients are compile-time constant-bank operands)
        float* rz = reinterpret_cast<float*>(&r[0][0]);
#pragma unroll
        for (int f = 0; f < kFields; ++f)
#pragma unroll
          for (int c2 = 0; c2 < n1; ++c2)
            rz[f * CP * 2 + c2] = fmaf(c_Dwf[N][c2 * n1 + c], T.fz[f], rz[f * CP * 2 + c2]);
        rz[(1 * CP * 2) + c] += T.su;
        rz[(2 * CP * 2) + c] += T.sv;
        rz[(3 * CP * 2) + c] += T.sw;
      }
      if (n1 < CW) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) {
          myX[f * FS + n1] = 0.f;
          myY[f * FS + n1] = 0.f;
        }
      }
    } else if (part) {
#pragma unroll
      for (int f = 0; f < kFields; ++f)
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          myX[f * FS + c] = 0.f;
          myY[f * FS + c] = 0.f;
        }
    }
    __syncthreads();
    // x and y contractions from shared memory, two nodes per packed FMA
    const float* rowX = sX + kk * SK + j * n1 * CW;  // + f*FS + m*CW + c
    const float* rowY = sY + kk * SK + i * n1 * CW;
#pragma unroll
    for (int f = 0; f < kFields; ++f)
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        const float2 dx = make_float2(Dwi[m], Dwi[m]);
        const float2 dy = make_float2(Dwj[m], Dwj[m]);
#pragma unroll
        for (int p = 0; p < CP; ++p) {
          const float2 vx = *reinterpret_cast<const float2*>(rowX + f * FS + m * CW + 2 * p);
          const float2 vy = *reinterpret_cast<const float2*>(rowY + f * FS + m * CW + 2 * p);
          r[f][p] = __ffma2_rn(dx, vx, r[f][p]);
          r[f][p] = __ffma2_rn(dy, vy, r[f][p]);
        }
      }
    // vertical DSS: the top node of layer k and the bottom node of layer k+1
    float* rr = reinterpret_cast<float*>(&r[0][0]);
    if (part) {
#pragma unroll
      for (int f = 0; f < kFields; ++f) sT[(f * KL + kk) * Nq + ab] = rr[f * CP * 2 + N];
    }
    if (part && kk == 0 && ch > 0) {
#pragma unroll
      for (int f = 0; f < kFields; ++f) rr[f * CP * 2] += sP[f * Nq + ab];
    }
    __syncthreads();
    if (part && kk > 0) {
#pragma unroll
      for (int f = 0; f < kFields; ++f) rr[f * CP * 2] += sT[(f * KL + kk - 1) * Nq + ab];
    }
    if (part && kk == KL - 1) {
#pragma unroll
      for (int f = 0; f < kFields; ++f) sP[f * Nq + ab] = rr[f * CP * 2 + N];
    }
    if (act) {
      float* dst = rc + ((long long)((long long)col * Nq + ab) * kFields) * A.NZr + kz0;
      const bool top = (k == A.nz - 1);
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        float* df = dst + (long long)f * A.NZr;
        if (N == 4) {
          *reinterpret_cast<float4*>(df) = make_float4(rr[f * CP * 2 + 0], rr[f * CP * 2 + 1],
                                                       rr[f * CP * 2 + 2], rr[f * CP * 2 + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < N; ++c) df[c] = rr[f * CP * 2 + c];
        }
        if (top) df[N] = rr[f * CP * 2 + N];
      }
    }
    __syncthreads();
  }
}

template <int N, int KL, int MB>
__global__ void __launch_bounds__(KL * (N + 1) * (N + 1), MB)
volume_pencil_mixed(const VolArgs A) {
  extern __shared__ __align__(16) float smem[];
  pencil_body<N, KL>(A, blockIdx.x, smem, threadIdx.x);
}

template <int N, int KL>
static size_t pencil_smem() {
  constexpr int n1 = N + 1, Nq = n1 * n1;
  return sizeof(float) * (2 * kFields * KL * pencil_sk(N) + kFields * KL * Nq + kFields * Nq);
}

template <int N, int KL, int MB>
static int launch_pencil(const VolArgs& A, cudaStream_t st) {
  const size_t sm = pencil_smem<N, KL>();
  static DeviceOnce attr;
  int rc = device_once(attr, [&] {
    SEM_CUDA_TRY(cudaFuncSetAttribute(volume_pencil_mixed<N, KL, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return SEM_OK;
  });
  if (rc) return rc;
  ProfScope ps("volume_mixed", st);
  volume_pencil_mixed<N, KL, MB><<<A.Ncol, KL * (N + 1) * (N + 1), sm, st>>>(A);
  return SEM_OK;
}

// Line-exchange variant of the mixed-form element kernel (same thread
// mapping, z-line ownership, z contraction and vertical DSS as pencil_body;
// the same sums, added in another order).  The x and y contractions are done
// by line owners: once the x and y flux components of every node of the chunk
// are in shared memory, thread (kk, L) contracts the whole x-line (j, c) = L
// and the whole y-line (i, c) = L of layer kk with the weak-derivative matrix
// and writes the results back onto the nodes it read (no other thread touches
// them in that phase); the z-line owner then adds both to its register-held z
// contraction.  Node (i, j, c), field f of layer kk sits at
// kk LS + (i + n1 j) LW + f n1 + c.  With LW odd and LS = 32 / KL (mod 32),
// every access of the three phases is a 32-bit access free of bank conflicts
// for N = 4 (consecutive threads: consecutive layers, then lines).
template <int N>
__host__ __device__ constexpr int lines_lw() { return (kFields * (N + 1)) | 1; }
template <int N, int KL>
__host__ __device__ constexpr int lines_ls() {
  return (N + 1) * (N + 1) * lines_lw<N>() +
         ((32 / KL - ((N + 1) * (N + 1) * lines_lw<N>()) % 32) % 32 + 32) % 32;
}
template <int N, int KL>
__host__ __device__ constexpr int lines_smem_floats() {
  return 2 * KL * lines_ls<N, KL>() + kFields * KL * (N + 1) * (N + 1) + 2 * kFields * (N + 1) * (N + 1);
}

// Horizontal Smagorinsky stress (Sec. 4) of one layer chunk, added to the
// z-line owners' residuals rz (momentum rows) inside the element kernel, so
// the state is not read again and the residual not re-written by a separate
// pass.  Same steps and thread roles as the separate stress pass: z-line
// owners form u, v, w; x-/y-line owners differentiate their lines; z-line
// owners form nu_t = (C_s Delta)^2 |S_h| and the weighted fluxes of rho tau;
// line owners contract them in weak form; z-line owners add them up.  The
// components live in sX and sY (free once the inviscid add-back is done).
template <int N, int KL, int LWV, int LSV>
__device__ __forceinline__ void smag_phases(const VolArgs& A, float* smem, const bool act, const int kk,
                                            const int ab, const int lc, const int lo, const int hm,
                                            const int kz0, const int lev, const float wi, const float wj,
                                            const float sxk, const float syk, float (&rz)[kFields][N + 1]) {
  constexpr int n1 = N + 1;
  float* zV = smem + kk * LSV + ab * LWV;   // this thread's z-line, + comp n1 + c
  const float cs2 = A.smag[lev][0], gx = A.smag[lev][1], gy = A.smag[lev][2];
  float rho[n1];
  __syncthreads();   // every add-back has read its fluxes: the buffers are free
  if (act) {
#pragma unroll
    for (int c = 0; c < n1; ++c) {
      const int kz = kz0 + c;
      float v[kFields];
      load_node<N>(A, hm, kz, v);
      rho[c] = __ldg(A.ref4 + kz).y + v[0];
      const float inv = __frcp_rn(rho[c]);
      zV[0 * n1 + c] = v[1] * inv;
      zV[1 * n1 + c] = v[2] * inv;
      zV[2 * n1 + c] = v[3] * inv;
    }
  }
  __syncthreads();
  if (act) {
    // derivatives along the x-line (nodes (m, lo, lc)) and the y-line (nodes (lo, m, lc))
    float* bx = smem + kk * LSV + lo * n1 * LWV + lc;
    float* by = smem + kk * LSV + lo * LWV + lc;
#pragma unroll
    for (int cp = 0; cp < 3; ++cp) {
      float F[n1], G[n1];
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        F[m] = bx[m * LWV + cp * n1];
        G[m] = by[m * n1 * LWV + cp * n1];
      }
#pragma unroll
      for (int o = 0; o < n1; ++o) {
        float ax_ = 0.f, ay_ = 0.f;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          ax_ = fmaf(c_Df[N][o * n1 + m], F[m], ax_);
          ay_ = fmaf(c_Df[N][o * n1 + m], G[m], ay_);
        }
        bx[o * LWV + (3 + cp) * n1] = ax_ * gx;
        by[o * n1 * LWV + (6 + cp) * n1] = ay_ * gy;
      }
    }
  }
  __syncthreads();
  if (act) {
    // eddy viscosity and weighted fluxes of rho tau at the thread's nodes
#pragma unroll
    for (int c = 0; c < n1; ++c) {
      const float ux = zV[3 * n1 + c], vx = zV[4 * n1 + c], wx = zV[5 * n1 + c];
      const float uy = zV[6 * n1 + c], vy = zV[7 * n1 + c], wy = zV[8 * n1 + c];
      const float sxy = 0.5f * (uy + vx);
      const float s2 = 2.f * (ux * ux + vy * vy + 2.f * sxy * sxy);
      const float nut = cs2 * (s2 > 0.f ? s2 * rsqrtf(s2) : 0.f);
      const float kv = rho[c] * nut;
      const float wc = c_wf[N][c];
      const float ax = wj * wc * sxk, ay = wi * wc * syk;
      zV[3 * n1 + c] = ax * (-2.f * kv * ux);
      zV[4 * n1 + c] = ax * (-2.f * kv * sxy);
      zV[5 * n1 + c] = ax * (-kv * wx);
      zV[6 * n1 + c] = ay * (-2.f * kv * sxy);
      zV[7 * n1 + c] = ay * (-2.f * kv * vy);
      zV[8 * n1 + c] = ay * (-kv * wy);
    }
  }
  __syncthreads();
  if (act) {
    // weak contraction of the line's fluxes, written back onto its nodes
    float* bx = smem + kk * LSV + lo * n1 * LWV + lc;
    float* by = smem + kk * LSV + lo * LWV + lc;
#pragma unroll
    for (int cp = 0; cp < 3; ++cp) {
      float F[n1], G[n1];
#pragma unroll
      for (int m = 0; m < n1; ++m) {
        F[m] = bx[m * LWV + (3 + cp) * n1];
        G[m] = by[m * n1 * LWV + (6 + cp) * n1];
      }
#pragma unroll
      for (int o = 0; o < n1; ++o) {
        float ax_ = 0.f, ay_ = 0.f;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          ax_ = fmaf(c_Dwf[N][o * n1 + m], F[m], ax_);
          ay_ = fmaf(c_Dwf[N][o * n1 + m], G[m], ay_);
        }
        bx[o * LWV + (3 + cp) * n1] = ax_;
        by[o * n1 * LWV + (6 + cp) * n1] = ay_;
      }
    }
  }
  __syncthreads();
  if (act) {
#pragma unroll
    for (int cp = 0; cp < 3; ++cp)
#pragma unroll
      for (int c = 0; c < n1; ++c) rz[1 + cp][c] += zV[(3 + cp) * n1 + c] + zV[(6 + cp) * n1 + c];
  }
}

// Body shared by the single-mesh kernel (one CTA per column) and the batched
// persistent kernel.  Threads t >= KL (N+1)^2 of a larger CTA take part in
// the barriers only.
// TMA (kind 4): the state runs of the CTA's non-hanging column lines are
// staged in shared memory by bulk copies (cp.async.bulk, one per field and
// line: the 16-byte-aligned window of at most KL N + 1 + 3 floats around the
// chunk's levels), completing on an mbarrier; the copies of chunk ch + 1 are
// issued once every thread has read chunk ch's staged values and run under
// chunk ch's line exchange.  Hanging lines, a state array that is not 16-byte
// aligned and a window that would run past the end of the array take the
// plain loads.  The values, hence the arithmetic, are those of the plain
// kernel.  The waits are bounded: a wait that runs out sets bit 2 of the
// status word, waits once more for the copies in flight and leaves the
// column's remaining chunks unwritten.
template <int N, int KL>
__host__ __device__ constexpr int lines_tma_sw() { return (KL * N + 1 + 3 + 3) / 4 * 4; }
template <int N, int KL>
__host__ __device__ constexpr int lines_tma_stage_off() { return (lines_smem_floats<N, KL>() + 3) / 4 * 4; }
template <int N, int KL>
__host__ __device__ constexpr int lines_tma_smem_floats() {
  return lines_tma_stage_off<N, KL>() + kFields * (N + 1) * (N + 1) * lines_tma_sw<N, KL>() + 4;
}

template <int N, int KL, bool SMAG = false, bool WARP = false, bool TMA = false>
__device__ __forceinline__ void lines_body(const VolArgs& A, const int col, float* smem, const int t) {
  constexpr int n1 = N + 1, Nq = n1 * n1;
  constexpr int LW = lines_lw<N>(), LS = lines_ls<N, KL>();
  // SMAG: the stress phases keep 9 components per node (u, v, w, their x and
  // y derivatives, then the weighted fluxes) in sX and sY, reused as one
  // buffer with layer stride LSV
  constexpr int LWV = (9 * n1) | 1;
  constexpr int LSV = Nq * LWV + ((32 / KL - (Nq * LWV) % 32) % 32 + 32) % 32;
  static_assert(!SMAG || LSV <= 2 * LS, "stress components do not fit the flux buffers");
  float* sX = smem;                       // [kk][LS]: x fluxes, then x contractions
  float* sY = sX + KL * LS;               // [kk][LS]: the same for y
  float* sT = sY + KL * LS;               // [f][kk][ab]: z part of the top-node residual
  float* sP = sT + kFields * KL * Nq;     // [2][f][ab]: top-node carry between chunks
  const bool part = t < KL * Nq;
  const int kk = t % KL, ab = part ? t / KL : 0;
  const int i = ab % n1, j = ab / n1;
  const int lc = ab % n1, lo = ab / n1;   // exchange phase: x-line (j, c) = (lo, lc), y-line (i, c) = (lo, lc)
  const int lev = A.col_level[col];
  const float* geo = A.geof[lev];
  const float sx = geo[4], sy = geo[5], sz = geo[6], J = geo[3];
  const int hm = part ? A.hmap[(long long)col * Nq + ab] : 0;
  const float wi = c_wf[N][i], wj = c_wf[N][j];
  float* rc = (float*)A.rc;
  const int nchunk = (A.nz + KL - 1) / KL;
  // TMA staging: window of field f, line ab at sQ + (f Nq + ab) SW; thread
  // t < 5 Nq issues the copy of (field t / Nq, line t mod Nq)
  static_assert(!TMA || (KL >= kFields && !SMAG && !WARP), "TMA staging needs a thread per field and line");
  constexpr int SW = lines_tma_sw<N, KL>();
  float* sQ = smem + lines_tma_stage_off<N, KL>();
  const uint32_t bar = TMA ? tcg::smem_u32(sQ + kFields * Nq * SW) : 0u;
  const float* qf = (const float*)A.q;
  const long long qtot = (long long)kFields * A.NG;
  const bool tma_ok = TMA && (((uintptr_t)A.q & 15) == 0);
  // whether chunk chn's window of line hq fits the array (the last field's is the furthest)
  auto staged = [&](int hq, int chn) {
    const int nl = min(KL, A.nz - chn * KL) * N + 1;
    return tma_ok && hq >= 0 &&
           ((((long long)(kFields - 1) * A.NG + (long long)hq * A.NZ + chn * KL * N + nl + 3) & ~3ll) <= qtot);
  };
  auto issue = [&](int chn) {
    if (t < kFields * Nq) {
      const int f = t / Nq, abq = t - (t / Nq) * Nq;
      const int hq = A.hmap[(long long)col * Nq + abq];
      if (staged(hq, chn)) {
        const int nl = min(KL, A.nz - chn * KL) * N + 1;
        const long long off = (long long)f * A.NG + (long long)hq * A.NZ + chn * KL * N;
        const long long ws = off & ~3ll, we = (off + nl + 3) & ~3ll;
        const uint32_t bytes = (uint32_t)((we - ws) * 4);
        tcg::fence_async_smem();
        tcg::mbar_expect_tx(bar, bytes);
        tcg::bulk_g2s(tcg::smem_u32(sQ + (f * Nq + abq) * SW), qf + ws, bytes, bar);
      }
    }
  };
  if constexpr (TMA) {
    if (t == 0) tcg::mbar_init(bar, 1);
    __syncthreads();
    issue(0);
    __syncthreads();
    if (t == 0) tcg::mbar_arrive(bar);
  }
  for (int ch = 0; ch < nchunk; ++ch) {
    const int k = ch * KL + kk;
    const bool act = part && k < A.nz;
    const int kz0 = k * N;
    const float hk = act ? __ldg(A.hzk32 + k) : 0.f;   // layer thickness
    // this thread's staged window (TMA): its offset inside the window per field
    bool st_line = false;
    int dwin = 0;
    if constexpr (TMA) {
      if (!__syncthreads_and(tcg::mbar_wait(bar, (uint32_t)(ch & 1)))) {
        // a wait ran out: record it, let the copies in flight land, stop
        if (t == 0) atomicOr(A.status, 4);
        tcg::mbar_wait(bar, (uint32_t)(ch & 1));
        __syncthreads();
        break;
      }
      st_line = part && staged(hm, ch);
      dwin = (int)(((long long)hm * A.NZ + ch * KL * N) & 3);
    }
    float rz[kFields][n1];
#pragma unroll
    for (int f = 0; f < kFields; ++f)
#pragma unroll
      for (int c = 0; c < n1; ++c) rz[f][c] = 0.f;
    float* zX = sX + kk * LS + ab * LW;   // this thread's z-line, + f n1 + c
    float* zY = sY + kk * LS + ab * LW;
    if (act) {
#pragma unroll
      for (int c = 0; c < n1; ++c) {
        float v[kFields];
        const int kz = kz0 + c;
        if (TMA && st_line) {
          // the staged window: field f starts (f NG) mod 4 floats later
#pragma unroll
          for (int f = 0; f < kFields; ++f)
            v[f] = sQ[(f * Nq + ab) * SW + ((dwin + (int)(((long long)f * A.NG) & 3)) & 3) + kk * N + c];
        } else {
          load_node<N>(A, hm, kz, v);
        }
        const float wc = c_wf[N][c];
        NodeTerms T;
        float wJn = wi * wj * wc * J * hk;
        if constexpr (!WARP) {
          node_terms(A, v, kz, wj * wc * sx * hk, wi * wc * sy * hk, wi * wj * sz, wJn, T);
        } else {
          // warped layers: metric of the node and the reference state at its height
          const float* mt = A.metric32 + ((((long long)col * Nq + ab) * A.nz + k) * n1 + c) * 3;
          const float zx = __ldg(mt), zy = __ldg(mt + 1), zz = __ldg(mt + 2);
          const float hx = geo[0], hy = geo[1];
          const float4 ra = hm >= 0 ? __ldg(A.ref4G + (long long)hm * A.NZ + kz)
                                    : __ldg(A.ref4H + (long long)(-1 - hm) * A.NZ + kz);
          wJn = wi * wj * wc * sz * zz;
          node_terms_w(A, v, ra, wj * wc * 0.5f * hy * zz, wi * wc * 0.5f * hx * zz, wi * wj * sz,
                       -wi * wj * 0.5f * hy * zx, -wi * wj * 0.5f * hx * zy, wJn, T);
        }
#pragma unroll
        for (int f = 0; f < kFields; ++f) {
          zX[f * n1 + c] = T.fx[f];
          zY[f * n1 + c] = T.fy[f];
        }
#pragma unroll
        for (int f = 0; f < kFields; ++f)
#pragma unroll
          for (int c2 = 0; c2 < n1; ++c2) rz[f][c2] = fmaf(c_Dwf[N][c2 * n1 + c], T.fz[f], rz[f][c2]);
        rz[1][c] += T.su;
        rz[2][c] += T.sv;
        rz[3][c] += T.sw;
        if (A.spg32) {
          // absorbing layer (Sec. 4): -R(z) q' at the node, weighted like the sources
          const float wR = wJn * __ldg(A.spg32 + kz);
#pragma unroll
          for (int f = 0; f < kFields; ++f) rz[f][c] = fmaf(-wR, v[f], rz[f][c]);
        }
      }
      if constexpr (!SMAG) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) sT[(f * KL + kk) * Nq + ab] = rz[f][N];
      }
    }
    __syncthreads();
    // every thread has read chunk ch's staged values: the next chunk's copies
    // run under this chunk's line exchange
    if (TMA && ch + 1 < nchunk) issue(ch + 1);
    if (act) {
      // x-line (lo, lc): nodes (m, lo, lc), m = 0..N
      float* bx = sX + kk * LS + lo * n1 * LW + lc;
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        float F[n1];
#pragma unroll
        for (int m = 0; m < n1; ++m) F[m] = bx[m * LW + f * n1];
#pragma unroll
        for (int i2 = 0; i2 < n1; ++i2) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < n1; ++m) acc = fmaf(c_Dwf[N][i2 * n1 + m], F[m], acc);
          bx[i2 * LW + f * n1] = acc;
        }
      }
      // y-line (lo, lc): nodes (lo, m, lc)
      float* by = sY + kk * LS + lo * LW + lc;
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        float F[n1];
#pragma unroll
        for (int m = 0; m < n1; ++m) F[m] = by[m * n1 * LW + f * n1];
#pragma unroll
        for (int j2 = 0; j2 < n1; ++j2) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < n1; ++m) acc = fmaf(c_Dwf[N][j2 * n1 + m], F[m], acc);
          by[j2 * n1 * LW + f * n1] = acc;
        }
      }
    }
    __syncthreads();
    // all of the next chunk's transaction counts are registered
    if (TMA && ch + 1 < nchunk && t == 0) tcg::mbar_arrive(bar);
    if constexpr (SMAG) {
      if (act) {
#pragma unroll
        for (int f = 0; f < kFields; ++f)
#pragma unroll
          for (int c = 0; c < n1; ++c) rz[f][c] += zX[f * n1 + c] + zY[f * n1 + c];
      }
      smag_phases<N, KL, LWV, LSV>(A, smem, act, kk, ab, lc, lo, hm, kz0, lev, wi, wj, sx * hk, sy * hk, rz);
      // the full top-node value of each layer, for the layer above
      if (act) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) sT[(f * KL + kk) * Nq + ab] = rz[f][N];
      }
      __syncthreads();
    }
    if (act) {
      if constexpr (!SMAG) {
#pragma unroll
        for (int f = 0; f < kFields; ++f)
#pragma unroll
          for (int c = 0; c < n1; ++c) rz[f][c] += zX[f * n1 + c] + zY[f * n1 + c];
      }
      // vertical DSS: the bottom node takes the full top-node value of the
      // layer below (its z part from sT, its x and y parts still in sX, sY;
      // with SMAG all of it from sT), summed as z + (x + y) like the value
      // the layer below forms itself and hands on between chunks, so that
      // the result does not depend on where the chunks split the column
      if (kk > 0 && SMAG) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) rz[f][0] += sT[(f * KL + kk - 1) * Nq + ab];
      } else if (kk > 0) {
        const float* pX = sX + (kk - 1) * LS + ab * LW;
        const float* pY = sY + (kk - 1) * LS + ab * LW;
#pragma unroll
        for (int f = 0; f < kFields; ++f)
          rz[f][0] += sT[(f * KL + kk - 1) * Nq + ab] + (pX[f * n1 + N] + pY[f * n1 + N]);
      } else if (ch > 0) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) rz[f][0] += sP[((ch - 1) & 1) * kFields * Nq + f * Nq + ab];
      }
      if (kk == KL - 1) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) sP[(ch & 1) * kFields * Nq + f * Nq + ab] = rz[f][N];
      }
      float* dst = rc + ((long long)((long long)col * Nq + ab) * kFields) * A.NZr + kz0;
      const bool top = (k == A.nz - 1);
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        float* df = dst + (long long)f * A.NZr;
        if (N == 4) {
          *reinterpret_cast<float4*>(df) = make_float4(rz[f][0], rz[f][1], rz[f][2], rz[f][3]);
        } else {
#pragma unroll
          for (int c = 0; c < N; ++c) df[c] = rz[f][c];
        }
        if (top) df[N] = rz[f][N];
      }
    }
    if (ch + 1 < nchunk) __syncthreads();
  }
}

template <int N, int KL, int MB>
__global__ void __launch_bounds__(KL * (N + 1) * (N + 1), MB)
volume_lines_mixed(const VolArgs A) {
  extern __shared__ __align__(16) float smem[];
  lines_body<N, KL>(A, blockIdx.x, smem, threadIdx.x);
}

// The same with the state staged by bulk copies (TMA, kind 4).
template <int N, int KL, int MB>
__global__ void __launch_bounds__(KL * (N + 1) * (N + 1), MB)
volume_lines_tma(const VolArgs A) {
  extern __shared__ __align__(16) float smem[];
  lines_body<N, KL, false, false, true>(A, blockIdx.x, smem, threadIdx.x);
}

// The same on warped layers (non-affine elements).
template <int N, int KL, int MB>
__global__ void __launch_bounds__(KL * (N + 1) * (N + 1), MB)
volume_lines_warp(const VolArgs A) {
  extern __shared__ __align__(16) float smem[];
  lines_body<N, KL, false, true>(A, blockIdx.x, smem, threadIdx.x);
}

// The same with the horizontal Smagorinsky stress added (N = 4 variants).
template <int N, int KL, int MB>
__global__ void __launch_bounds__(KL * (N + 1) * (N + 1), MB)
volume_lines_smag(const VolArgs A) {
  extern __shared__ __align__(16) float smem[];
  lines_body<N, KL, true>(A, blockIdx.x, smem, threadIdx.x);
}

// ---------------------------------------------------------------------------
// Mixed form, the paper's equation set (Sec. 2: mass in flux form; momentum
// and potential temperature in advective form, in the primitive perturbation
// variables rho', u, v, w, theta'): line-exchange element kernel.
//
// Same thread roles and contraction skeleton as lines_body, with a different
// pointwise part.  The z-line owner forms at each node of its line the
// weighted mass-flux components and the five quantities u, v, w, p', theta';
// the x- and y-line owners apply the weak derivative to their line's mass
// flux and the strong derivative D to the five quantities; the z-line owner
// takes the z derivatives from the quantities it kept in registers and forms
// the advective residuals node by node, as volume_column does for this set.
// A layer's top-node residual is complete only after that combination, so it
// passes to the layer above through shared memory after one more barrier.
// W: warped layers, as volume_column's warped branch: the weak mass flux is the
// contravariant one (the z component takes the x and y fluxes with the weights
// of J grad zeta), the strong derivatives are taken at constant height
// (d/dx = 2/hx (d/dxi - z_xi/z_zeta d/dzeta) and so on), and the reference
// state is the one at each node's height.
template <int N>
__host__ __device__ constexpr int nc_lw() { return (6 * (N + 1)) | 1; }
template <int N, int KL>
__host__ __device__ constexpr int nc_ls() {
  return (N + 1) * (N + 1) * nc_lw<N>() + ((32 / KL - ((N + 1) * (N + 1) * nc_lw<N>()) % 32) % 32 + 32) % 32;
}
template <int N, int KL>
__host__ __device__ constexpr int nc_smem_floats() {
  return 2 * KL * nc_ls<N, KL>() + kFields * KL * (N + 1) * (N + 1) + 2 * kFields * (N + 1) * (N + 1) +
         2 * (N + 1) * KL * (N + 1) * (N + 1) + 2 * 5 * (KL * N + 1);
}

template <int N, int KL, bool WARP = false>
__device__ __forceinline__ void lines_nc_body(const VolArgs& A, const int col, float* smem, const int t) {
  constexpr int n1 = N + 1, Nq = n1 * n1;
  constexpr int LW = nc_lw<N>(), LS = nc_ls<N, KL>();
  float* sX = smem;                       // [kk][LS]: per line ab, [6][n1]: mass flux x, u, v, w, p', theta'
  float* sY = sX + KL * LS;               // [kk][LS]: the same for y
  float* sT = sY + KL * LS;               // [f][kk][ab]: full top-node residual of each layer
  float* sP = sT + kFields * KL * Nq;     // [2][f][ab]: top-node carry between chunks
  float* sV = sP + 2 * kFields * Nq;      // [2][c][t]: 1 / rho and rho' of the thread's nodes
  constexpr int NL = KL * N + 1;          // levels of a chunk
  float* sR = sV + 2 * n1 * KL * Nq;      // [2][5][NL]: the chunk's reference rows, double-buffered:
                                          // theta0, p0, rho0, 1/(rho theta)0, dtheta0/dz
  const bool part = t < KL * Nq;
  const int kk = t % KL, ab = part ? t / KL : 0;
  const int i = ab % n1, j = ab / n1;
  const int lc = ab % n1, lo = ab / n1;   // exchange phase: x-line (j, c) = (lo, lc), y-line (i, c) = (lo, lc)
  const int lev = A.col_level[col];
  const float* geo = A.geof[lev];
  const float sx = geo[4], sy = geo[5], sz = geo[6], J = geo[3];
  const float gx = 2.f / geo[0], gy = 2.f / geo[1];
  constexpr int NT = KL * Nq;
  const int hm = part ? A.hmap[(long long)col * Nq + ab] : 0;
  const float wi = c_wf[N][i], wj = c_wf[N][j];
  const float fc = A.ff, g = A.gf;
  const float hx = geo[0], hy = geo[1];
  float* rc = (float*)A.rc;
  const int nchunk = (A.nz + KL - 1) / KL;
  // W: reference row at a node's own height; metric terms z_xi, z_eta, z_zeta of a node
  auto ref_at = [&](int kz) {
    return hm >= 0 ? A.refG32 + ((long long)hm * A.NZ + kz) * kRef
                   : A.refH32 + ((long long)(-1 - hm) * A.NZ + kz) * kRef;
  };
  auto metric_at = [&](int k, int c) {
    return A.metric32 + ((((long long)col * Nq + ab) * A.nz + k) * n1 + c) * 3;
  };
  // reference rows of chunk chn into buffer chn & 1 (levels past the top repeat it)
  auto stage_ref = [&](int chn) {
    float* R = sR + (chn & 1) * 5 * NL;
    for (int e = t; e < 5 * NL; e += blockDim.x) {
      const int f = e / NL, z = e - (e / NL) * NL;
      const int kz = min(chn * KL * N + z, A.NZ - 1);
      constexpr int fld[5] = {0, 2, 3, 6, 5};
      R[e] = __ldg(A.ref32 + (long long)kz * kRef + fld[f]);
    }
  };
  if constexpr (!WARP) {
    stage_ref(0);
    __syncthreads();
  }
  for (int ch = 0; ch < nchunk; ++ch) {
    const int k = ch * KL + kk;
    const bool act = part && k < A.nz;
    const int kz0 = k * N;
    const float hk = act ? __ldg(A.hzk32 + k) : 1.f;   // layer thickness
    const float* R = sR + (ch & 1) * 5 * NL + kk * N;   // + f NL + c
    float qz[5][n1];   // u, v, w, p', theta' on this thread's z-line
    float rm[n1];      // z part of the weak mass-flux contraction
#pragma unroll
    for (int c = 0; c < n1; ++c) {
      rm[c] = 0.f;
#pragma unroll
      for (int f = 0; f < 5; ++f) qz[f][c] = 0.f;
    }
    float* zX = sX + kk * LS + ab * LW;   // this thread's z-line, + s n1 + c
    float* zY = sY + kk * LS + ab * LW;
    if (act) {
#pragma unroll
      for (int c = 0; c < n1; ++c) {
        float v[kFields];
        const int kz = kz0 + c;
        load_node<N>(A, hm, kz, v);
        const float wc = c_wf[N][c];
        float th0, p0, rho0, inv_rt0, ax, ay, cxw = 0.f, cyw = 0.f;
        if constexpr (!WARP) {
          th0 = R[c], p0 = R[NL + c], rho0 = R[2 * NL + c], inv_rt0 = R[3 * NL + c];
          ax = wj * wc * sx * hk;
          ay = wi * wc * sy * hk;
        } else {
          // reference row: theta0, pi0, p0, rho0 | (rho theta)0, dtheta0/dz, 1/(rho theta)0, z
          const float* rf = ref_at(kz);
          const float4 r0 = __ldg(reinterpret_cast<const float4*>(rf));
          const float4 r1 = __ldg(reinterpret_cast<const float4*>(rf + 4));
          th0 = r0.x, p0 = r0.z, rho0 = r0.w, inv_rt0 = r1.z;
          const float* mt = metric_at(k, c);
          const float zx = __ldg(mt), zy = __ldg(mt + 1), zz = __ldg(mt + 2);
          ax = wj * wc * 0.5f * hy * zz;        // weighted J grad xi . e_x
          ay = wi * wc * 0.5f * hx * zz;        // weighted J grad eta . e_y
          cxw = -0.5f * hy * zx * wi * wj;      // weighted J grad zeta . e_x
          cyw = -0.5f * hx * zy * wi * wj;      // weighted J grad zeta . e_y
        }
        const float rp = v[0], u = v[1], vv = v[2], w = v[3], thp = v[4];
        const float rho = rho0 + rp;
        const float inv = __frcp_rn(rho);
        const float rtp = fmaf(rho0, thp, rp * (th0 + thp));   // (rho theta)'
        const float pp = p0 * pow1p_m1(rtp * inv_rt0, A.bin, A.gammaf);
        zX[c] = rho * u * ax;
        zY[c] = rho * vv * ay;
        float Fz = rho * w * (wi * wj * sz);
        if constexpr (WARP) Fz = fmaf(rho * u, cxw, fmaf(rho * vv, cyw, Fz));
#pragma unroll
        for (int c2 = 0; c2 < n1; ++c2) rm[c2] = fmaf(c_Dwf[N][c2 * n1 + c], Fz, rm[c2]);
        qz[0][c] = u;
        qz[1][c] = vv;
        qz[2][c] = w;
        qz[3][c] = pp;
        qz[4][c] = thp;
        sV[c * NT + t] = inv;
        sV[(n1 + c) * NT + t] = rp;
#pragma unroll
        for (int f = 0; f < 5; ++f) {
          zX[(f + 1) * n1 + c] = qz[f][c];
          zY[(f + 1) * n1 + c] = qz[f][c];
        }
      }
    }
    __syncthreads();
    // the next chunk's reference rows load under this chunk's line exchange
    if (!WARP && ch + 1 < nchunk) stage_ref(ch + 1);
    if (act) {
      // x-line (lo, lc): nodes (m, lo, lc); slot 0 weak, slots 1..5 strong
      float* bx = sX + kk * LS + lo * n1 * LW + lc;
      float* by = sY + kk * LS + lo * LW + lc;
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        float F[n1];
#pragma unroll
        for (int m = 0; m < n1; ++m) F[m] = bx[m * LW + s * n1];
#pragma unroll
        for (int i2 = 0; i2 < n1; ++i2) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < n1; ++m)
            acc = fmaf(s == 0 ? c_Dwf[N][i2 * n1 + m] : c_Df[N][i2 * n1 + m], F[m], acc);
          bx[i2 * LW + s * n1] = acc;
        }
      }
      // y-line (lo, lc): nodes (lo, m, lc)
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        float F[n1];
#pragma unroll
        for (int m = 0; m < n1; ++m) F[m] = by[m * n1 * LW + s * n1];
#pragma unroll
        for (int j2 = 0; j2 < n1; ++j2) {
          float acc = 0.f;
#pragma unroll
          for (int m = 0; m < n1; ++m)
            acc = fmaf(s == 0 ? c_Dwf[N][j2 * n1 + m] : c_Df[N][j2 * n1 + m], F[m], acc);
          by[j2 * n1 * LW + s * n1] = acc;
        }
      }
    }
    __syncthreads();
    // residuals of the bottom and top nodes (kept for the vertical DSS); the
    // inner nodes' go to the residual array as they are formed
    float rb[kFields], rt[kFields];
    float* dst = rc + ((long long)((long long)col * Nq + ab) * kFields) * A.NZr + kz0;
    if (act) {
      const float gz = 2.f / hk;
      const float wJ1 = wi * wj * J * hk;
#pragma unroll
      for (int c = 0; c < n1; ++c) {
        // derivatives of u, v, w, p', theta' at node c: x, y from the line
        // owners, z from this thread's own line
        float dx[5], dy[5], dz[5];
        float wJ, th0dz;
        if constexpr (!WARP) {
#pragma unroll
          for (int f = 0; f < 5; ++f) {
            float a = 0.f;
#pragma unroll
            for (int m = 0; m < n1; ++m) a = fmaf(c_Df[N][c * n1 + m], qz[f][m], a);
            dx[f] = zX[(f + 1) * n1 + c] * gx;
            dy[f] = zY[(f + 1) * n1 + c] * gy;
            dz[f] = a * gz;
          }
          wJ = wJ1 * c_wf[N][c];
          th0dz = R[4 * NL + c];
        } else {
          const float* mt = metric_at(k, c);
          const float zx = __ldg(mt), zy = __ldg(mt + 1), zz = __ldg(mt + 2);
          const float gzw = 1.f / zz, rzx = zx / zz, rzy = zy / zz;
#pragma unroll
          for (int f = 0; f < 5; ++f) {
            float a = 0.f;
#pragma unroll
            for (int m = 0; m < n1; ++m) a = fmaf(c_Df[N][c * n1 + m], qz[f][m], a);
            dx[f] = (zX[(f + 1) * n1 + c] - rzx * a) * gx;
            dy[f] = (zY[(f + 1) * n1 + c] - rzy * a) * gy;
            dz[f] = a * gzw;
          }
          wJ = wi * wj * c_wf[N][c] * sz * zz;
          th0dz = __ldg(ref_at(kz0 + c) + 5);
        }
        const float u = qz[0][c], vv = qz[1][c], w = qz[2][c], inv = sV[c * NT + t];
        float adv[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) adv[f] = fmaf(w, dz[f], fmaf(vv, dy[f], u * dx[f]));
        const float r[kFields] = {rm[c] + zX[c] + zY[c], wJ * (-adv[0] - dx[3] * inv + fc * vv),
                                  wJ * (-adv[1] - dy[3] * inv - fc * u),
                                  wJ * (-adv[2] - dz[3] * inv - sV[(n1 + c) * NT + t] * inv * g), wJ * (-w * th0dz - adv[4])};
#pragma unroll
        for (int f = 0; f < kFields; ++f) {
          if (c == 0) rb[f] = r[f];
          else if (c == N) rt[f] = r[f];
          else dst[(long long)f * A.NZr + c] = r[f];
        }
      }
#pragma unroll
      for (int f = 0; f < kFields; ++f) sT[(f * KL + kk) * Nq + ab] = rt[f];
    }
    __syncthreads();
    if (act) {
      // vertical DSS: the bottom node takes the full top-node value of the
      // layer below (this chunk: sT; the previous chunk's last layer: sP)
      if (kk > 0) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) rb[f] += sT[(f * KL + kk - 1) * Nq + ab];
      } else if (ch > 0) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) rb[f] += sP[((ch - 1) & 1) * kFields * Nq + f * Nq + ab];
      }
      if (kk == KL - 1) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) sP[(ch & 1) * kFields * Nq + f * Nq + ab] = rt[f];
      }
      const bool top = (k == A.nz - 1);
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        dst[(long long)f * A.NZr] = rb[f];
        if (top) dst[(long long)f * A.NZr + N] = rt[f];
      }
    }
  }
}

template <int N, int KL, int MB>
__global__ void __launch_bounds__(KL * (N + 1) * (N + 1), MB)
volume_lines_nc(const VolArgs A) {
  extern __shared__ __align__(16) float smem[];
  lines_nc_body<N, KL>(A, blockIdx.x, smem, threadIdx.x);
}

// The same on warped layers (non-affine elements).
template <int N, int KL, int MB>
__global__ void __launch_bounds__(KL * (N + 1) * (N + 1), MB)
volume_lines_nc_warp(const VolArgs A) {
  extern __shared__ __align__(16) float smem[];
  lines_nc_body<N, KL, true>(A, blockIdx.x, smem, threadIdx.x);
}

// ---------------------------------------------------------------------------
// Tensor-core variant of the line-exchange element kernel (kind 2, order 4).
//
// The x and y contractions of a layer chunk run on the fifth-generation
// tensor cores instead of the line owners' FMAs: with the rows of an MMA
// operand the (line, field, layer) triples of one direction and its K the
// N+1 = 5 nodes of a line (padded to 8), the contraction with the weak
// derivative matrix is D[row][n] = sum_k A[row][k] B[n][k], B[n][k] =
// w_k D_kn (padded to 16 x 8).  One chunk of KL = 4 layers has 500 rows per
// direction: 4 tiles of M = 128, 8 MMAs (tcgen05.mma kind::tf32, N = 16,
// K = 8) per product.  float32 accuracy needs three products per tile
// (A_hi B_hi + A_lo B_hi + A_hi B_lo with hi = the value rounded to tf32 and
// lo = the rest, "3xTF32"), so 24 MMAs per chunk, issued by one thread, with
// the accumulators in tensor memory (128 columns per CTA).  The z-line
// owners write the flux components as hi and lo parts into the K-major
// operand layout (core matrices of 8 rows x 16 bytes, no swizzle); after the
// MMAs each warp reads its 32 lanes of every tile (tcgen05.ld) and scatters
// the 5 outputs of its rows onto the nodes' positions of the line-exchange
// layout (reusing the operand buffers), from where the z-line owners add
// them up as in lines_body.  Everything else (pointwise terms, z contraction
// on registers, absorbing layer, vertical direct stiffness summation,
// residual stores) is lines_body's.  Waits on the MMA completion barrier are
// bounded; a wait that runs out sets bit 4 of the status word.

constexpr int kTcKL = 4, kTcThreads = 128, kTcRows = 512, kTcCols = 128;
constexpr int kTcOpBytes = kTcRows * 32;   // one operand (512 rows x 8 tf32)
__host__ __device__ constexpr size_t tc_smem_bytes() {
  // A: x hi, x lo, y hi, y lo; B: hi, lo; sT, sP; barrier and TMEM address
  return 4 * kTcOpBytes + 2 * 512 + sizeof(float) * (kFields * kTcKL * 25 + 2 * kFields * 25) + 16;
}

template <int MB>
__global__ void __launch_bounds__(kTcThreads, MB) volume_lines_tc(const VolArgs A) {
  constexpr int N = 4, n1 = 5, Nq = 25, KL = kTcKL;
  constexpr int LW = lines_lw<N>(), LS = lines_ls<N, KL>();
  static_assert(KL * LS * 4 <= 2 * kTcOpBytes, "staging must fit two operand buffers");
  extern __shared__ __align__(1024) unsigned char tsm[];
  unsigned char* opA = tsm;                                   // [4][kTcOpBytes]
  unsigned char* opB = tsm + 4 * kTcOpBytes;                  // [2][512]
  float* sT = reinterpret_cast<float*>(opB + 1024);           // [f][kk][ab]
  float* sP = sT + kFields * KL * Nq;                         // [2][f][ab]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sP + 2 * kFields * Nq);
  uint32_t* taddr_s = reinterpret_cast<uint32_t*>(mbar + 1);
  float* stX = reinterpret_cast<float*>(opA);                 // staging after the MMAs
  float* stY = reinterpret_cast<float*>(opA + 2 * kTcOpBytes);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int col = blockIdx.x;
  // zero the operands (their K padding stays zero), write B = w_k D_kn
  for (int q = t; q < kTcOpBytes; q += kTcThreads) reinterpret_cast<uint32_t*>(opA)[q] = 0u;
  for (int q = t; q < 256; q += kTcThreads) reinterpret_cast<uint32_t*>(opB)[q] = 0u;
  __syncthreads();
  {
    const int nn = t >> 3, k = t & 7;   // 128 threads: rows n = 0..15, k = 0..7
    const float v = (nn < n1 && k < n1) ? c_Dwf[N][nn * n1 + k] : 0.f;
    const float hi = tcg::tf32_rna(v);
    *reinterpret_cast<float*>(opB + tcg::aoff(nn, k)) = hi;
    *reinterpret_cast<float*>(opB + 512 + tcg::aoff(nn, k)) = v - hi;
  }
  if (warp == 0) {
    tcg::alloc(taddr_s, kTcCols);
  }
  if (t == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tcg::smem_u32(mbar)));
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t taddr = *taddr_s;
  const uint32_t bar = tcg::smem_u32(mbar);

  const bool part = t < KL * Nq;
  const int kk = t % KL, ab = part ? t / KL : 0;
  const int i = ab % n1, j = ab / n1;
  const int lev = A.col_level[col];
  const float* geo = A.geof[lev];
  const float sx = geo[4], sy = geo[5], sz = geo[6], J = geo[3];
  const int hm = part ? A.hmap[(long long)col * Nq + ab] : 0;
  const float wi = c_wf[N][i], wj = c_wf[N][j];
  float* rc = (float*)A.rc;
  const int nchunk = (A.nz + KL - 1) / KL;
  bool ok = true;
  for (int ch = 0; ch < nchunk && ok; ++ch) {
    const int k = ch * KL + kk;
    const bool act = part && k < A.nz;
    const int kz0 = k * N;
    const float hk = act ? __ldg(A.hzk32 + k) : 0.f;
    float rz[kFields][n1];
#pragma unroll
    for (int f = 0; f < kFields; ++f)
#pragma unroll
      for (int c = 0; c < n1; ++c) rz[f][c] = 0.f;
    if (act) {
#pragma unroll
      for (int c = 0; c < n1; ++c) {
        float v[kFields];
        const int kz = kz0 + c;
        load_node<N>(A, hm, kz, v);
        const float wc = c_wf[N][c];
        NodeTerms T;
        node_terms(A, v, kz, wj * wc * sx * hk, wi * wc * sy * hk, wi * wj * sz, wi * wj * wc * J * hk, T);
#pragma unroll
        for (int f = 0; f < kFields; ++f) {
          const int rx = kk + 4 * (f + 5 * (c + 5 * j)), ry = kk + 4 * (f + 5 * (c + 5 * i));
          const float xh = tcg::tf32_rna(T.fx[f]), yh = tcg::tf32_rna(T.fy[f]);
          *reinterpret_cast<float*>(opA + tcg::aoff(rx, i)) = xh;
          *reinterpret_cast<float*>(opA + kTcOpBytes + tcg::aoff(rx, i)) = T.fx[f] - xh;
          *reinterpret_cast<float*>(opA + 2 * kTcOpBytes + tcg::aoff(ry, j)) = yh;
          *reinterpret_cast<float*>(opA + 3 * kTcOpBytes + tcg::aoff(ry, j)) = T.fy[f] - yh;
        }
#pragma unroll
        for (int f = 0; f < kFields; ++f)
#pragma unroll
          for (int c2 = 0; c2 < n1; ++c2) rz[f][c2] = fmaf(c_Dwf[N][c2 * n1 + c], T.fz[f], rz[f][c2]);
        rz[1][c] += T.su;
        rz[2][c] += T.sv;
        rz[3][c] += T.sw;
        if (A.spg32) {
          const float wR = (wi * wj * wc * J * hk) * __ldg(A.spg32 + kz);
#pragma unroll
          for (int f = 0; f < kFields; ++f) rz[f][c] = fmaf(-wR, v[f], rz[f][c]);
        }
      }
#pragma unroll
      for (int f = 0; f < kFields; ++f) sT[(f * KL + kk) * Nq + ab] = rz[f][N];
    }
    // the operands are complete: make them visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t == 0) {
      constexpr uint32_t id = tcg::idesc_tf32(128, 16);
      const uint32_t a0 = tcg::smem_u32(opA), b0 = tcg::smem_u32(opB);
      const uint64_t bh = tcg::sdesc(b0, 128, 256), bl = tcg::sdesc(b0 + 512, 128, 256);
#pragma unroll
      for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int tl = 0; tl < 4; ++tl) {
          const uint32_t dcol = taddr + (uint32_t)((d * 4 + tl) * 16);
          const uint32_t ah = a0 + (uint32_t)(2 * d * kTcOpBytes + tl * 4096);
          const uint64_t dah = tcg::sdesc(ah, 128, 256), dal = tcg::sdesc(ah + kTcOpBytes, 128, 256);
          tcg::mma_tf32(dcol, dah, bh, id, 0);
          tcg::mma_tf32(dcol, dal, bh, id, 1);
          tcg::mma_tf32(dcol, dah, bl, id, 1);
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(bar) : "memory");
    }
    ok = __syncthreads_and(tcg::mbar_wait(bar, (uint32_t)(ch & 1)));   // the same answer in every thread
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
      // each warp: its 32 lanes (rows) of the 8 tiles; scatter the 5 outputs
#pragma unroll
      for (int d = 0; d < 2; ++d)
#pragma unroll
        for (int tl = 0; tl < 4; ++tl) {
          float o[8];
          tcg::ld8(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)((d * 4 + tl) * 16), o);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const int r = tl * 128 + 32 * warp + lane;
          if (r < 500) {
            const int rk = r % 4, rf = (r / 4) % 5, rcn = (r / 20) % 5, rl = r / 100;
            float* st = (d == 0 ? stX : stY) + rk * LS + rf * n1 + rcn;
#pragma unroll
            for (int nn = 0; nn < n1; ++nn) st[(d == 0 ? nn + n1 * rl : rl + n1 * nn) * LW] = o[nn];
          }
        }
    } else if (lane == 0) {
      atomicOr(A.status, 4);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (!ok) break;
    if (act) {
      const float* zX = stX + kk * LS + ab * LW;
      const float* zY = stY + kk * LS + ab * LW;
#pragma unroll
      for (int f = 0; f < kFields; ++f)
#pragma unroll
        for (int c = 0; c < n1; ++c) rz[f][c] += zX[f * n1 + c] + zY[f * n1 + c];
      if (kk > 0) {
        const float* pX = stX + (kk - 1) * LS + ab * LW;
        const float* pY = stY + (kk - 1) * LS + ab * LW;
        // z + (x + y), as the layer below forms its top-node value
#pragma unroll
        for (int f = 0; f < kFields; ++f)
          rz[f][0] += sT[(f * KL + kk - 1) * Nq + ab] + (pX[f * n1 + N] + pY[f * n1 + N]);
      } else if (ch > 0) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) rz[f][0] += sP[((ch - 1) & 1) * kFields * Nq + f * Nq + ab];
      }
      if (kk == KL - 1) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) sP[(ch & 1) * kFields * Nq + f * Nq + ab] = rz[f][N];
      }
      float* dst = rc + ((long long)((long long)col * Nq + ab) * kFields) * A.NZr + kz0;
      const bool top = (k == A.nz - 1);
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        float* df = dst + (long long)f * A.NZr;
        *reinterpret_cast<float4*>(df) = make_float4(rz[f][0], rz[f][1], rz[f][2], rz[f][3]);
        if (top) df[N] = rz[f][N];
      }
    }
    // the staging (operand) buffers are read: the next chunk may write them
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(kTcCols));
}

template <int MB>
static int launch_lines_tc(const VolArgs& A, cudaStream_t st) {
  const size_t sm = tc_smem_bytes();
  static DeviceOnce attr;
  int rc = device_once(attr, [&] {
    SEM_CUDA_TRY(cudaFuncSetAttribute(volume_lines_tc<MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return SEM_OK;
  });
  if (rc) return rc;
  ProfScope ps("volume_mixed", st);
  volume_lines_tc<MB><<<A.Ncol, kTcThreads, sm, st>>>(A);
  return SEM_OK;
}

template <int N, int KL, int MB>
static int launch_lines_smag(const VolArgs& A, cudaStream_t st) {
  const size_t sm = sizeof(float) * lines_smem_floats<N, KL>();
  static DeviceOnce attr;
  int rc = device_once(attr, [&] {
    SEM_CUDA_TRY(cudaFuncSetAttribute(volume_lines_smag<N, KL, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return SEM_OK;
  });
  if (rc) return rc;
  ProfScope ps("volume_mixed", st);
  volume_lines_smag<N, KL, MB><<<A.Ncol, KL * (N + 1) * (N + 1), sm, st>>>(A);
  return SEM_OK;
}

template <int N, int KL, int MB>
static int launch_lines(const VolArgs& A, cudaStream_t st) {
  const size_t sm = sizeof(float) * lines_smem_floats<N, KL>();
  static DeviceOnce attr;
  int rc = device_once(attr, [&] {
    SEM_CUDA_TRY(cudaFuncSetAttribute(volume_lines_mixed<N, KL, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SEM_CUDA_TRY(cudaFuncSetAttribute(volume_lines_warp<N, KL, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return SEM_OK;
  });
  if (rc) return rc;
  ProfScope ps("volume_mixed", st);
  if (A.metric32)
    volume_lines_warp<N, KL, MB><<<A.Ncol, KL * (N + 1) * (N + 1), sm, st>>>(A);
  else
    volume_lines_mixed<N, KL, MB><<<A.Ncol, KL * (N + 1) * (N + 1), sm, st>>>(A);
  return SEM_OK;
}

template <int N, int KL, int MB>
static int launch_lines_tma(const VolArgs& A, cudaStream_t st) {
  constexpr size_t sm = sizeof(float) * lines_tma_smem_floats<N, KL>();
  static DeviceOnce attr;
  int rc = device_once(attr, [&] {
    SEM_CUDA_TRY(cudaFuncSetAttribute(volume_lines_tma<N, KL, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return SEM_OK;
  });
  if (rc) return rc;
  ProfScope ps("volume_mixed", st);
  volume_lines_tma<N, KL, MB><<<A.Ncol, KL * (N + 1) * (N + 1), sm, st>>>(A);
  return SEM_OK;
}

template <int N, int KL, int MB>
static int launch_lines_nc(const VolArgs& A, cudaStream_t st) {
  constexpr size_t sm = sizeof(float) * nc_smem_floats<N, KL>();
  static DeviceOnce attr;
  int rc = device_once(attr, [&] {
    SEM_CUDA_TRY(cudaFuncSetAttribute(volume_lines_nc<N, KL, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    SEM_CUDA_TRY(cudaFuncSetAttribute(volume_lines_nc_warp<N, KL, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return SEM_OK;
  });
  if (rc) return rc;
  ProfScope ps("volume_mixed", st);
  if (A.metric32)
    volume_lines_nc_warp<N, KL, MB><<<A.Ncol, KL * (N + 1) * (N + 1), sm, st>>>(A);
  else
    volume_lines_nc<N, KL, MB><<<A.Ncol, KL * (N + 1) * (N + 1), sm, st>>>(A);
  return SEM_OK;
}

// Launch variants of the pencil kernel: layers per CTA (KL) and the minimum
// resident CTAs per SM the register allocation is sized for (MB).  The
// autotuner (sem_autotune) times them on a mesh and keeps the fastest.
struct PencilVariant {
  int N, KL, MB;
  int (*launch)(const VolArgs&, cudaStream_t);
  int kind;         // 0: z-pencil volume_pencil_mixed; 1: line-exchange volume_lines_mixed;
                    // 2: line exchange with the x, y contractions on tensor cores (volume_lines_tc);
                    // 4: line exchange with the state staged by bulk copies (volume_lines_tma);
                    // 5: line exchange for the paper's equation set (volume_lines_nc)
  int (*launch_smag)(const VolArgs&, cudaStream_t);   // with the stress added; null: none
};
static const PencilVariant kPencil[] = {
    {2, 16, 2, launch_pencil<2, 16, 2>},    {2, 16, 4, launch_lines<2, 16, 4>, 1},
    {2, 32, 2, launch_lines<2, 32, 2>, 1},
    {3, 16, 2, launch_pencil<3, 16, 2>},    {3, 16, 2, launch_lines<3, 16, 2>, 1},
    {3, 8, 4, launch_lines<3, 8, 4>, 1},    {3, 8, 6, launch_lines<3, 8, 6>, 1},
    {4, 8, 2, launch_pencil<4, 8, 2>},      {4, 16, 2, launch_pencil<4, 16, 2>},
    {4, 16, 2, launch_lines<4, 16, 2>, 1, launch_lines_smag<4, 16, 2>},
    {4, 8, 4, launch_lines<4, 8, 4>, 1, launch_lines_smag<4, 8, 4>},
    {4, 8, 2, launch_lines<4, 8, 2>, 1, launch_lines_smag<4, 8, 2>},
    {4, 4, 8, launch_lines<4, 4, 8>, 1, launch_lines_smag<4, 4, 8>},
    {4, kTcKL, 3, launch_lines_tc<3>, 2},
    {4, 8, 3, launch_lines<4, 8, 3>, 1, launch_lines_smag<4, 8, 3>},
    {4, 8, 3, launch_lines_tma<4, 8, 3>, 4},  {4, 8, 2, launch_lines_tma<4, 8, 2>, 4},
    {5, 8, 2, launch_pencil<5, 8, 2>},      {5, 8, 2, launch_lines<5, 8, 2>, 1},
    {5, 4, 4, launch_lines<5, 4, 4>, 1},
    {6, 4, 2, launch_pencil<6, 4, 2>},      {6, 8, 1, launch_lines<6, 8, 1>, 1},
    {6, 4, 2, launch_lines<6, 4, 2>, 1},
    // the paper's equation set
    {2, 16, 4, launch_lines_nc<2, 16, 4>, 5}, {3, 8, 4, launch_lines_nc<3, 8, 4>, 5},
    {4, 8, 3, launch_lines_nc<4, 8, 3>, 5},   {4, 8, 2, launch_lines_nc<4, 8, 2>, 5},
    {4, 6, 4, launch_lines_nc<4, 6, 4>, 5},   {4, 16, 2, launch_lines_nc<4, 16, 2>, 5},
    {5, 4, 3, launch_lines_nc<5, 4, 3>, 5},   {6, 4, 2, launch_lines_nc<6, 4, 2>, 5},
};
constexpr int kNumPencil = sizeof(kPencil) / sizeof(kPencil[0]);

// default choice before tuning: the line-exchange variant (kind 1, or 5 for
// the paper's set) with the most layers per CTA that fit nz (ties: more CTAs
// per SM), else the fewest layers
static int pencil_default(int N, int nz, int kind = 1) {
  int best = -1;
  for (int v = 0; v < kNumPencil; ++v) {
    if (kPencil[v].N != N || kPencil[v].kind != kind) continue;
    if (best < 0) { best = v; continue; }
    const PencilVariant& a = kPencil[v];
    const PencilVariant& b = kPencil[best];
    const int fa = a.KL <= nz, fb = b.KL <= nz;
    if (fa != fb ? fa > fb : (a.KL != b.KL ? (fa ? a.KL > b.KL : a.KL < b.KL) : a.MB > b.MB)) best = v;
  }
  return best;
}

static int launch_pencil_n(const VolArgs& A, int N, int nz, cudaStream_t st, int variant = -1,
                           bool smag = false) {
  if (variant < 0 || variant >= kNumPencil || kPencil[variant].N != N || kPencil[variant].kind == 5)
    variant = pencil_default(N, nz);
  // warped layers: the line-exchange kernels only
  if (A.metric32 && variant >= 0 && kPencil[variant].kind != 1) variant = pencil_default(N, nz);
  if (variant < 0) return fail(SEM_ERR_UNSUPPORTED, "order N not compiled");
  if (smag) return kPencil[variant].launch_smag(A, st);
  return kPencil[variant].launch(A, st);
}

// The paper's set, mixed form: the line-exchange rows (kind 5), box or
// warped layers.
static int launch_nc_n(const VolArgs& A, int N, int nz, cudaStream_t st, int variant = -1) {
  if (variant < 0 || variant >= kNumPencil || kPencil[variant].N != N || kPencil[variant].kind != 5)
    variant = pencil_default(N, nz, 5);
  if (variant < 0) return fail(SEM_ERR_UNSUPPORTED, "order N not compiled");
  return kPencil[variant].launch(A, st);
}

// Mixed conservative set on a line-exchange variant: the element kernel adds
// the absorbing layer itself (it holds every node's state), and, where the
// variant has a stress-adding form, the horizontal Smagorinsky stress too;
// the physics pass leaves out what it added (sponge_done, smag_done).
static int element_terms(Mesh& m, const sem_params& p, VolArgs& A, bool& sponge_done, bool& smag_done) {
  sponge_done = smag_done = false;
  // warped layers: the physics pass adds every term (at each node's height)
  if (p.eqset != SEM_EQ_CONSERVATIVE || m.warped()) return SEM_OK;
  int v = m.pencil_variant;
  if (v < 0 || v >= kNumPencil || kPencil[v].N != m.N) v = pencil_default(m.N, m.nz);
  if (v < 0 || (kPencil[v].kind != 1 && kPencil[v].kind != 4)) return SEM_OK;
  if (p.sponge_gamma > 0.0) {
    const int rc = ensure_sponge(m, p);
    if (rc) return rc;
    A.spg32 = m.dev->spg32;
    sponge_done = true;
  }
  if (p.smag_cs > 0.0 && kPencil[v].launch_smag) {
    for (int l = 0; l < kLev; ++l) {
      const double hx = m.hx(l), hy = m.hy(l);
      const double csd = p.smag_cs * (hx + hy) / (2.0 * m.N);
      A.smag[l][0] = (float)(csd * csd);
      A.smag[l][1] = (float)(2.0 / hx);
      A.smag[l][2] = (float)(2.0 / hy);
    }
    smag_done = true;
  }
  return SEM_OK;
}

static VolArgs make_vol_args(Mesh& m, const sem_params& p, const void* q, bool mixed, void* scratch) {
  DeviceTables& D = *m.dev;
  VolArgs A;
  A.q = q;
  A.rc = scratch ? scratch : D.scratch;
  A.hmap = D.hmap;
  A.hang_h = D.hang_h;
  A.hang_w = mixed ? (const void*)D.hang_w32 : (const void*)D.hang_w;
  A.col_level = D.col_level;
  A.ref = D.ref;
  A.ref32 = D.ref32;
  A.hzk = D.hzk;
  A.hzk32 = D.hzk32;
  A.ref4 = reinterpret_cast<const float4*>(D.ref32 + (size_t)m.NZ * kRef);
  A.spg32 = nullptr;
  A.status = D.status;
  const bool w = m.warped();
  A.metric = w ? D.metric : nullptr;
  A.metric32 = w ? D.metric32 : nullptr;
  A.refG = D.refG;
  A.refH = D.refH;
  A.refG32 = D.refG32;
  A.refH32 = D.refH32;
  A.ref4G = reinterpret_cast<const float4*>(D.ref4G);
  A.ref4H = reinterpret_cast<const float4*>(D.ref4H);
  A.Ncol = (int)m.Ncol();
  A.nz = m.nz;
  A.NZ = m.NZ;
  A.NZr = m.NZr();
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
  {
    double cb = 1.0;
    for (int k = 1; k <= 7; ++k) {
      cb *= (A.gamma - (k - 1)) / k;
      A.bin[k - 1] = (float)cb;
    }
    A.bin[7] = 0.f;
  }
  for (int l = 0; l < kLev; ++l) {
    const double hx = m.hx(l), hy = m.hy(l), hz = 1.0;   // per unit layer thickness
    const double g[8] = {hx, hy, hz, hx * hy * hz * 0.125, hy * hz * 0.25, hx * hz * 0.25,
                         hx * hy * 0.25, 0.0};
    for (int k = 0; k < 8; ++k) {
      A.geo[l][k] = g[k];
      A.geof[l][k] = (float)g[k];
    }
  }
  return A;
}

static int grid_cap(long long work, int per_sm = 8) {
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (work + 255) / 256;
  long long cap = (long long)nsm * per_sm;
  return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

// ---------------------------------------------------------------------------
// Mixed form, increment form of the SSP-RK3 step (sem_step_mixed).
//
// With d_s = q_s - q_n the three stages are
//   d_1 = dt L(q_n),  d_2 = 1/4 d_1 + 1/4 dt L(q_1),  d_3 = 2/3 d_2 + 2/3 dt L(q_2),
//   q_{n+1} = q_n + d_3.
// The increments are float32; the state q_n is float64 and receives one
// float64 addition per value and step.  Stages 0 and 1 write d and the
// float32 mirror q_n32 + d of the next stage state; stage 2 writes q_{n+1} and
// its mirror.
struct IncArgs {
  const float* rc;
  const int* qt_ptr;
  const int* qt_src;
  const float* qt_w;
  const int4* qt_rec_src;
  const float4* qt_rec_w;
  const float* Minv_h;
  const float* Minv_z;
  const float* Minv_g;  // warped layers: inverse lumped mass per node, else null
  const float* q32;   // mirror of q_n
  float* d;           // increment, updated in place
  float* qs32;        // stages 0, 1: mirror of the next stage state
  double* q;          // stage 2: float64 state, updated in place
  float* q32_out;     // stage 2: mirror of q_{n+1}
  float cdt, bcoef;
  int NG, NZ, NZr;
  int* status;
};

template <int STAGE, bool WARP = false>
__device__ __forceinline__ void inc_body(const IncArgs& A, const int gidx, int& bad) {
  const int h = (int)((unsigned)gidx / (unsigned)A.NZ);
  const int kz = gidx - h * A.NZ;
  // Stages 1 and 2 update d or q in place: their values are loaded before
  // the gather and before any store, so that the loads are not ordered after
  // the stores of the other fields and their latency overlaps the gather's.
  float dprev[kFields], q32v[kFields];
  double qv[kFields];
#pragma unroll
  for (int fl = 0; fl < kFields; ++fl) {
    const long long o = (long long)fl * A.NG + gidx;
    if (STAGE > 0) dprev[fl] = A.d[o];
    if (STAGE == 1) q32v[fl] = __ldg(A.q32 + o);
    if (STAGE == 2) qv[fl] = A.q[o];
  }
  // warped layers: the lumped mass per node (it does not factorise)
  const float s = WARP ? A.cdt * __ldg(A.Minv_g + gidx) : A.cdt * (__ldg(A.Minv_h + h) * __ldg(A.Minv_z + kz));
  const bool lid = (kz == 0) || (kz == A.NZ - 1);
  float acc[kFields] = {0, 0, 0, 0, 0};
  // Q_h^T gather, in the order of the CSR lists: from the compact record
  // (sources and weights known after one load each), else from the lists
  const int4 s4 = __ldg(A.qt_rec_src + h);
  if (s4.x >= 0) {
    const float4 w4 = __ldg(A.qt_rec_w + h);
    const int src[4] = {s4.x, s4.y, s4.z, s4.w};
    const float ww[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (src[e] < 0) break;
      const float* p = A.rc + (long long)src[e] * kFields * A.NZr + kz;
#pragma unroll
      for (int fl = 0; fl < kFields; ++fl) acc[fl] = fmaf(ww[e], __ldg(p + fl * A.NZr), acc[fl]);
    }
  } else {
    const int beg = __ldg(A.qt_ptr + h), end = __ldg(A.qt_ptr + h + 1);
    for (int e = beg; e < end; ++e) {
      const float w = __ldg(A.qt_w + e);
      const float* p = A.rc + (long long)__ldg(A.qt_src + e) * kFields * A.NZr + kz;
#pragma unroll
      for (int fl = 0; fl < kFields; ++fl) acc[fl] = fmaf(w, __ldg(p + fl * A.NZr), acc[fl]);
    }
  }
#pragma unroll
  for (int fl = 0; fl < kFields; ++fl) {
    const long long o = (long long)fl * A.NG + gidx;
    const float inc = (fl == 3 && lid) ? 0.f : acc[fl] * s;
    const float dn = (STAGE == 0) ? inc : fmaf(A.bcoef, dprev[fl], inc);
    if (STAGE < 2) {
      A.d[o] = dn;
      A.qs32[o] = (STAGE == 0 ? __ldg(A.q32 + o) : q32v[fl]) + dn;
    } else {
      const double qn = qv[fl] + f2d_bits(dn);
      A.q[o] = qn;
      A.q32_out[o] = d2f_bits(qn);
      bad |= nonfinite_bits(qn);
    }
  }
}

template <int STAGE, bool WARP = false>
__global__ void __launch_bounds__(256) dss_inc(const IncArgs A) {
  int bad = 0;
  for (int gidx = blockIdx.x * blockDim.x + threadIdx.x; gidx < A.NG; gidx += gridDim.x * blockDim.x)
    inc_body<STAGE, WARP>(A, gidx, bad);
  if (STAGE == 2 && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(A.status, 1);
}

int launch_step_mixed(Mesh& m, const sem_params& p, double* q, float* q32, float* work32, double dt,
                      cudaStream_t st) {
  int rc = upload_basis_constants();
  if (rc) return rc;
  DeviceTables& D = *m.dev;
  float* d = work32;
  float* qs32 = work32 + (size_t)kFields * m.NG;
  for (int stage = 0; stage < 3; ++stage) {
    // element work on the stage state's mirror
    VolArgs A = make_vol_args(m, p, stage == 0 ? (const void*)q32 : (const void*)qs32, true, nullptr);
    bool sponge_done = false, smag_done = false;
    if ((rc = element_terms(m, p, A, sponge_done, smag_done))) return rc;
    if (p.eqset == SEM_EQ_CONSERVATIVE) {
      if ((rc = launch_pencil_n(A, m.N, m.nz, st, m.pencil_variant, smag_done))) return rc;
    } else {
      // the paper's set (same residual layout)
      if ((rc = launch_nc_n(A, m.N, m.nz, st, m.nc_variant))) return rc;
    }
    SEM_CUDA_TRY(cudaGetLastError());
    if (physics_on(p) &&
        (rc = launch_physics(m, p, A.q, true, nullptr, p.time + (stage == 0 ? 0.0 : (stage == 1 ? dt : 0.5 * dt)),
                             st, sponge_done, smag_done)))
      return rc;
    IncArgs B;
    B.rc = (const float*)D.scratch;
    B.qt_ptr = D.qt_ptr;
    B.qt_src = D.qt_src;
    B.qt_w = D.qt_w32;
    B.qt_rec_src = reinterpret_cast<const int4*>(D.qt_rec_src);
    B.qt_rec_w = reinterpret_cast<const float4*>(D.qt_rec_w);
    B.Minv_h = D.Minv_h32;
    B.Minv_z = D.Minv_z32;
    B.Minv_g = m.warped() ? D.Minv_g32 : nullptr;
    B.q32 = q32;
    B.d = d;
    B.qs32 = qs32;
    B.q = q;
    B.q32_out = q32;
    const double cs[3] = {1.0, 0.25, 2.0 / 3.0};
    B.cdt = (float)(cs[stage] * dt);
    B.bcoef = (float)cs[stage];
    B.NG = (int)m.NG;
    B.NZ = m.NZ;
    B.NZr = m.NZr();
    B.status = D.status;
    ProfScope ps("dss_inc_mixed", st);
    const int blocks = grid_cap(m.NG, 64);
    if (B.Minv_g) {
      if (stage == 0) dss_inc<0, true><<<blocks, 256, 0, st>>>(B);
      else if (stage == 1) dss_inc<1, true><<<blocks, 256, 0, st>>>(B);
      else dss_inc<2, true><<<blocks, 256, 0, st>>>(B);
    } else {
      if (stage == 0) dss_inc<0><<<blocks, 256, 0, st>>>(B);
      else if (stage == 1) dss_inc<1><<<blocks, 256, 0, st>>>(B);
      else dss_inc<2><<<blocks, 256, 0, st>>>(B);
    }
    SEM_CUDA_TRY(cudaGetLastError());
  }
  return SEM_OK;
}

// Rows of the variant table for a mesh and equation set: the conservative
// set's kernels (kinds 0, 1, 2, 4; warped layers: kind 1 only) or the paper's
// set's (kind 5).
static bool tune_row(const Mesh& m, int eqset, int v) {
  if (kPencil[v].N != m.N) return false;
  if (eqset != SEM_EQ_CONSERVATIVE) return kPencil[v].kind == 5;
  if (kPencil[v].kind == 5) return false;
  return !m.warped() || kPencil[v].kind == 1;
}

// Autotuner: time every element-kernel variant compiled for the mesh's order
// and the parameters' equation set on the given state (float32 mirror) and
// keep the fastest for this mesh and set.
int autotune_pencil(Mesh& m, const sem_params& p, const float* q32, int reps, sem_tune_out* out,
                    cudaStream_t st) {
  int rc = upload_basis_constants();
  if (rc) return rc;
  const int eqset = p.eqset;
  VolArgs A = make_vol_args(m, p, q32, true, nullptr);
  cudaEvent_t e0, e1;
  SEM_CUDA_TRY(cudaEventCreate(&e0));
  SEM_CUDA_TRY(cudaEventCreate(&e1));
  int best = -1;
  float best_ms = 0.f;
  out->n_variants = 0;
  for (int v = 0; v < kNumPencil && out->n_variants < SEM_TUNE_MAX; ++v) {
    if (!tune_row(m, eqset, v)) continue;
    for (int w = 0; w < 2; ++w) kPencil[v].launch(A, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) kPencil[v].launch(A, st);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(SEM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    const int k = out->n_variants++;
    out->layers_per_cta[k] = kPencil[v].KL;
    out->min_ctas_per_sm[k] = kPencil[v].MB;
    out->kind[k] = kPencil[v].kind;
    out->ms[k] = ms;
    if (best < 0 || ms < best_ms) {
      best = v;
      best_ms = ms;
      out->chosen = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) return fail(SEM_ERR_UNSUPPORTED, "no variant for this order");
  (eqset == SEM_EQ_CONSERVATIVE ? m.pencil_variant : m.nc_variant) = best;
  return SEM_OK;
}

// Row `row` of the autotuner's table for the mesh's order and the equation
// set (-1: default).
int select_pencil(Mesh& m, int eqset, int row) {
  int& sel = eqset == SEM_EQ_CONSERVATIVE ? m.pencil_variant : m.nc_variant;
  if (row == -1) {
    sel = -1;
    return SEM_OK;
  }
  int k = 0;
  for (int v = 0; v < kNumPencil && k < SEM_TUNE_MAX; ++v) {
    if (!tune_row(m, eqset, v)) continue;   // the rows sem_autotune lists
    if (k == row) {
      sel = v;
      return SEM_OK;
    }
    ++k;
  }
  return fail(SEM_ERR_ARG, "autotune_select: row outside the variant table of this order");
}

// ---------------------------------------------------------------------------
// Batched mixed-form steps over many independent meshes (sem_batch_*).
//
// One persistent element kernel per stage: CTAs of kBatchThreads threads pull
// (instance, column) tiles, costliest first, from an atomic counter and run
// the pencil body for the tile's order N (layers per CTA fixed per N so that
// KL (N+1)^2 <= kBatchThreads).  One gather/increment kernel per stage runs
// over the concatenated global nodes of all instances.  With graphs enabled
// the nine launches of a step (3 x counter reset, element, increment) are
// captured once and replayed with one cudaGraphLaunch per step.
// Layers per CTA for order N in a CTA of BT threads: as many as fit, at most 16.
__host__ __device__ constexpr int batch_kl(int N, int BT) {
  return (BT / ((N + 1) * (N + 1))) < 16 ? (BT / ((N + 1) * (N + 1))) : 16;
}

template <int BT, int MB>
__global__ void __launch_bounds__(BT, MB)
volume_batch_mixed(const VolArgs* __restrict__ insts, const int* __restrict__ inst_N,
                   const int2* __restrict__ tiles, int ntiles, int* counter) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_tile;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) break;
    const int2 tl = tiles[tile];
    const VolArgs& A = insts[tl.x];
    switch (inst_N[tl.x]) {
      case 2: lines_body<2, batch_kl(2, BT)>(A, tl.y, smem, threadIdx.x); break;
      case 3: lines_body<3, batch_kl(3, BT)>(A, tl.y, smem, threadIdx.x); break;
      case 4: lines_body<4, batch_kl(4, BT)>(A, tl.y, smem, threadIdx.x); break;
      case 5: lines_body<5, batch_kl(5, BT)>(A, tl.y, smem, threadIdx.x); break;
      case 6: lines_body<6, batch_kl(6, BT)>(A, tl.y, smem, threadIdx.x); break;
      default: break;
    }
  }
}

// The same queue with the paper's equation set (the line-exchange body of
// volume_lines_nc).
template <int BT, int MB>
__global__ void __launch_bounds__(BT, MB)
volume_batch_nc(const VolArgs* __restrict__ insts, const int* __restrict__ inst_N,
                const int2* __restrict__ tiles, int ntiles, int* counter) {
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_tile;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) break;
    const int2 tl = tiles[tile];
    const VolArgs& A = insts[tl.x];
    switch (inst_N[tl.x]) {
      case 2: lines_nc_body<2, batch_kl(2, BT)>(A, tl.y, smem, threadIdx.x); break;
      case 3: lines_nc_body<3, batch_kl(3, BT)>(A, tl.y, smem, threadIdx.x); break;
      case 4: lines_nc_body<4, batch_kl(4, BT)>(A, tl.y, smem, threadIdx.x); break;
      case 5: lines_nc_body<5, batch_kl(5, BT)>(A, tl.y, smem, threadIdx.x); break;
      case 6: lines_nc_body<6, batch_kl(6, BT)>(A, tl.y, smem, threadIdx.x); break;
      default: break;
    }
  }
}

template <int BT>
static size_t batch_smem() {
  size_t m = lines_smem_floats<2, batch_kl(2, BT)>();
  m = std::max(m, (size_t)lines_smem_floats<3, batch_kl(3, BT)>());
  m = std::max(m, (size_t)lines_smem_floats<4, batch_kl(4, BT)>());
  m = std::max(m, (size_t)lines_smem_floats<5, batch_kl(5, BT)>());
  m = std::max(m, (size_t)lines_smem_floats<6, batch_kl(6, BT)>());
  return m * sizeof(float);
}
template <int BT>
static size_t batch_smem_nc() {
  size_t m = nc_smem_floats<2, batch_kl(2, BT)>();
  m = std::max(m, (size_t)nc_smem_floats<3, batch_kl(3, BT)>());
  m = std::max(m, (size_t)nc_smem_floats<4, batch_kl(4, BT)>());
  m = std::max(m, (size_t)nc_smem_floats<5, batch_kl(5, BT)>());
  m = std::max(m, (size_t)nc_smem_floats<6, batch_kl(6, BT)>());
  return m * sizeof(float);
}

// Launch configurations of the batched element kernel (threads per CTA and
// the CTAs per SM its registers are sized for), for the conservative set and
// for the paper's set; chosen by timing at set-up, per set.
struct BatchVariant {
  int BT, MB;
  void (*kernel)(const VolArgs*, const int*, const int2*, int, int*);
  size_t (*smem)();
  void (*kernel_nc)(const VolArgs*, const int*, const int2*, int, int*);
  size_t (*smem_nc)();
};
static const BatchVariant kBatch[] = {
    {400, 1, volume_batch_mixed<400, 1>, batch_smem<400>, volume_batch_nc<400, 1>, batch_smem_nc<400>},
    {200, 2, volume_batch_mixed<200, 2>, batch_smem<200>, volume_batch_nc<200, 2>, batch_smem_nc<200>},
    {200, 3, volume_batch_mixed<200, 3>, batch_smem<200>, volume_batch_nc<200, 3>, batch_smem_nc<200>},
    {256, 2, volume_batch_mixed<256, 2>, batch_smem<256>, volume_batch_nc<256, 2>, batch_smem_nc<256>},
};
constexpr int kNumBatch = sizeof(kBatch) / sizeof(kBatch[0]);

template <int STAGE>
__global__ void __launch_bounds__(256)
dss_inc_batch(const IncArgs* __restrict__ insts, const int* __restrict__ off, int ninst, int total,
              int* status) {
  int bad = 0;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total; g += gridDim.x * blockDim.x) {
    int lo = 0, hi = ninst - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(off + mid) <= g) lo = mid; else hi = mid - 1;
    }
    inc_body<STAGE>(insts[lo], g - __ldg(off + lo), bad);
  }
  if (STAGE == 2 && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, 1);
}


struct BatchImpl {
  std::vector<Mesh*> meshes;
  int total_nodes = 0;
  VolArgs* d_vol = nullptr;   // [2][n]: stage 0 (reads q32), stages 1-2 (read the stage mirror)
  IncArgs* d_inc = nullptr;   // [3][n]
  int* d_N = nullptr;
  int2* d_tiles = nullptr;
  int ntiles = 0;
  int* d_off = nullptr;
  int* d_counter = nullptr;   // [3]
  int* d_status = nullptr;
  cudaStream_t cap = nullptr;
  // branch streams: instances with their own launches whose column residuals
  // are small enough (kBranchBytes) run side by side (each keeps its stage
  // order), forked from and joined to the step's stream; larger ones run one
  // after another on it, so that their residuals stay in L2 between the
  // element and the gather kernel
  std::vector<char> branch;
  std::vector<cudaStream_t> br;
  std::vector<cudaEvent_t> br_done;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<const void*> key;  // arrays and dt the device tables were built for
  std::vector<double> key_dt;
  double key_par[8] = {0};
  int nsm = 152;
  std::vector<IncArgs> h_inc;  // host copy of the increment-kernel arguments [3][n]
  int nsmall = 0;
  int eq = SEM_EQ_CONSERVATIVE;  // equation set of the current tables and graph
  int variant[2] = {-1, -1};     // batched element-kernel configuration (kBatch), per set
  std::vector<char> big;     // instances launched with their own tuned kernel
  std::vector<VolArgs> h_vol;  // host copy of the element-kernel arguments [2][n]
  float variant_ms[2][kNumBatch] = {{0}};
};

static void batch_free(BatchImpl* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaStream_t x : b->br) cudaStreamDestroy(x);
  for (cudaEvent_t x : b->br_done) cudaEventDestroy(x);
  if (b->fork) cudaEventDestroy(b->fork);
  void* ptrs[] = {b->d_vol, b->d_inc, b->d_N, b->d_tiles, b->d_off, b->d_counter, b->d_status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

int batch_create(Mesh* const* meshes, int n, void** out) {
  int rc = upload_basis_constants();
  if (rc) return rc;
  BatchImpl* b = new BatchImpl();
  b->meshes.assign(meshes, meshes + n);
  long long tot = 0;
  std::vector<int> Ns(n), off(n);
  std::vector<std::pair<long long, int2>> tiles;
  int dev0 = 0, nsm0 = 152;
  cudaGetDevice(&dev0);
  cudaDeviceGetAttribute(&nsm0, cudaDevAttrMultiProcessorCount, dev0);
  b->big.assign(n, 0);
  for (int k = 0; k < n; ++k) {
    Mesh& m = *meshes[k];
    if (m.warped()) {
      batch_free(b);
      delete b;
      return fail(SEM_ERR_UNSUPPORTED, "batched steps of warped meshes are not built");
    }
    if ((rc = ensure_device(m))) { batch_free(b); delete b; return rc; }
    Ns[k] = m.N;
    // meshes with enough columns to fill the GPU keep their own tuned
    // launches; the rest share the persistent column queue and one
    // concatenated gather/increment launch
    if (m.Ncol() >= 2LL * nsm0) {
      b->big[k] = 1;
      off[k] = (int)tot;
      continue;
    }
    off[k] = (int)tot;
    tot += m.NG;
    const long long cost = (long long)(m.N + 1) * (m.N + 1) * (m.N + 1) * m.nz;
    for (int c = 0; c < (int)m.Ncol(); ++c) tiles.push_back({cost, make_int2(k, c)});
  }
  for (int k = 0; k < n; ++k)
    if (meshes[k]->NG * kFields >= (1ll << 31)) {
      delete b;
      return fail(SEM_ERR_ARG, "mesh too large for 32-bit indexing");
    }
  b->total_nodes = (int)tot;
  std::stable_sort(tiles.begin(), tiles.end(),
                   [](const std::pair<long long, int2>& x, const std::pair<long long, int2>& y) { return x.first > y.first; });
  std::vector<int2> tl(tiles.size());
  for (size_t t = 0; t < tiles.size(); ++t) tl[t] = tiles[t].second;
  b->ntiles = (int)tl.size();
  cudaError_t e = cudaMalloc((void**)&b->d_vol, sizeof(VolArgs) * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_inc, sizeof(IncArgs) * 3 * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_N, sizeof(int) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_tiles, sizeof(int2) * (tl.size() ? tl.size() : 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_off, sizeof(int) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_counter, sizeof(int) * 3);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_N, Ns.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tl.empty())
    e = cudaMemcpy(b->d_tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice);
  std::vector<int> soff;
  for (int k = 0; k < n; ++k)
    if (!b->big[k]) soff.push_back(off[k]);
  b->nsmall = (int)soff.size();
  if (e == cudaSuccess && !soff.empty())
    e = cudaMemcpy(b->d_off, soff.data(), sizeof(int) * soff.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  {
    constexpr long long kBranchBytes = 16ll << 20;
    b->branch.assign(n, 0);
    int nbig = 0;
    for (int k = 0; k < n; ++k) {
      const Mesh& m = *meshes[k];
      b->branch[k] = b->big[k] && m.Ncol() * m.Nq * kFields * m.NZr() * (long long)sizeof(float) <= kBranchBytes;
      nbig += b->branch[k];
    }
    const int nbr = std::min(nbig, 4);
    if (nbr > 0 && e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int i = 0; i < nbr && e == cudaSuccess; ++i) {
      cudaStream_t x = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->br.push_back(x);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) b->br_done.push_back(ev);
    }
  }
  for (int v = 0; v < kNumBatch && e == cudaSuccess; ++v) {
    e = cudaFuncSetAttribute(kBatch[v].kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kBatch[v].smem());
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kBatch[v].kernel_nc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kBatch[v].smem_nc());
  }
  if (e != cudaSuccess) {
    batch_free(b);
    delete b;
    return fail(SEM_ERR_CUDA, std::string("batch set-up: ") + cudaGetErrorString(e));
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  *out = b;
  return SEM_OK;
}

void batch_destroy(void* h) {
  BatchImpl* b = (BatchImpl*)h;
  if (!b) return;
  batch_free(b);
  delete b;
}

static void batch_volume(BatchImpl* b, int v, const VolArgs* vol, int* counter, cudaStream_t st) {
  const BatchVariant& V = kBatch[v];
  const int vgrid = std::min(b->ntiles, b->nsm * V.MB);
  if (b->eq == SEM_EQ_CONSERVATIVE)
    V.kernel<<<vgrid, V.BT, V.smem(), st>>>(vol, b->d_N, b->d_tiles, b->ntiles, counter);
  else
    V.kernel_nc<<<vgrid, V.BT, V.smem_nc(), st>>>(vol, b->d_N, b->d_tiles, b->ntiles, counter);
}

// time every configuration of the element kernel on stage-0 inputs (side
// effect: the meshes' residual scratch) and keep the fastest
static int batch_tune(BatchImpl* b, cudaStream_t st) {
  cudaEvent_t e0, e1;
  SEM_CUDA_TRY(cudaEventCreate(&e0));
  SEM_CUDA_TRY(cudaEventCreate(&e1));
  float best = 0.f;
  for (int v = 0; v < kNumBatch; ++v) {
    cudaMemsetAsync(b->d_counter, 0, sizeof(int), st);
    batch_volume(b, v, b->d_vol, b->d_counter, st);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) {
      cudaMemsetAsync(b->d_counter, 0, sizeof(int), st);
      batch_volume(b, v, b->d_vol, b->d_counter, st);
    }
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(SEM_ERR_CUDA, std::string("batch tuning: ") + cudaGetErrorString(e));
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const int q = b->eq == SEM_EQ_CONSERVATIVE ? 0 : 1;
    b->variant_ms[q][v] = ms / 3.f;
    if (b->variant[q] < 0 || b->variant_ms[q][v] < best) {
      best = b->variant_ms[q][v];
      b->variant[q] = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return SEM_OK;
}

static void batch_enqueue(BatchImpl* b, cudaStream_t st) {
  const int n = (int)b->meshes.size();
  const int igrid = std::max(1, std::min((b->total_nodes + 255) / 256, b->nsm * 64));
  const int nbr = (int)b->br.size();
  if (nbr > 0) {
    cudaEventRecord(b->fork, st);
    for (int i = 0; i < nbr; ++i) cudaStreamWaitEvent(b->br[i], b->fork, 0);
  }
  // instances with their own launches: all three stages, on a branch stream
  // or on the step's stream
  int bi = 0;
  for (int k = 0; k < n; ++k) {
    if (!b->big[k]) continue;
    cudaStream_t s2 = b->branch[k] ? b->br[bi++ % nbr] : st;
    Mesh& m = *b->meshes[k];
    for (int stage = 0; stage < 3; ++stage) {
      if (b->eq == SEM_EQ_CONSERVATIVE)
        launch_pencil_n(b->h_vol[(stage == 0 ? 0 : n) + k], m.N, m.nz, s2, m.pencil_variant);
      else
        launch_nc_n(b->h_vol[(stage == 0 ? 0 : n) + k], m.N, m.nz, s2, m.nc_variant);
      const IncArgs& B = b->h_inc[stage * n + k];
      const int blocks = grid_cap(B.NG, 64);   // as in the single-mesh step
      if (stage == 0) dss_inc<0><<<blocks, 256, 0, s2>>>(B);
      else if (stage == 1) dss_inc<1><<<blocks, 256, 0, s2>>>(B);
      else dss_inc<2><<<blocks, 256, 0, s2>>>(B);
    }
  }
  // the others: persistent column queue and concatenated increment kernel
  for (int stage = 0; stage < 3; ++stage) {
    if (b->ntiles > 0) {
      cudaMemsetAsync(b->d_counter + stage, 0, sizeof(int), st);
      batch_volume(b, b->variant[b->eq == SEM_EQ_CONSERVATIVE ? 0 : 1], b->d_vol + (stage == 0 ? 0 : n),
                   b->d_counter + stage, st);
    }
    const int ns = b->nsmall;
    if (ns > 0 && b->total_nodes > 0) {
      if (stage == 0) dss_inc_batch<0><<<igrid, 256, 0, st>>>(b->d_inc, b->d_off, ns, b->total_nodes, b->d_status);
      else if (stage == 1) dss_inc_batch<1><<<igrid, 256, 0, st>>>(b->d_inc + ns, b->d_off, ns, b->total_nodes, b->d_status);
      else dss_inc_batch<2><<<igrid, 256, 0, st>>>(b->d_inc + 2 * ns, b->d_off, ns, b->total_nodes, b->d_status);
    }
  }
  for (int i = 0; i < nbr; ++i) {
    cudaEventRecord(b->br_done[i], b->br[i]);
    cudaStreamWaitEvent(st, b->br_done[i], 0);
  }
}

int batch_step_mixed(void* h, const sem_params& p, double* const* q, float* const* q32,
                     float* const* work32, const double* dt, int use_graph, cudaStream_t st) {
  BatchImpl* b = (BatchImpl*)h;
  if (physics_on(p))
    return fail(SEM_ERR_UNSUPPORTED, "batched step: no Smagorinsky stress or absorbing layer (smag_cs, sponge_gamma)");
  const int n = (int)b->meshes.size();
  std::vector<const void*> key;
  for (int k = 0; k < n; ++k) {
    key.push_back(q[k]);
    key.push_back(q32[k]);
    key.push_back(work32[k]);
  }
  std::vector<double> kdt(dt, dt + n);
  const double par[8] = {p.g, p.f, p.R_d, p.c_p, p.p00, p.theta_s, p.N_bv, (double)p.eqset};
  const bool same = key == b->key && kdt == b->key_dt && std::memcmp(par, b->key_par, sizeof(par)) == 0;
  if (!same) {
    b->eq = p.eqset;
    std::vector<VolArgs> vol(2 * n);
    std::vector<IncArgs> inc(3 * n);
    for (int k = 0; k < n; ++k) {
      Mesh& m = *b->meshes[k];
      int rc = ensure_reference(m, p);
      if (rc) return rc;
      float* qs32 = work32[k] + (size_t)kFields * m.NG;
      vol[k] = make_vol_args(m, p, q32[k], true, nullptr);
      vol[n + k] = make_vol_args(m, p, qs32, true, nullptr);
      DeviceTables& D = *m.dev;
      const double cs[3] = {1.0, 0.25, 2.0 / 3.0};
      for (int s = 0; s < 3; ++s) {
        IncArgs& B = inc[s * n + k];
        B.rc = (const float*)D.scratch;
        B.qt_ptr = D.qt_ptr;
        B.qt_src = D.qt_src;
        B.qt_w = D.qt_w32;
        B.qt_rec_src = reinterpret_cast<const int4*>(D.qt_rec_src);
        B.qt_rec_w = reinterpret_cast<const float4*>(D.qt_rec_w);
        B.Minv_h = D.Minv_h32;
        B.Minv_z = D.Minv_z32;
        B.Minv_g = nullptr;   // batched meshes are box meshes
        B.q32 = q32[k];
        B.d = work32[k];
        B.qs32 = qs32;
        B.q = q[k];
        B.q32_out = q32[k];
        B.cdt = (float)(cs[s] * dt[k]);
        B.bcoef = (float)cs[s];
        B.NG = (int)m.NG;
        B.NZ = m.NZ;
        B.NZr = m.NZr();
        B.status = b->d_status;
      }
    }
    // the previous graph may still read the old tables
    SEM_CUDA_TRY(cudaStreamSynchronize(st));
    SEM_CUDA_TRY(cudaMemcpy(b->d_vol, vol.data(), sizeof(VolArgs) * vol.size(), cudaMemcpyHostToDevice));
    // device copy: small instances only, [3][nsmall]
    std::vector<IncArgs> sinc;
    for (int s2 = 0; s2 < 3; ++s2)
      for (int k = 0; k < n; ++k)
        if (!b->big[k]) sinc.push_back(inc[s2 * n + k]);
    if (!sinc.empty())
      SEM_CUDA_TRY(cudaMemcpy(b->d_inc, sinc.data(), sizeof(IncArgs) * sinc.size(), cudaMemcpyHostToDevice));
    b->h_inc = inc;
    b->h_vol = vol;
    for (int k = 0; k < n; ++k)
      if (b->big[k] && (p.eqset == SEM_EQ_CONSERVATIVE ? b->meshes[k]->pencil_variant
                                                       : b->meshes[k]->nc_variant) < 0) {
        sem_tune_out tout;
        std::memset(&tout, 0, sizeof(tout));
        int rc = autotune_pencil(*b->meshes[k], p, q32[k], 3, &tout, st);
        if (rc) return rc;
      }
    b->key = key;
    b->key_dt = kdt;
    std::memcpy(b->key_par, par, sizeof(par));
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (b->graph) {
      cudaGraphDestroy(b->graph);
      b->graph = nullptr;
    }
    if (b->variant[b->eq == SEM_EQ_CONSERVATIVE ? 0 : 1] < 0 && b->ntiles > 0) {
      int rc = batch_tune(b, st);
      if (rc) return rc;
    }
  }
  if (!use_graph) {
    ProfScope ps("batch_step_mixed", st);
    batch_enqueue(b, st);
    SEM_CUDA_TRY(cudaGetLastError());
    return SEM_OK;
  }
  if (!b->exec) {
    SEM_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    batch_enqueue(b, b->cap);
    cudaError_t e = cudaStreamEndCapture(b->cap, &b->graph);
    if (e != cudaSuccess) return fail(SEM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    SEM_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  ProfScope ps("batch_step_mixed_graph", st);
  SEM_CUDA_TRY(cudaGraphLaunch(b->exec, st));
  return SEM_OK;
}

int batch_tuning(void* h, int* variant, int* bt, int* mb, float* ms, int max) {
  BatchImpl* b = (BatchImpl*)h;
  const int q = b->eq == SEM_EQ_CONSERVATIVE ? 0 : 1;
  *variant = b->variant[q];
  for (int v = 0; v < kNumBatch && v < max; ++v) {
    bt[v] = kBatch[v].BT;
    mb[v] = kBatch[v].MB;
    ms[v] = b->variant_ms[q][v];
  }
  return kNumBatch < max ? kNumBatch : max;
}

int batch_status(void* h, int* status, cudaStream_t st) {
  BatchImpl* b = (BatchImpl*)h;
  int v = 0;
  SEM_CUDA_TRY(cudaMemcpyAsync(&v, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SEM_CUDA_TRY(cudaMemsetAsync(b->d_status, 0, sizeof(int), st));
  SEM_CUDA_TRY(cudaStreamSynchronize(st));
  *status = v ? SEM_ERR_NUMERIC : SEM_OK;
  return SEM_OK;
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
  if (m.NG * kFields >= (1ll << 31)) return fail(SEM_ERR_ARG, "mesh too large for 32-bit node indexing");
  DeviceTables& D = *m.dev;
  const bool mixed = p.precision == SEM_PREC_MIXED;
  const float* qs32 = s.qs32;
  if (mixed && !qs32) {
    // no caller mirror: make one in the mesh scratch
    if ((rc = launch_mirror(s.qs, D.mirror, (long long)kFields * m.NG, st))) return rc;
    qs32 = D.mirror;
  }
  VolArgs A = make_vol_args(m, p, mixed ? (const void*)qs32 : (const void*)s.qs, mixed, s.scratch);
  const int eq = p.eqset;
  bool sponge_done = false, smag_done = false;
  if (mixed && eq == SEM_EQ_CONSERVATIVE) {
    if ((rc = element_terms(m, p, A, sponge_done, smag_done))) return rc;
    if ((rc = launch_pencil_n(A, m.N, m.nz, st, m.pencil_variant, smag_done))) return rc;
  } else if (mixed) {
    if ((rc = launch_nc_n(A, m.N, m.nz, st, m.nc_variant))) return rc;
  } else switch (m.N) {
    case 2: launch_volume_fp64<2>(A, eq, st); break;
    case 3: launch_volume_fp64<3>(A, eq, st); break;
    case 4: launch_volume_fp64<4>(A, eq, st); break;
    case 5: launch_volume_fp64<5>(A, eq, st); break;
    case 6: launch_volume_fp64<6>(A, eq, st); break;
    default: return fail(SEM_ERR_UNSUPPORTED, "order N not compiled");
  }
  SEM_CUDA_TRY(cudaGetLastError());
  if (physics_on(p) &&
      (rc = launch_physics(m, p, mixed ? (const void*)qs32 : (const void*)s.qs, mixed, s.scratch, s.time, st,
                           sponge_done, smag_done)))
    return rc;
  DssArgs B;
  B.rc = s.scratch ? s.scratch : D.scratch;
  B.qt_ptr = D.qt_ptr;
  B.qt_src = D.qt_src;
  B.qt_w = mixed ? (const void*)D.qt_w32 : (const void*)D.qt_w;
  B.Minv_h = mixed ? (const void*)D.Minv_h32 : (const void*)D.Minv_h;
  B.Minv_z = mixed ? (const void*)D.Minv_z32 : (const void*)D.Minv_z;
  B.qt_rec_unit = reinterpret_cast<const int4*>(D.qt_rec_unit);
  B.qt_rec_src = reinterpret_cast<const int4*>(D.qt_rec_src);
  B.qt_rec_w = reinterpret_cast<const float4*>(D.qt_rec_w);
  B.Minv_g = !m.warped() ? nullptr : (mixed ? (const void*)D.Minv_g32 : (const void*)D.Minv_g);
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
  B.NZr = m.NZr();
  B.status = D.status;
  {
    ProfScope ps(mixed ? "dss_rk_mixed" : "dss_rk_fp64", st);
    if (mixed && B.Minv_g)
      dss_stage_mixed<true><<<grid_cap(m.NG, 64), 256, 0, st>>>(B);
    else if (mixed)
      dss_stage_mixed<<<grid_cap(m.NG, 64), 256, 0, st>>>(B);
    else {
      const size_t sm = sizeof(double) * m.NZ;
      if (sm > 48 * 1024) return fail(SEM_ERR_UNSUPPORTED, "more than 6144 vertical levels");
      if (s.rhs_only)
        dss_stage_fp64<0><<<grid_cap(m.NG), 256, sm, st>>>(B);
      else if (s.a == 0.0 && s.b == 1.0)
        dss_stage_fp64<1><<<grid_cap(m.NG), 256, sm, st>>>(B);
      else if (s.a == 0.75 && s.b == 0.25)
        dss_stage_fp64<3><<<grid_cap(m.NG), 256, sm, st>>>(B);
      else
        dss_stage_fp64<2><<<grid_cap(m.NG), 256, sm, st>>>(B);
    }
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
  int rc = check_params(p);   // the same validation as sem_rhs
  if (rc) return rc;
  Mesh& m = mh->m;
  const size_t need = (size_t)m.Ncol() * m.Nq * kFields * m.NZr() * sizeof(double);
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
  // the terms of the paper's runs keep per-mesh tables that are allocated on first use
  if (physics_on(*p)) return fail(SEM_ERR_UNSUPPORTED, "sem_rhs_noalloc: smag_cs, sponge_gamma and heat_q0 must be 0");
  // new reference-state parameters are uploaded with a synchronous copy,
  // which a stream capture would not record: refuse that case
  if (reference_stale(m, *p)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    SEM_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(SEM_ERR_ARG, "sem_rhs_noalloc: new reference-state parameters during stream capture; "
                               "make one call with them before capturing");
  }
  if ((rc = ensure_reference(m, *p))) return rc;
  void* scratch = nullptr;
  if ((rc = noalloc_scratch_address(dev, &scratch))) return rc;
  StageArgs s{nullptr, q, rhs, nullptr, nullptr, 0.0, 0.0, 1.0, 1, scratch};
  s.time = p->time;
  return launch_rhs_stage(m, *p, s, st);
}
