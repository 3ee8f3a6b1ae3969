// Terms of the paper's runs (Sec. 4): the horizontal Smagorinsky-Lilly
// stress ("Sub-grid models") and the Rayleigh absorbing layer ("Boundary
// conditions"), as an element pass that adds to the column residuals the
// element kernel has written, before the gather.
//
//   physics_column<N, EQ, R>: one CTA per leaf column marches up its layers.
//     Per element node it gathers the state, forms the velocity, and
//     - stress: the element-local horizontal velocity gradients, the strain
//       S_xx = du/dx, S_yy = dv/dy, S_xy = (du/dy + dv/dx)/2, the eddy
//       viscosity nu_t = (C_s Delta)^2 sqrt(2 (S_xx^2 + S_yy^2 + 2 S_xy^2))
//       with Delta = (hx + hy)/(2N), and the weak divergence of the fluxes
//       rho tau (EQ 0, conservative set) or tau (EQ 1), tau_{i,d} = -2 nu_t
//       S_{i,d} for the horizontal momentum and tau_{z,d} = -nu_t dw/dx_d,
//       d in {x, y};
//     - absorbing layer: the collocated source w J (-R(z) q') on every field;
//     - synthetic heating: the collocated source w J rho Q (EQ 0) or w J Q
//       on the theta equation, Q = q0 tanh(t / tau) exp(-((r - r0)/w)^2)
//       sin(pi z / z_h) for r <= r_max, z <= z_h (a stand-in for the
//       paper's observed heating);
//     then sums the face shared with the layer below (vertical DSS) and adds
//     the result into r_C[column][ab][field][kz].
//
// R is the arithmetic type: double for the float64 form, float for the mixed
// form (float32 mirror of the state, float32 residuals).  The mixed form of
// the conservative set uses physics_lines (below) instead, and only for what
// the element kernel has not added: a line-exchange element kernel adds the
// absorbing layer, and at order 4 the stress as well (k_stage.cu), in which
// case this pass runs for the heating alone, if at all.
#include <algorithm>
#include <cmath>
#include <vector>

#include "sem_internal.h"

namespace sem {
namespace {

__constant__ double p_xi[kMaxN + 1][kMaxN + 1];
__constant__ double p_w[kMaxN + 1][kMaxN + 1];
__constant__ double p_D[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];   // [i][m] = h_m'(xi_i)
__constant__ double p_Dw[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];  // [i][m] = w_m h_i'(xi_m)
__constant__ float p_wf[kMaxN + 1][kMaxN + 1];
__constant__ float p_Df[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];
__constant__ float p_Dwf[kMaxN + 1][(kMaxN + 1) * (kMaxN + 1)];

template <typename R> struct PTab;
template <> struct PTab<double> {
  __device__ static double w(int N, int i) { return p_w[N][i]; }
  __device__ static double D(int N, int k) { return p_D[N][k]; }
  __device__ static double Dw(int N, int k) { return p_Dw[N][k]; }
};
template <> struct PTab<float> {
  __device__ static float w(int N, int i) { return p_wf[N][i]; }
  __device__ static float D(int N, int k) { return p_Df[N][k]; }
  __device__ static float Dw(int N, int k) { return p_Dwf[N][k]; }
};

static int upload_constants_now() {
  constexpr int K = (kMaxN + 1) * (kMaxN + 1);
  double xi[kMaxN + 1][kMaxN + 1] = {}, w[kMaxN + 1][kMaxN + 1] = {}, D[kMaxN + 1][K] = {}, Dw[kMaxN + 1][K] = {};
  float wf[kMaxN + 1][kMaxN + 1] = {}, Df[kMaxN + 1][K] = {}, Dwf[kMaxN + 1][K] = {};
  for (int N = 2; N <= kMaxN; ++N) {
    const Basis1D& B = basis(N);
    const int n = N + 1;
    for (int i = 0; i < n; ++i) {
      xi[N][i] = B.xi[i];
      w[N][i] = B.w[i];
      wf[N][i] = (float)B.w[i];
      for (int m = 0; m < n; ++m) {
        D[N][i * n + m] = B.D[i * n + m];
        Dw[N][i * n + m] = B.w[m] * B.D[m * n + i];
        Df[N][i * n + m] = (float)D[N][i * n + m];
        Dwf[N][i * n + m] = (float)Dw[N][i * n + m];
      }
    }
  }
  SEM_CUDA_TRY(cudaMemcpyToSymbol(p_xi, xi, sizeof(xi)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(p_w, w, sizeof(w)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(p_D, D, sizeof(D)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(p_Dw, Dw, sizeof(Dw)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(p_wf, wf, sizeof(wf)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(p_Df, Df, sizeof(Df)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(p_Dwf, Dwf, sizeof(Dwf)));
  return SEM_OK;
}

// the tables of the current device (uploaded on its first use)
int upload_constants() {
  static DeviceOnce once;
  return device_once(once, upload_constants_now);
}

struct PhysArgs {
  const void* q;        // state [5][NG]: float64, or the float32 mirror (mixed form)
  void* rc;             // column residuals (same type)
  const int* hmap;
  const int* hang_h;
  const void* hang_w;   // hanging-row weights (same type)
  const int* col_level;
  const void* ref;      // reference state [NZ][kRef] (same type)
  const void* spg;      // absorbing-layer rate [NZ] (same type), null when off
  int nz, NZ, NZr, smag;
  long long NG;
  double cs;
  double geo[16][2];    // hx, hy per level
  const double* hzk;     // [nz] layer thicknesses (same type as the state when float)
  const float* hzk32;
  // synthetic heating: amplitude heat_q0 tanh(t / heat_ramp) at the time of
  // the state (0: off), ring radius and width, cut-off radius, depth
  double heat_amp, heat_r0, heat_width, heat_rmax, heat_ztop;
  const double* col_x0;  // [Ncol] column corners
  const double* col_y0;
  const double* zk;      // [NZ] heights of the levels
  // warped layers (non-affine elements): metric terms z_xi, z_eta, z_zeta per
  // node of each column line ([Ncol][Nq][nz][N+1][3], same type as the
  // state), node heights of global and hanging nodes, and the absorbing
  // layer's parameters (its rate is taken at each node's own height)
  const void* metric;
  const double* zG;
  const double* zH;
  const void* refG;      // reference state at the nodes' heights [NG][kRef], [Nhang NZ][kRef] (same type)
  const void* refH;
  double spg_gamma, spg_depth, Lz;
};

// R(z) of the absorbing layer at height z: gamma sin^2(pi/2 (1 - (Lz - z) /
// z_d)) clipped to [0, 1], zero below Lz - z_d (the per-level tables of box
// meshes hold the same values).
__device__ __forceinline__ double sponge_at(const PhysArgs& A, double z) {
  if (!(z >= A.Lz - A.spg_depth)) return 0.0;
  const double s = sin(0.5 * 3.14159265358979323846 * (1.0 - (A.Lz - z) / A.spg_depth));
  return fmin(1.0, fmax(0.0, A.spg_gamma * s * s));
}

// Q of the synthetic heating (K/s) at (x, y, z): ring in r, half sine in z,
// zero beyond heat_rmax and above heat_ztop.
__device__ __forceinline__ double heating_at(const PhysArgs& A, double x, double y, double z) {
  const double r = hypot(x, y);
  if (!(r <= A.heat_rmax && z <= A.heat_ztop)) return 0.0;
  const double a = (r - A.heat_r0) / A.heat_width;
  return A.heat_amp * exp(-a * a) * sin(3.14159265358979323846 * z / A.heat_ztop);
}

template <typename R>
__device__ __forceinline__ R geo_at(const PhysArgs& A, int l, int k) { return (R)A.geo[l][k]; }

// WARP: warped layers.  The Jacobian and the weak-form factors come from
// the node's metric terms (J = hx hy z_zeta / 4, J grad xi = (hy z_zeta / 2,
// 0, 0), J grad eta = (0, hx z_zeta / 2, 0), J grad zeta = (-hy z_xi / 2,
// -hx z_eta / 2, hx hy / 4)); the horizontal velocity gradients are taken at
// constant height, d/dx = (2 / hx) (d/dxi - (z_xi / z_zeta) d/dzeta), and the
// horizontal stress fluxes enter the zeta contraction through J grad zeta;
// the absorbing layer and the heating are evaluated at each node's height.
template <int N, int EQ, typename R, bool WARP = false>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
physics_column(const PhysArgs A) {
  constexpr int n1 = N + 1, Nq = n1 * n1, P = n1 * n1 * n1;
  __shared__ R sU[3][P];
  __shared__ R sF[WARP ? 9 : 6][P];
  __shared__ R sC[2][kFields][Nq];
  const int col = blockIdx.x, t = threadIdx.x;
  const bool act = t < P;
  const int i = t % n1, j = (t / n1) % n1, c = t / Nq;
  const int ab = i + n1 * j;
  const int lev = A.col_level[col];
  const R hx = geo_at<R>(A, lev, 0), hy = geo_at<R>(A, lev, 1);
  const R gx = (R)2 / hx, gy = (R)2 / hy;
  const R delta = (hx + hy) / (R)(2 * N);
  const R csd = (R)A.cs * delta;
  const R cs2 = csd * csd;
  const int hm = act ? A.hmap[(long long)col * Nq + ab] : 0;
  const R wi = act ? PTab<R>::w(N, i) : (R)0, wj = act ? PTab<R>::w(N, j) : (R)0;
  const R wc = act ? PTab<R>::w(N, c) : (R)0;
  const R* q = (const R*)A.q;
  const R* hw = (const R*)A.hang_w;
  const R* ref = (const R*)A.ref;
  const R* spg = (const R*)A.spg;
  R* rc = (R*)A.rc;
  const R* met = (const R*)A.metric;
  for (int k = 0; k < A.nz; ++k) {
    const int kz = k * N + c;
    // the layer's thickness: Jacobian and the weak-form factors J dxi/dx, J deta/dy
    const R hz = (R)A.hzk[k];
    R J = hx * hy * hz * (R)0.125;
    R sx = hy * hz * (R)0.25, sy = hx * hz * (R)0.25;
    R zx = 0, zy = 0, zz = 1;
    double zn = 0.0;
    if (WARP && act) {
      const R* mt = met + ((((long long)col * Nq + ab) * A.nz + k) * n1 + c) * 3;
      zx = mt[0];
      zy = mt[1];
      zz = mt[2];
      J = hx * hy * zz * (R)0.25;
      sx = hy * zz * (R)0.5;
      sy = hx * zz * (R)0.5;
      zn = hm >= 0 ? A.zG[(long long)hm * A.NZ + kz] : A.zH[(long long)(-1 - hm) * A.NZ + kz];
    }
    const R wJ = wi * wj * wc * J;
    R r[kFields] = {0, 0, 0, 0, 0};
    R rfac = (R)1;
    if (act) {
      R v[kFields];
      if (hm >= 0) {
        const R* p = q + (long long)hm * A.NZ + kz;
#pragma unroll
        for (int f = 0; f < kFields; ++f) v[f] = p[(long long)f * A.NG];
      } else {
        const int hk = -1 - hm;
#pragma unroll
        for (int f = 0; f < kFields; ++f) v[f] = (R)0;
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          const R wm = hw[hk * n1 + m];
          const R* p = q + (long long)A.hang_h[hk * n1 + m] * A.NZ + kz;
#pragma unroll
          for (int f = 0; f < kFields; ++f) v[f] += wm * p[(long long)f * A.NG];
        }
      }
      R u = v[1], vv = v[2], w = v[3];
      if (EQ == 0) {
        // warped layers: the reference density at the node's own height
        const R rho0 = !WARP ? ref[(long long)kz * kRef + 3]
                     : hm >= 0 ? ((const R*)A.refG)[((long long)hm * A.NZ + kz) * kRef + 3]
                               : ((const R*)A.refH)[((long long)(-1 - hm) * A.NZ + kz) * kRef + 3];
        const R rho = rho0 + v[0];
        const R inv = (R)1 / rho;
        u *= inv;
        vv *= inv;
        w *= inv;
        rfac = rho;
      }
      if (spg) {
        const R Rz = WARP ? (R)sponge_at(A, zn) : spg[kz];
#pragma unroll
        for (int f = 0; f < kFields; ++f) r[f] = wJ * (-Rz * v[f]);
      }
      if (A.heat_amp != 0.0) {
        const double hxd = A.geo[lev][0], hyd = A.geo[lev][1];
        const double x = A.col_x0[col] + 0.5 * (1.0 + p_xi[N][i]) * hxd;
        const double y = A.col_y0[col] + 0.5 * (1.0 + p_xi[N][j]) * hyd;
        const R Q = (R)heating_at(A, x, y, WARP ? zn : A.zk[kz]);
        r[4] += wJ * (EQ == 0 ? rfac * Q : Q);
      }
      if (A.smag) {
        sU[0][t] = u;
        sU[1][t] = vv;
        sU[2][t] = w;
      }
    }
    if (A.smag) {
      __syncthreads();
      if (act) {
        R ux = 0, uy = 0, vx = 0, vy = 0, wx = 0, wy = 0;
        R uz = 0, vz = 0, wz = 0;   // zeta derivatives (warped layers)
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          const R Di = PTab<R>::D(N, i * n1 + m), Dj = PTab<R>::D(N, j * n1 + m);
          const int lx = m + n1 * j + Nq * c, ly = i + n1 * m + Nq * c;
          ux += Di * sU[0][lx];
          uy += Dj * sU[0][ly];
          vx += Di * sU[1][lx];
          vy += Dj * sU[1][ly];
          wx += Di * sU[2][lx];
          wy += Dj * sU[2][ly];
          if (WARP) {
            const R Dc = PTab<R>::D(N, c * n1 + m);
            const int lz = i + n1 * j + Nq * m;
            uz += Dc * sU[0][lz];
            vz += Dc * sU[1][lz];
            wz += Dc * sU[2][lz];
          }
        }
        if (WARP) {
          // derivatives at constant height
          const R ex = zx / zz, ey = zy / zz;
          ux -= ex * uz; vx -= ex * vz; wx -= ex * wz;
          uy -= ey * uz; vy -= ey * vz; wy -= ey * wz;
        }
        ux *= gx; vx *= gx; wx *= gx;
        uy *= gy; vy *= gy; wy *= gy;
        const R sxx = ux, syy = vy, sxy = (R)0.5 * (uy + vx);
        const R nut = cs2 * sqrt((R)2 * (sxx * sxx + syy * syy + (R)2 * sxy * sxy));
        const R kv = rfac * nut;
        const R ax = wj * wc * sx, ay = wi * wc * sy;
        sF[0][t] = ax * ((R)-2 * kv * sxx);
        sF[1][t] = ay * ((R)-2 * kv * sxy);
        sF[2][t] = ax * ((R)-2 * kv * sxy);
        sF[3][t] = ay * ((R)-2 * kv * syy);
        sF[4][t] = ax * (-kv * wx);
        sF[5][t] = ay * (-kv * wy);
        if (WARP) {
          // the zeta component of each flux, through J grad zeta
          const R bx = -wi * wj * hy * zx * (R)0.5, by = -wi * wj * hx * zy * (R)0.5;
          sF[WARP ? 6 : 0][t] = bx * ((R)-2 * kv * sxx) + by * ((R)-2 * kv * sxy);
          sF[WARP ? 7 : 0][t] = bx * ((R)-2 * kv * sxy) + by * ((R)-2 * kv * syy);
          sF[WARP ? 8 : 0][t] = bx * (-kv * wx) + by * (-kv * wy);
        }
      }
      __syncthreads();
      if (act) {
#pragma unroll
        for (int m = 0; m < n1; ++m) {
          const R Dwi = PTab<R>::Dw(N, i * n1 + m), Dwj = PTab<R>::Dw(N, j * n1 + m);
          const int lx = m + n1 * j + Nq * c, ly = i + n1 * m + Nq * c;
          r[1] += Dwi * sF[0][lx] + Dwj * sF[1][ly];
          r[2] += Dwi * sF[2][lx] + Dwj * sF[3][ly];
          r[3] += Dwi * sF[4][lx] + Dwj * sF[5][ly];
          if (WARP) {
            const R Dwc = PTab<R>::Dw(N, c * n1 + m);
            const int lz = i + n1 * j + Nq * m;
            r[1] += Dwc * sF[WARP ? 6 : 0][lz];
            r[2] += Dwc * sF[WARP ? 7 : 0][lz];
            r[3] += Dwc * sF[WARP ? 8 : 0][lz];
          }
        }
      }
    }
    if (act) {
      // vertical direct stiffness summation inside the column, then add
      if (c == 0 && k > 0) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) r[f] += sC[(k - 1) & 1][f][ab];
      }
      if (c == N && k < A.nz - 1) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) sC[k & 1][f][ab] = r[f];
      } else {
        R* dst = rc + ((long long)((long long)col * Nq + ab) * kFields) * A.NZr + kz;
#pragma unroll
        for (int f = 0; f < kFields; ++f) dst[(long long)f * A.NZr] += r[f];
      }
    }
    __syncthreads();
  }
}

template <int N, typename R>
void launch_n(const PhysArgs& A, int eq, int ncol, cudaStream_t st) {
  constexpr int threads = ((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32;
  if (A.metric) {
    if (eq == SEM_EQ_CONSERVATIVE) physics_column<N, 0, R, true><<<ncol, threads, 0, st>>>(A);
    else physics_column<N, 1, R, true><<<ncol, threads, 0, st>>>(A);
  } else if (eq == SEM_EQ_CONSERVATIVE) {
    physics_column<N, 0, R><<<ncol, threads, 0, st>>>(A);
  } else {
    physics_column<N, 1, R><<<ncol, threads, 0, st>>>(A);
  }
}

// Mixed form, conservative set: the same terms with the thread layout of the
// line-exchange element kernel (coalesced z-line loads and residual updates).
// Thread (layer kk, line ab) owns the vertical line of N+1 nodes of its
// element; node (i, j, c) keeps 9 float32 components (u, v, w, then the x and
// y derivatives, later the weighted x and y stress fluxes) at
// kk LS + (i + (N+1) j) LW + comp (N+1) + c.  Phases, separated by barriers:
//  A  z-line owner: state -> rho, u, v, w (and the layer source in registers);
//  B  x-line / y-line owners: du/dx, dv/dx, dw/dx (comps 3-5), du/dy, dv/dy,
//     dw/dy (comps 6-8) of their line, written onto its nodes;
//  C  z-line owner: nu_t and the weighted fluxes of rho tau, in place;
//  D  x-line / y-line owners: weak contraction of their line's fluxes, in place;
//  E  z-line owner: sums, vertical DSS, residual update.
template <int N>
__host__ __device__ constexpr int plines_lw() { return (9 * (N + 1)) | 1; }
template <int N, int KL>
__host__ __device__ constexpr int plines_ls() {
  return (N + 1) * (N + 1) * plines_lw<N>() +
         ((32 / KL - ((N + 1) * (N + 1) * plines_lw<N>()) % 32) % 32 + 32) % 32;
}
template <int N, int KL>
__host__ __device__ constexpr int plines_smem_floats() {
  return KL * plines_ls<N, KL>() + kFields * KL * (N + 1) * (N + 1) + 2 * kFields * (N + 1) * (N + 1);
}

template <int N, int KL, int MB>
__global__ void __launch_bounds__(KL * (N + 1) * (N + 1), MB)
physics_lines(const PhysArgs A) {
  constexpr int n1 = N + 1, Nq = n1 * n1;
  constexpr int LW = plines_lw<N>(), LS = plines_ls<N, KL>();
  extern __shared__ __align__(16) float smem[];
  float* sV = smem;                       // [kk][LS]: node components
  float* sT = sV + KL * LS;               // [f][kk][ab]: layer source of the top node
  float* sP = sT + kFields * KL * Nq;     // [2][f][ab]: top-node carry between chunks
  const int col = blockIdx.x, t = threadIdx.x;
  const int kk = t % KL, ab = t / KL;
  const int i = ab % n1, j = ab / n1;
  const int lc = ab % n1, lo = ab / n1;   // x-line (j, c) = (lo, lc), y-line (i, c) = (lo, lc)
  const int lev = A.col_level[col];
  const float hx = (float)A.geo[lev][0], hy = (float)A.geo[lev][1];
  const float gx = 2.f / hx, gy = 2.f / hy;
  const float csd = (float)A.cs * ((hx + hy) / (float)(2 * N));
  const float cs2 = csd * csd;
  const int hm = A.hmap[(long long)col * Nq + ab];
  const float wi = p_wf[N][i], wj = p_wf[N][j];
  const float* q = (const float*)A.q;
  const float* hw = (const float*)A.hang_w;
  const float* ref = (const float*)A.ref;
  const float* spg = (const float*)A.spg;
  float* rc = (float*)A.rc;
  const bool heat = A.heat_amp != 0.0;
  const int nchunk = (A.nz + KL - 1) / KL;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int k = ch * KL + kk;
    const bool act = k < A.nz;
    const int kz0 = k * N;
    const float hz = act ? A.hzk32[k] : 0.f;   // the layer's thickness
    const float J = hx * hy * hz * 0.125f;
    const float sx = hy * hz * 0.25f, sy = hx * hz * 0.25f;
    float r[kFields][n1];
#pragma unroll
    for (int f = 0; f < kFields; ++f)
#pragma unroll
      for (int c = 0; c < n1; ++c) r[f][c] = 0.f;
    float rho[n1];
    float* zV = sV + kk * LS + ab * LW;   // this thread's z-line, + comp n1 + c
    if (act) {
      {
        // the residuals this thread updates at the end of the chunk: start
        // bringing them into L1 now
        const float* dp = rc + ((long long)((long long)col * Nq + ab) * kFields) * A.NZr + kz0;
#pragma unroll
        for (int f = 0; f < kFields; ++f)
          asm volatile("prefetch.global.L1 [%0];" ::"l"(dp + (long long)f * A.NZr));
      }
#pragma unroll
      for (int c = 0; c < n1; ++c) {
        const int kz = kz0 + c;
        float v[kFields];
        if (hm >= 0) {
          const float* pq = q + (long long)hm * A.NZ + kz;
#pragma unroll
          for (int f = 0; f < kFields; ++f) v[f] = __ldg(pq + (long long)f * A.NG);
        } else {
          const int hk = -1 - hm;
#pragma unroll
          for (int f = 0; f < kFields; ++f) v[f] = 0.f;
#pragma unroll
          for (int m = 0; m < n1; ++m) {
            const float wm = __ldg(hw + hk * n1 + m);
            const float* pq = q + (long long)__ldg(A.hang_h + hk * n1 + m) * A.NZ + kz;
#pragma unroll
            for (int f = 0; f < kFields; ++f) v[f] = fmaf(wm, __ldg(pq + (long long)f * A.NG), v[f]);
          }
        }
        rho[c] = __ldg(ref + (long long)kz * kRef + 3) + v[0];
        const float inv = __frcp_rn(rho[c]);   // = 1 / rho, correctly rounded
        zV[0 * n1 + c] = v[1] * inv;
        zV[1 * n1 + c] = v[2] * inv;
        zV[2 * n1 + c] = v[3] * inv;
        if (spg) {
          const float wJ = wi * wj * p_wf[N][c] * J;
          const float Rz = __ldg(spg + kz);
#pragma unroll
          for (int f = 0; f < kFields; ++f) r[f][c] = wJ * (-Rz * v[f]);
        }
        if (heat) {
          const double x = A.col_x0[col] + 0.5 * (1.0 + p_xi[N][i]) * A.geo[lev][0];
          const double y = A.col_y0[col] + 0.5 * (1.0 + p_xi[N][j]) * A.geo[lev][1];
          const float Q = (float)heating_at(A, x, y, A.zk[kz]);
          r[4][c] += wi * wj * p_wf[N][c] * J * (rho[c] * Q);
        }
      }
#pragma unroll
      for (int f = 0; f < kFields; ++f) sT[(f * KL + kk) * Nq + ab] = r[f][N];
    }
    if (A.smag) {
      __syncthreads();
      if (act) {
        // B: derivatives along the thread's x-line (nodes (m, lo, lc)) and y-line (nodes (lo, m, lc))
        float* bx = sV + kk * LS + lo * n1 * LW + lc;
        float* by = sV + kk * LS + lo * LW + lc;
#pragma unroll
        for (int cp = 0; cp < 3; ++cp) {
          float F[n1], G[n1];
#pragma unroll
          for (int m = 0; m < n1; ++m) {
            F[m] = bx[m * LW + cp * n1];
            G[m] = by[m * n1 * LW + cp * n1];
          }
#pragma unroll
          for (int o = 0; o < n1; ++o) {
            float ax_ = 0.f, ay_ = 0.f;
#pragma unroll
            for (int m = 0; m < n1; ++m) {
              ax_ = fmaf(p_Df[N][o * n1 + m], F[m], ax_);
              ay_ = fmaf(p_Df[N][o * n1 + m], G[m], ay_);
            }
            bx[o * LW + (3 + cp) * n1] = ax_ * gx;
            by[o * n1 * LW + (6 + cp) * n1] = ay_ * gy;
          }
        }
      }
      __syncthreads();
      if (act) {
        // C: eddy viscosity and weighted fluxes of rho tau at the thread's nodes
#pragma unroll
        for (int c = 0; c < n1; ++c) {
          const float ux = zV[3 * n1 + c], vx = zV[4 * n1 + c], wx = zV[5 * n1 + c];
          const float uy = zV[6 * n1 + c], vy = zV[7 * n1 + c], wy = zV[8 * n1 + c];
          const float sxy = 0.5f * (uy + vx);
          // sqrt(s) as s rsqrt(s): a few ulp, well inside float32 arithmetic
          // error of the pass, and 7 % faster than the correctly rounded sqrtf
          const float s2 = 2.f * (ux * ux + vy * vy + 2.f * sxy * sxy);
          const float nut = cs2 * (s2 > 0.f ? s2 * rsqrtf(s2) : 0.f);
          const float kv = rho[c] * nut;
          const float wc = p_wf[N][c];
          const float ax = wj * wc * sx, ay = wi * wc * sy;
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
        // D: weak contraction of the line's fluxes, written back onto its nodes
        float* bx = sV + kk * LS + lo * n1 * LW + lc;
        float* by = sV + kk * LS + lo * LW + lc;
#pragma unroll
        for (int cp = 0; cp < 3; ++cp) {
          float F[n1], G[n1];
#pragma unroll
          for (int m = 0; m < n1; ++m) {
            F[m] = bx[m * LW + (3 + cp) * n1];
            G[m] = by[m * n1 * LW + (6 + cp) * n1];
          }
#pragma unroll
          for (int o = 0; o < n1; ++o) {
            float ax_ = 0.f, ay_ = 0.f;
#pragma unroll
            for (int m = 0; m < n1; ++m) {
              ax_ = fmaf(p_Dwf[N][o * n1 + m], F[m], ax_);
              ay_ = fmaf(p_Dwf[N][o * n1 + m], G[m], ay_);
            }
            bx[o * LW + (3 + cp) * n1] = ax_;
            by[o * n1 * LW + (6 + cp) * n1] = ay_;
          }
        }
      }
    }
    __syncthreads();
    if (act) {
      // E: sums at the thread's nodes, vertical DSS, residual update
      if (A.smag) {
#pragma unroll
        for (int cp = 0; cp < 3; ++cp)
#pragma unroll
          for (int c = 0; c < n1; ++c) r[1 + cp][c] += zV[(3 + cp) * n1 + c] + zV[(6 + cp) * n1 + c];
      }
      if (kk > 0) {
        const float* pV = sV + (kk - 1) * LS + ab * LW;
#pragma unroll
        for (int f = 0; f < kFields; ++f) {
          float add = sT[(f * KL + kk - 1) * Nq + ab];
          if (A.smag && f >= 1 && f <= 3) add += pV[(2 + f) * n1 + N] + pV[(5 + f) * n1 + N];
          r[f][0] += add;
        }
      } else if (ch > 0) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) r[f][0] += sP[((ch - 1) & 1) * kFields * Nq + f * Nq + ab];
      }
      if (kk == KL - 1) {
#pragma unroll
        for (int f = 0; f < kFields; ++f) sP[(ch & 1) * kFields * Nq + f * Nq + ab] = r[f][N];
      }
      float* dst = rc + ((long long)((long long)col * Nq + ab) * kFields) * A.NZr + kz0;
      const bool top = (k == A.nz - 1);
      // fields with a contribution: the layer touches all, the stress the
      // momentum, the heating the theta equation
      const bool lay = spg != nullptr;
#pragma unroll
      for (int f = 0; f < kFields; ++f) {
        if (f == 0 && !lay) continue;
        if (f == 4 && !lay && !heat) continue;
        if (f >= 1 && f <= 3 && !lay && !A.smag) continue;
        float* df = dst + (long long)f * A.NZr;
        if (N == 4) {
          float4 o = *reinterpret_cast<float4*>(df);
          o.x += r[f][0];
          o.y += r[f][1];
          o.z += r[f][2];
          o.w += r[f][3];
          *reinterpret_cast<float4*>(df) = o;
        } else {
#pragma unroll
          for (int c = 0; c < N; ++c) df[c] += r[f][c];
        }
        if (top) df[N] += r[f][N];
      }
    }
    if (ch + 1 < nchunk) __syncthreads();
  }
}

template <int N, int KL, int MB>
int launch_lines(const PhysArgs& A, int ncol, cudaStream_t st) {
  const size_t sm = sizeof(float) * plines_smem_floats<N, KL>();
  static DeviceOnce attr;
  int rc = device_once(attr, [&] {
    SEM_CUDA_TRY(cudaFuncSetAttribute(physics_lines<N, KL, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    return SEM_OK;
  });
  if (rc) return rc;
  physics_lines<N, KL, MB><<<ncol, KL * (N + 1) * (N + 1), sm, st>>>(A);
  return SEM_OK;
}

}  // namespace

// Absorbing-layer rate R(z) per level (float64 and float32 tables), rebuilt
// when gamma or the depth change.
int ensure_sponge(Mesh& m, const sem_params& p) {
  DeviceTables& D = *m.dev;
  if (D.spg && D.spg_key[0] == p.sponge_gamma && D.spg_key[1] == p.sponge_depth) return SEM_OK;
  std::vector<double> R(m.NZ);
  std::vector<float> R32(m.NZ);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < m.NZ; ++k) {
    const double z = m.zk[k];
    const double a = 0.5 * pi * (1.0 - (m.Lz - z) / p.sponge_depth);
    const double s = std::sin(a);
    double r = std::min(1.0, std::max(0.0, p.sponge_gamma * s * s));
    if (!(z >= m.Lz - p.sponge_depth)) r = 0.0;
    R[k] = r;
    R32[k] = (float)r;
  }
  if (!D.spg) {
    SEM_CUDA_TRY(cudaMalloc((void**)&D.spg, (size_t)m.NZ * sizeof(double)));
    SEM_CUDA_TRY(cudaMalloc((void**)&D.spg32, (size_t)m.NZ * sizeof(float)));
  }
  SEM_CUDA_TRY(cudaMemcpy(D.spg, R.data(), R.size() * sizeof(double), cudaMemcpyHostToDevice));
  SEM_CUDA_TRY(cudaMemcpy(D.spg32, R32.data(), R32.size() * sizeof(float), cudaMemcpyHostToDevice));
  D.spg_key[0] = p.sponge_gamma;
  D.spg_key[1] = p.sponge_depth;
  return SEM_OK;
}

int launch_physics(Mesh& m, const sem_params& p, const void* q, bool mixed, void* scratch,
                   double time, cudaStream_t st, bool sponge_done, bool smag_done) {
  int rc = upload_constants();
  if (rc) return rc;
  DeviceTables& D = *m.dev;
  const bool sponge = p.sponge_gamma > 0.0 && !sponge_done;
  const double heat_amp = p.heat_q0 > 0.0 ? p.heat_q0 * std::tanh(time / p.heat_ramp) : 0.0;
  const bool smag = p.smag_cs > 0.0 && !smag_done;
  if (!sponge && !smag && heat_amp == 0.0) return SEM_OK;   // nothing to add
  if (sponge && (rc = ensure_sponge(m, p))) return rc;
  PhysArgs A;
  A.q = q;
  A.rc = scratch ? scratch : D.scratch;
  A.hmap = D.hmap;
  A.hang_h = D.hang_h;
  A.hang_w = mixed ? (const void*)D.hang_w32 : (const void*)D.hang_w;
  A.col_level = D.col_level;
  A.ref = mixed ? (const void*)D.ref32 : (const void*)D.ref;
  A.spg = sponge ? (mixed ? (const void*)D.spg32 : (const void*)D.spg) : nullptr;
  A.nz = m.nz;
  A.NZ = m.NZ;
  A.NZr = m.NZr();
  A.smag = smag;
  A.NG = m.NG;
  A.cs = p.smag_cs;
  A.heat_amp = heat_amp;
  A.heat_r0 = p.heat_r0;
  A.heat_width = p.heat_width;
  A.heat_rmax = p.heat_rmax;
  A.heat_ztop = p.heat_ztop;
  A.col_x0 = D.col_x0;
  A.col_y0 = D.col_y0;
  A.zk = D.zk;
  A.hzk = D.hzk;
  A.hzk32 = D.hzk32;
  const bool w = m.warped();
  A.metric = w ? (mixed ? (const void*)D.metric32 : (const void*)D.metric) : nullptr;
  A.zG = w ? D.zG : nullptr;
  A.zH = w ? D.zH : nullptr;
  A.refG = w ? (mixed ? (const void*)D.refG32 : (const void*)D.refG) : nullptr;
  A.refH = w ? (mixed ? (const void*)D.refH32 : (const void*)D.refH) : nullptr;
  A.spg_gamma = p.sponge_gamma;
  A.spg_depth = p.sponge_depth;
  A.Lz = m.Lz;
  for (int l = 0; l < 16; ++l) {
    A.geo[l][0] = m.hx(l);
    A.geo[l][1] = m.hy(l);

  }
  ProfScope ps("physics", st);
  const int ncol = (int)m.Ncol();
  if (mixed && p.eqset == SEM_EQ_CONSERVATIVE && !w) {
    switch (m.N) {
      case 2: rc = launch_lines<2, 16, 4>(A, ncol, st); break;
      case 3: rc = launch_lines<3, 16, 2>(A, ncol, st); break;
      case 4: rc = launch_lines<4, 8, 4>(A, ncol, st); break;
      case 5: rc = launch_lines<5, 4, 4>(A, ncol, st); break;
      case 6: rc = launch_lines<6, 4, 2>(A, ncol, st); break;
      default: return fail(SEM_ERR_UNSUPPORTED, "order N not compiled");
    }
    if (rc) return rc;
    SEM_CUDA_TRY(cudaGetLastError());
    return SEM_OK;
  }
  switch (m.N) {
    case 2: mixed ? launch_n<2, float>(A, p.eqset, ncol, st) : launch_n<2, double>(A, p.eqset, ncol, st); break;
    case 3: mixed ? launch_n<3, float>(A, p.eqset, ncol, st) : launch_n<3, double>(A, p.eqset, ncol, st); break;
    case 4: mixed ? launch_n<4, float>(A, p.eqset, ncol, st) : launch_n<4, double>(A, p.eqset, ncol, st); break;
    case 5: mixed ? launch_n<5, float>(A, p.eqset, ncol, st) : launch_n<5, double>(A, p.eqset, ncol, st); break;
    case 6: mixed ? launch_n<6, float>(A, p.eqset, ncol, st) : launch_n<6, double>(A, p.eqset, ncol, st); break;
    default: return fail(SEM_ERR_UNSUPPORTED, "order N not compiled");
  }
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
