// Criterion, diagnostics and coordinate kernels.
//
//   adapt_column<N, EQ>: Sec. 3.1 threshold criterion.  One CTA per leaf
//     column; per element the velocity magnitude at every local node (hanging
//     nodes interpolated as in the modified DSS), its maximum, and the flag
//       +1 if max > threshold(lvl+1) and lvl < lvl_max,
//       -1 if max <= threshold(lvl) and lvl > 0, else 0.
//     The speed is evaluated with explicitly rounded float64 operations
//     (sqrt(U U + V V + W W) / rho in that order, no contraction into FMA) so
//     that the decision is taken in float64 exactly as written.
//   diag_level: Sec. 4.2 diagnostics, one CTA per vertical level: maximum
//     horizontal speed and the mass-weighted mean speed over the horizontal
//     sub-domain |x|, |y| <= half_width, reduced in a fixed order.
#include "sem_internal.h"

namespace sem {

struct AdaptArgs {
  const double* q;
  const int* hmap;
  const int* hang_h;
  const double* hang_w;
  const int* col_level;
  const double* ref;
  int8_t* flags;
  double* cmax;
  int nz, NZ;
  long long NG;
  int lvl_max;
  double thr[SEM_MAX_THRESHOLDS];
};

template <int N, int EQ>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
adapt_column(const AdaptArgs A) {
  constexpr int n1 = N + 1, Nq = n1 * n1, P = n1 * n1 * n1;
  constexpr int NW = (P + 31) / 32;
  __shared__ double red[NW];
  const int col = blockIdx.x, t = threadIdx.x;
  const bool act = t < P;
  const int i = t % n1, j = (t / n1) % n1, c = t / Nq;
  const int ab = i + n1 * j;
  const int hm = act ? A.hmap[(long long)col * Nq + ab] : 0;
  const int lev = A.col_level[col];
  for (int k = 0; k < A.nz; ++k) {
    double s = 0.0;
    if (act) {
      const int kz = k * N + c;
      double v[4] = {0, 0, 0, 0};
      if (hm >= 0) {
        const double* p = A.q + (long long)hm * A.NZ + kz;
        for (int f = 0; f < 4; ++f) v[f] = p[(long long)f * A.NG];
      } else {
        const int h = -1 - hm;
        for (int m = 0; m <= N; ++m) {
          const double w = A.hang_w[h * n1 + m];
          const double* p = A.q + (long long)A.hang_h[h * n1 + m] * A.NZ + kz;
          for (int f = 0; f < 4; ++f) v[f] = __dadd_rn(v[f], __dmul_rn(w, p[(long long)f * A.NG]));
        }
      }
      double ss = __dadd_rn(__dadd_rn(__dmul_rn(v[1], v[1]), __dmul_rn(v[2], v[2])), __dmul_rn(v[3], v[3]));
      s = __dsqrt_rn(ss);
      if (EQ == 0) s = __ddiv_rn(s, __dadd_rn(A.ref[(long long)kz * kRef + 3], v[0]));
    }
    // block maximum over the element's nodes
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((t & 31) == 0) red[t >> 5] = s;
    __syncthreads();
    if (t == 0) {
      double mx = red[0];
      for (int w = 1; w < NW; ++w) mx = fmax(mx, red[w]);
      const long long e = (long long)col * A.nz + k;
      int flag = 0;
      if (lev < A.lvl_max && mx > A.thr[lev]) flag = 1;
      else if (lev > 0 && mx <= A.thr[lev - 1]) flag = -1;
      A.flags[e] = (int8_t)flag;
      if (A.cmax) A.cmax[e] = mx;
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
                 cudaStream_t st) {
  DeviceTables& D = *m.dev;
  AdaptArgs A;
  A.q = q;
  A.hmap = D.hmap;
  A.hang_h = D.hang_h;
  A.hang_w = D.hang_w;
  A.col_level = D.col_level;
  A.ref = D.ref;
  A.flags = flags;
  A.cmax = cmax;
  A.nz = m.nz;
  A.NZ = m.NZ;
  A.NG = m.NG;
  A.lvl_max = p.lvl_max;
  for (int k = 0; k < SEM_MAX_THRESHOLDS; ++k) A.thr[k] = p.thresholds[k];
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
           double* out /*[NZ][4]*/) {
  __shared__ double s_max[256], s_num[256], s_den[256];
  const int kz = blockIdx.x;
  const double rho0 = ref[(long long)kz * kRef + 3];
  double mx = 0.0, num = 0.0, den = 0.0;
  for (long long h = threadIdx.x; h < NH; h += blockDim.x) {
    if (!(fabs(xh[h]) <= hw + 1e-6 && fabs(yh[h]) <= hw + 1e-6)) continue;
    const long long g = h * NZ + kz;
    const double U = q[NG + g], V = q[2 * NG + g];
    double s = sqrt(U * U + V * V);
    if (eq == 0) s = s / (rho0 + q[g]);
    mx = fmax(mx, s);
    num += Mh[h] * s;
    den += Mh[h];
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
__global__ void coords_kernel(const double* xh, const double* yh, const double* zk, long long NH,
                              int NZ, double* xyz) {
  const long long NG = NH * NZ;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < NG;
       g += (long long)gridDim.x * blockDim.x) {
    const long long h = g / NZ;
    const int k = (int)(g - h * NZ);
    xyz[g] = xh[h];
    xyz[NG + g] = yh[h];
    xyz[2 * NG + g] = zk[k];
  }
}

int launch_coords(Mesh& m, double* xyz, cudaStream_t st) {
  DeviceTables& D = *m.dev;
  long long blocks = std::min<long long>((m.NG + 255) / 256, 152 * 16);
  coords_kernel<<<(int)blocks, 256, 0, st>>>(D.xh, D.yh, D.zk, m.NH, m.NZ, xyz);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}

}  // namespace sem
