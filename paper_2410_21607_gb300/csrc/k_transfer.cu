// Solution transfer to an adapted mesh (Algorithm 3, "refine and coarsen
// marked elements").  The paper does not state the transfer operator; the
// one used:
//   1. new element values: unchanged columns copy theirs; a refined column's
//      children evaluate the parent polynomial at their nodes (horizontal
//      child interpolation P_a (x) P_b, z unchanged); a coarsened column takes
//      the exact L2 projection of its four children,
//      q = 1/4 sum_{a,b} (R_a (x) R_b) q_ab,  R_c = M^-1 P_c^T M  (M the exact
//      1-D mass matrix; the z direction is common to parent and children);
//   2. projection onto the continuous, hanging-node-constrained space,
//      (Q^T W Q) q_G = Q^T W q_L with W the LGL quadrature weights times the
//      Jacobian.  Q^T W Q = A_h (x) M_z: diagonal (the lumped mass) except on
//      the coarse-side nodes that hanging rows couple; those small coupled
//      blocks are solved by a Jacobi-preconditioned conjugate gradient, one
//      CTA per (block, field, level), with a bounded iteration count.
// The projection keeps every continuous field (refinement changes nothing)
// and the lumped total of every field.
#include <algorithm>
#include <numeric>

#include "sem_internal.h"

namespace sem {

__constant__ double c_P[kMaxN + 1][2][(kMaxN + 1) * (kMaxN + 1)];  // child interpolation
__constant__ double c_R[kMaxN + 1][2][(kMaxN + 1) * (kMaxN + 1)];  // child L2 projection
__constant__ double c_tw[kMaxN + 1][kMaxN + 1];                     // LGL weights

static int upload_transfer_constants_now() {
  static double P[kMaxN + 1][2][(kMaxN + 1) * (kMaxN + 1)] = {};
  static double R[kMaxN + 1][2][(kMaxN + 1) * (kMaxN + 1)] = {};
  static double W[kMaxN + 1][kMaxN + 1] = {};
  for (int N = 2; N <= kMaxN; ++N) {
    const Basis1D& B = basis(N);
    const int n = N + 1;
    // inverse of the exact mass matrix (Gauss-Jordan, SPD, tiny)
    std::vector<double> M = B.Mex, Mi(n * n, 0.0);
    for (int i = 0; i < n; ++i) Mi[i * n + i] = 1.0;
    for (int col = 0; col < n; ++col) {
      int piv = col;
      for (int r = col + 1; r < n; ++r)
        if (std::fabs(M[r * n + col]) > std::fabs(M[piv * n + col])) piv = r;
      for (int q = 0; q < n; ++q) {
        std::swap(M[col * n + q], M[piv * n + q]);
        std::swap(Mi[col * n + q], Mi[piv * n + q]);
      }
      double d = M[col * n + col];
      for (int q = 0; q < n; ++q) {
        M[col * n + q] /= d;
        Mi[col * n + q] /= d;
      }
      for (int r = 0; r < n; ++r) {
        if (r == col) continue;
        double f = M[r * n + col];
        for (int q = 0; q < n; ++q) {
          M[r * n + q] -= f * M[col * n + q];
          Mi[r * n + q] -= f * Mi[col * n + q];
        }
      }
    }
    for (int c = 0; c < 2; ++c) {
      // R_c = M^-1 P_c^T M
      std::vector<double> T(n * n, 0.0);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
          for (int q = 0; q < n; ++q) T[i * n + j] += B.P[c][q * n + i] * B.Mex[q * n + j];
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          double s = 0.0;
          for (int q = 0; q < n; ++q) s += Mi[i * n + q] * T[q * n + j];
          R[N][c][i * n + j] = s;
          P[N][c][i * n + j] = B.P[c][i * n + j];
        }
    }
    for (int i = 0; i < n; ++i) W[N][i] = B.w[i];
  }
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_P, P, sizeof(P)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_R, R, sizeof(R)));
  SEM_CUDA_TRY(cudaMemcpyToSymbol(c_tw, W, sizeof(W)));
  return SEM_OK;
}

// the tables of the current device (uploaded on its first use)
static int upload_transfer_constants() {
  static DeviceOnce once;
  return device_once(once, upload_transfer_constants_now);
}

struct TrArgs {
  const double* qold;
  const int* old_hmap;
  const int* old_hang_h;
  const double* old_hang_w;
  long long old_NG;
  const int* org;      // [Ncol][6]
  const int* new_level;
  double* out;         // new scratch [Ncol][Nq][5][NZ]
  int nz, NZ;
  double Lx, Ly, Lz;
  int nx, ny;
  const double* hzk;   // [nz] layer thicknesses
};

template <int N>
__device__ __forceinline__ void gather_old(const TrArgs& A, int col, int ab, int kz, double v[kFields]) {
  constexpr int n1 = N + 1, Nq = n1 * n1;
  const int hm = A.old_hmap[(long long)col * Nq + ab];
  if (hm >= 0) {
    for (int f = 0; f < kFields; ++f) v[f] = A.qold[(long long)f * A.old_NG + (long long)hm * A.NZ + kz];
  } else {
    const int k = -1 - hm;
    for (int f = 0; f < kFields; ++f) v[f] = 0.0;
    for (int m = 0; m <= N; ++m) {
      const double w = A.old_hang_w[k * n1 + m];
      const long long o = (long long)A.old_hang_h[k * n1 + m] * A.NZ + kz;
      for (int f = 0; f < kFields; ++f) v[f] += w * A.qold[(long long)f * A.old_NG + o];
    }
  }
}

template <int N>
__global__ void __launch_bounds__(((N + 1) * (N + 1) * (N + 1) + 31) / 32 * 32)
transfer_local(const TrArgs A) {
  constexpr int n1 = N + 1, Nq = n1 * n1, P = n1 * n1 * n1;
  __shared__ double sQ[4][kFields][P];
  __shared__ double sC[2][kFields][Nq];
  const int col = blockIdx.x, t = threadIdx.x;
  const bool act = t < P;
  const int i = t % n1, j = (t / n1) % n1, c = t / Nq;
  const int ab = i + n1 * j;
  const int* o = A.org + (long long)col * 6;
  const int kind = o[0];
  const int lev = A.new_level[col];
  const double hx = A.Lx / (double)((long long)A.nx << lev);
  const double hy = A.Ly / (double)((long long)A.ny << lev);
  const double wJ1 = act ? c_tw[N][i] * c_tw[N][j] * c_tw[N][c] * hx * hy * 0.125 : 0.0;  // per unit thickness
  const int nsrc = kind == 2 ? 4 : 1;
  for (int k = 0; k < A.nz; ++k) {
    const int kz = k * N + c;
    if (act) {
      for (int s = 0; s < nsrc; ++s) {
        double v[kFields];
        gather_old<N>(A, o[1 + s], ab, kz, v);
        for (int f = 0; f < kFields; ++f) sQ[s][f][t] = v[f];
      }
    }
    __syncthreads();
    double r[kFields] = {0, 0, 0, 0, 0};
    if (act) {
      if (kind == 0) {
        for (int f = 0; f < kFields; ++f) r[f] = sQ[0][f][t];
      } else if (kind == 1) {
        const int ca = o[5] & 1, cb = o[5] >> 1;
        for (int m = 0; m < n1; ++m)
          for (int n = 0; n < n1; ++n) {
            const double w = c_P[N][ca][i * n1 + m] * c_P[N][cb][j * n1 + n];
            for (int f = 0; f < kFields; ++f) r[f] += w * sQ[0][f][m + n1 * n + Nq * c];
          }
      } else {
        for (int s = 0; s < 4; ++s) {
          const int ca = s & 1, cb = s >> 1;
          for (int m = 0; m < n1; ++m)
            for (int n = 0; n < n1; ++n) {
              const double w = 0.25 * c_R[N][ca][i * n1 + m] * c_R[N][cb][j * n1 + n];
              for (int f = 0; f < kFields; ++f) r[f] += w * sQ[s][f][m + n1 * n + Nq * c];
            }
        }
      }
      const double wJ = wJ1 * A.hzk[k];
      for (int f = 0; f < kFields; ++f) r[f] *= wJ;
      if (c == 0 && k > 0)
        for (int f = 0; f < kFields; ++f) r[f] += sC[(k - 1) & 1][f][ab];
      if (c == N && k < A.nz - 1) {
        for (int f = 0; f < kFields; ++f) sC[k & 1][f][ab] = r[f];
      } else {
        double* dst = A.out + ((long long)((long long)col * Nq + ab) * kFields) * A.NZ + kz;
        for (int f = 0; f < kFields; ++f) dst[(long long)f * A.NZ] = r[f];
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
transfer_gather(const double* sc, const int* qt_ptr, const int* qt_src, const double* qt_w,
                const double* Minv_h, const double* Minv_z, const int* coupled, long long NG,
                int NZ, double* q) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < NG;
       g += (long long)gridDim.x * blockDim.x) {
    const long long h = g / NZ;
    const int kz = (int)(g - h * NZ);
    const int beg = qt_ptr[h], end = qt_ptr[h + 1];
    double acc[kFields] = {0, 0, 0, 0, 0};
    for (int e = beg; e < end; ++e) {
      const double w = qt_w[e];
      const double* p = sc + (long long)qt_src[e] * kFields * NZ + kz;
      for (int f = 0; f < kFields; ++f) acc[f] += w * p[(long long)f * NZ];
    }
    // coupled nodes keep b / M_z(kz) as the right-hand side of their block solve
    const double s = coupled[h] ? Minv_z[kz] : Minv_h[h] * Minv_z[kz];
    for (int f = 0; f < kFields; ++f) q[(long long)f * NG + g] = acc[f] * s;
  }
}

__device__ double block_sum(double v, double* red) {
  const int t = threadIdx.x;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// one CTA per (component, field, level); dynamic smem 5 n doubles
__global__ void __launch_bounds__(256)
transfer_cg(const int* comp_ptr, const int* nodes, const int* A_ptr, const int* A_col,
            const double* A_val, long long NG, int NZ, double* q, int max_iter, int* status) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  const int comp = blockIdx.x;
  const int f = blockIdx.y / NZ, kz = blockIdx.y % NZ;
  const int beg = comp_ptr[comp], n = comp_ptr[comp + 1] - beg;
  double* x = sm;
  double* r = sm + n;
  double* p = sm + 2 * n;
  double* Ap = sm + 3 * n;
  double* dinv = sm + 4 * n;
  const int t = threadIdx.x;
  double bb = 0.0;
  for (int a = t; a < n; a += blockDim.x) {
    const int row = beg + a;
    double d = 0.0;
    for (int e = A_ptr[row]; e < A_ptr[row + 1]; ++e)
      if (A_col[e] == a) d = A_val[e];
    dinv[a] = 1.0 / d;
    const double b = q[(long long)f * NG + (long long)nodes[row] * NZ + kz];
    r[a] = b;            // rhs stored in r until x0 is formed
    bb += b * b;
  }
  bb = block_sum(bb, red);
  for (int a = t; a < n; a += blockDim.x) x[a] = r[a] * dinv[a];
  __syncthreads();
  // r = b - A x0
  for (int a = t; a < n; a += blockDim.x) {
    const int row = beg + a;
    double s = 0.0;
    for (int e = A_ptr[row]; e < A_ptr[row + 1]; ++e) s += A_val[e] * x[A_col[e]];
    Ap[a] = r[a] - s;
  }
  __syncthreads();
  double rz = 0.0;
  for (int a = t; a < n; a += blockDim.x) {
    r[a] = Ap[a];
    p[a] = r[a] * dinv[a];
    rz += r[a] * p[a];
  }
  rz = block_sum(rz, red);
  const double tol2 = 1e-30 * bb;
  int it = 0;
  for (; it < max_iter; ++it) {
    double rr = 0.0;
    for (int a = t; a < n; a += blockDim.x) rr += r[a] * r[a];
    rr = block_sum(rr, red);
    if (rr <= tol2) break;
    double pAp = 0.0;
    for (int a = t; a < n; a += blockDim.x) {
      const int row = beg + a;
      double s = 0.0;
      for (int e = A_ptr[row]; e < A_ptr[row + 1]; ++e) s += A_val[e] * p[A_col[e]];
      Ap[a] = s;
      pAp += p[a] * s;
    }
    pAp = block_sum(pAp, red);
    const double alpha = rz / pAp;
    double rz2 = 0.0;
    for (int a = t; a < n; a += blockDim.x) {
      x[a] += alpha * p[a];
      r[a] -= alpha * Ap[a];
      rz2 += r[a] * r[a] * dinv[a];
    }
    rz2 = block_sum(rz2, red);
    const double beta = rz2 / rz;
    rz = rz2;
    for (int a = t; a < n; a += blockDim.x) p[a] = r[a] * dinv[a] + beta * p[a];
    __syncthreads();
  }
  if (it == max_iter && t == 0) atomicOr(status, 2);
  for (int a = t; a < n; a += blockDim.x)
    q[(long long)f * NG + (long long)nodes[beg + a] * NZ + kz] = x[a];
}

// Build the coupled blocks of A_h = Q_h^T W_h Q_h on the host (once per mesh).
static int build_coupled_blocks(Mesh& m) {
  DeviceTables& D = *m.dev;
  if (D.tr_coupled) return SEM_OK;
  const int n1 = m.N + 1;
  const Basis1D& B = basis(m.N);
  const long long nh = m.NH;
  std::vector<int> parent(nh);
  std::iota(parent.begin(), parent.end(), 0);
  auto find = [&](int x) {
    while (parent[x] != x) x = parent[x] = parent[parent[x]];
    return x;
  };
  std::vector<char> coupled(nh, 0);
  const long long nhang = (long long)m.hang_h.size() / n1;
  for (long long k = 0; k < nhang; ++k) {
    int first = -1, cnt = 0;
    for (int q = 0; q < n1; ++q)
      if (m.hang_w[k * n1 + q] != 0.0) ++cnt;
    if (cnt < 2) continue;
    for (int q = 0; q < n1; ++q) {
      if (m.hang_w[k * n1 + q] == 0.0) continue;
      int h = m.hang_h[k * n1 + q];
      coupled[h] = 1;
      if (first < 0) first = h;
      else parent[find(h)] = find(first);
    }
  }
  // components in order of their smallest node
  std::vector<int> comp_of(nh, -1), order;
  std::vector<std::vector<int>> comps;
  for (long long h = 0; h < nh; ++h) {
    if (!coupled[h]) continue;
    int r = find((int)h);
    if (comp_of[r] < 0) {
      comp_of[r] = (int)comps.size();
      comps.emplace_back();
    }
    comps[comp_of[r]].push_back((int)h);
  }
  std::vector<int> local(nh, -1), cid(nh, -1);
  std::vector<int> comp_ptr(1, 0), nodes;
  for (size_t c = 0; c < comps.size(); ++c) {
    for (size_t a = 0; a < comps[c].size(); ++a) {
      local[comps[c][a]] = (int)a;
      cid[comps[c][a]] = (int)c;
      nodes.push_back(comps[c][a]);
    }
    comp_ptr.push_back((int)nodes.size());
  }
  // assemble rows of A_h for the coupled nodes
  std::vector<std::vector<std::pair<int, double>>> rows(nodes.size());
  auto row_of = [&](int h) { return comp_ptr[cid[h]] + local[h]; };
  auto add = [&](int h, int g, double v) {
    auto& R = rows[row_of(h)];
    int lc = local[g];
    for (auto& e : R)
      if (e.first == lc) { e.second += v; return; }
    R.push_back({lc, v});
  };
  for (long long c = 0; c < m.Ncol(); ++c) {
    const int l = m.leaves[c].l;
    for (int ab = 0; ab < m.Nq; ++ab) {
      const double W = B.w[ab % n1] * B.w[ab / n1] * m.hx(l) * m.hy(l) * 0.25;
      const int v = m.hmap[c * m.Nq + ab];
      if (v >= 0) {
        if (coupled[v]) add(v, v, W);
      } else {
        const int k = -1 - v;
        for (int q = 0; q < n1; ++q) {
          const double wq = m.hang_w[(size_t)k * n1 + q];
          if (wq == 0.0) continue;
          const int hq = m.hang_h[(size_t)k * n1 + q];
          if (!coupled[hq]) continue;  // delta rows only touch uncoupled nodes
          for (int r = 0; r < n1; ++r) {
            const double wr = m.hang_w[(size_t)k * n1 + r];
            if (wr == 0.0) continue;
            add(hq, m.hang_h[(size_t)k * n1 + r], wq * wr * W);
          }
        }
      }
    }
  }
  std::vector<int> A_ptr(1, 0), A_col;
  std::vector<double> A_val;
  for (auto& R : rows) {
    std::sort(R.begin(), R.end());
    for (auto& e : R) {
      A_col.push_back(e.first);
      A_val.push_back(e.second);
    }
    A_ptr.push_back((int)A_col.size());
  }
  std::vector<int> cpl(nh);
  for (long long h = 0; h < nh; ++h) cpl[h] = coupled[h];
  D.n_comp = (int)comps.size();
  D.max_comp = 0;
  for (auto& c : comps) D.max_comp = std::max<int>(D.max_comp, (int)c.size());
  auto up = [](auto*& dst, const auto& v) -> int {
    using T = typename std::decay<decltype(v[0])>::type;
    size_t n = v.empty() ? 1 : v.size();
    SEM_CUDA_TRY(cudaMalloc((void**)&dst, n * sizeof(T)));
    if (!v.empty()) SEM_CUDA_TRY(cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return SEM_OK;
  };
  int rc;
  if ((rc = up(D.tr_comp_ptr, comp_ptr)) || (rc = up(D.tr_nodes, nodes)) || (rc = up(D.tr_A_ptr, A_ptr)) ||
      (rc = up(D.tr_A_col, A_col)) || (rc = up(D.tr_A_val, A_val)) || (rc = up(D.tr_coupled, cpl)))
    return rc;
  return SEM_OK;
}

template <int N>
static void launch_local(const TrArgs& A, int ncol, cudaStream_t st) {
  constexpr int P = (N + 1) * (N + 1) * (N + 1);
  transfer_local<N><<<ncol, (P + 31) / 32 * 32, 0, st>>>(A);
}

int launch_transfer(Mesh& o, Mesh& m, const double* qold, double* qnew, cudaStream_t st) {
  int rc = upload_transfer_constants();
  if (rc) return rc;
  if ((rc = build_coupled_blocks(m))) return rc;
  DeviceTables& D = *m.dev;
  DeviceTables& Do = *o.dev;
  if (o.NZ != m.NZ || o.N != m.N) return fail(SEM_ERR_ARG, "meshes differ in N or layering");
  TrArgs A;
  A.qold = qold;
  A.old_hmap = Do.hmap;
  A.old_hang_h = Do.hang_h;
  A.old_hang_w = Do.hang_w;
  A.old_NG = o.NG;
  A.org = D.org;
  A.new_level = D.col_level;
  A.out = (double*)D.scratch;
  A.nz = m.nz;
  A.NZ = m.NZ;
  A.Lx = m.Lx;
  A.Ly = m.Ly;
  A.Lz = m.Lz;
  A.nx = m.nx;
  A.ny = m.ny;
  A.hzk = D.hzk;
  const int nc = (int)m.Ncol();
  switch (m.N) {
    case 2: launch_local<2>(A, nc, st); break;
    case 3: launch_local<3>(A, nc, st); break;
    case 4: launch_local<4>(A, nc, st); break;
    case 5: launch_local<5>(A, nc, st); break;
    case 6: launch_local<6>(A, nc, st); break;
    default: return fail(SEM_ERR_UNSUPPORTED, "order N not compiled");
  }
  SEM_CUDA_TRY(cudaGetLastError());
  long long blocks = std::min<long long>((m.NG + 255) / 256, 152 * 8);
  transfer_gather<<<(int)blocks, 256, 0, st>>>((const double*)D.scratch, D.qt_ptr, D.qt_src, D.qt_w,
                                              D.Minv_h, D.Minv_z, D.tr_coupled, m.NG, m.NZ, qnew);
  SEM_CUDA_TRY(cudaGetLastError());
  if (D.n_comp > 0) {
    const size_t smem = (size_t)5 * D.max_comp * sizeof(double);
    if (smem > 200 * 1024) return fail(SEM_ERR_UNSUPPORTED, "coupled 2:1 block too large for one CTA");
    SEM_CUDA_TRY(cudaFuncSetAttribute(transfer_cg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(D.n_comp, kFields * m.NZ);
    transfer_cg<<<grid, 256, smem, st>>>(D.tr_comp_ptr, D.tr_nodes, D.tr_A_ptr, D.tr_A_col, D.tr_A_val,
                                         m.NG, m.NZ, qnew, 500, D.status);
    SEM_CUDA_TRY(cudaGetLastError());
  }
  return SEM_OK;
}

}  // namespace sem
