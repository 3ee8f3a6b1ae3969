// Host topology of the column-structured non-conforming mesh (bookkeeping
// only; every field operation runs in the CUDA kernels).
//
// Sec. 3.1 of the paper refines horizontally and by whole columns, so the
// mesh is a horizontal quadtree forest (one root per base column) extruded
// through nz layers that every column shares.  Hence the constraint matrix
// of the modified DSS factorises as Q = Q_h (x) I_z: a local node (a, b, c)
// of column k, layer e maps to global node (h, kz) with kz = e N + c and h
// given by the column's horizontal map.  Horizontal global nodes are
//   * interior nodes of a column,
//   * nodes of a column side shared with a same-level neighbour (or owned by
//     the coarse side of a 2:1 face),
//   * grid vertices that are not in the interior of a coarser side.
// A side node of a column whose neighbour across that side is coarser (and a
// vertex in the interior of a coarser side) is hanging: its row of Q_h holds
// the coarse side's N+1 Lagrange basis values at its position (Sec. 3.1,
// "the values of the local solution at hanging nodes contribute to the
// global solution through interpolation").
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "sem_internal.h"

namespace sem {

// ---------------------------------------------------------------------------
// 1-D LGL basis
static void legendre_pair(int n, double x, double& pn, double& pnm1) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { pn = 1.0; pnm1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pnm1 = p0;
}

double lagrange(const std::vector<double>& xi, int j, double x) {
  double v = 1.0;
  for (size_t m = 0; m < xi.size(); ++m)
    if ((int)m != j) v *= (x - xi[m]) / (xi[j] - xi[m]);
  return v;
}

static Basis1D make_basis(int N) {
  Basis1D B;
  B.N = N;
  const int n = N + 1;
  B.xi.assign(n, 0.0);
  B.w.assign(n, 0.0);
  // Newton iteration x <- x - (x P_N - P_{N-1}) / ((N+1) P_N), whose fixed
  // points are the LGL nodes, started from Chebyshev-Gauss-Lobatto points.
  for (int i = 0; i < n; ++i) {
    double x = -std::cos(M_PI * i / N);
    for (int it = 0; it < 200; ++it) {
      double pn, pm;
      legendre_pair(N, x, pn, pm);
      double dx = (x * pn - pm) / (n * pn);
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    B.xi[i] = x;
  }
  B.xi[0] = -1.0;
  B.xi[N] = 1.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.5 * (B.xi[i] - B.xi[N - i]);
    B.xi[i] = s;
  }
  if (N % 2 == 0) B.xi[N / 2] = 0.0;
  for (int i = 0; i < n; ++i) {
    double pn, pm;
    legendre_pair(N, B.xi[i], pn, pm);
    B.w[i] = 2.0 / (N * (N + 1.0) * pn * pn);
  }
  for (int i = 0; i < n; ++i) {
    double s = 0.5 * (B.w[i] + B.w[N - i]);
    B.w[i] = s;
  }
  // derivative matrix from barycentric weights
  std::vector<double> lam(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int m = 0; m < n; ++m)
      if (m != j) lam[j] /= (B.xi[j] - B.xi[m]);
  B.D.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      double d = (lam[j] / lam[i]) / (B.xi[i] - B.xi[j]);
      B.D[i * n + j] = d;
      diag -= d;
    }
    B.D[i * n + i] = diag;
  }
  for (int c = 0; c < 2; ++c) {
    B.P[c].assign(n * n, 0.0);
    for (int i = 0; i < n; ++i) {
      double x = 0.5 * (B.xi[i] + 2.0 * c - 1.0);
      for (int j = 0; j < n; ++j) B.P[c][i * n + j] = lagrange(B.xi, j, x);
    }
  }
  // exact mass matrix with an (N+2)-point Gauss-Legendre rule
  const int ng = N + 2;
  std::vector<double> gx(ng), gw(ng);
  for (int i = 0; i < ng; ++i) {
    double x = -std::cos(M_PI * (i + 0.75) / (ng + 0.5));
    for (int it = 0; it < 100; ++it) {
      double pn, pm;
      legendre_pair(ng, x, pn, pm);
      double dp = ng * (x * pn - pm) / (x * x - 1.0);
      double dx = pn / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    double pn, pm;
    legendre_pair(ng, x, pn, pm);
    double dp = ng * (x * pn - pm) / (x * x - 1.0);
    gx[i] = x;
    gw[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  B.Mex.assign(n * n, 0.0);
  for (int g = 0; g < ng; ++g)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        B.Mex[i * n + j] += gw[g] * lagrange(B.xi, i, gx[g]) * lagrange(B.xi, j, gx[g]);
  return B;
}

const Basis1D& basis(int N) {
  static std::mutex mu;
  static Basis1D cache[kMaxN + 1];
  std::lock_guard<std::mutex> lk(mu);
  if (cache[N].N != N) cache[N] = make_basis(N);
  return cache[N];
}

// ---------------------------------------------------------------------------
static inline uint64_t spread16(uint64_t v) {
  uint64_t x = v & 0xFFFFFFFFull;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}
static inline uint64_t morton_key(const Leaf& f) {
  // position of the leaf's lower-left corner on a 2^16-times finer grid
  uint64_t X = (uint64_t)f.i << (16 - f.l), Y = (uint64_t)f.j << (16 - f.l);
  return spread16(X) | (spread16(Y) << 1);
}

struct Grid {
  int NX = 0, NY = 0, L = 0;
  bool px = true, py = true;
  std::vector<int> owner;
  int at(long X, long Y) const {   // owner of cell (X, Y), -1 outside a closed side
    if (X < 0 || X >= NX) {
      if (!px) return -1;
      X = ((X % NX) + NX) % NX;
    }
    if (Y < 0 || Y >= NY) {
      if (!py) return -1;
      Y = ((Y % NY) + NY) % NY;
    }
    return owner[(size_t)X * NY + Y];
  }
};

static int make_grid(const Mesh& m, const std::vector<Leaf>& leaves, Grid& G) {
  int L = 0;
  for (auto& f : leaves) L = std::max(L, f.l);
  if (L > 12) return fail(SEM_ERR_TOPOLOGY, "refinement level above 12");
  G.L = L;
  G.NX = m.nx << L;
  G.NY = m.ny << L;
  G.px = m.px;
  G.py = m.py;
  G.owner.assign((size_t)G.NX * G.NY, -1);
  for (size_t c = 0; c < leaves.size(); ++c) {
    const Leaf& f = leaves[c];
    if (f.l < 0 || f.i < 0 || f.j < 0 || f.i >= (m.nx << f.l) || f.j >= (m.ny << f.l))
      return fail(SEM_ERR_TOPOLOGY, "leaf outside the base grid");
    int s = 1 << (L - f.l);
    for (int X = f.i * s; X < (f.i + 1) * s; ++X)
      for (int Y = f.j * s; Y < (f.j + 1) * s; ++Y) {
        int& o = G.owner[(size_t)X * G.NY + Y];
        if (o != -1) return fail(SEM_ERR_TOPOLOGY, "leaves overlap");
        o = (int)c;
      }
  }
  for (int o : G.owner)
    if (o < 0) return fail(SEM_ERR_TOPOLOGY, "leaves do not cover the domain");
  return SEM_OK;
}

// owners of the one-cell ring around a leaf (face and corner neighbours)
static void ring(const Grid& G, const Leaf& f, std::vector<int>& out) {
  out.clear();
  int s = 1 << (G.L - f.l);
  long X0 = (long)f.i * s, X1 = X0 + s, Y0 = (long)f.j * s, Y1 = Y0 + s;
  auto add = [&](long X, long Y) {
    int o = G.at(X, Y);
    if (o >= 0 && std::find(out.begin(), out.end(), o) == out.end()) out.push_back(o);
  };
  for (long X = X0 - 1; X <= X1; ++X) {
    add(X, Y0 - 1);
    add(X, Y1);
  }
  for (long Y = Y0; Y < Y1; ++Y) {
    add(X0 - 1, Y);
    add(X1, Y);
  }
}

int check_leaves(const Mesh& m) {
  Grid G;
  int rc = make_grid(m, m.leaves, G);
  if (rc) return rc;
  std::vector<int> nb;
  for (size_t c = 0; c < m.leaves.size(); ++c) {
    ring(G, m.leaves[c], nb);
    for (int d : nb)
      if (d != (int)c && std::abs(m.leaves[d].l - m.leaves[c].l) > 1)
        return fail(SEM_ERR_TOPOLOGY, "mesh is not 2:1 balanced");
  }
  return SEM_OK;
}

// ---------------------------------------------------------------------------
// global numbering
namespace {
struct Pending {
  int col, ab;
  uint64_t keys[kMaxN + 1];
  double w[kMaxN + 1];
};
inline uint64_t vkey(long X, long Y) {
  return (0ull << 62) | ((uint64_t)X << 25) | (uint64_t)Y;
}
inline uint64_t skey(int orient, long X, long Y, int lev, int idx) {
  return (1ull << 62) | ((uint64_t)orient << 61) | ((uint64_t)lev << 57) |
         ((uint64_t)idx << 50) | ((uint64_t)X << 25) | (uint64_t)Y;
}
}  // namespace

int build_mesh(Mesh& m) {
  const int N = m.N;
  const int n1 = N + 1;
  if (N < 2 || N > kMaxN) return fail(SEM_ERR_UNSUPPORTED, "order N must be in 2..6");
  std::stable_sort(m.leaves.begin(), m.leaves.end(),
                   [](const Leaf& a, const Leaf& b) { return morton_key(a) < morton_key(b); });
  Grid G;
  int rc = make_grid(m, m.leaves, G);
  if (rc) return rc;
  rc = check_leaves(m);
  if (rc) return rc;
  if (((long)G.NX >= (1l << 25)) || ((long)G.NY >= (1l << 25)) || m.leaves.size() >= (1ull << 40))
    return fail(SEM_ERR_ARG, "mesh too large");
  m.Lf = G.L;
  m.Nq = n1 * n1;
  m.P = n1 * n1 * n1;
  m.NZ = m.nz * N + 1;
  const Basis1D& B = basis(N);
  const long ncol = (long)m.leaves.size();
  m.hmap.assign((size_t)ncol * m.Nq, 0);
  std::unordered_map<uint64_t, int> id;
  id.reserve((size_t)ncol * m.Nq);
  std::vector<Pending> pend;
  m.xh.clear();
  m.yh.clear();
  const double hxf = m.Lx / G.NX, hyf = m.Ly / G.NY;
  auto wrapx = [&](double x) {
    if (m.px) {
      if (x >= 0.5 * m.Lx - 1e-9 * m.Lx) x -= m.Lx;
      if (std::fabs(x + 0.5 * m.Lx) < 1e-9 * m.Lx) x = -0.5 * m.Lx;
    }
    return x;
  };
  auto wrapy = [&](double y) {
    if (m.py) {
      if (y >= 0.5 * m.Ly - 1e-9 * m.Ly) y -= m.Ly;
      if (std::fabs(y + 0.5 * m.Ly) < 1e-9 * m.Ly) y = -0.5 * m.Ly;
    }
    return y;
  };
  auto modx = [&](long X) { return m.px ? ((X % G.NX) + G.NX) % G.NX : X; };
  auto mody = [&](long Y) { return m.py ? ((Y % G.NY) + G.NY) % G.NY : Y; };
  long nonconf = 0;

  // hanging row on the side of coarse leaf d (orient 0: side at constant X
  // running in Y from T0 = start, 1: at constant Y running in X); t is the
  // reference coordinate of the point on that side.
  auto coarse_side_row = [&](Pending& p, int orient, long line, long T0, int dl, double t) {
    long S = 1l << (G.L - dl);
    for (int q = 0; q <= N; ++q) {
      uint64_t k;
      if (q == 0 || q == N) {
        long T = T0 + (q == N ? S : 0);
        k = orient == 0 ? vkey(modx(line), mody(T)) : vkey(modx(T), mody(line));
      } else {
        k = orient == 0 ? skey(0, modx(line), mody(T0), dl, q) : skey(1, modx(T0), mody(line), dl, q);
      }
      p.keys[q] = k;
      double v = lagrange(B.xi, q, t);
      for (int r = 0; r <= N; ++r)
        if (t == B.xi[r]) v = (r == q) ? 1.0 : 0.0;
      p.w[q] = v;
    }
  };

  for (long c = 0; c < ncol; ++c) {
    const Leaf& f = m.leaves[c];
    const int s = 1 << (G.L - f.l);
    const long X0 = (long)f.i * s, X1 = X0 + s, Y0 = (long)f.j * s, Y1 = Y0 + s;
    const double x0 = -0.5 * m.Lx + f.i * m.hx(f.l), y0 = -0.5 * m.Ly + f.j * m.hy(f.l);
    for (int b = 0; b <= N; ++b) {
      for (int a = 0; a <= N; ++a) {
        const int ab = a + n1 * b;
        const bool eX = (a == 0 || a == N), eY = (b == 0 || b == N);
        uint64_t key = 0;
        bool hanging = false;
        Pending p{};
        p.col = (int)c;
        p.ab = ab;
        if (!eX && !eY) {
          // inside the cross-section: no key (numbered below without the map)
        } else if (eX && eY) {
          long X = a == 0 ? X0 : X1, Y = b == 0 ? Y0 : Y1;
          int cells[4] = {G.at(X - 1, Y - 1), G.at(X, Y - 1), G.at(X - 1, Y), G.at(X, Y)};
          for (int q = 0; q < 4 && !hanging; ++q) {
            int d = cells[q];
            if (d < 0 || m.leaves[d].l >= f.l) continue;
            const Leaf& g = m.leaves[d];
            long S = 1l << (G.L - g.l);
            long dX0 = (long)g.i * S, dY0 = (long)g.j * S;
            // offset of the vertex from the coarse leaf's corner (periodic)
            long ox = X - dX0, oy = Y - dY0;
            if (m.px) ox = ((ox % G.NX) + G.NX) % G.NX;
            if (m.py) oy = ((oy % G.NY) + G.NY) % G.NY;
            if (ox > S) ox -= G.NX;
            if (oy > S) oy -= G.NY;
            bool cornerx = (ox == 0 || ox == S), cornery = (oy == 0 || oy == S);
            if (cornerx && cornery) continue;
            hanging = true;
            if (cornerx)
              coarse_side_row(p, 0, dX0 + ox, dY0, g.l, 2.0 * oy / S - 1.0);
            else
              coarse_side_row(p, 1, dY0 + oy, dX0, g.l, 2.0 * ox / S - 1.0);
          }
          if (!hanging) key = vkey(modx(X), mody(Y));
        } else {
          int orient = eX ? 0 : 1;
          long line = eX ? (a == 0 ? X0 : X1) : (b == 0 ? Y0 : Y1);
          int idx = eX ? b : a;
          long T0 = eX ? Y0 : X0;
          int d = eX ? G.at(a == 0 ? X0 - 1 : X1, Y0) : G.at(X0, b == 0 ? Y0 - 1 : Y1);
          if (d >= 0 && m.leaves[d].l < f.l) {
            const Leaf& g = m.leaves[d];
            long S = 1l << (G.L - g.l);
            long dT0 = eX ? (long)g.j * S : (long)g.i * S;
            long off = T0 - dT0;
            long NT = eX ? G.NY : G.NX;
            off = ((off % NT) + NT) % NT;
            int child = (int)(off / s);
            hanging = true;
            coarse_side_row(p, orient, line, dT0, g.l, 0.5 * (B.xi[idx] + 2.0 * child - 1.0));
          } else {
            if (d >= 0 && m.leaves[d].l > f.l && idx == 1) ++nonconf;
            key = orient == 0 ? skey(0, modx(line), mody(T0), f.l, idx)
                              : skey(1, modx(T0), mody(line), f.l, idx);
          }
        }
        if (hanging) {
          m.hmap[(size_t)c * m.Nq + ab] = -1 - (int)pend.size();
          pend.push_back(p);
        } else {
          // a node inside the column's cross-section belongs to it alone: a
          // new index without the map; a shared one is looked up (and
          // numbered on first sight) in one map operation
          int h = (int)m.xh.size();
          bool fresh = true;
          if (eX || eY) {
            auto ins = id.try_emplace(key, h);
            fresh = ins.second;
            h = ins.first->second;
          }
          if (fresh) {
            m.xh.push_back(wrapx(x0 + 0.5 * (1.0 + B.xi[a]) * m.hx(f.l)));
            m.yh.push_back(wrapy(y0 + 0.5 * (1.0 + B.xi[b]) * m.hy(f.l)));
          }
          m.hmap[(size_t)c * m.Nq + ab] = h;
        }
      }
    }
  }
  (void)hxf;
  (void)hyf;
  m.NH = (long long)m.xh.size();
  m.NG = m.NH * m.NZ;
  m.n_nonconf_sides = nonconf;
  m.hang_h.assign(pend.size() * n1, 0);
  m.hang_w.assign(pend.size() * n1, 0.0);
  for (size_t k = 0; k < pend.size(); ++k) {
    for (int q = 0; q <= N; ++q) {
      auto it = id.find(pend[k].keys[q]);
      if (it == id.end()) {
        if (pend[k].w[q] == 0.0) { m.hang_h[k * n1 + q] = 0; m.hang_w[k * n1 + q] = 0.0; continue; }
        return fail(SEM_ERR_TOPOLOGY, "hanging node refers to a hanging node (chained constraint)");
      }
      m.hang_h[k * n1 + q] = it->second;
      m.hang_w[k * n1 + q] = pend[k].w[q];
    }
  }
  // transposed constraint (gather lists), sorted by (h, source): the sources
  // are visited in increasing order, so one counting pass by h and a stable
  // scatter give that order without a comparison sort
  auto each_entry = [&](auto&& emit) {
    for (long c = 0; c < ncol; ++c)
      for (int ab = 0; ab < m.Nq; ++ab) {
        const int v = m.hmap[(size_t)c * m.Nq + ab];
        const int src = (int)(c * m.Nq + ab);
        if (v >= 0) {
          emit(v, src, 1.0);
        } else {
          const int k = -1 - v;
          for (int q = 0; q <= N; ++q)
            if (m.hang_w[(size_t)k * n1 + q] != 0.0) emit(m.hang_h[(size_t)k * n1 + q], src, m.hang_w[(size_t)k * n1 + q]);
        }
      }
  };
  m.qt_ptr.assign(m.NH + 1, 0);
  each_entry([&](int h, int, double) { m.qt_ptr[h + 1]++; });
  for (long long h = 0; h < m.NH; ++h) m.qt_ptr[h + 1] += m.qt_ptr[h];
  m.qt_src.resize(m.qt_ptr[m.NH]);
  m.qt_w.resize(m.qt_ptr[m.NH]);
  {
    std::vector<int> next(m.qt_ptr.begin(), m.qt_ptr.end() - 1);
    each_entry([&](int h, int src, double w) {
      const int e = next[h]++;
      m.qt_src[e] = src;
      m.qt_w[e] = w;
    });
  }
  // lumped mass factors
  m.Mh.assign(m.NH, 0.0);
  for (long long h = 0; h < m.NH; ++h)
    for (int e = m.qt_ptr[h]; e < m.qt_ptr[h + 1]; ++e) {
      int src = m.qt_src[e];
      int c = src / m.Nq, ab = src % m.Nq;
      int a = ab % n1, b = ab / n1;
      int l = m.leaves[c].l;
      m.Mh[h] += m.qt_w[e] * B.w[a] * B.w[b] * m.hx(l) * m.hy(l) * 0.25;
    }
  m.Mz.assign(m.NZ, 0.0);
  m.zk.assign(m.NZ, 0.0);
  for (int k = 0; k < m.nz; ++k)
    for (int c = 0; c <= N; ++c) {
      m.Mz[k * N + c] += B.w[c] * m.hz(k) * 0.5;
      m.zk[k * N + c] = m.zf[k] + 0.5 * (1.0 + B.xi[c]) * m.hz(k);
    }
  m.zk[0] = 0.0;
  m.zk[m.NZ - 1] = m.Lz;
  for (long long h = 0; h < m.NH; ++h)
    if (!(m.Mh[h] > 0.0)) return fail(SEM_ERR_TOPOLOGY, "non-positive lumped mass");
  if (m.warped()) return build_warp(m);
  return SEM_OK;
}

// ---------------------------------------------------------------------------
// one adaptation pass (Sec. 3.1; Remark 3.1; 2:1 balance)
int adapt_leaves(const Mesh& old, const int8_t* flags, std::vector<Leaf>& out,
                 std::vector<Origin>& origin) {
  const auto& L = old.leaves;
  const long ncol = (long)L.size();
  Grid G;
  int rc = make_grid(old, L, G);
  if (rc) return rc;
  std::vector<int> colflag(ncol, -1), target(ncol);
  for (long c = 0; c < ncol; ++c) {
    int mx = -1;
    for (int k = 0; k < old.nz; ++k) {
      int v = flags[c * old.nz + k];
      if (v < -1 || v > 1) return fail(SEM_ERR_ARG, "flags must be -1, 0 or 1");
      mx = std::max(mx, v);
    }
    colflag[c] = mx;
    target[c] = L[c].l + ((mx > 0 && L[c].l < old.lvl_max) ? 1 : 0);
  }
  std::vector<std::vector<int>> nb(ncol);
  for (long c = 0; c < ncol; ++c) {
    ring(G, L[c], nb[c]);
    nb[c].erase(std::remove(nb[c].begin(), nb[c].end(), (int)c), nb[c].end());
  }
  // refinement propagates until every neighbour pair differs by at most one
  std::vector<int> work;
  for (long c = 0; c < ncol; ++c) work.push_back((int)c);
  while (!work.empty()) {
    int c = work.back();
    work.pop_back();
    for (int d : nb[c]) {
      if (target[d] < target[c] - 1) {
        target[d] = target[c] - 1;
        work.push_back(d);
      }
    }
  }
  // complete sibling groups whose four columns are flagged -1 everywhere
  auto leaf_at = [&](int l, int i, int j) -> int {
    if (l > G.L) return -1;
    int s = 1 << (G.L - l);
    int o = G.owner[(size_t)(i * s) * G.NY + (size_t)(j * s)];
    return (L[o].l == l && L[o].i == i && L[o].j == j) ? o : -1;
  };
  std::vector<int> group(ncol, -1);
  std::vector<std::array<int, 4>> groups;
  for (long c = 0; c < ncol; ++c) {
    const Leaf& f = L[c];
    if (f.l == 0 || group[c] >= 0 || colflag[c] != -1 || target[c] != f.l) continue;
    int pi = f.i >> 1, pj = f.j >> 1;
    std::array<int, 4> sib;
    bool ok = true;
    for (int q = 0; q < 4 && ok; ++q) {
      sib[q] = leaf_at(f.l, 2 * pi + (q & 1), 2 * pj + (q >> 1));
      ok = sib[q] >= 0 && colflag[sib[q]] == -1 && target[sib[q]] == f.l;
    }
    if (!ok) continue;
    for (int q = 0; q < 4; ++q) group[sib[q]] = (int)groups.size();
    groups.push_back(sib);
  }
  std::vector<char> gok(groups.size(), 1);
  bool changed = true;
  while (changed) {
    changed = false;
    for (size_t g = 0; g < groups.size(); ++g) {
      if (!gok[g]) continue;
      int l = L[groups[g][0]].l;
      for (int q = 0; q < 4 && gok[g]; ++q)
        for (int d : nb[groups[g][q]]) {
          if (group[d] == (int)g) continue;
          int fin = (group[d] >= 0 && gok[group[d]]) ? target[d] - 1 : target[d];
          if (fin > l) {
            gok[g] = 0;
            changed = true;
            break;
          }
        }
    }
  }
  out.clear();
  origin.clear();
  std::vector<char> emitted(groups.size(), 0);
  for (long c = 0; c < ncol; ++c) {
    const Leaf& f = L[c];
    int g = group[c];
    if (g >= 0 && gok[g]) {
      if (!emitted[g]) {
        emitted[g] = 1;
        out.push_back({f.l - 1, f.i >> 1, f.j >> 1});
        Origin o{};
        o.kind = 2;
        for (int q = 0; q < 4; ++q) o.src[q] = groups[g][q];
        origin.push_back(o);
      }
    } else if (target[c] > f.l) {
      for (int q = 0; q < 4; ++q) {
        out.push_back({f.l + 1, 2 * f.i + (q & 1), 2 * f.j + (q >> 1)});
        Origin o{};
        o.kind = 1;
        o.src[0] = (int)c;
        o.a = q & 1;
        o.b = q >> 1;
        origin.push_back(o);
      }
    } else {
      out.push_back(f);
      Origin o{};
      o.kind = 0;
      o.src[0] = (int)c;
      origin.push_back(o);
    }
  }
  return SEM_OK;
}

}  // namespace sem
