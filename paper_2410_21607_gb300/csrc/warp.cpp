// Warped layers: non-affine hexahedral elements (host geometry).
//
// Every node of the box mesh moves vertically to
//   z = zeta + A sin(2 pi kx (x + Lx/2) / Lx) sin(2 pi ky (y + Ly/2) / Ly) sin(pi zeta / Lz),
// which keeps the lids flat and the lateral periodicity and curves the layer
// surfaces.  The heights of the global nodes come from the warp; a hanging
// line takes the interpolation of its coarse neighbour's lines (the same
// constraint as the state, Sec. 3.1), so hanging nodes lie on the coarse
// face and the mesh stays watertight.  Each element is the isoparametric
// image of the reference cube through its nodal coordinates (Sec. 3's
// tensor-product LGL basis): x and y stay affine, x = x0 + (1 + xi) hx / 2,
// y = y0 + (1 + eta) hy / 2, and the height is the element's polynomial
// z(xi, eta, zeta), so the metric at a node needs z_xi, z_eta, z_zeta, the
// derivatives of the element's nodal heights by the LGL derivative matrix:
//   J = hx hy z_zeta / 4,
//   J grad xi   = (hy/2 z_zeta, 0, 0),
//   J grad eta  = (0, hx/2 z_zeta, 0),
//   J grad zeta = (-hy/2 z_xi, -hx/2 z_eta, hx hy / 4).
// These satisfy the discrete metric identities exactly (the derivative
// operators along different reference directions commute).  The lumped mass
// no longer factorises into horizontal and vertical parts: M = Q^T (w J) per
// global node.
#include <cmath>

#include "sem_internal.h"

namespace sem {

double warp_height(const Mesh& m, double x, double y, double zeta) {
  const double pi = 3.14159265358979323846;
  return zeta + m.warp_A * std::sin(2.0 * pi * m.warp_kx * (x + 0.5 * m.Lx) / m.Lx) *
                    std::sin(2.0 * pi * m.warp_ky * (y + 0.5 * m.Ly) / m.Ly) * std::sin(pi * zeta / m.Lz);
}

int build_warp(Mesh& m) {
  const Basis1D& B = basis(m.N);
  const int N = m.N, n1 = N + 1, Nq = m.Nq, NZ = m.NZ, nz = m.nz;
  const long long ncol = m.Ncol();
  const long long nhang = (long long)m.hang_h.size() / n1;
  m.zG.assign((size_t)m.NG, 0.0);
  for (long long h = 0; h < m.NH; ++h)
    for (int kz = 0; kz < NZ; ++kz) m.zG[(size_t)h * NZ + kz] = warp_height(m, m.xh[h], m.yh[h], m.zk[kz]);
  m.zH.assign((size_t)nhang * NZ, 0.0);
  for (long long k = 0; k < nhang; ++k)
    for (int kz = 0; kz < NZ; ++kz) {
      double z = 0.0;
      for (int q = 0; q < n1; ++q)
        z += m.hang_w[(size_t)k * n1 + q] * m.zG[(size_t)m.hang_h[(size_t)k * n1 + q] * NZ + kz];
      m.zH[(size_t)k * NZ + kz] = z;
    }
  auto zline = [&](long long c, int ab, int kz) {
    const int v = m.hmap[(size_t)c * Nq + ab];
    return v >= 0 ? m.zG[(size_t)v * NZ + kz] : m.zH[(size_t)(-1 - v) * NZ + kz];
  };
  // metric [col][ab][k][c][3] = z_xi, z_eta, z_zeta at node (a, b, c) of layer k,
  // and the lumped mass contribution of every column-line node
  m.metric.assign((size_t)ncol * Nq * nz * n1 * 3, 0.0);
  std::vector<double> mline((size_t)ncol * Nq * NZ, 0.0);
  for (long long c = 0; c < ncol; ++c) {
    const int l = m.leaves[c].l;
    const double hx = m.hx(l), hy = m.hy(l);
    for (int k = 0; k < nz; ++k)
      for (int b = 0; b < n1; ++b)
        for (int a = 0; a < n1; ++a)
          for (int cc = 0; cc < n1; ++cc) {
            const int kz = k * N + cc;
            double zx = 0.0, zy = 0.0, zz = 0.0;
            for (int q = 0; q < n1; ++q) {
              zx += B.D[a * n1 + q] * zline(c, q + n1 * b, kz);
              zy += B.D[b * n1 + q] * zline(c, a + n1 * q, kz);
              zz += B.D[cc * n1 + q] * zline(c, a + n1 * b, k * N + q);
            }
            if (!(zz > 0.0)) return fail(SEM_ERR_ARG, "the warp folds an element (non-positive Jacobian)");
            const int ab = a + n1 * b;
            double* mt = &m.metric[((((size_t)c * Nq + ab) * nz + k) * n1 + cc) * 3];
            mt[0] = zx;
            mt[1] = zy;
            mt[2] = zz;
            mline[((size_t)c * Nq + ab) * NZ + kz] += B.w[a] * B.w[b] * B.w[cc] * hx * hy * 0.25 * zz;
          }
  }
  m.Mg.assign((size_t)m.NG, 0.0);
  for (long long h = 0; h < m.NH; ++h)
    for (int e = m.qt_ptr[h]; e < m.qt_ptr[h + 1]; ++e)
      for (int kz = 0; kz < NZ; ++kz)
        m.Mg[(size_t)h * NZ + kz] += m.qt_w[e] * mline[(size_t)m.qt_src[e] * NZ + kz];
  for (size_t g = 0; g < m.Mg.size(); ++g)
    if (!(m.Mg[g] > 0.0)) return fail(SEM_ERR_TOPOLOGY, "non-positive lumped mass");
  return SEM_OK;
}

}  // namespace sem
