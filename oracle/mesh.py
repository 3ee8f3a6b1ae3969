"""Brute-force hexahedral LGL mesh with hanging nodes (Sec. 3 and 3.1).

The domain is the box [-Lx/2, Lx/2] x [-Ly/2, Ly/2] x [0, Lz] split into a
base grid of nx x ny columns of nz hexahedra.  Refinement is horizontal only
and always takes a whole column (Sec. 3.1, "Refining an element"), so a mesh is
a list of leaf columns (level, i, j): column (i, j) of the 2^level-times finer
horizontal grid.  Element e = column c, layer k  ->  e = c * nz + k.

Global nodes and the constraint matrix Q are built by brute force from node
coordinates, following the modified DSS described at the end of Sec. 3.1:

* a local node is *hanging* when it lies on the boundary of a coarser element
  at a point where that coarser element has no node of its own;
* every other local node position is a global node (periodic images merged);
* the row of Q for a non-hanging local node is the unit vector of its global
  node; the row of a hanging node holds the coarser element's basis functions
  evaluated at the node (its interpolation onto the non-hanging nodes), with
  any hanging coarse node substituted recursively.

The local element vector is q_L = Q q_G and the assembled residual is Q^T r_L.

Warped layers (non-affine elements): with warp = (A, kx, ky) the layer
surfaces are curved, every node of the box mesh moving vertically to
    z = zeta + A sin(2 pi kx (x + Lx/2) / Lx) sin(2 pi ky (y + Ly/2) / Ly) sin(pi zeta / Lz),
which keeps the lids flat and the lateral periodicity.  Topology (global
nodes, Q) is built on the box coordinates; the heights of the global nodes
come from the warp and the local heights are z_L = Q z_G, so that hanging
nodes lie on the coarse side's face (the mesh stays watertight).  Every
element is the isoparametric image of the reference cube through its nodal
coordinates: at each node the Jacobian matrix dx_d/dxi_i comes from the
derivative matrix applied to the element's coordinates, and its inverse
gives d xi_i / dx_d and the derivative operators
    G_d[k, l] = sum_i (d xi_i / dx_d)(x_k) d psi_l / d xi_i (xi_k),
with the quadrature weights w_k det(dx/dxi)(x_k).  Without a warp the
elements are the axis-aligned boxes and the operators are the closed forms
of element_ops.

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np
import scipy.sparse as sp

from . import basis


class OracleMesh:
    def __init__(self, Lx, Ly, Lz, nx, ny, nz, N, leaves=None,
                 periodic=(True, True), z_faces=None, warp=None):
        self.Lx, self.Ly, self.Lz = float(Lx), float(Ly), float(Lz)
        self.nx, self.ny, self.nz, self.N = int(nx), int(ny), int(nz), int(N)
        # layer faces 0 = z_0 < z_1 < ... < z_nz = Lz (uniform by default; a
        # stretched grid gives its own): every element stays an axis-aligned box
        if z_faces is None:
            self.zf = np.array([k * (self.Lz / self.nz) for k in range(self.nz)] + [self.Lz])
        else:
            self.zf = np.asarray(z_faces, dtype=np.float64)
            if (self.zf.shape != (self.nz + 1,) or self.zf[0] != 0.0 or self.zf[-1] != self.Lz
                    or np.any(np.diff(self.zf) <= 0)):
                raise ValueError("z_faces must rise strictly from 0 to Lz (nz + 1 values)")
        self.hzk = np.diff(self.zf)
        self.periodic = tuple(bool(p) for p in periodic)
        if leaves is None:
            leaves = [(0, i, j) for j in range(ny) for i in range(nx)]
        self.leaves = [tuple(int(v) for v in t) for t in leaves]
        self._check_tiling()
        self.xi, self.w = basis.lgl_nodes_weights(self.N)
        self.warp = None if warp is None else tuple(float(v) for v in warp)
        self._build_elements()
        self._build_global_nodes()
        if self.warp is not None:
            self._apply_warp()

    # ------------------------------------------------------------------
    def _check_tiling(self):
        """Every base column is covered exactly once by the leaves."""
        lmax = max(l for l, _, _ in self.leaves)
        s = 1 << lmax
        cover = np.zeros((self.nx * s, self.ny * s), dtype=np.int64)
        for l, i, j in self.leaves:
            f = 1 << (lmax - l)
            if not (0 <= i < self.nx << l and 0 <= j < self.ny << l):
                raise ValueError(f"leaf {(l, i, j)} outside the base grid")
            cover[i * f:(i + 1) * f, j * f:(j + 1) * f] += 1
        if not np.all(cover == 1):
            raise ValueError("leaves do not tile the domain exactly once")

    def column_box(self, c):
        l, i, j = self.leaves[c]
        hx = self.Lx / (self.nx << l)
        hy = self.Ly / (self.ny << l)
        return (-0.5 * self.Lx + i * hx, hx, -0.5 * self.Ly + j * hy, hy, l)

    def _build_elements(self):
        N, nz = self.N, self.nz
        n1 = N + 1
        self.P = n1 ** 3
        self.Ncol = len(self.leaves)
        self.Ne = self.Ncol * nz
        ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1),
                                 indexing="ij")
        # local index l = i + (N+1)(j + (N+1)k)  (Sec. 3)
        li = np.zeros(self.P, dtype=np.int64)
        lj = np.zeros(self.P, dtype=np.int64)
        lk = np.zeros(self.P, dtype=np.int64)
        for i in range(n1):
            for j in range(n1):
                for k in range(n1):
                    l = i + n1 * (j + n1 * k)
                    li[l], lj[l], lk[l] = i, j, k
        self.li, self.lj, self.lk = li, lj, lk
        X = np.zeros((self.Ne, self.P, 3))
        box = np.zeros((self.Ne, 6))
        level = np.zeros(self.Ne, dtype=np.int64)
        col = np.zeros(self.Ne, dtype=np.int64)
        layer = np.zeros(self.Ne, dtype=np.int64)
        for c in range(self.Ncol):
            x0, hx, y0, hy, l = self.column_box(c)
            for k in range(nz):
                e = c * nz + k
                z0, hz = self.zf[k], self.hzk[k]
                X[e, :, 0] = x0 + 0.5 * (1.0 + self.xi[li]) * hx
                X[e, :, 1] = y0 + 0.5 * (1.0 + self.xi[lj]) * hy
                X[e, :, 2] = z0 + 0.5 * (1.0 + self.xi[lk]) * hz
                box[e] = (x0, hx, y0, hy, z0, hz)
                level[e], col[e], layer[e] = l, c, k
        self.X, self.box, self.level, self.col, self.layer = X, box, level, col, layer
        w = self.w
        # quadrature weight times Jacobian at every local node: w_i w_j w_k J
        J = box[:, 1] * box[:, 3] * box[:, 5] / 8.0
        self.wJ = (w[li] * w[lj] * w[lk])[None, :] * J[:, None]

    # ------------------------------------------------------------------
    def _wrap(self, pts):
        """Map periodic coordinates into [-L/2, L/2)."""
        pts = pts.copy()
        for d, L in ((0, self.Lx), (1, self.Ly)):
            if self.periodic[d]:
                v = pts[..., d] + 0.5 * L
                v = v - np.floor(v / L) * L
                v = np.where(np.abs(v - L) < 1e-9 * L, 0.0, v)
                v = np.where(np.abs(v) < 1e-9 * L, 0.0, v)
                pts[..., d] = v - 0.5 * L
        return pts

    def _ref_coord(self, x, x0, h):
        """Reference coordinate of x in [x0, x0+h], snapped onto the LGL nodes."""
        r = 2.0 * (x - x0) / h - 1.0
        for a in self.xi:
            r = np.where(np.abs(r - a) < 1e-11, a, r)
        return r

    def _build_global_nodes(self):
        N, nz = self.N, self.nz
        NL = self.Ne * self.P
        Xw = self._wrap(self.X.reshape(NL, 3))
        levels_l = np.repeat(self.level, self.P)
        # --- hanging detection: for each coarser column, the finer local nodes
        # inside its closed horizontal rectangle lie on its boundary ---------
        hang_of = -np.ones(NL, dtype=np.int64)       # coarse column index
        tol = 1e-9 * min(self.Lx, self.Ly)
        for c in range(self.Ncol):
            x0, hx, y0, hy, l = self.column_box(c)
            finer = np.nonzero(levels_l > l)[0]
            if finer.size == 0:
                continue
            p = Xw[finer]
            inside = np.ones(len(finer), dtype=bool)
            shifted = np.zeros((len(finer), 2))
            for d, (a0, h, L) in enumerate(((x0, hx, self.Lx), (y0, hy, self.Ly))):
                v = p[:, d]
                ok = (v >= a0 - tol) & (v <= a0 + h + tol)
                sh = np.zeros_like(v)
                if self.periodic[d]:
                    for s in (-L, L):
                        vs = v + s
                        oks = (vs >= a0 - tol) & (vs <= a0 + h + tol)
                        sh = np.where(~ok & oks, s, sh)
                        ok = ok | oks
                inside &= ok
                shifted[:, d] = v + sh
            idx = finer[inside]
            if idx.size == 0:
                continue
            rx = self._ref_coord(shifted[inside, 0], x0, hx)
            ry = self._ref_coord(shifted[inside, 1], y0, hy)
            on_x = np.isin(rx, self.xi)
            on_y = np.isin(ry, self.xi)
            hanging = ~(on_x & on_y)
            for q in idx[hanging]:
                if hang_of[q] >= 0 and hang_of[q] != c:
                    raise RuntimeError("node hangs on two coarser columns")
                hang_of[q] = c
        self.hang_of = hang_of
        # --- distinct positions of the non-hanging nodes -> global nodes ---
        free = np.nonzero(hang_of < 0)[0]
        scale = 1e-4  # metres; node spacings are kilometres
        keys = np.round(Xw[free] / scale).astype(np.int64)
        uniq, inv = np.unique(keys, axis=0, return_inverse=True)
        inv = inv.reshape(-1)
        NG = len(uniq)
        XG = np.zeros((NG, 3))
        XG[inv] = Xw[free]
        # guard against one position split across two rounding cells
        spread = np.abs(Xw[free] - XG[inv]).max() if free.size else 0.0
        if spread > 1e-6:
            raise RuntimeError("inconsistent node coordinates")
        order = np.lexsort((XG[:, 0], XG[:, 1], XG[:, 2]))
        XG = XG[order]
        rank = np.empty(NG, dtype=np.int64)
        rank[order] = np.arange(NG)
        gid = -np.ones(NL, dtype=np.int64)
        gid[free] = rank[inv]
        self.NG, self.XG = NG, XG
        # --- rows of Q, hanging rows by (recursive) interpolation ---------
        rows = {}

        def row(q, depth=0):
            if depth > 8:
                raise RuntimeError("constraint chain too deep")
            if gid[q] >= 0:
                return {int(gid[q]): 1.0}
            if q in rows:
                return rows[q]
            c = hang_of[q]
            x0, hx, y0, hy, _ = self.column_box(c)
            pz = Xw[q, 2]
            k = min(max(int(np.searchsorted(self.zf, pz, side="right")) - 1, 0), nz - 1)
            e = c * nz + k
            pxy = Xw[q, :2].copy()
            for d, (a0, h, L) in enumerate(((x0, hx, self.Lx), (y0, hy, self.Ly))):
                if self.periodic[d]:
                    for s in (0.0, -L, L):
                        if a0 - tol <= pxy[d] + s <= a0 + h + tol:
                            pxy[d] += s
                            break
            rx = self._ref_coord(np.array([pxy[0]]), x0, hx)
            ry = self._ref_coord(np.array([pxy[1]]), y0, hy)
            rz = self._ref_coord(np.array([pz]), self.zf[k], self.hzk[k])
            hx_ = basis.lagrange_eval(self.xi, rx)[0]
            hy_ = basis.lagrange_eval(self.xi, ry)[0]
            hz_ = basis.lagrange_eval(self.xi, rz)[0]
            out = {}
            for lc in range(self.P):
                v = hx_[self.li[lc]] * hy_[self.lj[lc]] * hz_[self.lk[lc]]
                if v == 0.0:
                    continue
                for g, wv in row(e * self.P + lc, depth + 1).items():
                    out[g] = out.get(g, 0.0) + v * wv
            rows[q] = out
            return out

        # non-hanging rows are unit vectors; only hanging rows need row()
        ri, ci, vv = [free], [gid[free]], [np.ones(free.size)]
        for q in np.nonzero(hang_of >= 0)[0]:
            items = [(g, v) for g, v in row(int(q)).items() if v != 0.0]
            ri.append(np.full(len(items), q))
            ci.append(np.array([g for g, _ in items], dtype=np.int64))
            vv.append(np.array([v for _, v in items]))
        ri, ci, vv = np.concatenate(ri), np.concatenate(ci), np.concatenate(vv)
        self.Q = sp.csr_matrix((vv, (ri, ci)), shape=(NL, NG))
        self.QT = self.Q.T.tocsr()
        self.gid = gid
        self.n_hanging = int(np.sum(hang_of >= 0))
        # lumped global mass, built through the same Q^T (Sec. 3.1)
        self.M = self.QT @ self.wJ.reshape(NL)
        self.z_bottom = np.abs(XG[:, 2]) < 1e-9 * self.Lz
        self.z_top = np.abs(XG[:, 2] - self.Lz) < 1e-9 * self.Lz

    # ------------------------------------------------------------------
    def warp_height(self, x, y, zeta):
        """Height of the point (x, y, zeta) of the box under the warp."""
        A, kx, ky = self.warp
        return zeta + A * (np.sin(2 * np.pi * kx * (x + 0.5 * self.Lx) / self.Lx)
                           * np.sin(2 * np.pi * ky * (y + 0.5 * self.Ly) / self.Ly)
                           * np.sin(np.pi * zeta / self.Lz))

    def _apply_warp(self):
        """Heights of the global nodes from the warp, local heights Q z_G, and
        the isoparametric metric at every local node of every element."""
        self.XG_box = self.XG.copy()
        self.XG = self.XG.copy()
        self.XG[:, 2] = self.warp_height(self.XG[:, 0], self.XG[:, 1], self.XG[:, 2])
        self.X = self.X.copy()
        self.X[:, :, 2] = (self.Q @ self.XG[:, 2]).reshape(self.Ne, self.P)
        D = basis.derivative_matrix(self.N)
        I = np.eye(self.N + 1)
        Dref = (np.kron(I, np.kron(I, D)), np.kron(I, np.kron(D, I)), np.kron(D, np.kron(I, I)))
        self.G_elem = np.zeros((self.Ne, 3, self.P, self.P))
        w3 = self.w[self.li] * self.w[self.lj] * self.w[self.lk]
        self.detJ = np.zeros((self.Ne, self.P))
        for e in range(self.Ne):
            # Jm[k, d, i] = d x_d / d xi_i at node k
            Jm = np.stack([np.stack([Dref[i] @ self.X[e, :, d] for i in range(3)], axis=1)
                           for d in range(3)], axis=1)
            det = np.linalg.det(Jm)
            if np.any(det <= 0):
                raise ValueError("the warp folds an element (non-positive Jacobian)")
            inv = np.linalg.inv(Jm)          # inv[k, i, d] = d xi_i / d x_d
            for d in range(3):
                self.G_elem[e, d] = sum(inv[:, i, d][:, None] * Dref[i] for i in range(3))
            self.detJ[e] = det
        self.wJ = w3[None, :] * self.detJ
        NL = self.Ne * self.P
        self.M = self.QT @ self.wJ.reshape(NL)
        self.z_bottom = np.abs(self.XG[:, 2]) < 1e-9 * self.Lz
        self.z_top = np.abs(self.XG[:, 2] - self.Lz) < 1e-9 * self.Lz

    # ------------------------------------------------------------------
    def to_local(self, qG):
        """Scatter: q_L = Q q_G.  qG: (F, NG) -> (F, Ne, P)."""
        qG = np.atleast_2d(qG)
        return np.stack([self.Q @ f for f in qG]).reshape(len(qG), self.Ne, self.P)

    def assemble(self, rL):
        """Gather: R_G = Q^T r_L.  rL: (F, Ne, P) -> (F, NG)."""
        return np.stack([self.QT @ f.reshape(-1) for f in rL])

    def element_ops(self, level, layer=0):
        """Dense derivative operators G_d[k, l] = d psi_l / d x_d at node k
        for the elements of a refinement level and a layer.

        For an axis-aligned element the map is affine, d xi / dx = 2 / hx, so
        G_x = (2/hx) I (x) I (x) D with D[m, i] = h_i'(xi_m), in the ordering
        l = i + (N+1)(j + (N+1)k) (i fastest); G_z has the layer's thickness.
        """
        l = level
        hx = self.Lx / (self.nx << l)
        hy = self.Ly / (self.ny << l)
        D = basis.derivative_matrix(self.N)
        I = np.eye(self.N + 1)
        Gx = (2.0 / hx) * np.kron(I, np.kron(I, D))
        Gy = (2.0 / hy) * np.kron(I, np.kron(D, I))
        Gz = (2.0 / self.hzk[layer]) * np.kron(D, np.kron(I, I))
        return Gx, Gy, Gz

    def op_groups(self):
        """(level, element indices, (G_x, G_y, G_z)) for every group of
        elements that share their derivative operators (level and layer);
        with a warp every element is its own group."""
        if self.warp is not None:
            for e in range(self.Ne):
                yield int(self.level[e]), np.array([e]), tuple(self.G_elem[e])
            return
        for lev in np.unique(self.level):
            for k in range(self.nz):
                es = np.nonzero((self.level == lev) & (self.layer == k))[0]
                if es.size:
                    yield int(lev), es, self.element_ops(int(lev), k)

    def column_levels(self):
        return np.array([l for l, _, _ in self.leaves], dtype=np.int64)
