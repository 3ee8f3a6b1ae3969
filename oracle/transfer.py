"""Solution transfer between meshes when columns are refined or coarsened.

The paper refines and coarsens marked elements (Algorithm 3) without stating
how the solution moves to the new mesh.  The reading used here:
* a refined element's children take the parent's polynomial evaluated at their
  nodes (interpolation; exact, since the children's space contains it);
* a coarsened parent takes the L2 projection of its four children's
  polynomials onto its own space, M a = int psi_i q dV, integrated exactly
  (Gauss-Legendre with N+2 points per direction on every child);
* unchanged elements keep their local values;
* the new global values are the projection of the new element values onto
  the continuous, hanging-node-constrained space (Sec. 3.1), with the LGL
  quadrature as inner product:  (Q^T W Q) q_G = Q^T W q_L,  W = diag(w J).
  Q^T W Q is diagonal (= the lumped mass M) except between the coarse-face
  nodes that hanging rows of Q couple.
This reproduces every field that is already continuous (q_L = Q q_G'
gives q_G = q_G'), so refining a column changes nothing, and, because the
rows of Q sum to one, it keeps the lumped total sum_g M_g q_g = sum_l w_l J_l
q_l.  Interpolation and L2 projection both keep the integral of every field,
and LGL quadrature is exact for the degree-N polynomials involved, so the
lumped total of each field is unchanged by a transfer.  (A plain
mass-weighted average Q^T W q_L / M would also conserve, but it shifts a
continuous field at the coarse nodes of every 2:1 face.)

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import basis
from .mesh import OracleMesh


def _tensor_eval(xi, rx, ry, rz):
    """T[p, l] = psi_l at reference points (rx, ry, rz)[p]; l = i + n(j + n k)."""
    Hx = basis.lagrange_eval(xi, rx)
    Hy = basis.lagrange_eval(xi, ry)
    Hz = basis.lagrange_eval(xi, rz)
    n = len(xi)
    T = np.einsum("pk,pj,pi->pkji", Hz, Hy, Hx).reshape(len(rx), n ** 3)
    return T


def transfer(old, new_leaves, origin, qG_old):
    """Move the global state qG_old (F, NG_old) of mesh `old` to the new leaves."""
    new = OracleMesh(old.Lx, old.Ly, old.Lz, old.nx, old.ny, old.nz, old.N,
                     leaves=new_leaves, periodic=old.periodic, z_faces=old.zf)
    xi = old.xi
    nz, P = old.nz, old.P
    qL_old = old.to_local(qG_old)               # (F, Ne_old, P)
    F = qL_old.shape[0]
    qL_new = np.zeros((F, new.Ne, P))
    g, gw = basis.gauss_legendre(old.N + 2)
    GX, GY, GZ = np.meshgrid(g, g, g, indexing="ij")
    GW = (gw[:, None, None] * gw[None, :, None] * gw[None, None, :]).reshape(-1)
    gx, gy, gz = GX.reshape(-1), GY.reshape(-1), GZ.reshape(-1)
    for cn, org in enumerate(origin):
        for k in range(nz):
            en = cn * nz + k
            if org[0] == "same":
                qL_new[:, en] = qL_old[:, org[1] * nz + k]
            elif org[0] == "refine":
                _, c, a, b = org
                eo = c * nz + k
                x0, hx, y0, hy = old.box[eo][:4]
                X = new.X[en]
                rx = 2.0 * (X[:, 0] - x0) / hx - 1.0
                ry = 2.0 * (X[:, 1] - y0) / hy - 1.0
                rz = xi[new.lk]
                T = _tensor_eval(xi, rx, ry, rz)
                qL_new[:, en] = qL_old[:, eo] @ T.T
            else:
                sib = org[1]
                x0, hx, y0, hy, z0, hz = new.box[en]
                M1 = basis.exact_mass_matrix(old.N)
                M3 = np.kron(M1, np.kron(M1, M1)) * (hx * hy * hz / 8.0)
                rhs = np.zeros((F, P))
                for c in sib:
                    eo = c * nz + k
                    cx0, chx, cy0, chy, cz0, chz = old.box[eo]
                    Tc = _tensor_eval(xi, gx, gy, gz)           # child basis at its Gauss pts
                    vals = qL_old[:, eo] @ Tc.T                  # (F, nGauss)
                    px = cx0 + 0.5 * (1.0 + gx) * chx
                    py = cy0 + 0.5 * (1.0 + gy) * chy
                    Tp = _tensor_eval(xi, 2.0 * (px - x0) / hx - 1.0,
                                      2.0 * (py - y0) / hy - 1.0, gz)
                    Jc = chx * chy * chz / 8.0
                    rhs += (vals * (GW * Jc)[None, :]) @ Tp
                qL_new[:, en] = np.linalg.solve(M3, rhs.T).T
    return new, project_continuous(new, qL_new)


def project_continuous(mesh, qL):
    """Solve (Q^T W Q) q_G = Q^T W q_L for every field; qL (F, Ne, P)."""
    W = sp.diags(mesh.wJ.reshape(-1))
    A = (mesh.QT @ W @ mesh.Q).tocsc()
    b = mesh.assemble(qL * mesh.wJ[None])
    lu = spla.splu(A)
    return np.stack([lu.solve(bf) for bf in b])
