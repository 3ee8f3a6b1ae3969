"""Pins of the oracle's brute-force mesh and hanging-node constraint Q (Sec. 3.1)."""
import numpy as np
import pytest

from oracle import basis, mesh
from oracle.transfer import _tensor_eval


def ring_leaves(nx, ny, ci, cj):
    """Base nx x ny with column (ci, cj) refined once."""
    out = [(0, i, j) for j in range(ny) for i in range(nx) if (i, j) != (ci, cj)]
    out += [(1, 2 * ci + a, 2 * cj + b) for b in (0, 1) for a in (0, 1)]
    return out


def two_level_leaves():
    """4x4 base, 2x2 block refined once, one of its children refined again."""
    leaves = []
    for j in range(4):
        for i in range(4):
            if 1 <= i <= 2 and 1 <= j <= 2:
                continue
            leaves.append((0, i, j))
    for j in range(2, 6):
        for i in range(2, 6):
            if (i, j) == (3, 3):
                continue
            leaves.append((1, i, j))
    leaves += [(2, 6 + a, 6 + b) for b in (0, 1) for a in (0, 1)]
    return leaves


@pytest.mark.parametrize("N", [2, 3, 4])
def test_uniform_counts(N):
    m = mesh.OracleMesh(60e3, 40e3, 10e3, 3, 2, 2, N)
    assert m.NG == (3 * N) * (2 * N) * (2 * N + 1)
    assert m.n_hanging == 0
    m2 = mesh.OracleMesh(60e3, 40e3, 10e3, 3, 2, 2, N, periodic=(False, False))
    assert m2.NG == (3 * N + 1) * (2 * N + 1) * (2 * N + 1)


def test_hanging_count_single_refined_column():
    N, nz = 4, 2
    m = mesh.OracleMesh(300e3, 300e3, 12e3, 3, 3, nz, N, leaves=ring_leaves(3, 3, 1, 1))
    # 4 sides x 2 fine elements x (N+1-2 positions off coarse nodes) x (N+1) z x nz
    assert m.n_hanging == 4 * 2 * (N - 1) * (N + 1) * nz
    np.testing.assert_allclose(np.asarray(m.Q.sum(axis=1)).ravel(), 1.0, atol=1e-14)


@pytest.mark.parametrize("N", [3, 4])
@pytest.mark.parametrize("leaves_fn", ["ring", "two_level"])
def test_Q_reproduces_global_polynomials(N, leaves_fn):
    """Non-periodic mesh: Q applied to a degree-N global polynomial gives its
    values at every local node, hanging ones included."""
    if leaves_fn == "ring":
        nx, leaves = 3, ring_leaves(3, 3, 1, 1)
    else:
        nx, leaves = 4, two_level_leaves()
    m = mesh.OracleMesh(80e3, 80e3, 10e3, nx, nx, 2, N, leaves=leaves,
                        periodic=(False, False))
    rng = np.random.default_rng(7)
    C = rng.normal(size=(N + 1, N + 1, 2))

    def f(X):
        x, y, z = X[..., 0] / 40e3, X[..., 1] / 40e3, X[..., 2] / 10e3
        out = np.zeros_like(x)
        for a in range(N + 1):
            for b in range(N + 1):
                out += C[a, b, 0] * x ** a * y ** b + C[a, b, 1] * x ** b * z ** a
        return out

    qL = m.to_local(f(m.XG))[0]
    np.testing.assert_allclose(qL, f(m.X), rtol=0, atol=1e-11 * np.abs(f(m.X)).max())
    # a degree N+1 polynomial is not reproduced at hanging nodes
    g = lambda X: (X[..., 0] / 40e3) ** (N + 1) + (X[..., 1] / 40e3) ** (N + 1)
    qL = m.to_local(g(m.XG))[0]
    assert np.abs(qL - g(m.X)).max() > 1e-8


def test_Q_makes_field_continuous_across_2to1_faces():
    """For random global values, each element's polynomial and its neighbour's
    agree on the shared (non-conforming) faces: sample points on every face of
    every fine element and evaluate from both sides."""
    N = 4
    m = mesh.OracleMesh(80e3, 80e3, 10e3, 4, 4, 2, N, leaves=two_level_leaves())
    rng = np.random.default_rng(3)
    qL = m.to_local(rng.normal(size=m.NG))[0]
    xi = m.xi
    worst = 0.0
    t = rng.uniform(-1, 1, size=(12, 2))
    for e in range(m.Ne):
        x0, hx, y0, hy, z0, hz = m.box[e]
        for side in range(4):
            s, u = t[:, 0], t[:, 1]
            if side < 2:
                px = np.full_like(s, x0 + (hx if side else 0.0))
                py = y0 + 0.5 * (1 + s) * hy
            else:
                py = np.full_like(s, y0 + (hy if side == 3 else 0.0))
                px = x0 + 0.5 * (1 + s) * hx
            pz = z0 + 0.5 * (1 + u) * hz
            Te = _tensor_eval(xi, 2 * (px - x0) / hx - 1, 2 * (py - y0) / hy - 1, u)
            mine = Te @ qL[e]
            # the neighbour containing a point just outside the face
            eps = 1e-3
            qx = px + (eps if side == 1 else -eps if side == 0 else 0.0)
            qy = py + (eps if side == 3 else -eps if side == 2 else 0.0)
            for p in range(len(s)):
                X = (qx[p] + 40e3) % 80e3 - 40e3
                Y = (qy[p] + 40e3) % 80e3 - 40e3
                for e2 in range(m.Ne):
                    a0, ahx, b0, bhy, c0, chz = m.box[e2]
                    if a0 <= X <= a0 + ahx and b0 <= Y <= b0 + bhy and c0 <= pz[p] <= c0 + chz:
                        # evaluate e2 at the face point (wrapped into e2's frame)
                        fx = px[p] + (X - qx[p])
                        fy = py[p] + (Y - qy[p])
                        T2 = _tensor_eval(xi, [2 * (fx - a0) / ahx - 1], [2 * (fy - b0) / bhy - 1],
                                          [2 * (pz[p] - c0) / chz - 1])
                        worst = max(worst, abs(float((T2 @ qL[e2])[0]) - mine[p]))
                        break
    assert worst < 1e-11


def test_lumped_mass_is_volume():
    m = mesh.OracleMesh(80e3, 80e3, 10e3, 4, 4, 2, 4, leaves=two_level_leaves())
    assert abs(m.M.sum() - 80e3 * 80e3 * 10e3) < 1e-9 * 80e3 * 80e3 * 10e3
    assert np.all(m.M > 0)


def test_tiling_validation():
    with pytest.raises(ValueError):
        mesh.OracleMesh(80e3, 80e3, 10e3, 2, 2, 1, 4,
                        leaves=[(0, 0, 0), (0, 1, 0), (0, 0, 1)])
