"""Pins of the oracle's right-hand side (Eqs. mass_split..ent_split, Sec. 3)."""
import numpy as np
import pytest
import sympy as sy

from oracle import mesh, refstate, rhs
from oracle.rk import step_generic
from synth.vortex import vortex_state, random_state
from tests.test_oracle_mesh import two_level_leaves

PRM = refstate.Params()


def small_nc_mesh():
    return mesh.OracleMesh(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=two_level_leaves())


@pytest.mark.parametrize("eqset", ["C", "NC"])
@pytest.mark.parametrize("nc", [False, True])
def test_rest_state_is_exactly_steady(eqset, nc):
    m = small_nc_mesh() if nc else mesh.OracleMesh(300e3, 300e3, 12e3, 3, 3, 2, 4)
    T = rhs.rhs(m, np.zeros((5, m.NG)), PRM, eqset)
    assert np.all(T == 0.0)


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_free_stream_preserved_on_nonconforming_mesh(eqset):
    m = small_nc_mesh()
    prm = refstate.Params(f=0.0)
    ref = refstate.reference_state(m.XG[:, 2], prm)
    q = np.zeros((5, m.NG))
    if eqset == "C":
        q[1], q[2] = 7.0 * ref["rho0"], -3.0 * ref["rho0"]
    else:
        q[1], q[2] = 7.0, -3.0
    T = rhs.rhs(m, q, prm, eqset)
    scale = np.abs(rhs.rhs(m, random_state(m.XG, 12e3, 1, eqset), prm, eqset)).max(axis=1)
    assert np.all(np.abs(T).max(axis=1) <= 1e-12 * scale)


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_mass_conserved_to_roundoff_across_2to1_faces(eqset):
    m = small_nc_mesh()
    T = rhs.rhs(m, random_state(m.XG, 12e3, 2, eqset), PRM, eqset)
    tot = np.sum(m.M * T[0])
    assert abs(tot) <= 1e-13 * np.sum(np.abs(m.M * T[0]))
    if eqset == "C":  # (rho theta)' is conserved too
        assert abs(np.sum(m.M * T[4])) <= 1e-13 * np.sum(np.abs(m.M * T[4]))


def test_weak_equals_assembled_strong_divergence_on_conforming_mesh():
    """On a conforming periodic mesh, summation by parts makes the assembled
    weak divergence equal to the mass-weighted average of the element-wise
    strong divergence (the face terms of a continuous flux cancel)."""
    m = mesh.OracleMesh(300e3, 300e3, 12e3, 3, 3, 3, 4)
    q = random_state(m.XG, 12e3, 5)
    T = rhs.rhs(m, q, PRM, "C")
    qL = m.to_local(q)
    G = m.element_ops(0)
    div = sum(qL[1 + d] @ G[d].T for d in range(3))        # strong d(rho u_d)/dx_d
    strong = m.assemble((m.wJ * div)[None])[0] / m.M
    np.testing.assert_allclose(T[0], -strong, atol=1e-12 * np.abs(strong).max())


def _mms(eqset, n, N=4, stretch=0.0, warp=None):
    """Max relative error of the oracle tendency against the exact one for a
    smooth periodic manufactured state on an n x n x n mesh (layer faces
    stretched by tests.helpers.stretched_faces when stretch > 0; warped
    layers, OracleMesh's warp, when warp is given)."""
    Lx, Lz = 40e3, 10e3
    x, y, z = sy.symbols("x y z", real=True)
    g, f, gam = PRM.g, PRM.f, PRM.gamma
    N2 = PRM.N_bv ** 2
    th0 = PRM.theta_s * sy.exp(N2 * z / g)
    pi0 = 1 + g * g / (PRM.c_p * PRM.theta_s * N2) * (sy.exp(-N2 * z / g) - 1)
    p0 = PRM.p00 * pi0 ** (PRM.c_p / PRM.R_d)
    rho0 = PRM.p00 * pi0 ** (PRM.c_v / PRM.R_d) / (PRM.R_d * th0)
    kx = 2 * sy.pi / Lx
    s = sy.sin(sy.pi * z / Lz)
    rp = 1e-3 * sy.sin(kx * x) * sy.cos(kx * y) * sy.cos(sy.pi * z / Lz)
    u = 10 * sy.cos(kx * x) * sy.sin(kx * y) + 3
    v = -8 * sy.sin(kx * x + 0.3) * sy.cos(kx * y) + 2
    w = 0.5 * sy.sin(kx * (x + y)) * s
    thp = 0.5 * sy.cos(kx * x) * sy.cos(kx * y - 0.2) * (1 + z / Lz)
    rho = rho0 + rp
    rtp = rho0 * thp + rp * (th0 + thp)
    pp = p0 * ((1 + rtp / (rho0 * th0)) ** gam - 1)
    div = lambda F: sy.diff(F[0], x) + sy.diff(F[1], y) + sy.diff(F[2], z)
    if eqset == "C":
        U, V, W = rho * u, rho * v, rho * w
        rt = rho0 * th0 + rtp
        state = [rp, U, V, W, rtp]
        tend = [-div((U, V, W)),
                -div((U * u + pp, U * v, U * w)) + f * V,
                -div((V * u, V * v + pp, V * w)) - f * U,
                -div((W * u, W * v, W * w + pp)) - rp * g,
                -div((rt * u, rt * v, rt * w))]
    else:
        adv = lambda q: u * sy.diff(q, x) + v * sy.diff(q, y) + w * sy.diff(q, z)
        state = [rp, u, v, w, thp]
        tend = [-div((rho * u, rho * v, rho * w)),
                -adv(u) - sy.diff(pp, x) / rho + f * v,
                -adv(v) - sy.diff(pp, y) / rho - f * u,
                -adv(w) - sy.diff(pp, z) / rho - rp / rho * g,
                -w * sy.diff(th0, z) - adv(thp)]
    from tests.helpers import stretched_faces
    m = mesh.OracleMesh(Lx, Lx, Lz, n, n, n, N,
                        z_faces=stretched_faces(Lz, n, stretch) if stretch > 0 else None, warp=warp)
    X = m.XG
    ev = lambda e: np.broadcast_to(sy.lambdify((x, y, z), e, "numpy")(X[:, 0], X[:, 1], X[:, 2]),
                                   (m.NG,)).astype(float)
    q = np.stack([ev(e) for e in state])
    Tx = np.stack([ev(e) for e in tend])
    T = rhs.rhs(m, q, PRM, eqset)
    lid = m.z_bottom | m.z_top
    err = []
    for k in range(5):
        sel = ~lid if k == 3 else np.ones(m.NG, bool)
        d, r, wm = T[k][sel] - Tx[k][sel], Tx[k][sel], m.M[sel]
        err.append(np.sqrt(np.sum(wm * d * d) / np.sum(wm * r * r)))
    return np.array(err)


@pytest.mark.slow
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_manufactured_solution_convergence(eqset):
    """Mass-weighted L2 error of every tendency against the exact one falls at
    about the order of the basis (N = 4) when the mesh is halved."""
    e4, e8 = _mms(eqset, 4), _mms(eqset, 8)
    rate = np.log2(e4 / e8)
    assert np.all(e8 < 1e-3), e8
    assert np.all(rate >= 3.5), rate


def test_rk3_stability_polynomial():
    for lam_dt in [-0.3, -1.0 + 0.5j, 0.7j, -2.4]:
        got = step_generic(lambda q: lam_dt * q, np.complex128(1.0), 1.0)
        zz = lam_dt
        assert abs(got - (1 + zz + zz ** 2 / 2 + zz ** 3 / 6)) < 1e-15


def test_rk_step_keeps_rest_and_conserves_mass():
    from oracle.rk import rk_step
    m = small_nc_mesh()
    q = vortex_state(m.XG, 12e3)
    q1 = rk_step(m, PRM, q, 1.0)
    assert abs(np.sum(m.M * (q1[0] - q[0]))) <= 1e-13 * np.sum(m.M * np.abs(q[0]))
    assert np.all(rk_step(m, PRM, np.zeros_like(q), 1.0) == 0.0)
