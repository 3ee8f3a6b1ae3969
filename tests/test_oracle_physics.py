"""Pins of the oracle's optional terms of the paper's runs (Sec. 4): the
Rayleigh absorbing layer and the horizontal Smagorinsky-Lilly stress.

Each pin is a property the discretisation must have, not a retyping of the
formula: closed-form tendencies of fields the element polynomials hold
exactly (they fix the factors 2 and sqrt(2), the gradient scale, the filter
width and the sign), the kinetic-energy identity of the weak stress
divergence (it fixes the pairing of fluxes with test-function gradients) and
the pointwise action of the lumped collocated sponge.
"""
import numpy as np
import pytest

from oracle import mesh, refstate, rhs
from synth.vortex import random_state
from tests.test_oracle_mesh import two_level_leaves

L, LZ = 300e3, 12e3


def visc_tendency(m, q, prm, eqset="C"):
    """Tendency of the added terms alone (rhs with them minus rhs without)."""
    off = refstate.Params(f=prm.f)
    return rhs.rhs(m, q, prm, eqset) - rhs.rhs(m, q, off, eqset)


def test_sponge_rate_profile():
    prm = refstate.Params(sponge_gamma=0.8, sponge_depth=4000.0)
    z = np.array([LZ, LZ - 2000.0, LZ - 4000.0, LZ - 6000.0, 0.0])
    R = rhs.sponge_rate(z, LZ, prm)
    # gamma sin^2(pi/2) at the lid, gamma sin^2(pi/4) half-way, zero at and
    # below the bottom of the layer (where the literal formula would rise again)
    np.testing.assert_allclose(R, [0.8, 0.4, 0.0, 0.0, 0.0], atol=1e-15)
    strong = refstate.Params(sponge_gamma=3.0)
    assert rhs.sponge_rate(np.array([LZ]), LZ, strong)[0] == 1.0     # clipped to 1


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_lumped_sponge_acts_pointwise_on_a_conforming_mesh(eqset):
    """A collocated source assembled with the lumped mass is the pointwise
    value at every global node: -R(z) q' for every field."""
    m = mesh.OracleMesh(L, L, LZ, 3, 3, 3, 4)
    prm = refstate.Params(sponge_gamma=0.01, sponge_depth=6000.0)
    q = random_state(m.XG, LZ, 3, eqset)
    T = visc_tendency(m, q, prm, eqset)
    expect = -rhs.sponge_rate(m.XG[:, 2], LZ, prm)[None, :] * q
    expect[3, m.z_bottom | m.z_top] = 0.0
    np.testing.assert_allclose(T, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())
    assert np.count_nonzero(expect[0]) > 0 and np.all(expect[:, m.XG[:, 2] < LZ - 6000.0] == 0.0)


def _interior(m, Ly=L):
    x, y = m.XG[:, 0], m.XG[:, 1]
    return (np.abs(np.abs(x) - L / 2) > 1.0) & (np.abs(np.abs(y) - Ly / 2) > 1.0)


def _polynomial_state(m, u, v, w):
    """Conservative state with rho' = 0, momentum rho0(z) times the velocity."""
    rho0 = refstate.reference_state(m.XG[:, 2], refstate.Params())["rho0"]
    q = np.zeros((5, m.NG))
    q[1], q[2], q[3] = rho0 * u, rho0 * v, rho0 * w
    return q, rho0


@pytest.mark.parametrize("nx", [3, 4])
def test_smagorinsky_closed_form_tendencies(nx):
    """Velocities of degree <= 2 in x, y: the stress flux is a polynomial the
    quadrature integrates exactly, so at interior nodes the tendency equals
    the analytic -div(rho tau) to round-off.  C_s is chosen so that
    C_s Delta = L0 with Delta = (hx + hy) / (2N)."""
    N, Ly = 4, 0.8 * L                   # hx != hy: Delta is their mean over N
    m = mesh.OracleMesh(L, Ly, LZ, nx, nx, 2, N, periodic=(False, False))
    L0 = 500.0
    prm = refstate.Params(f=0.0, smag_cs=L0 / ((L / nx + Ly / nx) / (2 * N)))
    x, y = m.XG[:, 0], m.XG[:, 1]
    inner = _interior(m, Ly) & ~(m.z_bottom | m.z_top)
    a, b = 2e-5, 1e-11                   # u_x = a + 2 b x > 0 on the box
    # 1. u = a x + b x^2: nu_t = sqrt(2) L0^2 u_x, d(rho u)/dt = 4 sqrt(2) rho0 L0^2 u_x u_xx
    q, rho0 = _polynomial_state(m, a * x + b * x ** 2, 0 * x, 0 * x)
    T = visc_tendency(m, q, prm)
    ux = a + 2 * b * x
    exp1 = 4 * np.sqrt(2) * rho0 * L0 ** 2 * ux * (2 * b)
    np.testing.assert_allclose(T[1, inner], exp1[inner], rtol=1e-9)
    assert np.abs(T[2:4, inner]).max() <= 1e-9 * np.abs(exp1).max()
    # 2. the same along y for v
    q, rho0 = _polynomial_state(m, 0 * y, a * y + b * y ** 2, 0 * y)
    T = visc_tendency(m, q, prm)
    exp2 = 4 * np.sqrt(2) * rho0 * L0 ** 2 * (a + 2 * b * y) * (2 * b)
    np.testing.assert_allclose(T[2, inner], exp2[inner], rtol=1e-9)
    # 3. shear u = c (y + L)^2: S_xy = c (y + L), nu_t = 2 L0^2 S_xy,
    #    d(rho u)/dt = d/dy (4 rho0 L0^2 S_xy^2) = 8 rho0 L0^2 c^2 (y + L)
    c = 1e-10
    q, rho0 = _polynomial_state(m, c * (y + L) ** 2, 0 * y, 0 * y)
    T = visc_tendency(m, q, prm)
    exp3 = 8 * rho0 * L0 ** 2 * c ** 2 * (y + L)
    np.testing.assert_allclose(T[1, inner], exp3[inner], rtol=1e-9)
    # the v equation sees d/dx of the same stress, which is zero
    assert np.abs(T[2, inner]).max() <= 1e-9 * np.abs(exp3).max()
    # 4. vertical velocity diffused by the horizontal viscosity of u = a x:
    #    w = d x^2, d(rho w)/dt = d/dx (rho0 nu_t 2 d x) = 2 sqrt(2) rho0 L0^2 a d
    d = 1e-10
    q, rho0 = _polynomial_state(m, a * x, 0 * x, d * x ** 2)
    T = visc_tendency(m, q, prm)
    exp4 = 2 * np.sqrt(2) * rho0 * L0 ** 2 * a * d
    np.testing.assert_allclose(T[3, inner], exp4[inner], rtol=1e-9)


def _energy_identity(m, q, prm, eqset):
    """Sum over global nodes of u . R_visc (assembled, before the lid rule)
    and the quadrature of -rho nu_t (2 S_h:S_h + |grad_h w|^2)."""
    off = refstate.Params(f=prm.f)
    qL = m.to_local(q)
    dr = rhs.element_residual(m, qL, prm, eqset) - rhs.element_residual(m, qL, off, eqset)
    R = m.assemble(dr)
    ref = refstate.reference_state(m.XG[:, 2], prm)
    if eqset == "C":
        rho = ref["rho0"] + q[0]
        vel = q[1:4] / rho
    else:
        vel = q[1:4]
    lhs = np.sum(vel * R[1:4])
    # right-hand side from element-local gradients
    refl = refstate.reference_state(m.X[:, :, 2], prm)
    rhsum = 0.0
    for lev, es, G in m.op_groups():
        if eqset == "C":
            rl = refl["rho0"][es] + qL[0, es]
            ul, vl, wl = qL[1, es] / rl, qL[2, es] / rl, qL[3, es] / rl
        else:
            rl = 1.0
            ul, vl, wl = qL[1, es], qL[2, es], qL[3, es]
        du = [ul @ G[dd].T for dd in range(2)]
        dv = [vl @ G[dd].T for dd in range(2)]
        dw = [wl @ G[dd].T for dd in range(2)]
        sxx, syy, sxy = du[0], dv[1], 0.5 * (du[1] + dv[0])
        ss = sxx ** 2 + syy ** 2 + 2 * sxy ** 2
        delta = (L / (m.nx << int(lev)) + L / (m.ny << int(lev))) / (2 * m.N)
        nut = (prm.smag_cs * delta) ** 2 * np.sqrt(2 * ss)
        rhsum += np.sum(m.wJ[es] * rl * nut * (2 * ss + dw[0] ** 2 + dw[1] ** 2))
    return lhs, -rhsum


@pytest.mark.parametrize("eqset,nc", [("C", False), ("NC", False), ("NC", True)])
def test_smagorinsky_energy_identity_and_dissipation(eqset, nc):
    """The weak stress divergence paired with the (continuous) velocity is
    minus the quadrature of rho nu_t (2 S_h:S_h + |grad_h w|^2) <= 0.  Holds
    on non-conforming meshes for the velocity set, where the velocity is the
    interpolated field itself."""
    m = (mesh.OracleMesh(L, L, LZ, 4, 4, 2, 4, leaves=two_level_leaves()) if nc
         else mesh.OracleMesh(L, L, LZ, 3, 3, 2, 4))
    prm = refstate.Params(smag_cs=0.21)
    q = random_state(m.XG, LZ, 8, eqset)
    lhs, rhs_ = _energy_identity(m, q, prm, eqset)
    assert rhs_ < 0.0
    assert abs(lhs - rhs_) <= 1e-10 * abs(rhs_)


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_physics_keep_mass_conservation_and_rest_state(eqset):
    m = mesh.OracleMesh(L, L, LZ, 4, 4, 2, 4, leaves=two_level_leaves())
    prm = refstate.Params(smag_cs=0.21, sponge_gamma=0.01)
    T = rhs.rhs(m, np.zeros((5, m.NG)), prm, eqset)
    assert np.all(T == 0.0)
    q = random_state(m.XG, LZ, 4, eqset)
    Tv = visc_tendency(m, q, refstate.Params(smag_cs=0.21), eqset)
    # the stress acts on momentum only
    assert np.all(Tv[0] == 0.0) and np.all(Tv[4] == 0.0)


# ---------------------------------------------------------------------------
# synthetic heating source and the stage times


def test_heating_rate_profile():
    prm = refstate.Params(heat_q0=0.005, time=1e6)
    zt, r0, rmax = prm.heat_ztop, prm.heat_r0, prm.heat_rmax
    Q = rhs.heating_rate(np.array([r0, 0.0, r0 + 1e3, rmax + 1.0, r0]),
                         np.array([0.0, r0, 0.0, 0.0, 0.0]),
                         np.array([zt / 2, zt / 2, zt / 2, zt / 2, zt + 1.0]), prm)
    ring = np.exp(-(1e3 / prm.heat_width) ** 2)
    np.testing.assert_allclose(Q, [0.005, 0.005, 0.005 * ring, 0.0, 0.0], rtol=1e-14, atol=1e-18)
    # the tanh ramp: nothing at t = 0, tanh(1) of the peak at t = tau
    assert rhs.heating_rate(np.array([r0]), np.array([0.0]), np.array([zt / 2]), prm.at(0.0))[0] == 0.0
    np.testing.assert_allclose(
        rhs.heating_rate(np.array([r0]), np.array([0.0]), np.array([zt / 2]), prm.at(prm.heat_ramp)),
        0.005 * np.tanh(1.0), rtol=1e-14)


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_lumped_heating_acts_pointwise_on_a_conforming_mesh(eqset):
    m = mesh.OracleMesh(200e3, 200e3, 18e3, 4, 4, 3, 4)
    prm = refstate.Params(heat_q0=0.004, time=900.0)
    T = rhs.rhs(m, np.zeros((5, m.NG)), prm, eqset)
    Q = rhs.heating_rate(m.XG[:, 0], m.XG[:, 1], m.XG[:, 2], prm)
    fac = refstate.reference_state(m.XG[:, 2], prm)["rho0"] if eqset == "C" else 1.0
    np.testing.assert_allclose(T[4], fac * Q, rtol=1e-12, atol=1e-15 * np.abs(fac * Q).max())
    assert np.all(T[:4] == 0.0) and np.count_nonzero(Q) > 0


def test_rk3_stage_times_integrate_quadratic_forcing_exactly():
    """SSP-RK3 with the stage times (t, t + dt, t + dt/2) is Simpson's rule on
    a pure forcing dq/dt = g(t), exact for quadratics."""
    from oracle.rk import step_generic
    t0, dt = 3.0, 0.7
    g = lambda q, t: 3.0 * t ** 2 - 2.0 * t + 1.0
    exact = (t0 + dt) ** 3 - (t0 + dt) ** 2 + (t0 + dt) - (t0 ** 3 - t0 ** 2 + t0)
    assert abs(step_generic(g, 0.0, dt, t0) - exact) <= 1e-13 * abs(exact)


def test_heating_enters_the_step_at_the_stage_times():
    """One short step from rest with the heating on: the theta change is the
    stage-time quadrature of the forcing (the dynamics answer at O(dt^2))."""
    from oracle.rk import rk_step
    m = mesh.OracleMesh(200e3, 200e3, 18e3, 4, 4, 3, 4)
    prm = refstate.Params(heat_q0=0.004, heat_ramp=0.05, time=0.01)
    dt = 0.02
    q1 = rk_step(m, prm, np.zeros((5, m.NG)), dt)
    rho0 = refstate.reference_state(m.XG[:, 2], prm)["rho0"]
    Qs = [rhs.heating_rate(m.XG[:, 0], m.XG[:, 1], m.XG[:, 2], prm.at(prm.time + c * dt)) for c in (0, 1, 0.5)]
    simpson = dt * (Qs[0] + Qs[1] + 4 * Qs[2]) / 6
    np.testing.assert_allclose(q1[4], rho0 * simpson, rtol=1e-5, atol=1e-5 * np.abs(rho0 * simpson).max())


# ---------------------------------------------------------------------------
# warped layers (non-affine elements): the same properties with the general
# isoparametric metric

WARP = (600.0, 1, 1)


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_warped_sponge_and_heating_act_pointwise_at_the_node_heights(eqset):
    """On a conforming warped mesh the lumped collocated sources are the
    pointwise values at each global node's own height (a level height in
    their place fails: the layer surfaces are curved)."""
    m = mesh.OracleMesh(L, L, LZ, 3, 3, 3, 4, warp=WARP)
    z = m.XG[:, 2]
    prm = refstate.Params(sponge_gamma=0.01, sponge_depth=6000.0)
    q = random_state(m.XG, LZ, 3, eqset)
    T = visc_tendency(m, q, prm, eqset)
    expect = -rhs.sponge_rate(z, LZ, prm)[None, :] * q
    expect[3, m.z_bottom | m.z_top] = 0.0
    np.testing.assert_allclose(T, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())
    # the curved layer surfaces put the nodes of one level at different
    # heights, inside the layer where the rate varies
    zb = m.XG_box[:, 2]
    level = np.abs(zb - zb[np.argmin(np.abs(zb - (LZ - 3000.0)))]) < 1e-6
    assert np.ptp(z[level]) > 100.0 and np.ptp(expect[0][level]) > 0.0
    hm = mesh.OracleMesh(200e3, 200e3, 18e3, 4, 4, 3, 4, warp=WARP)
    hp = refstate.Params(heat_q0=0.004, time=900.0)
    Th = rhs.rhs(hm, np.zeros((5, hm.NG)), hp, eqset)
    Q = rhs.heating_rate(hm.XG[:, 0], hm.XG[:, 1], hm.XG[:, 2], hp)
    fac = refstate.reference_state(hm.XG[:, 2], hp)["rho0"] if eqset == "C" else 1.0
    np.testing.assert_allclose(Th[4], fac * Q, rtol=1e-12, atol=1e-15 * np.abs(fac * Q).max())
    assert np.all(Th[:4] == 0.0) and np.count_nonzero(Q) > 0


@pytest.mark.parametrize("eqset,nc", [("C", False), ("NC", False), ("NC", True)])
def test_warped_smagorinsky_energy_identity_and_dissipation(eqset, nc):
    """The stress's energy identity with horizontal gradients taken at
    constant height through the warped metric: it fixes the pairing of the
    horizontal fluxes with the zeta derivatives of the test functions."""
    m = (mesh.OracleMesh(L, L, LZ, 4, 4, 2, 4, leaves=two_level_leaves(), warp=WARP) if nc
         else mesh.OracleMesh(L, L, LZ, 3, 3, 2, 4, warp=WARP))
    prm = refstate.Params(smag_cs=0.21)
    q = random_state(m.XG, LZ, 8, eqset)
    lhs, rhs_ = _energy_identity(m, q, prm, eqset)
    assert rhs_ < 0.0
    assert abs(lhs - rhs_) <= 1e-10 * abs(rhs_)


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_warped_physics_keep_mass_conservation_and_rest_state(eqset):
    m = mesh.OracleMesh(L, L, LZ, 4, 4, 2, 4, leaves=two_level_leaves(), warp=WARP)
    prm = refstate.Params(smag_cs=0.21, sponge_gamma=0.01)
    assert np.all(rhs.rhs(m, np.zeros((5, m.NG)), prm, eqset) == 0.0)
    q = random_state(m.XG, LZ, 4, eqset)
    Tv = visc_tendency(m, q, refstate.Params(smag_cs=0.21), eqset)
    assert np.all(Tv[0] == 0.0) and np.all(Tv[4] == 0.0)
    assert np.abs(Tv[1:4]).max() > 0.0
