"""Pins of the oracle's alternative criterion variables (Sec. 3.1's C^l; the
vorticity and potential-vorticity candidates the paper names in Sec. 1 and
Sec. 5): closed forms for rigid rotation in the stratified reference state,
the vortex's prescribed peak vorticity, and the per-level choice of variable.
"""
import numpy as np
import pytest

from oracle import adapt, mesh, refstate
from synth.vortex import VortexSpec, vortex_state, gaussian_vortex_scale
from tests.test_oracle_mesh import two_level_leaves

PRM = refstate.Params()


def rotation_state(m, omega, eqset="C"):
    """Rigid rotation u = -omega y, v = omega x in the reference state."""
    ref = refstate.reference_state(m.XG[:, 2], PRM)
    x, y = m.XG[:, 0], m.XG[:, 1]
    q = np.zeros((5, m.NG))
    fac = ref["rho0"] if eqset == "C" else 1.0
    q[1], q[2] = -omega * y * fac, omega * x * fac
    return q


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_rigid_rotation_vorticity_and_pv(eqset):
    m = mesh.OracleMesh(300e3, 300e3, 12e3, 3, 3, 2, 4, periodic=(False, False))
    om = 3e-5
    q = rotation_state(m, om, eqset)
    zeta = adapt.criterion_vorticity(m, q, PRM, eqset)
    np.testing.assert_allclose(zeta, 2 * om, rtol=1e-9)
    # PV = (2 omega + f) dtheta0/dz / rho0, theta0 = theta_s exp(N^2 z / g)
    ref = refstate.reference_state(m.X[:, :, 2], PRM)
    pv_exact = (2 * om + PRM.f) * ref["dtheta0"] / ref["rho0"]
    pv = adapt.criterion_pv(m, q, PRM, eqset)
    np.testing.assert_allclose(pv, pv_exact, rtol=1e-6)
    # extra stratification theta' = a z (conservative set: (rho theta)' = rho0 a z)
    a = 2e-3
    q2 = q.copy()
    q2[4] = a * m.XG[:, 2] * (refstate.reference_state(m.XG[:, 2], PRM)["rho0"] if eqset == "C" else 1.0)
    pv2 = adapt.criterion_pv(m, q2, PRM, eqset)
    np.testing.assert_allclose(pv2, (2 * om + PRM.f) * (ref["dtheta0"] + a) / ref["rho0"], rtol=1e-6)
    # rest state: only the planetary vorticity
    pv0 = adapt.criterion_pv(m, np.zeros((5, m.NG)), PRM, eqset)
    np.testing.assert_allclose(pv0, PRM.f * ref["dtheta0"] / ref["rho0"], rtol=1e-6)
    assert np.all(adapt.criterion_vorticity(m, np.zeros((5, m.NG)), PRM, eqset) == 0.0)


def test_vortex_peak_vorticity():
    """The vortex's surface vorticity peak (the Gaussian's amplitude, fixed by
    v_max = 20 m/s at 50 km) is what the criterion sees at the centre."""
    spec = VortexSpec(noise_K=0.0)
    zeta0 = gaussian_vortex_scale(spec.vmax, spec.rmw)[1]
    m = mesh.OracleMesh(800e3, 800e3, 24e3, 24, 24, 2, 4)   # taper at 200 km far from the edge
    q = vortex_state(m.XG, 24e3, spec)
    zeta = adapt.criterion_vorticity(m, q, PRM)
    near = (np.hypot(m.X[:, :, 0], m.X[:, :, 1]) < 1.0) & (m.X[:, :, 2] < 1.0)
    assert near.any()
    np.testing.assert_allclose(zeta[near], zeta0, rtol=0.02)
    assert abs(zeta.max() - zeta0) <= 0.03 * zeta0


def test_per_level_variables():
    """threshold(l+1) is compared with variables[l]: a level-0 element follows
    the speed, a level-1 element refines by vorticity and coarsens by speed."""
    m = mesh.OracleMesh(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=two_level_leaves())
    q = vortex_state(m.XG, 12e3, VortexSpec(noise_K=0.0))
    s = adapt.criterion_speed(m, q, PRM).max(axis=1)
    z = adapt.criterion_vorticity(m, q, PRM).max(axis=1)
    thr = [5.0, 5e-4]
    fl, cmax = adapt.criterion_flags(m, q, PRM, thr, 2, variables=["speed", "vorticity"])
    for e in range(m.Ne):
        lv = m.level[e]
        if lv == 0:
            want = 1 if s[e] > thr[0] else 0
            assert cmax[e] == s[e]
        else:
            want = 1 if (lv < 2 and z[e] > thr[1]) else (-1 if s[e] <= thr[0] else 0)
        assert fl[e] == want, e
    assert set(np.unique(fl[m.level == 1])) >= {1} or set(np.unique(fl[m.level == 1])) >= {-1}
    # all-speed default unchanged
    f0, c0 = adapt.criterion_flags(m, q, PRM, [5.0, 10.0], 2)
    f1, c1 = adapt.criterion_flags(m, q, PRM, [5.0, 10.0], 2, variables=["speed", "speed"])
    assert np.array_equal(f0, f1) and np.array_equal(c0, c1)


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_warped_vorticity_is_taken_at_constant_height(eqset):
    """On warped layers u = -omega y + a z, v = omega x + b z: the vertical
    vorticity at constant height is exactly 2 omega, which holds only if the
    horizontal derivatives carry the metric's correction -(z_xi / z_zeta)
    d/dzeta (without it the shear a, b leaks in through the tilted layers).
    The rigid rotation's potential vorticity (2 omega + f) dtheta0/dz / rho0
    holds to 2e-4: the exponential theta0 is interpolated along curved
    elements."""
    m = mesh.OracleMesh(300e3, 300e3, 12e3, 3, 3, 2, 4, periodic=(False, False), warp=(600.0, 1, 1))
    om, a, b = 3e-5, 2e-3, -1e-3
    ref = refstate.reference_state(m.XG[:, 2], PRM)
    x, y, z = m.XG[:, 0], m.XG[:, 1], m.XG[:, 2]
    fac = ref["rho0"] if eqset == "C" else 1.0
    q = np.zeros((5, m.NG))
    q[1], q[2] = (-om * y + a * z) * fac, (om * x + b * z) * fac
    zeta = adapt.criterion_vorticity(m, q, PRM, eqset)
    np.testing.assert_allclose(zeta, 2 * om, rtol=1e-9)
    # without the shear the potential vorticity has the rigid-rotation value
    qr = rotation_state(m, om, eqset)
    refl = refstate.reference_state(m.X[:, :, 2], PRM)
    np.testing.assert_allclose(adapt.criterion_pv(m, qr, PRM, eqset),
                               (2 * om + PRM.f) * refl["dtheta0"] / refl["rho0"], rtol=2e-4)
