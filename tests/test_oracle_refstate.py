"""Pins of the oracle's hydrostatic reference state (Sec. 2, eqs. rho_split,
theta_split, p_split and hydro_bal) against what the physics fixes, not
against its own closed forms:

- the hydrostatic balance dp0/dz = -rho0 g, checked by central differences
  of the oracle's p0 at several heights (a wrong exponent in rho0 or p0, a
  wrong sign in pi0, or a wrong scale height fails it);
- the ideal gas law p = rho R_d T with T = theta pi and the Exner function
  pi = (p / p00)^(R_d / c_p), evaluated from the oracle's p0, rho0 and theta0
  (the equation of state of Sec. 2);
- the buoyancy frequency: (g / theta0) dtheta0/dz = N_bv^2 at every height
  (central differences), and the table's dtheta0/dz against the same
  difference;
- the surface values theta0(0) = theta_s, pi0(0) = 1, p0(0) = p00, and a
  positive Exner pressure up to the top of the deepest box (24 km);
- the pressure perturbation p' against p00 (R_d rho theta / p00)^gamma - p0
  evaluated directly in extended precision.
"""
import numpy as np
import pytest

from oracle import refstate

PRM = refstate.Params()
Z = np.array([0.0, 250.0, 1000.0, 5000.0, 11000.0, 17500.0, 23500.0])


def _fd(fun, z, h):
    """Fourth-order central difference of fun at z with step h."""
    return (-fun(z + 2 * h) + 8 * fun(z + h) - 8 * fun(z - h) + fun(z - 2 * h)) / (12 * h)


@pytest.mark.parametrize("prm", [PRM, refstate.Params(theta_s=290.0, N_bv=0.012),
                                 refstate.Params(R_d=287.05, c_p=1005.7, p00=1.0e5, g=9.80665)])
def test_hydrostatic_balance_by_finite_differences(prm):
    zc = Z[1:]                       # keep z - 2h >= 0
    dp = _fd(lambda z: refstate.reference_state(z, prm)["p0"], zc, 50.0)
    rho0 = refstate.reference_state(zc, prm)["rho0"]
    np.testing.assert_allclose(dp, -rho0 * prm.g, rtol=1e-8)


@pytest.mark.parametrize("prm", [PRM, refstate.Params(theta_s=290.0, N_bv=0.012)])
def test_ideal_gas_law_and_exner_function(prm):
    r = refstate.reference_state(Z, prm)
    T0 = r["theta0"] * r["pi0"]
    np.testing.assert_allclose(r["p0"], r["rho0"] * prm.R_d * T0, rtol=1e-13)
    np.testing.assert_allclose(r["pi0"], (r["p0"] / prm.p00) ** (prm.R_d / prm.c_p), rtol=1e-13)
    np.testing.assert_allclose(r["rhotheta0"], r["rho0"] * r["theta0"], rtol=1e-15)


def test_buoyancy_frequency_and_theta_gradient():
    zc = Z[1:]
    th = lambda z: refstate.reference_state(z, PRM)["theta0"]
    dth = _fd(th, zc, 50.0)
    np.testing.assert_allclose(PRM.g / th(zc) * dth, PRM.N_bv ** 2, rtol=1e-9)
    np.testing.assert_allclose(refstate.reference_state(zc, PRM)["dtheta0"], dth, rtol=1e-9)


def test_surface_values_and_positive_exner_pressure():
    r = refstate.reference_state(np.array([0.0]), PRM)
    assert r["theta0"][0] == PRM.theta_s
    assert r["pi0"][0] == 1.0
    assert abs(r["p0"][0] - PRM.p00) <= 1e-12 * PRM.p00
    top = refstate.reference_state(np.array([24e3]), PRM)
    # 1 + g^2/(c_p theta_s N^2) (exp(-N^2 z/g) - 1) at 24 km: 0.3067
    assert 0.30 < top["pi0"][0] < 0.31
    zz = np.linspace(0.0, 24e3, 97)
    r = refstate.reference_state(zz, PRM)
    assert np.all(np.diff(r["p0"]) < 0) and np.all(np.diff(r["rho0"]) < 0)
    assert np.all(np.diff(r["theta0"]) > 0)


def test_pressure_perturbation_against_the_equation_of_state():
    from decimal import Decimal, getcontext
    getcontext().prec = 40
    r = refstate.reference_state(Z, PRM)
    rng = np.random.default_rng(7)
    for k in range(len(Z)):
        for x in np.concatenate([rng.uniform(-0.05, 0.05, 3), [1e-9, -3e-7, 0.3]]):
            rt = r["rhotheta0"][k] * (1.0 + x)
            pp = refstate.pressure_perturbation(rt - r["rhotheta0"][k], r["rhotheta0"][k], r["p0"][k], PRM.gamma)
            # p = p00 (R_d rho theta / p00)^gamma, in 40 digits
            D = Decimal
            g = D(PRM.c_p) / D(PRM.c_p - PRM.R_d)
            p = D(PRM.p00) * ((D(PRM.R_d) * D(rt) / D(PRM.p00)).ln() * g).exp()
            p0 = D(PRM.p00) * ((D(PRM.R_d) * D(r["rhotheta0"][k]) / D(PRM.p00)).ln() * g).exp()
            exact = float(p - p0)
            assert abs(pp - exact) <= 1e-12 * abs(exact) + 1e-12 * float(p0) * 1e-9, (k, x, pp, exact)
