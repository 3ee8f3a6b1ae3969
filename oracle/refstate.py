"""Hydrostatic reference state (Eqs. rho_split, theta_split, p_split, hydro_bal).

Sec. 2 splits rho, theta and p into a z-only hydrostatic part plus a
fluctuation, with dp0/dz = -rho0 g.  The paper takes the background from a
sounding that is not available; the reference state used here is the
constant Brunt-Vaisala-frequency atmosphere (theta0(0) = theta_s, buoyancy
frequency N_bv), written in closed form:

    theta0(z) = theta_s exp(N_bv^2 z / g)
    pi0(z)    = 1 + g^2 / (c_p theta_s N_bv^2) (exp(-N_bv^2 z / g) - 1)
    p0        = p00 pi0^(c_p / R_d)
    rho0      = p00 pi0^(c_v / R_d) / (R_d theta0)
    (rho theta)0 = rho0 theta0

which satisfies c_p theta0 dpi0/dz = -g, i.e. dp0/dz = -rho0 g exactly, and the
ideal gas law p = rho R_d T with T = theta pi, pi = (p / p00)^(R_d / c_p)
(Sec. 2).

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np


class Params:
    """Physical constants (Sec. 2: g = 9.81; the gas constants are unstated
    in the paper, the values below are the ones used throughout), and the
    sub-grid and absorbing-layer terms of the paper's runs (Sec. 4), off by
    default: smag_cs is the Smagorinsky coefficient C_s (the paper's 0.21),
    sponge_gamma and sponge_depth the Rayleigh layer's gamma and z_d (the
    paper's 1.0 and 4 km), heat_* the synthetic heating source (off at
    heat_q0 = 0) and time the time of the state."""

    def __init__(self, g=9.81, R_d=287.0, c_p=1004.0, p00=1.0e5, f=5.0e-5,
                 theta_s=300.0, N_bv=0.01, smag_cs=0.0, sponge_gamma=0.0, sponge_depth=4000.0,
                 heat_q0=0.0, heat_r0=27.5e3, heat_width=10.0e3, heat_rmax=60.0e3,
                 heat_ztop=15.0e3, heat_ramp=600.0, time=0.0):
        self.g, self.R_d, self.c_p, self.p00 = g, R_d, c_p, p00
        self.c_v = c_p - R_d
        self.gamma = c_p / self.c_v
        self.f, self.theta_s, self.N_bv = f, theta_s, N_bv
        self.smag_cs, self.sponge_gamma, self.sponge_depth = smag_cs, sponge_gamma, sponge_depth
        # synthetic latent-heating source (stand-in for the paper's observed
        # heating, Sec. 4): peak rate heat_q0 (K/s) on the ring r = heat_r0
        self.heat_q0, self.heat_r0, self.heat_width = heat_q0, heat_r0, heat_width
        self.heat_rmax, self.heat_ztop, self.heat_ramp = heat_rmax, heat_ztop, heat_ramp
        self.time = time

    def at(self, time):
        """A copy with the state's time set (the heating depends on it)."""
        import copy
        c = copy.copy(self)
        c.time = time
        return c


def reference_state(z, prm):
    """theta0, pi0, p0, rho0, (rho theta)0 and d theta0/dz at heights z."""
    z = np.asarray(z, dtype=np.float64)
    g, N2 = prm.g, prm.N_bv ** 2
    theta0 = prm.theta_s * np.exp(N2 * z / g)
    pi0 = 1.0 + g * g / (prm.c_p * prm.theta_s * N2) * (np.exp(-N2 * z / g) - 1.0)
    p0 = prm.p00 * pi0 ** (prm.c_p / prm.R_d)
    rho0 = prm.p00 * pi0 ** (prm.c_v / prm.R_d) / (prm.R_d * theta0)
    rhotheta0 = rho0 * theta0
    dtheta0 = theta0 * N2 / g
    return dict(theta0=theta0, pi0=pi0, p0=p0, rho0=rho0,
                rhotheta0=rhotheta0, dtheta0=dtheta0)


def pressure_perturbation(rhotheta_pert, rhotheta0, p0, gamma):
    """p' = p - p0 with p = p00 (R_d rho theta / p00)^gamma.

    Since p0 = p00 (R_d (rho theta)0 / p00)^gamma:
        p' = p0 ((1 + (rho theta)'/(rho theta)0)^gamma - 1)
           = p0 expm1(gamma log1p((rho theta)' / (rho theta)0)),
    which is exactly zero for a zero perturbation.
    """
    return p0 * np.expm1(gamma * np.log1p(rhotheta_pert / rhotheta0))
