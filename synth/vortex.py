"""Balanced axisymmetric warm-core vortex (the initial condition of Sec. 4).

The tangential wind follows the paper's profile
    vbar(r, z) = V(r) exp(-z^sigma / (sigma D1^sigma)) exp(-(r / D2)^6),
sigma = 2, D1 = 5823 m, D2 = 200 km, w = 0.  V(r) is the wind of a Gaussian
vorticity distribution zeta(r) = zeta0 exp(-(r/L)^2):
    V(r) = zeta0 L^2 / (2 r) (1 - exp(-(r/L)^2)),
whose maximum sits at r = x* L with x* the root of 2x^2 e^{-x^2} = 1 - e^{-x^2}
(x* ~ 1.12091); L and zeta0 follow from the requested radius and value of the
maximum wind.

Density and potential temperature are put in gradient-wind and hydrostatic
balance with the iteration the paper describes (alternate between the two
balances until converged), on a fine (r, z) grid:
    p(r, z)   = p_bg(z) - int_r^Rmax rho (v^2/r' + f v) dr'
    rho(r, z) = rho_bg(z) - (1/g) d(p - p_bg)/dz
starting from rho = rho_bg.  The background is the constant buoyancy-frequency
atmosphere (theta_s, N_bv).  Values at nodes are bilinear interpolants of the
grid fields.  Seeded potential-temperature noise, uniform in [-amp, amp] K, is
drawn per node from splitmix64 keyed by (seed, node coordinates rounded to
1 mm), so it does not depend on how either side numbers its nodes.
"""
from dataclasses import dataclass
import functools

import numpy as np
from scipy.interpolate import RegularGridInterpolator

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x):
    with np.errstate(over="ignore"):
        x = (x + np.uint64(0x9E3779B97F4A7C15)) & _MASK64
        z = x
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _MASK64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _MASK64
        return z ^ (z >> np.uint64(31))


def splitmix64_uniform(seed, xyz):
    """U[0,1) per point from splitmix64 keyed by (seed, coordinates in mm)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    keys = np.round(xyz * 1000.0).astype(np.int64).view(np.uint64)
    h = _splitmix64(np.full(keys.shape[0], np.uint64(seed)))
    for d in range(3):
        h = _splitmix64(h ^ keys[:, d])
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass(frozen=True)
class VortexSpec:
    vmax: float = 20.0          # m/s
    rmw: float = 50.0e3         # m
    D1: float = 5823.0          # m
    D2: float = 200.0e3         # m
    sigma: float = 2.0
    f: float = 5.0e-5           # 1/s
    theta_s: float = 300.0      # K
    N_bv: float = 0.01          # 1/s
    g: float = 9.81
    R_d: float = 287.0
    c_p: float = 1004.0
    p00: float = 1.0e5
    noise_K: float = 0.1
    seed: int = 20241028
    xc: float = 0.0
    yc: float = 0.0
    u0: float = 0.0             # uniform background wind added to the vortex (m/s)
    v0: float = 0.0


def gaussian_vortex_scale(vmax, rmw):
    """(L, zeta0) of the Gaussian-vorticity vortex with maximum vmax at rmw."""
    x = 1.1
    for _ in range(60):
        e = np.exp(-x * x)
        F = 1.0 - e - 2.0 * x * x * e
        dF = 2.0 * x * e - 4.0 * x * e + 4.0 * x ** 3 * e
        x -= F / dF
    L = rmw / x
    zeta0 = 2.0 * vmax * rmw / (L * L * (1.0 - np.exp(-x * x)))
    return L, zeta0, x


def _background(z, s):
    g, N2 = s.g, s.N_bv ** 2
    c_v = s.c_p - s.R_d
    th = s.theta_s * np.exp(N2 * z / g)
    pi = 1.0 + g * g / (s.c_p * s.theta_s * N2) * (np.exp(-N2 * z / g) - 1.0)
    p = s.p00 * pi ** (s.c_p / s.R_d)
    rho = s.p00 * pi ** (c_v / s.R_d) / (s.R_d * th)
    return th, p, rho


def tangential_wind(r, z, s):
    L, zeta0, _ = gaussian_vortex_scale(s.vmax, s.rmw)
    r = np.asarray(r, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        V = np.where(r > 0, zeta0 * L * L / (2.0 * r) * (1.0 - np.exp(-(r / L) ** 2)), 0.0)
    return (V * np.exp(-np.asarray(z) ** s.sigma / (s.sigma * s.D1 ** s.sigma))
            * np.exp(-(r / s.D2) ** 6))


@functools.lru_cache(maxsize=8)
def _balanced_grid(s, Rmax, Lz, dr=250.0, dz=25.0):
    nr = int(np.ceil(Rmax / dr)) + 2
    nzg = int(np.ceil(Lz / dz)) + 1
    r = np.arange(nr) * dr
    z = np.linspace(0.0, Lz, nzg)
    R, Z = np.meshgrid(r, z, indexing="ij")
    v = tangential_wind(R, Z, s)
    with np.errstate(invalid="ignore", divide="ignore"):
        cen = np.where(R > 0, v * v / R, 0.0) + s.f * v
    th_bg, p_bg, rho_bg = _background(z, s)
    rho = np.broadcast_to(rho_bg, R.shape).copy()
    for _ in range(50):
        A = rho * cen
        # I(r) = int_r^Rmax A dr' by the trapezoid rule from the outer edge
        seg = 0.5 * (A[1:] + A[:-1]) * dr
        I = np.zeros_like(A)
        I[:-1] = np.cumsum(seg[::-1], axis=0)[::-1]
        dp = -I                                  # p - p_bg
        rho_new = rho_bg[None, :] - np.gradient(dp, z, axis=1, edge_order=2) / s.g
        change = np.max(np.abs(rho_new - rho)) / np.max(rho_bg)
        rho = rho_new
        if change < 1e-13:
            break
    p = p_bg[None, :] + dp
    c_v = s.c_p - s.R_d
    rhotheta = s.p00 / s.R_d * (p / s.p00) ** (c_v / s.c_p)
    rhotheta_bg = s.p00 / s.R_d * (p_bg / s.p00) ** (c_v / s.c_p)
    drho = rho - rho_bg[None, :]
    drt = rhotheta - rhotheta_bg[None, :]
    return (RegularGridInterpolator((r, z), drho), RegularGridInterpolator((r, z), drt))


def vortex_state(xyz, Lz, spec=VortexSpec(), eqset="C", Rmax=None):
    """Initial state at nodes xyz (NG, 3): array (5, NG) in the variables of `eqset`.

    eqset "C": (rho', rho u, rho v, rho w, (rho theta)');
    eqset "NC": (rho', u, v, w, theta').  Perturbations are relative to the
    constant-N background of `spec`.
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    x, y, z = xyz[:, 0] - spec.xc, xyz[:, 1] - spec.yc, xyz[:, 2]
    r = np.hypot(x, y)
    if Rmax is None:
        Rmax = float(r.max()) + 1000.0
    fr, ft = _balanced_grid(spec, float(np.ceil(Rmax / 1000.0) * 1000.0), float(Lz))
    pts = np.stack([r, np.clip(z, 0.0, Lz)], axis=1)
    drho = fr(pts)
    drt = ft(pts)
    th_bg, _, rho_bg = _background(z, spec)
    rho = rho_bg + drho
    vb = tangential_wind(r, z, spec)
    with np.errstate(invalid="ignore", divide="ignore"):
        s_ = np.where(r > 0, y / r, 0.0)
        c_ = np.where(r > 0, x / r, 0.0)
    u, v, w = -vb * s_ + spec.u0, vb * c_ + spec.v0, np.zeros_like(vb)
    dth = spec.noise_K * (2.0 * splitmix64_uniform(spec.seed, xyz) - 1.0)
    Tp = drt + rho * dth
    if eqset == "C":
        return np.stack([drho, rho * u, rho * v, rho * w, Tp])
    thp = (Tp - drho * th_bg) / rho
    return np.stack([drho, u, v, w, thp])


def random_state(xyz, Lz, seed, eqset="C", amp=1.0, spec=VortexSpec()):
    """A vortex state plus seeded random perturbations of every field.

    Used by parity tests to excite all terms (nonzero w away from the lids,
    large density and theta perturbations).  The draws are keyed by node
    coordinates, like the theta noise."""
    q = vortex_state(xyz, Lz, spec, eqset)
    scale = np.array([2e-3, 2.0, 2.0, 0.5, 0.5]) * amp
    for f in range(5):
        u = splitmix64_uniform(int(seed) * 8 + f + 1, xyz)
        q[f] = q[f] + scale[f] * (2.0 * u - 1.0)
    z = np.asarray(xyz)[:, 2]
    lid = (np.abs(z) < 1e-6) | (np.abs(z - Lz) < 1e-6)
    q[3, lid] = 0.0
    return q
