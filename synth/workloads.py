"""Named synthetic workloads (mesh sizes, time step, step counts).

The paper's own case (an 800 x 800 x 20 km domain forced by observed latent
heating over a sounding, Sec. 4) needs data that is not available; these
workloads keep its ingredients that matter for the solver's cost and numerics:
order-4 LGL hexahedra, the warm-core vortex family of Sec. 4, doubly periodic
lateral boundaries and the velocity-magnitude threshold criterion of
Sec. 4.1.  The time steps keep the acoustic Courant number near 0.35 on the
smallest LGL spacing (0.1727 h for N = 4).
"""
from dataclasses import dataclass, field
from typing import Tuple


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    N: int
    Lx: float
    Ly: float
    Lz: float
    dt: float
    steps: int
    lvl_max: int = 0
    thresholds: Tuple[float, ...] = ()
    t_amr_steps: int = 0
    refine_radius: float = 0.0
    refine_levels: int = 0
    vmax: float = 20.0
    rmw: float = 50.0e3
    notes: str = field(default="", compare=False)

    @property
    def n_elements_base(self):
        return self.nx * self.ny * self.nz


WORKLOADS = {
    "uniform-6x6x4-N4": Workload(
        "uniform-6x6x4-N4", 6, 6, 4, 4, 600e3, 600e3, 24e3, dt=1.0, steps=10,
        notes="18,000 local nodes; small case the oracle finishes in seconds"),
    "uniform-64x64x16-N4": Workload(
        "uniform-64x64x16-N4", 64, 64, 16, 4, 2048e3, 2048e3, 24e3, dt=0.25, steps=100,
        notes="65,536 elements, 8,192,000 local nodes, 4,259,840 global nodes"),
    "amr-32x32x8-N4-L3": Workload(
        "amr-32x32x8-N4-L3", 32, 32, 8, 4, 600e3, 600e3, 24e3, dt=0.4, steps=500,
        lvl_max=3, thresholds=(5.0, 10.0, 15.0), t_amr_steps=50,
        refine_radius=150e3, refine_levels=3,
        notes="geometric level-3 refinement inside r < 150 km, 2:1 balanced"),
    "amr-8x8x4-N4-L2": Workload(
        "amr-8x8x4-N4-L2", 8, 8, 4, 4, 600e3, 600e3, 24e3, dt=1.0, steps=50,
        lvl_max=2, thresholds=(5.0, 10.0), t_amr_steps=25,
        refine_radius=150e3, refine_levels=2,
        notes="reduced-size adaptive case for oracle comparison"),
}


@dataclass(frozen=True)
class Instance:
    """One member of the batched workload."""
    nx: int
    nz: int
    N: int
    L: float
    Lz: float
    vmax: float
    rmw: float
    levels: int
    dt: float


def lgl_min_gap(N):
    """Smallest LGL node spacing on [-1, 1] as a fraction of the element width."""
    import numpy as np
    x = -np.cos(np.pi * np.arange(N + 1) / N)
    for _ in range(60):            # Newton on (1 - x^2) P_N'(x) = 0, interior nodes
        P = np.polynomial.legendre.Legendre.basis(N)
        dP, d2P = P.deriv(), P.deriv(2)
        f = (1 - x * x) * dP(x)
        df = -2 * x * dP(x) + (1 - x * x) * d2P(x)
        step = np.zeros_like(x)
        step[1:-1] = f[1:-1] / df[1:-1]
        x = x - step
    return float(np.min(np.diff(np.sort(x)))) / 2.0


def batched_instances(seed=4, count=16):
    """The 16-instance batched workload: seeded base sizes 8..48 (nz = nx/4),
    orders 3..6, v_max 15..40 m/s, radius of maximum wind 30..80 km and 0..3
    levels of geometric refinement inside r < 3 RMW; 600 km boxes for nx >= 16,
    300 km below.  dt keeps the acoustic Courant number at 0.35 on the finest
    LGL spacing (vertical or horizontal)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = int(rng.integers(2, 13)) * 4          # 8 .. 48
        nz = max(nx // 4, 2)
        N = int(rng.integers(3, 7))
        vmax = float(rng.uniform(15.0, 40.0))
        rmw = float(rng.uniform(30e3, 80e3))
        levels = int(rng.integers(0, 4))
        L = 600e3 if nx >= 16 else 300e3
        Lz = 24e3
        g = lgl_min_gap(N)
        h = min(L / (nx << levels), Lz / nz)
        dt = 0.35 * g * h / 347.0
        out.append(Instance(nx, nz, N, L, Lz, vmax, rmw, levels, dt))
    return out


def geometric_flags(leaves, nx, nz, L, radius, lvl_max):
    """Refinement flags (+1) for every element of a column whose centre lies
    within `radius` of the domain centre, below lvl_max; 0 elsewhere."""
    import numpy as np
    fl = np.zeros(len(leaves) * nz, dtype=np.int8)
    for c, (l, i, j) in enumerate(leaves):
        h = L / (nx << l)
        xc = -0.5 * L + (i + 0.5) * h
        yc = -0.5 * L + (j + 0.5) * h
        if l < lvl_max and np.hypot(xc, yc) < radius:
            fl[c * nz:(c + 1) * nz] = 1
    return fl


def translating_vortices(count=10, seed=7):
    """Seeded vortices for the learned-schedule experiment on a 150 km box:
    v_max 20..32 m/s, radius of maximum wind 14..22 km, outer taper 45 km so
    the vortex fits the periodic box, centre within 40 km of the middle, and a
    uniform background wind of 6..14 m/s in a random direction that carries
    it across element boundaries.  No theta noise (the inviscid
    discretisation amplifies grid-scale noise over a few hundred steps)."""
    import numpy as np
    from .vortex import VortexSpec
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        ang = rng.uniform(0, 2 * np.pi)
        sp = rng.uniform(6, 14)
        out.append(VortexSpec(vmax=float(rng.uniform(20, 32)), rmw=float(rng.uniform(14e3, 22e3)),
                              D2=45e3, u0=float(sp * np.cos(ang)), v0=float(sp * np.sin(ang)),
                              noise_K=0.0, xc=float(rng.uniform(-40e3, 40e3)),
                              yc=float(rng.uniform(-40e3, 40e3)), seed=10 + k))
    return out
