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
