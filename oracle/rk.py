"""Explicit third-order Runge-Kutta time integration (Sec. 4, "Time integration").

The paper names an explicit third-order RK scheme with a constant time step
but not which one; the three-stage strong-stability-preserving scheme of Shu
and Osher is used:
    q1      = qn + dt L(qn)
    q2      = 3/4 qn + 1/4 (q1 + dt L(q1))
    q_{n+1} = 1/3 qn + 2/3 (q2 + dt L(q2))
Each stage is q_out = a qn + b qs + c dt L(qs) with the coefficients below.

Test infrastructure only (see oracle/__init__.py).
"""
from .rhs import rhs

SSP_RK3 = ((0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0))


def stage_update(stage, qn, qs, dt, L_qs):
    a, b, c = SSP_RK3[stage]
    return a * qn + b * qs + c * dt * L_qs


def step_generic(L, qn, dt):
    """One SSP-RK3 step of dq/dt = L(q) for any callable L."""
    qs = qn
    for s in range(3):
        qs = stage_update(s, qn, qs, dt, L(qs))
    return qs


def rk_stage(mesh, prm, stage, qn, qs, dt, eqset="C"):
    return stage_update(stage, qn, qs, dt, rhs(mesh, qs, prm, eqset))


def rk_step(mesh, prm, qn, dt, eqset="C"):
    return step_generic(lambda q: rhs(mesh, q, prm, eqset), qn, dt)
