"""Explicit third-order Runge-Kutta time integration (Sec. 4, "Time integration").

The paper names an explicit third-order RK scheme with a constant time step
but not which one; the three-stage strong-stability-preserving scheme of Shu
and Osher is used:
    q1      = qn + dt L(qn)
    q2      = 3/4 qn + 1/4 (q1 + dt L(q1))
    q_{n+1} = 1/3 qn + 2/3 (q2 + dt L(q2))
Each stage is q_out = a qn + b qs + c dt L(qs) with the coefficients below;
the stage states approximate the solution at t_n, t_n + dt and t_n + dt/2,
the times at which L is evaluated (only the heating source depends on time).

Test infrastructure only (see oracle/__init__.py).
"""
from .rhs import rhs

SSP_RK3 = ((0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0))
STAGE_TIMES = (0.0, 1.0, 0.5)


def stage_update(stage, qn, qs, dt, L_qs):
    a, b, c = SSP_RK3[stage]
    return a * qn + b * qs + c * dt * L_qs


def step_generic(L, qn, dt, t=0.0):
    """One SSP-RK3 step of dq/dt = L(q, t) from time t for any callable L
    (a callable of q alone is accepted too)."""
    import inspect
    timed = len(inspect.signature(L).parameters) >= 2
    qs = qn
    for s in range(3):
        Lq = L(qs, t + STAGE_TIMES[s] * dt) if timed else L(qs)
        qs = stage_update(s, qn, qs, dt, Lq)
    return qs


def rk_stage(mesh, prm, stage, qn, qs, dt, eqset="C"):
    """Stage `stage` of the step from prm.time (the time of qn)."""
    return stage_update(stage, qn, qs, dt,
                        rhs(mesh, qs, prm.at(prm.time + STAGE_TIMES[stage] * dt), eqset))


def rk_step(mesh, prm, qn, dt, eqset="C"):
    """One step from prm.time (the time of qn)."""
    return step_generic(lambda q, t: rhs(mesh, q, prm.at(t), eqset), qn, dt, prm.time)
