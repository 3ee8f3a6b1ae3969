"""Parity at the benchmark's full size (64 x 64 x 16 elements, N = 4,
2048 x 2048 x 24 km, 4,259,840 global nodes) in the launch configuration
bench.py times (autotuned element kernel, increment-form mixed step), against
one full SSP-RK3 step of the CPU oracle at every node; plus the float64 stage
at 1e-12.  The oracle builds the 8.2 M-node mesh by brute force (about a
minute).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from oracle import mesh as om, refstate, rhs as orhs, rk as ork  # noqa: E402
from synth.vortex import vortex_state  # noqa: E402

from tests.helpers import group_rel_l2, node_perm  # noqa: E402

PRM = refstate.Params()
L, LZ, NX, NZ, N, DT = 2048e3, 24e3, 64, 16, 4, 0.25


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_21607_gb300 import build
    build.build()
    from paper_2410_21607_gb300 import sem as s
    return s


@pytest.fixture(scope="module")
def pair(sem):
    m = sem.sem_mesh_create(L, L, LZ, NX, NX, NZ, N)
    o = om.OracleMesh(L, L, LZ, NX, NX, NZ, N)
    perm = node_perm(sem.sem_mesh_coords_host(m), o.XG)
    q_o = vortex_state(o.XG, LZ)
    return m, o, perm, q_o


def full(q, z, eqset="C"):
    ref = refstate.reference_state(z, PRM)
    out = q.copy()
    out[0] += ref["rho0"]
    out[4] += ref["rhotheta0"] if eqset == "C" else ref["theta0"]
    return out


def test_fullsize_mixed_step_matches_oracle(sem, pair):
    m, o, perm, q_o = pair
    q_ref = ork.rk_step(o, PRM, q_o, DT)
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q = torch.from_numpy(np.ascontiguousarray(q_o[:, perm])).cuda()
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    sem.sem_autotune(m, p, q32, 2)
    sem.sem_step_mixed(m, p, q, q32, work, DT)
    torch.cuda.synchronize()
    got = q.cpu().numpy()
    z = o.XG[perm, 2]
    err = group_rel_l2(full(got, z), full(q_ref[:, perm], z))
    assert np.all(err <= 1e-4), err
    inc = group_rel_l2(got - q_o[:, perm], q_ref[:, perm] - q_o[:, perm])
    assert np.all(inc <= 1e-4), inc       # the step's own increment, not only the state
    assert sem.sem_status(m) == 0


def test_fullsize_paper_set_mixed_step_matches_oracle(sem, pair):
    """The paper's equation set at full size: one mixed increment-form step
    (autotuned among that set's line-exchange variants) against one oracle
    step at every node, in the full fields and in the step's increment."""
    m, o, perm, _ = pair
    q_o = vortex_state(o.XG, LZ, eqset="NC")
    q_ref = ork.rk_step(o, PRM, q_o, DT, "NC")
    p = sem.sem_params_default(eqset=1, precision=sem.SEM_PREC_MIXED)
    q = torch.from_numpy(np.ascontiguousarray(q_o[:, perm])).cuda()
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    rows, _ = sem.sem_autotune(m, p, q32, 2)
    assert {r[3] for r in rows} == {5}
    sem.sem_step_mixed(m, p, q, q32, work, DT)
    torch.cuda.synchronize()
    got = q.cpu().numpy()
    z = o.XG[perm, 2]
    err = group_rel_l2(full(got, z, "NC"), full(q_ref[:, perm], z, "NC"))
    assert np.all(err <= 1e-4), err
    inc = group_rel_l2(got - q_o[:, perm], q_ref[:, perm] - q_o[:, perm])
    assert np.all(inc <= 1e-4), inc
    assert sem.sem_status(m) == 0


def test_fullsize_fp64_rhs_matches_oracle(sem, pair):
    """Float64 tendency at full size on the vortex plus seeded perturbations of
    every field (so that every tendency is O(1); for the bare vortex the mass
    tendency nearly cancels and its relative error measures the rounding order
    of the cancelling sum, 1e-11)."""
    from synth.vortex import random_state
    m, o, perm, _ = pair
    q_o = random_state(o.XG, LZ, 17)
    T_o = orhs.rhs(o, q_o, PRM)
    p = sem.sem_params_default()
    q = torch.from_numpy(np.ascontiguousarray(q_o[:, perm])).cuda()
    out = torch.empty_like(q)
    sem.sem_rhs(m, p, q, out)
    torch.cuda.synchronize()
    err = group_rel_l2(out.cpu().numpy(), T_o[:, perm])
    assert np.all(err <= 1e-12), err
