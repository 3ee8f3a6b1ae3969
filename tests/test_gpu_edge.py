"""GPU parity on the degenerate meshes of the method: a single periodic
column (every horizontal face shared by the element with itself), a single
walled column, one layer (the lid and the floor in the same element, a
layer chunk of one layer out of the kernels' 2 to 16), one column of
several layers at the highest order, and the smallest order (N = 2).

Same bars as tests/test_gpu_parity.py: float64 tendencies 1e-12, mixed form
1e-4 (tendencies, every element-kernel variant the autotuner lists, steps in
the full fields and in the change), criterion flags exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adapt, refstate, rhs as orhs, rk as ork  # noqa: E402
from synth.vortex import random_state, vortex_state  # noqa: E402
from tests.helpers import group_rel_l2  # noqa: E402
from tests.test_gpu_parity import dev, full_fields, host, increment_err, make_pair  # noqa: E402

PRM = refstate.Params()
EDGE = {
    "one-periodic-column-1x1x1-N4": dict(L=300e3, Lz=12e3, nx=1, nz=1, N=4),
    "one-walled-column-1x1x1-N3": dict(L=300e3, Lz=12e3, nx=1, nz=1, N=3, periodic=(False, False)),
    "one-layer-2x2x1-N2": dict(L=300e3, Lz=12e3, nx=2, nz=1, N=2),
    "one-column-1x1x5-N6": dict(L=300e3, Lz=12e3, nx=1, nz=5, N=6),
    "one-layer-3x3x1-N5": dict(L=300e3, Lz=12e3, nx=3, nz=1, N=5),
}


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_21607_gb300 import build
    build.build()
    from paper_2410_21607_gb300 import sem as s
    return s


@pytest.mark.parametrize("name", list(EDGE))
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_edge_rhs_both_forms_match_oracle(sem, name, eqset):
    m, o, X, perm = make_pair(sem, **EDGE[name])
    q_o = random_state(o.XG, o.Lz, 61, eqset)
    T_o = orhs.rhs(o, q_o, PRM, eqset)
    q = dev(q_o[:, perm])
    for prec, tol in ((0, 1e-12), (1, 1e-4)):
        p = sem.sem_params_default(eqset=0 if eqset == "C" else 1, precision=prec)
        out = torch.full_like(q, float("nan"))
        sem.sem_rhs(m, p, q, out)
        err = group_rel_l2(host(out), T_o[:, perm])
        assert np.all(err <= tol), (prec, err)
        rest = torch.full_like(q, 3.0)
        sem.sem_rhs(m, p, torch.zeros_like(q), rest)
        assert torch.count_nonzero(rest).item() == 0
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("name", list(EDGE))
def test_edge_every_variant_matches_oracle(sem, name):
    m, o, X, perm = make_pair(sem, **EDGE[name])
    q_o = random_state(o.XG, o.Lz, 62)
    T_o = orhs.rhs(o, q_o, PRM)
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    rows, _ = sem.sem_autotune(m, p, q32, 1)
    assert len(rows) >= 2
    for row in range(len(rows)):
        sem.sem_autotune_select(m, row)
        out = torch.full_like(q, float("nan"))
        sem.sem_rhs(m, p, q, out)
        assert np.all(group_rel_l2(host(out), T_o[:, perm]) <= 1e-4), rows[row]


@pytest.mark.parametrize("name", list(EDGE))
def test_edge_steps_and_criterion_match_oracle(sem, name):
    """Three SSP-RK3 steps of 1 s from the balanced vortex in both forms,
    then the speed criterion's flags on the result."""
    m, o, X, perm = make_pair(sem, **EDGE[name])
    q_o = vortex_state(o.XG, o.Lz)
    q_ref = q_o.copy()
    for _ in range(3):
        q_ref = ork.rk_step(o, PRM, q_ref, 1.0)
    z = X[:, 2]
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        q = dev(q_o[:, perm])
        p = sem.sem_params_default(precision=prec)
        if prec == 0:
            w1, w2 = torch.empty_like(q), torch.empty_like(q)
            for _ in range(3):
                sem.sem_step(m, p, q, w1, w2, 1.0)
        else:
            q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
            work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
            sem.sem_mirror(m, q, q32)
            for _ in range(3):
                sem.sem_step_mixed(m, p, q, q32, work, 1.0)
        got = host(q)
        assert np.all(group_rel_l2(full_fields(got, z), full_fields(q_ref[:, perm], z)) <= tol), prec
        assert np.all(increment_err(got, q_o[:, perm], q_ref[:, perm]) <= tol), prec
    thr = [2.0, 5.0, 10.0]
    fl_o, cmax_o = adapt.criterion_flags(o, q_ref, PRM, thr, 3)
    ps = sem.sem_params_default(thresholds=thr, lvl_max=3)
    flags = torch.empty(m.Ne, dtype=torch.int8, device="cuda")
    cmax = torch.empty(m.Ne, dtype=torch.float64, device="cuda")
    sem.sem_adapt_flags(m, ps, dev(q_ref[:, perm]), flags, cmax)
    lv = sem.sem_mesh_leaves_host(m)
    oleaf = {tuple(l): c for c, l in enumerate(o.leaves)}
    emap = np.array([oleaf[tuple(l)] * o.nz + k for l in lv for k in range(o.nz)])
    np.testing.assert_allclose(host(cmax), cmax_o[emap], rtol=1e-13)
    tie = np.min(np.abs(cmax_o[emap][:, None] - np.array(thr)[None]), axis=1) <= 1e-12 * max(thr)
    assert np.array_equal(host(flags)[~tie], fl_o[emap][~tie])
    assert sem.sem_status(m) == 0


def test_empty_batch_is_refused(sem):
    with pytest.raises(sem.SemError) as e:
        sem.sem_batch_create([])
    assert e.value.code == sem.SEM_ERR_ARG
