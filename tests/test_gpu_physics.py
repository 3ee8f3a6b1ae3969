"""GPU parity of the terms of the paper's runs (Sec. 4): the horizontal
Smagorinsky stress, the Rayleigh absorbing layer and the synthetic heating
source (with the stage times of the steps), through the C ABI, against the
oracle (oracle/rhs.py, oracle/rk.py).

The added terms are checked on their own (tendency with them minus tendency
without, on both sides) as well as in the total, so that a small term cannot
hide under the tolerance of the inviscid part.  Float64: total 1e-12, added
terms 1e-9 (the difference of two float64 tendencies).  Mixed: total 1e-4,
added terms ADDED_TOL of their own norm (the float32 rounding of the total
carries into the difference of the two mixed tendencies, so the bound on the
added terms is looser than on the total, but it is relative to the terms
themselves: a wrong term fails it whatever the size of the total).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mesh as om, refstate, rhs as orhs, rk as ork  # noqa: E402
from synth.vortex import random_state, vortex_state  # noqa: E402
from tests.helpers import group_rel_l2, node_perm  # noqa: E402
from tests.test_gpu_parity import MESHES, dev, full_fields, host, make_pair, two_level_leaves  # noqa: E402

PHYS = dict(smag_cs=0.21, sponge_gamma=0.02, sponge_depth=6000.0)
ADDED_TOL = 1e-3


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_21607_gb300 import build
    build.build()
    from paper_2410_21607_gb300 import sem as s
    return s


def _gpu_rhs(sem, m, q, eqset, prec, **phys):
    p = sem.sem_params_default(eqset=0 if eqset == "C" else 1, precision=prec, **phys)
    out = torch.empty_like(q)
    sem.sem_rhs(m, p, q, out)
    return host(out)


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_physics_rhs_fp64_matches_oracle(sem, name, eqset):
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = random_state(o.XG, o.Lz, 21, eqset)
    prm = refstate.Params(**PHYS)
    T_o = orhs.rhs(o, q_o, prm, eqset)
    dT_o = T_o - orhs.rhs(o, q_o, refstate.Params(), eqset)
    q = dev(q_o[:, perm])
    T = _gpu_rhs(sem, m, q, eqset, 0, **PHYS)
    dT = T - _gpu_rhs(sem, m, q, eqset, 0)
    assert np.all(group_rel_l2(T, T_o[:, perm]) <= 1e-12)
    err = group_rel_l2(dT, dT_o[:, perm])
    assert np.all(err <= 1e-9), err
    assert np.linalg.norm(dT_o[1]) > 0 and np.linalg.norm(dT_o[0]) > 0


@pytest.mark.parametrize("name", ["uniform-6x6x4-N4", "twolevel-N4", "stretched-twolevel-N4", "uniform-3x3x2-N2",
                                  "twolevel-N3-open", "uniform-5x4x3-N6"])
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_physics_rhs_mixed_matches_oracle(sem, name, eqset):
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = random_state(o.XG, o.Lz, 22, eqset)
    prm = refstate.Params(**PHYS)
    T_o = orhs.rhs(o, q_o, prm, eqset)
    dT_o = T_o - orhs.rhs(o, q_o, refstate.Params(), eqset)
    q = dev(q_o[:, perm])
    T = _gpu_rhs(sem, m, q, eqset, 1, **PHYS)
    dT = T - _gpu_rhs(sem, m, q, eqset, 1)
    assert np.all(group_rel_l2(T, T_o[:, perm]) <= 1e-4)
    ratio = group_rel_l2(T_o, 0 * T_o) / np.maximum(group_rel_l2(dT_o, 0 * dT_o), 1e-300)
    err = group_rel_l2(dT, dT_o[:, perm])
    assert np.all(err <= ADDED_TOL), (err, ratio)


def _spec(name):
    if name == "twolevel-17-layers-N4":   # several layer chunks per column for every variant
        return dict(L=300e3, Lz=24e3, nx=4, nz=17, N=4, leaves=two_level_leaves())
    return MESHES[name]


@pytest.mark.parametrize("name", ["twolevel-N4", "stretched-twolevel-N4", "twolevel-17-layers-N4",
                                  "uniform-5x4x3-N6"])
def test_physics_rhs_every_variant_matches_oracle(sem, name):
    """Mixed tendency with both terms through each element-kernel variant: an
    order-4 line-exchange variant adds both terms in the element kernel, other
    line-exchange variants the absorbing layer (the physics pass the stress),
    a z-pencil variant leaves both to the physics pass.  17 layers give every
    variant several layer chunks, so the carry of the top-node values (with
    the stress) between chunks is exercised."""
    m, o, X, perm = make_pair(sem, **_spec(name))
    q_o = random_state(o.XG, o.Lz, 24)
    T_o = orhs.rhs(o, q_o, refstate.Params(**PHYS))
    dT_o = T_o - orhs.rhs(o, q_o, refstate.Params())
    ratio = group_rel_l2(T_o, 0 * T_o) / np.maximum(group_rel_l2(dT_o, 0 * dT_o), 1e-300)
    q = dev(q_o[:, perm])
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    rows, _ = sem.sem_autotune(m, sem.sem_params_default(precision=1), q32, 1)
    kinds = set()
    for row in range(len(rows)):
        sem.sem_autotune_select(m, row)
        T = _gpu_rhs(sem, m, q, "C", 1, **PHYS)
        dT = T - _gpu_rhs(sem, m, q, "C", 1)
        assert np.all(group_rel_l2(T, T_o[:, perm]) <= 1e-4), rows[row]
        err = group_rel_l2(dT, dT_o[:, perm])
        assert np.all(err <= ADDED_TOL), (rows[row], err, ratio)
        kinds.add(rows[row][3])
    assert kinds == ({0, 1, 2, 4} if m.N == 4 else {0, 1})
    # the absorbing layer alone (no physics pass at all on a line variant)
    sp = dict(sponge_gamma=0.02, sponge_depth=6000.0)
    dS_o = orhs.rhs(o, q_o, refstate.Params(**sp)) - orhs.rhs(o, q_o, refstate.Params())
    sem.sem_autotune_select(m, -1)
    dS = _gpu_rhs(sem, m, q, "C", 1, **sp) - _gpu_rhs(sem, m, q, "C", 1)
    ratio = group_rel_l2(T_o, 0 * T_o) / np.maximum(group_rel_l2(dS_o, 0 * dS_o), 1e-300)
    err = group_rel_l2(dS, dS_o[:, perm])
    assert np.all(err <= ADDED_TOL), (err, ratio)
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("prec,name", [(0, "twolevel-N4"), (1, "twolevel-N4"), (1, "twolevel-17-layers-N4")])
def test_physics_steps_match_oracle(sem, prec, name):
    """Ten SSP-RK3 steps with both terms on a two-level mesh (1 s; 0.25 s on
    the 17-layer mesh, whose thin layers bound the acoustic step), in the
    float64 form (sem_step) and the mixed increment form (sem_step_mixed)."""
    m, o, X, perm = make_pair(sem, **_spec(name))
    dt = 0.25 if name == "twolevel-17-layers-N4" else 1.0
    q_o = vortex_state(o.XG, o.Lz)
    prm = refstate.Params(**PHYS)
    p = sem.sem_params_default(precision=prec, **PHYS)
    q = dev(q_o[:, perm])
    if prec == 0:
        w1, w2 = torch.empty_like(q), torch.empty_like(q)
        for _ in range(10):
            sem.sem_step(m, p, q, w1, w2, dt)
    else:
        q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
        work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
        sem.sem_mirror(m, q, q32)
        for _ in range(10):
            sem.sem_step_mixed(m, p, q, q32, work, dt)
    for _ in range(10):
        q_o = ork.rk_step(o, prm, q_o, dt)
    z = X[:, 2]
    err = group_rel_l2(full_fields(host(q), z), full_fields(q_o[:, perm], z))
    assert np.all(err <= (1e-12 if prec == 0 else 1e-4)), err
    pert = group_rel_l2(host(q), q_o[:, perm])       # the perturbation fields themselves
    assert np.all(pert <= (1e-10 if prec == 0 else 1e-3)), pert
    assert sem.sem_status(m) == 0


def test_physics_rejected_by_the_batched_step(sem):
    m = sem.sem_mesh_create(300e3, 300e3, 12e3, 3, 3, 2, 4)
    b = sem.sem_batch_create([m])
    q = torch.zeros(5, m.NG, dtype=torch.float64, device="cuda")
    q32 = torch.zeros(5, m.NG, dtype=torch.float32, device="cuda")
    work = torch.zeros(10, m.NG, dtype=torch.float32, device="cuda")
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED, smag_cs=0.21)
    with pytest.raises(sem.SemError) as e:
        sem.sem_batch_step_mixed(b, p, [q], [q32], [work], [1.0])
    assert e.value.code == sem.SEM_ERR_UNSUPPORTED


def test_bad_physics_params_rejected(sem):
    m = sem.sem_mesh_create(300e3, 300e3, 12e3, 3, 3, 2, 4)
    q = torch.zeros(5, m.NG, dtype=torch.float64, device="cuda")
    out = torch.empty_like(q)
    for bad in (dict(smag_cs=-0.1), dict(sponge_gamma=-1.0), dict(sponge_gamma=1.0, sponge_depth=0.0)):
        with pytest.raises(sem.SemError) as e:
            sem.sem_rhs(m, sem.sem_params_default(**bad), q, out)
        assert e.value.code == sem.SEM_ERR_ARG


HEAT = dict(heat_q0=0.005, heat_r0=27.5e3, heat_width=10e3, heat_rmax=60e3, heat_ztop=10e3, heat_ramp=5.0)


@pytest.mark.parametrize("name", ["uniform-6x6x4-N4", "twolevel-N4", "uniform-5x4x3-N6"])
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_heating_rhs_matches_oracle(sem, name, eqset):
    """Heating source at t = 3 s: float64 total 1e-12 and the source alone
    1e-10 (only the theta equation moves); mixed total 1e-4 and the source
    alone ADDED_TOL of its own norm."""
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = random_state(o.XG, o.Lz, 23, eqset)
    prm = refstate.Params(time=3.0, **HEAT)
    T_o = orhs.rhs(o, q_o, prm, eqset)
    dT_o = T_o - orhs.rhs(o, q_o, refstate.Params(), eqset)
    q = dev(q_o[:, perm])
    T = _gpu_rhs(sem, m, q, eqset, 0, time=3.0, **HEAT)
    dT = T - _gpu_rhs(sem, m, q, eqset, 0)
    assert np.all(group_rel_l2(T, T_o[:, perm]) <= 1e-12)
    assert np.linalg.norm(dT_o[4]) > 0
    assert np.linalg.norm(dT[4] - dT_o[4, perm]) <= 1e-10 * np.linalg.norm(dT_o[4])
    assert np.all(dT[:4] == 0.0)
    Tm = _gpu_rhs(sem, m, q, eqset, 1, time=3.0, **HEAT)
    dTm = Tm - _gpu_rhs(sem, m, q, eqset, 1)
    assert np.all(group_rel_l2(Tm, T_o[:, perm]) <= 1e-4)
    ratio = max(np.linalg.norm(T_o[4]) / np.linalg.norm(dT_o[4]), 1.0)
    assert np.linalg.norm(dTm[4] - dT_o[4, perm]) <= ADDED_TOL * np.linalg.norm(dT_o[4]), ratio


@pytest.mark.parametrize("prec", [0, 1])
def test_heating_steps_use_the_stage_times(sem, prec):
    """Ten steps of 1 s from t = 0 with a 5 s ramp: the source changes within
    a step, so the stage times (t, t + dt, t + dt/2) matter.  The state's
    increment over the run is compared (float64 1e-10, mixed 1e-4)."""
    m, o, X, perm = make_pair(sem, **MESHES["uniform-6x6x4-N4"])
    q0 = vortex_state(o.XG, o.Lz)
    q_o = q0.copy()
    p = sem.sem_params_default(precision=prec, **HEAT)
    q = dev(q0[:, perm])
    if prec == 1:
        q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
        work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
        sem.sem_mirror(m, q, q32)
    else:
        w1, w2 = torch.empty_like(q), torch.empty_like(q)
    for s in range(10):
        p.time = float(s)
        if prec == 1:
            sem.sem_step_mixed(m, p, q, q32, work, 1.0)
        else:
            sem.sem_step(m, p, q, w1, w2, 1.0)
        q_o = ork.rk_step(o, refstate.Params(time=float(s), **HEAT), q_o, 1.0)
    inc = group_rel_l2(host(q) - q0[:, perm], q_o[:, perm] - q0[:, perm])
    assert np.all(inc <= (1e-10 if prec == 0 else 1e-4)), inc
    assert sem.sem_status(m) == 0


def test_noalloc_refuses_the_optional_terms(sem):
    m = sem.sem_mesh_create(300e3, 300e3, 12e3, 3, 3, 2, 4)
    sem.sem_mesh_coords_host(m)
    q = torch.zeros(5, m.NG, dtype=torch.float64, device="cuda")
    out = torch.empty_like(q)
    sem.sem_rhs(m, sem.sem_params_default(), q, out)     # device tables exist now
    with pytest.raises(sem.SemError) as e:
        sem.sem_rhs_noalloc(m, sem.sem_params_default(heat_q0=0.01), q, out)
    assert e.value.code == sem.SEM_ERR_UNSUPPORTED
