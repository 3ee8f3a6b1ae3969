"""GPU parity on warped layers (non-affine elements): the right-hand side,
the stages and steps of both forms through the C ABI against the oracle's
general isoparametric discretisation (oracle/mesh.py, warp), on conforming
and non-conforming meshes.

Tolerances as in tests/test_gpu_parity.py: float64 1e-12 (tendencies), mixed
form 1e-4 (tendencies, states and their change over the steps).  The metric
terms are float64 tables on both forms' inputs (the mixed form reads them
rounded once to float32).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adapt, refstate, rhs as orhs, rk as ork  # noqa: E402
from synth.vortex import random_state, vortex_state  # noqa: E402
from tests.helpers import group_rel_l2  # noqa: E402
from tests.test_gpu_parity import dev, full_fields, host, increment_err, make_pair  # noqa: E402
from tests.test_oracle_mesh import two_level_leaves  # noqa: E402

PRM = refstate.Params()
WMESH = {
    "warped-4x4x2-N4": dict(L=300e3, Lz=12e3, nx=4, nz=2, N=4, warp=(700.0, 1, 1)),
    "warped-twolevel-N4": dict(L=300e3, Lz=12e3, nx=4, nz=2, N=4, leaves=two_level_leaves(), warp=(700.0, 1, 2)),
    "warped-twolevel-17-layers-N4": dict(L=300e3, Lz=24e3, nx=4, nz=17, N=4, leaves=two_level_leaves(),
                                         warp=(400.0, 2, 1)),
    "warped-twolevel-N3": dict(L=300e3, Lz=12e3, nx=4, nz=3, N=3, leaves=two_level_leaves(), warp=(700.0, 1, 1)),
}


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_21607_gb300 import build
    build.build()
    from paper_2410_21607_gb300 import sem as s
    return s


@pytest.mark.parametrize("name", list(WMESH))
@pytest.mark.parametrize("eqset", ["C", "NC"])
@pytest.mark.parametrize("prec", [0, 1])
def test_warped_rhs_matches_oracle(sem, name, eqset, prec):
    """Random perturbations of every field, and the balanced vortex (zero
    vertical velocity: a state on which only the metric's cross terms move
    the vertical fluxes)."""
    m, o, X, perm = make_pair(sem, **WMESH[name])
    for q_o in (random_state(o.XG, o.Lz, 51, eqset), vortex_state(o.XG, o.Lz, eqset=eqset)):
        T_o = orhs.rhs(o, q_o, PRM, eqset)
        p = sem.sem_params_default(eqset=0 if eqset == "C" else 1, precision=prec)
        q = dev(q_o[:, perm])
        out = torch.full_like(q, float("nan"))
        sem.sem_rhs(m, p, q, out)
        err = group_rel_l2(host(out), T_o[:, perm])
        assert np.all(err <= (1e-12 if prec == 0 else 1e-4)), err
    assert sem.sem_status(m) == 0


def test_warped_every_line_variant_matches_oracle(sem):
    """On warped meshes the autotuner lists the line-exchange variants only;
    each gives the mixed tendency within 1e-4 (several layer chunks)."""
    m, o, X, perm = make_pair(sem, **WMESH["warped-twolevel-17-layers-N4"])
    q_o = random_state(o.XG, o.Lz, 52)
    T_o = orhs.rhs(o, q_o, PRM)
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    rows, _ = sem.sem_autotune(m, p, q32, 1)
    assert len(rows) >= 2 and {r[3] for r in rows} == {1}
    for row in range(len(rows)):
        sem.sem_autotune_select(m, row)
        out = torch.full_like(q, float("nan"))
        sem.sem_rhs(m, p, q, out)
        assert np.all(group_rel_l2(host(out), T_o[:, perm]) <= 1e-4), rows[row]


@pytest.mark.parametrize("name", ["warped-twolevel-17-layers-N4", "warped-twolevel-N3", "warped-4x4x2-N4"])
def test_warped_every_paper_set_variant_matches_oracle(sem, name):
    """The paper's set on warped layers: every line-exchange variant of its
    table (kind 5) gives the mixed tendency within 1e-4 of the oracle, for a
    random state and for the balanced vortex."""
    m, o, X, perm = make_pair(sem, **WMESH[name])
    p = sem.sem_params_default(eqset=1, precision=sem.SEM_PREC_MIXED)
    states = (random_state(o.XG, o.Lz, 53, "NC"), vortex_state(o.XG, o.Lz, eqset="NC"))
    q32 = torch.empty((5, m.NG), dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, dev(states[0][:, perm]), q32)
    rows, _ = sem.sem_autotune(m, p, q32, 1)
    assert rows and {r[3] for r in rows} == {5}
    for row in list(range(len(rows))) + [-1]:
        sem.sem_autotune_select(m, row, eqset=1)
        for q_o in states:
            T_o = orhs.rhs(o, q_o, PRM, "NC")
            q = dev(q_o[:, perm])
            out = torch.full_like(q, float("nan"))
            sem.sem_rhs(m, p, q, out)
            err = group_rel_l2(host(out), T_o[:, perm])
            assert np.all(err <= 1e-4), (row, err)
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("name", ["warped-4x4x2-N4", "warped-twolevel-N4"])
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_warped_mixed_steps_both_sets_match_oracle(sem, name, eqset):
    """Five mixed increment-form steps of 1 s from the balanced vortex in
    either equation set: within 1e-4 of the oracle's steps in the full fields
    and in the change."""
    m, o, X, perm = make_pair(sem, **WMESH[name])
    q_o = vortex_state(o.XG, o.Lz, eqset=eqset)
    q_ref = q_o.copy()
    for _ in range(5):
        q_ref = ork.rk_step(o, PRM, q_ref, 1.0, eqset)
    q = dev(q_o[:, perm])
    p = sem.sem_params_default(eqset=0 if eqset == "C" else 1, precision=sem.SEM_PREC_MIXED)
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    for _ in range(5):
        sem.sem_step_mixed(m, p, q, q32, work, 1.0)
    got = host(q)
    z = X[:, 2]
    assert np.all(group_rel_l2(full_fields(got, z, eqset), full_fields(q_ref[:, perm], z, eqset)) <= 1e-4)
    assert np.all(increment_err(got, q_o[:, perm], q_ref[:, perm]) <= 1e-4)
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("name", ["warped-4x4x2-N4", "warped-twolevel-N4"])
@pytest.mark.parametrize("prec", [0, 1])
def test_warped_steps_match_oracle(sem, name, prec):
    """Five SSP-RK3 steps of 1 s from the balanced vortex: the float64 form
    (sem_step) within 1e-10 of the oracle's steps, the mixed increment form
    (sem_step_mixed) within 1e-4 in the full fields and in the change."""
    m, o, X, perm = make_pair(sem, **WMESH[name])
    q_o = vortex_state(o.XG, o.Lz)
    q_ref = q_o.copy()
    for _ in range(5):
        q_ref = ork.rk_step(o, PRM, q_ref, 1.0)
    q = dev(q_o[:, perm])
    p = sem.sem_params_default(precision=prec)
    if prec == 0:
        w1, w2 = torch.empty_like(q), torch.empty_like(q)
        for _ in range(5):
            sem.sem_step(m, p, q, w1, w2, 1.0)
    else:
        q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
        work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
        sem.sem_mirror(m, q, q32)
        for _ in range(5):
            sem.sem_step_mixed(m, p, q, q32, work, 1.0)
    got = host(q)
    z = X[:, 2]
    tol = 1e-10 if prec == 0 else 1e-4
    assert np.all(group_rel_l2(full_fields(got, z), full_fields(q_ref[:, perm], z)) <= tol)
    assert np.all(increment_err(got, q_o[:, perm], q_ref[:, perm]) <= tol)
    assert sem.sem_status(m) == 0


def test_warped_rest_state_mass_and_coordinates(sem):
    m, o, X, perm = make_pair(sem, **WMESH["warped-twolevel-N4"])
    M = sem.sem_mesh_mass_host(m)
    q = dev(random_state(o.XG, o.Lz, 5)[:, perm])
    out = torch.empty_like(q)
    for prec in (0, 1):
        for eq in (0, 1):
            z0 = torch.zeros_like(q)
            rest = torch.full_like(q, 7.0)
            sem.sem_rhs(m, sem.sem_params_default(eqset=eq, precision=prec), z0, rest)
            assert torch.count_nonzero(rest).item() == 0
        sem.sem_rhs(m, sem.sem_params_default(precision=prec), q, out)
        T = host(out)
        tol = 1e-13 if prec == 0 else 1e-6
        assert abs(np.sum(M * T[0])) <= tol * np.sum(np.abs(M * T[0]))
    xyz = torch.empty(3, m.NG, dtype=torch.float64, device="cuda")
    sem.sem_mesh_coords(m, xyz)
    assert np.array_equal(host(xyz), sem.sem_mesh_coords_host(m))


def test_warped_speed_criterion_and_diagnostics(sem):
    m, o, X, perm = make_pair(sem, **WMESH["warped-twolevel-N4"])
    q_o = vortex_state(o.XG, o.Lz)
    lv = sem.sem_mesh_leaves_host(m)
    oleaf = {tuple(l): c for c, l in enumerate(o.leaves)}
    emap = np.array([oleaf[tuple(l)] * o.nz + k for l in lv for k in range(o.nz)])
    thr = [5.0, 10.0, 15.0]
    fl_o, cmax_o = adapt.criterion_flags(o, q_o, PRM, thr, 3)
    p = sem.sem_params_default(thresholds=thr, lvl_max=3)
    flags = torch.empty(m.Ne, dtype=torch.int8, device="cuda")
    cmax = torch.empty(m.Ne, dtype=torch.float64, device="cuda")
    sem.sem_adapt_flags(m, p, dev(q_o[:, perm]), flags, cmax)
    np.testing.assert_allclose(host(cmax), cmax_o[emap], rtol=1e-14)
    tie = np.min(np.abs(cmax_o[emap][:, None] - np.array(thr)[None]), axis=1) <= 1e-12 * max(thr)
    assert np.array_equal(host(flags)[~tie], fl_o[emap][~tie])
    d = sem.sem_diag(m, p, dev(q_o[:, perm]), 150e3)
    sp = np.hypot(q_o[1], q_o[2]) / (refstate.reference_state(o.XG[:, 2], PRM)["rho0"] + q_o[0])
    assert abs(d["max_wind"] - sp.max()) <= 1e-12 * sp.max()


PHYS = dict(smag_cs=0.21, sponge_gamma=0.02, sponge_depth=6000.0)
HEAT = dict(heat_q0=0.005, heat_r0=27.5e3, heat_width=10e3, heat_rmax=60e3, heat_ztop=10e3, heat_ramp=5.0)
ADDED_TOL = 1e-3


def _gpu_rhs(sem, m, q, eqset, prec, **phys):
    p = sem.sem_params_default(eqset=0 if eqset == "C" else 1, precision=prec, **phys)
    out = torch.full_like(q, float("nan"))
    sem.sem_rhs(m, p, q, out)
    return host(out)


@pytest.mark.parametrize("name", ["warped-4x4x2-N4", "warped-twolevel-N4", "warped-twolevel-N3"])
@pytest.mark.parametrize("eqset", ["C", "NC"])
@pytest.mark.parametrize("terms", ["stress+layer", "heating"])
def test_warped_physics_rhs_matches_oracle(sem, name, eqset, terms):
    """The terms of the paper's runs on warped layers: horizontal stress at
    constant height (through the metric), absorbing layer and heating at
    each node's height.  Totals at 1e-12 (float64) and 1e-4 (mixed); the
    added terms alone at 1e-9 (float64) and ADDED_TOL of their own norm
    (mixed)."""
    m, o, X, perm = make_pair(sem, **WMESH[name])
    phys = dict(PHYS) if terms == "stress+layer" else dict(time=3.0, **HEAT)
    q_o = random_state(o.XG, o.Lz, 25, eqset)
    T_o = orhs.rhs(o, q_o, refstate.Params(**phys), eqset)
    dT_o = T_o - orhs.rhs(o, q_o, PRM, eqset)
    assert np.linalg.norm(dT_o) > 0
    q = dev(q_o[:, perm])
    for prec, tol, added in ((0, 1e-12, 1e-9), (1, 1e-4, ADDED_TOL)):
        T = _gpu_rhs(sem, m, q, eqset, prec, **phys)
        dT = T - _gpu_rhs(sem, m, q, eqset, prec)
        assert np.all(group_rel_l2(T, T_o[:, perm]) <= tol), prec
        for g in (slice(1, 4), slice(0, 1), slice(4, 5)):
            ref = np.linalg.norm(dT_o[g])
            if ref > 0:
                assert np.linalg.norm(dT[g] - dT_o[g][:, perm]) <= added * ref, (prec, g)
            else:
                assert np.all(dT[g] == 0.0), (prec, g)
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_warped_physics_steps_match_oracle(sem, prec):
    """Five steps of 1 s from the balanced vortex with the stress, the
    absorbing layer and the heating (stage times) on a warped 2:1 mesh."""
    m, o, X, perm = make_pair(sem, **WMESH["warped-twolevel-N4"])
    phys = dict(PHYS, **HEAT)
    q0 = vortex_state(o.XG, o.Lz)
    q_ref = q0.copy()
    for s_ in range(5):
        q_ref = ork.rk_step(o, refstate.Params(time=float(s_), **phys), q_ref, 1.0)
    q = dev(q0[:, perm])
    p = sem.sem_params_default(precision=prec, **phys)
    if prec == 0:
        w1, w2 = torch.empty_like(q), torch.empty_like(q)
    else:
        q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
        work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
        sem.sem_mirror(m, q, q32)
    for s_ in range(5):
        p.time = float(s_)
        if prec == 0:
            sem.sem_step(m, p, q, w1, w2, 1.0)
        else:
            sem.sem_step_mixed(m, p, q, q32, work, 1.0)
    got = host(q)
    tol = 1e-10 if prec == 0 else 1e-4
    assert np.all(group_rel_l2(full_fields(got, X[:, 2]), full_fields(q_ref[:, perm], X[:, 2])) <= tol)
    assert np.all(increment_err(got, q0[:, perm], q_ref[:, perm]) <= tol)
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_warped_checkpoint_resume_is_bitwise(sem, prec, tmp_path):
    """Four steps straight through equal two steps, a checkpoint, the mesh
    and state read back (warped layers rebuilt from the file), and two more."""
    m, o, X, perm = make_pair(sem, **WMESH["warped-twolevel-N4"])
    q0 = dev(vortex_state(o.XG, o.Lz)[:, perm])
    p = sem.sem_params_default(precision=prec)

    def steps(mesh, q, n):
        if prec == 0:
            w1, w2 = torch.empty_like(q), torch.empty_like(q)
            for _ in range(n):
                sem.sem_step(mesh, p, q, w1, w2, 1.0)
        else:
            q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
            work = torch.empty((10, mesh.NG), dtype=torch.float32, device="cuda")
            sem.sem_mirror(mesh, q, q32)
            for _ in range(n):
                sem.sem_step_mixed(mesh, p, q, q32, work, 1.0)
        return q

    a = steps(m, q0.clone(), 4)
    b = steps(m, q0.clone(), 2)
    path = tmp_path / "warped.ckpt"
    sem.sem_checkpoint_write(m, b, path, time=2.0, step=2)
    m2, t, s_ = sem.sem_checkpoint_read_mesh(path)
    c = torch.empty((5, m2.NG), dtype=torch.float64, device="cuda")
    sem.sem_checkpoint_read_state(path, m2, c)
    c = steps(m2, c, 2)
    torch.cuda.synchronize()
    assert torch.equal(a, c)
    box = sem.sem_mesh_create(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=two_level_leaves(), lvl_max=3)
    with pytest.raises(sem.SemError):          # written for the warped mesh
        sem.sem_checkpoint_read_state(path, box, c)


@pytest.mark.parametrize("name", ["warped-twolevel-N4", "warped-twolevel-N3"])
@pytest.mark.parametrize("eqset", ["C", "NC"])
@pytest.mark.parametrize("variables", [("vorticity",) * 3, ("pv",) * 3, ("speed", "vorticity", "pv")])
def test_warped_alternative_criteria_match_oracle(sem, name, eqset, variables):
    """Vorticity and potential vorticity on warped layers (derivatives at
    constant height through the node metric): element maxima within 1e-10
    of the oracle's and flags equal away from ties."""
    crit = {"speed": sem.SEM_CRIT_SPEED, "vorticity": sem.SEM_CRIT_VORTICITY, "pv": sem.SEM_CRIT_PV}
    m, o, X, perm = make_pair(sem, **WMESH[name])
    q_o = random_state(o.XG, o.Lz, 33, eqset, amp=0.2)
    lv = sem.sem_mesh_leaves_host(m)
    oleaf = {tuple(l): c for c, l in enumerate(o.leaves)}
    emap = np.array([oleaf[tuple(l)] * o.nz + k for l in lv for k in range(o.nz)])
    maxima = {v: adapt.CRITERIA[v](o, q_o, PRM, eqset).max(axis=1) for v in set(variables)}
    thr = [float(np.quantile(maxima[v], qq)) * (1 + 1e-6) for v, qq in zip(variables, (0.3, 0.6, 0.9))]
    fl_o, cmax_o = adapt.criterion_flags(o, q_o, PRM, thr, 3, eqset, variables=list(variables))
    p = sem.sem_params_default(eqset=0 if eqset == "C" else 1, thresholds=thr, lvl_max=3,
                               criterion=[crit[v] for v in variables])
    flags = torch.empty(m.Ne, dtype=torch.int8, device="cuda")
    cmax = torch.empty(m.Ne, dtype=torch.float64, device="cuda")
    sem.sem_adapt_flags(m, p, dev(q_o[:, perm]), flags, cmax)
    fl, cm = host(flags), host(cmax)
    np.testing.assert_allclose(cm, cmax_o[emap], rtol=1e-10, atol=1e-12 * np.abs(cmax_o).max())
    levels = o.level[emap]
    near = np.zeros(m.Ne, dtype=bool)
    for lvl in range(4):
        for t_idx in (lvl - 1, lvl):
            if 0 <= t_idx < 3:
                mx = maxima[variables[t_idx]][emap]
                near |= (levels == lvl) & (np.abs(mx - thr[t_idx]) <= 1e-9 * abs(thr[t_idx]))
    assert np.array_equal(fl[~near], fl_o[emap][~near])


def test_warped_refusals(sem):
    m, o, X, perm = make_pair(sem, **WMESH["warped-4x4x2-N4"])
    with pytest.raises(sem.SemError) as e:
        sem.sem_batch_create([m])
    assert e.value.code == sem.SEM_ERR_UNSUPPORTED
