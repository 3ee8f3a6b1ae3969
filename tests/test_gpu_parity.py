"""GPU parity: every C-ABI compute call against the CPU oracle on the same
seeded inputs.

Tolerances (relative L2 per field group {rho, momentum, theta}):
  FP64 form   <= 1e-12
  mixed form  <= 1e-4 on states after RK stages (full fields), and on
                 tendencies <= 1e-4 of the tendency norm
Flags of the criterion are integers decided in float64 on both sides: they
must agree exactly, except where the element maximum lies within 1e-12
(relative) of a threshold.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adapt, diag, mesh as om, refstate, rhs as orhs, rk as ork, transfer as otr  # noqa: E402
from synth.vortex import random_state, vortex_state, VortexSpec  # noqa: E402
from tests.helpers import group_rel_l2, node_perm, stretched_faces  # noqa: E402
from tests.test_oracle_mesh import two_level_leaves  # noqa: E402


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_21607_gb300 import build
    build.build()
    from paper_2410_21607_gb300 import sem as s
    return s


PRM = refstate.Params()


def make_pair(sem, L, Lz, nx, nz, N, leaves=None, periodic=(True, True), lvl_max=3, z_faces=None, warp=None):
    m = sem.sem_mesh_create(L, L, Lz, nx, nx, nz, N, leaves=leaves, periodic=periodic, lvl_max=lvl_max,
                            z_faces=z_faces, warp=warp)
    o = om.OracleMesh(L, L, Lz, nx, nx, nz, N, leaves=leaves, periodic=periodic, z_faces=z_faces, warp=warp)
    xyz = sem.sem_mesh_coords_host(m)
    perm = node_perm(xyz, o.XG)
    return m, o, xyz.T, perm


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def full_fields(q, z, eqset="C"):
    """Full (not perturbation) fields used by the state-level norms."""
    ref = refstate.reference_state(z, PRM)
    out = q.copy()
    out[0] += ref["rho0"]
    if eqset == "C":
        out[4] += ref["rhotheta0"]
    else:
        out[4] += ref["theta0"]
    return out


def increment_err(got, q0, ref):
    """Relative L2 error of the state's change (got - q0 against ref - q0)
    per field group: the dynamics, not the reference state that dominates
    the full fields."""
    return group_rel_l2(got - q0, ref - q0)


MESHES = {
    "uniform-6x6x4-N4": dict(L=600e3, Lz=24e3, nx=6, nz=4, N=4),
    "twolevel-N4": dict(L=300e3, Lz=12e3, nx=4, nz=2, N=4, leaves=two_level_leaves()),
    "twolevel-N3-open": dict(L=300e3, Lz=12e3, nx=4, nz=3, N=3, leaves=two_level_leaves(),
                             periodic=(False, False)),
    "uniform-5x4x3-N6": dict(L=500e3, Lz=12e3, nx=5, nz=3, N=6),
    "uniform-3x3x2-N2": dict(L=300e3, Lz=12e3, nx=3, nz=2, N=2),
    "twolevel-N5": dict(L=300e3, Lz=12e3, nx=4, nz=2, N=5, leaves=two_level_leaves()),
    # layers thickening upwards (top to bottom thickness 2.5), non-conforming
    "stretched-twolevel-N4": dict(L=300e3, Lz=12e3, nx=4, nz=3, N=4, leaves=two_level_leaves(),
                                  z_faces=stretched_faces(12e3, 3, 1.5)),
}


@pytest.mark.parametrize("name", list(MESHES))
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_rhs_fp64_matches_oracle(sem, name, eqset):
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = random_state(o.XG, o.Lz, 11, eqset)
    T_o = orhs.rhs(o, q_o, PRM, eqset)
    p = sem.sem_params_default(eqset=0 if eqset == "C" else 1)
    q = dev(q_o[:, perm])
    out = torch.empty_like(q)
    sem.sem_rhs(m, p, q, out)
    T = host(out)
    err = group_rel_l2(T, T_o[:, perm])
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("name", ["uniform-6x6x4-N4", "twolevel-N4", "stretched-twolevel-N4", "twolevel-N5"])
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_rhs_mixed_matches_oracle(sem, name, eqset):
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = random_state(o.XG, o.Lz, 12, eqset)
    T_o = orhs.rhs(o, q_o, PRM, eqset)
    p = sem.sem_params_default(eqset=0 if eqset == "C" else 1, precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    out = torch.empty_like(q)
    sem.sem_rhs(m, p, q, out)
    err = group_rel_l2(host(out), T_o[:, perm])
    assert np.all(err <= 1e-4), err


@pytest.mark.parametrize("name", ["twolevel-N4", "twolevel-17-layers-N4", "uniform-5x4x3-N6",
                                  "stretched-twolevel-N4", "twolevel-N5"])
def test_every_element_kernel_variant_matches_oracle(sem, name):
    """Each launch variant of the mixed element kernel (z-pencil and line
    exchange, every layers-per-CTA count) gives the
    mixed tendency within 1e-4 of the oracle.  17 layers make several layer
    chunks per column for every variant, so the carry of the top-face residual
    between chunks is exercised."""
    spec = dict(MESHES.get(name, {}))
    if name == "twolevel-17-layers-N4":
        spec = dict(L=300e3, Lz=24e3, nx=4, nz=17, N=4, leaves=two_level_leaves())
    m, o, X, perm = make_pair(sem, **spec)
    q_o = random_state(o.XG, o.Lz, 13)
    T_o = orhs.rhs(o, q_o, PRM)
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    rows, _ = sem.sem_autotune(m, p, q32, 1)
    assert len(rows) >= 2
    kinds = set()
    lines = []
    for row in list(range(len(rows))) + [-1]:
        sem.sem_autotune_select(m, row)
        out = torch.full_like(q, float("nan"))
        sem.sem_rhs(m, p, q, out)
        err = group_rel_l2(host(out), T_o[:, perm])
        assert np.all(err <= 1e-4), (row, rows[row] if row >= 0 else "default", err)
        if row >= 0:
            kinds.add(rows[row][3])
            if rows[row][3] in (1, 4):
                lines.append((rows[row], out.clone()))
    assert kinds == ({0, 1, 2, 4} if m.N == 4 else {0, 1})
    # the line-exchange variants do the same arithmetic per node whatever the
    # layers per CTA (the face shared by two chunks is summed as inside one)
    for r, o in lines[1:]:
        assert torch.equal(o, lines[0][1]), (r, lines[0][0])
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("name", ["twolevel-N4", "twolevel-17-layers-N4", "uniform-5x4x3-N6",
                                  "stretched-twolevel-N4", "twolevel-N5", "twolevel-N3-open",
                                  "uniform-3x3x2-N2"])
def test_every_paper_set_variant_matches_oracle(sem, name):
    """Each launch variant of the mixed element kernel of the paper's
    equation set (line exchange, kind 5) gives the mixed tendency within 1e-4
    of the oracle; 17 layers make several layer chunks per column, so the
    top-node carry between chunks is exercised, and two-level meshes give
    hanging lines.  The conservative set's choice is left as it was."""
    spec = dict(MESHES.get(name, {}))
    if name == "twolevel-17-layers-N4":
        spec = dict(L=300e3, Lz=24e3, nx=4, nz=17, N=4, leaves=two_level_leaves())
    m, o, X, perm = make_pair(sem, **spec)
    q_o = random_state(o.XG, o.Lz, 17, "NC")
    T_o = orhs.rhs(o, q_o, PRM, "NC")
    p = sem.sem_params_default(eqset=1, precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    rows, chosen = sem.sem_autotune(m, p, q32, 1)
    assert rows and {r[3] for r in rows} == {5}
    assert len(rows) == (4 if m.N == 4 else 1)
    outs = []
    for row in list(range(len(rows))) + [-1]:
        sem.sem_autotune_select(m, row, eqset=1)
        out = torch.full_like(q, float("nan"))
        sem.sem_rhs(m, p, q, out)
        err = group_rel_l2(host(out), T_o[:, perm])
        assert np.all(err <= 1e-4), (row, rows[row] if row >= 0 else "default", err)
        outs.append(out.clone())
    # the same arithmetic per node whatever the layers per CTA
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    assert sem.sem_status(m) == 0


def test_rest_state_exactly_steady_on_gpu(sem):
    m, o, X, perm = make_pair(sem, **MESHES["twolevel-N4"])
    for prec in (0, 1):
        for eq in (0, 1):
            p = sem.sem_params_default(eqset=eq, precision=prec)
            q = torch.zeros(5, m.NG, dtype=torch.float64, device="cuda")
            out = torch.full_like(q, 7.0)
            sem.sem_rhs(m, p, q, out)
            assert torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("prec", [0, 1])
def test_ten_rk3_steps_uniform_6x6x4(sem, prec):
    """The small workload: 10 SSP-RK3 steps at dt = 1 s on the 6x6x4 mesh."""
    m, o, X, perm = make_pair(sem, **MESHES["uniform-6x6x4-N4"])
    q_o = vortex_state(o.XG, o.Lz)
    q_ref = q_o.copy()
    for _ in range(10):
        q_ref = ork.rk_step(o, PRM, q_ref, 1.0)
    p = sem.sem_params_default(precision=prec)
    q = dev(q_o[:, perm])
    w1, w2 = torch.empty_like(q), torch.empty_like(q)
    for _ in range(10):
        sem.sem_step(m, p, q, w1, w2, 1.0)
    got = host(q)
    z = X[:, 2]
    err = group_rel_l2(full_fields(got, z), full_fields(q_ref[:, perm], z))
    tol = 1e-12 if prec == 0 else 1e-4
    assert np.all(err <= tol), err
    # the perturbation itself, and the change over the ten steps
    pert = group_rel_l2(got, q_ref[:, perm])
    assert np.all(pert <= (1e-11 if prec == 0 else 1e-3)), pert
    inc = increment_err(got, q_o[:, perm], q_ref[:, perm])
    assert np.all(inc <= (1e-10 if prec == 0 else 1e-4)), inc
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("stage", [0, 1, 2])
def test_rk_stage_on_nonconforming_mesh(sem, stage):
    m, o, X, perm = make_pair(sem, **MESHES["twolevel-N4"])
    qn_o = random_state(o.XG, o.Lz, 21)
    qs_o = random_state(o.XG, o.Lz, 22)
    ref = ork.rk_stage(o, PRM, stage, qn_o, qs_o, 0.7)
    p = sem.sem_params_default()
    qn, qs = dev(qn_o[:, perm]), dev(qs_o[:, perm])
    out = torch.empty_like(qn)
    sem.sem_rk_stage(m, p, stage, qn, qs, out, 0.7)
    err = group_rel_l2(host(out), ref[:, perm])
    assert np.all(err <= 1e-12), err


def test_mass_conservation_on_gpu(sem):
    m, o, X, perm = make_pair(sem, **MESHES["twolevel-N4"])
    M = sem.sem_mesh_mass_host(m)
    q = dev(random_state(o.XG, o.Lz, 5)[:, perm])
    out = torch.empty_like(q)
    for prec in (0, 1):
        sem.sem_rhs(m, sem.sem_params_default(precision=prec), q, out)
        T = host(out)
        tol = 1e-13 if prec == 0 else 1e-6
        assert abs(np.sum(M * T[0])) <= tol * np.sum(np.abs(M * T[0]))


@pytest.mark.parametrize("name", ["uniform-6x6x4-N4", "twolevel-N4"])
def test_adapt_flags_match_oracle(sem, name):
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = vortex_state(o.XG, o.Lz)
    lv = sem.sem_mesh_leaves_host(m)
    oleaf = {tuple(l): c for c, l in enumerate(o.leaves)}
    emap = np.array([oleaf[tuple(l)] * o.nz + k for l in lv for k in range(o.nz)])
    q = dev(q_o[:, perm])
    for thr in ([5.0, 10.0, 15.0], [2.0, 5.0, 7.5], [7.5, 15.0, 22.5]):
        fl_o, cmax_o = adapt.criterion_flags(o, q_o, PRM, thr, 3)
        p = sem.sem_params_default(thresholds=thr, lvl_max=3)
        flags = torch.empty(m.Ne, dtype=torch.int8, device="cuda")
        cmax = torch.empty(m.Ne, dtype=torch.float64, device="cuda")
        sem.sem_adapt_flags(m, p, q, flags, cmax)
        fl, cm = host(flags), host(cmax)
        np.testing.assert_allclose(cm, cmax_o[emap], rtol=1e-14)
        tie = np.min(np.abs(cmax_o[emap][:, None] - np.array(thr)[None]), axis=1) <= 1e-12 * max(thr)
        assert np.array_equal(fl[~tie], fl_o[emap][~tie])
        assert np.array_equal(sem.sem_adapt_flags_host(m, p, q), fl)


CRIT = {"speed": 0, "vorticity": 1, "pv": 2}


@pytest.mark.parametrize("name", ["uniform-6x6x4-N4", "twolevel-N4", "uniform-5x4x3-N6", "stretched-twolevel-N4"])
@pytest.mark.parametrize("eqset", ["C", "NC"])
@pytest.mark.parametrize("variables", [("vorticity",) * 3, ("pv",) * 3, ("speed", "vorticity", "pv")])
def test_adapt_flags_alternative_criteria_match_oracle(sem, name, eqset, variables):
    """Vorticity, potential vorticity and a per-level combination (Sec. 3.1's
    C^l): element maxima within 1e-10 and flags equal to the oracle's away
    from ties (the derivative sums are rounded in different orders)."""
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = random_state(o.XG, o.Lz, 31, eqset, amp=0.2)
    lv = sem.sem_mesh_leaves_host(m)
    oleaf = {tuple(l): c for c, l in enumerate(o.leaves)}
    emap = np.array([oleaf[tuple(l)] * o.nz + k for l in lv for k in range(o.nz)])
    # thresholds at quantiles of each level's variable, so that every flag occurs
    maxima = {v: adapt.CRITERIA[v](o, q_o, PRM, eqset).max(axis=1) for v in set(variables)}
    thr = [float(np.quantile(maxima[v], qq)) * (1 + 1e-6) for v, qq in zip(variables, (0.3, 0.6, 0.9))]
    fl_o, cmax_o = adapt.criterion_flags(o, q_o, PRM, thr, 3, eqset, variables=list(variables))
    p = sem.sem_params_default(eqset=0 if eqset == "C" else 1, thresholds=thr, lvl_max=3,
                               criterion=[CRIT[v] for v in variables])
    flags = torch.empty(m.Ne, dtype=torch.int8, device="cuda")
    cmax = torch.empty(m.Ne, dtype=torch.float64, device="cuda")
    sem.sem_adapt_flags(m, p, dev(q_o[:, perm]), flags, cmax)
    fl, cm = host(flags), host(cmax)
    np.testing.assert_allclose(cm, cmax_o[emap], rtol=1e-10, atol=1e-12 * np.abs(cmax_o).max())
    levels = o.level[emap]
    near = np.zeros(m.Ne, dtype=bool)
    for lvl in range(4):
        for t_idx in (lvl - 1, lvl):          # the coarsening and the refinement test
            if 0 <= t_idx < 3:
                mx = maxima[variables[t_idx]][emap]
                near |= (levels == lvl) & (np.abs(mx - thr[t_idx]) <= 1e-9 * abs(thr[t_idx]))
    assert np.array_equal(fl[~near], fl_o[emap][~near])
    assert len(set(fl.tolist())) >= 2


def test_transfer_matches_oracle(sem):
    """Refine by the criterion, then coarsen everything back: both transfers
    against the oracle's (interpolation, L2 projection, continuous projection)."""
    m, o, X, perm = make_pair(sem, L=600e3, Lz=24e3, nx=4, nz=2, N=4)
    q_o = vortex_state(o.XG, o.Lz)
    lv = [tuple(l) for l in sem.sem_mesh_leaves_host(m)]
    oleaf = {l: c for c, l in enumerate(o.leaves)}
    fl_o, _ = adapt.criterion_flags(o, q_o, PRM, [5.0, 10.0], 2)
    # flags in library element order
    fl_lib = np.array([fl_o[oleaf[l] * o.nz + k] for l in lv for k in range(o.nz)], dtype=np.int8)
    new = sem.sem_transfer_plan(m, fl_lib)
    new_o, org = adapt.update_leaves(o.leaves, fl_o, o.nz, 4, 4, 2)
    o2, q2_o = otr.transfer(o, new_o, org, q_o)
    perm2 = node_perm(sem.sem_mesh_coords_host(new), o2.XG)
    q = dev(q_o[:, perm])
    q2 = torch.empty(5, new.NG, dtype=torch.float64, device="cuda")
    sem.sem_transfer(m, new, q, q2)
    err = group_rel_l2(host(q2), q2_o[:, perm2])
    assert np.all(err <= 1e-12), err
    assert sem.sem_status(new) == 0
    # coarsen everything back
    back = sem.sem_transfer_plan(new, -np.ones(new.Ne, dtype=np.int8))
    q3 = torch.empty(5, back.NG, dtype=torch.float64, device="cuda")
    sem.sem_transfer(new, back, q2, q3)
    perm3 = node_perm(sem.sem_mesh_coords_host(back), o.XG)
    err = group_rel_l2(host(q3), q_o[:, perm3])
    assert np.all(err <= 1e-12), err


def test_transfer_coarsening_matches_oracle(sem):
    m, o, X, perm = make_pair(sem, **MESHES["twolevel-N4"])
    q_o = random_state(o.XG, o.Lz, 9)
    lv = [tuple(l) for l in sem.sem_mesh_leaves_host(m)]
    fl_lib = np.array([-1 if l[0] == 2 else (1 if l == (0, 0, 0) else 0)
                       for l in lv for _ in range(o.nz)], dtype=np.int8)
    oleaf = {tuple(l): c for c, l in enumerate(lv)}
    fl_o = np.zeros(o.Ne, dtype=np.int8)
    for c, l in enumerate(o.leaves):
        fl_o[c * o.nz:(c + 1) * o.nz] = fl_lib[oleaf[tuple(l)] * o.nz]
    new = sem.sem_transfer_plan(m, fl_lib)
    new_o, org = adapt.update_leaves(o.leaves, fl_o, o.nz, 4, 4, 3)
    o2, q2_o = otr.transfer(o, new_o, org, q_o)
    perm2 = node_perm(sem.sem_mesh_coords_host(new), o2.XG)
    q2 = torch.empty(5, new.NG, dtype=torch.float64, device="cuda")
    sem.sem_transfer(m, new, dev(q_o[:, perm]), q2)
    err = group_rel_l2(host(q2), q2_o[:, perm2])
    assert np.all(err <= 1e-12), err


@pytest.mark.parametrize("prec", [0, 1])
def test_adaptive_run_matches_oracle(sem, prec):
    """The whole adaptive cycle at reduced size: 8x8x4 base of a 600 km box
    (N = 4), geometric refinement to level 2 inside 150 km, thresholds
    [5, 10] m/s, 40 SSP-RK3 steps of 1 s with a remesh (criterion, topology
    update, transfer) after steps 20 and 40, on the GPU (float64 or mixed form)
    and in the oracle on its own meshes.  Flags are compared exactly away from
    ties; the meshes must stay identical; states at the end within 1e-10
    (float64) or 1e-4 (mixed) relative L2 of the full fields."""
    from synth.workloads import geometric_flags
    L, Lz, nx, nz, N, dt, lmax, thr = 600e3, 24e3, 8, 4, 4, 1.0, 2, [5.0, 10.0]
    m = sem.sem_mesh_create(L, L, Lz, nx, nx, nz, N, lvl_max=lmax)
    for _ in range(lmax):
        lv = [tuple(x) for x in sem.sem_mesh_leaves_host(m)]
        m = sem.sem_transfer_plan(m, geometric_flags(lv, nx, nz, L, 150e3, lmax))
    o = om.OracleMesh(L, L, Lz, nx, nx, nz, N, leaves=[tuple(x) for x in sem.sem_mesh_leaves_host(m)])
    q_o = vortex_state(o.XG, Lz)
    q = dev(q_o[:, node_perm(sem.sem_mesh_coords_host(m), o.XG)])
    p = sem.sem_params_default(precision=prec, thresholds=thr, lvl_max=lmax)
    ties = 0
    for cycle in range(2):
        if prec == 0:
            w1, w2 = torch.empty_like(q), torch.empty_like(q)
            for _ in range(20):
                sem.sem_step(m, p, q, w1, w2, dt)
        else:
            q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
            work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
            sem.sem_mirror(m, q, q32)
            for _ in range(20):
                sem.sem_step_mixed(m, p, q, q32, work, dt)
        for _ in range(20):
            q_o = ork.rk_step(o, PRM, q_o, dt)
        # criterion on both sides, in library element order
        lv = [tuple(x) for x in sem.sem_mesh_leaves_host(m)]
        oleaf = {tuple(l): c for c, l in enumerate(o.leaves)}
        emap = np.array([oleaf[l] * nz + k for l in lv for k in range(nz)])
        flags = torch.empty(m.Ne, dtype=torch.int8, device="cuda")
        cmax = torch.empty(m.Ne, dtype=torch.float64, device="cuda")
        sem.sem_adapt_flags(m, p, q, flags, cmax)
        fl_o, cmax_o = adapt.criterion_flags(o, q_o, PRM, thr, lmax)
        fl = host(flags)
        tie = np.min(np.abs(cmax_o[emap][:, None] - np.array(thr)[None]), axis=1) <= \
            (1e-12 if prec == 0 else 1e-5) * max(thr)
        assert np.array_equal(fl[~tie], fl_o[emap][~tie]), cycle
        ties += int(tie.sum())
        fl = fl_o[emap].astype(np.int8)      # identical meshes on both sides
        assert np.count_nonzero(fl) > 0
        new = sem.sem_transfer_plan(m, fl)
        new_o, org = adapt.update_leaves(o.leaves, fl_o, nz, nx, nx, lmax)
        assert sorted(tuple(x) for x in sem.sem_mesh_leaves_host(new)) == sorted(map(tuple, new_o))
        q2 = torch.empty(5, new.NG, dtype=torch.float64, device="cuda")
        sem.sem_transfer(m, new, q, q2)
        o, q_o = otr.transfer(o, new_o, org, q_o)
        m, q = new, q2
    perm = node_perm(sem.sem_mesh_coords_host(m), o.XG)
    z = o.XG[perm, 2]
    err = group_rel_l2(full_fields(host(q), z), full_fields(q_o[:, perm], z))
    assert np.all(err <= (1e-10 if prec == 0 else 1e-4)), err
    pert = group_rel_l2(host(q), q_o[:, perm])
    assert np.all(pert <= (1e-9 if prec == 0 else 1e-3)), pert
    assert ties <= 2
    assert sem.sem_status(m) == 0


def test_diag_matches_oracle(sem):
    m, o, X, perm = make_pair(sem, **MESHES["uniform-6x6x4-N4"])
    q_o = vortex_state(o.XG, o.Lz)
    d_o = diag.wind_diagnostics(o, q_o, PRM)
    d = sem.sem_diag(m, sem.sem_params_default(), dev(q_o[:, perm]))
    assert abs(d["max_wind"] - d_o["max_wind"]) <= 1e-12 * d_o["max_wind"]
    assert abs(d["max_mean_wind"] - d_o["max_mean_wind"]) <= 1e-12 * d_o["max_mean_wind"]


def test_coords_on_device_match_host(sem):
    m = sem.sem_mesh_create(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=two_level_leaves())
    xyz = torch.empty(3, m.NG, dtype=torch.float64, device="cuda")
    sem.sem_mesh_coords(m, xyz)
    assert np.array_equal(host(xyz), sem.sem_mesh_coords_host(m))


def test_nonfinite_state_sets_status(sem):
    m = sem.sem_mesh_create(300e3, 300e3, 12e3, 3, 3, 2, 4)
    q = torch.zeros(5, m.NG, dtype=torch.float64, device="cuda")
    q[1, 17] = float("nan")
    w1, w2 = torch.empty_like(q), torch.empty_like(q)
    sem.sem_step(m, sem.sem_params_default(), q, w1, w2, 1.0)
    assert sem.sem_status(m) == sem.SEM_ERR_NUMERIC
    assert sem.sem_status(m) == 0       # reading clears it


def test_fp64_second_stage_special_values(sem):
    """The float64 second SSP-RK3 stage forms qs / 4 from the bits of qs
    (exponent lowered by 2): against 3/4 qn + 1/4 qs + dt/4 R(qs) formed here
    from the library's float64 right-hand side, for stage states holding
    signed zeros and values near the bottom of the normal range; a
    non-finite stage state still raises the status."""
    m, o, X, perm = make_pair(sem, **MESHES["twolevel-N4"])
    qn = dev(random_state(o.XG, o.Lz, 81)[:, perm])
    qs = dev(random_state(o.XG, o.Lz, 82)[:, perm])
    qs[3, ::7] = 0.0
    qs[3, 3::7] = -0.0
    qs[1, ::11] = 3e-306
    qs[2, ::13] = -5e-307
    qs[0, ::17] = 1e-308          # its quarter is subnormal: the kernel gives zero
    p = sem.sem_params_default()
    R = torch.empty_like(qs)
    sem.sem_rhs(m, p, qs, R)
    dt = 0.5
    out = torch.empty_like(qs)
    sem.sem_rk_stage(m, p, 1, qn, qs, out, dt)
    want = 0.75 * host(qn) + 0.25 * host(qs) + (0.25 * dt) * host(R)
    got = host(out)
    scale = np.abs(want).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - want) <= 1e-14 * scale)
    assert sem.sem_status(m) == 0
    qs[4, 5] = float("inf")
    sem.sem_rk_stage(m, p, 1, qn, qs, out, dt)
    assert sem.sem_status(m) == sem.SEM_ERR_NUMERIC


def test_bad_arguments_are_rejected(sem):
    m = sem.sem_mesh_create(300e3, 300e3, 12e3, 3, 3, 2, 4)
    q = torch.zeros(5, m.NG, dtype=torch.float64, device="cuda")
    p = sem.sem_params_default()
    with pytest.raises(sem.SemError):
        sem.sem_rhs(m, p, q, q)                       # aliasing
    with pytest.raises(sem.SemError):
        sem.sem_rk_stage(m, p, 3, q, q, torch.empty_like(q), 1.0)
    p.eqset = 7
    with pytest.raises(sem.SemError):
        sem.sem_rhs(m, p, q, torch.empty_like(q))


def test_mixed_stage_with_mirrors_matches_oracle(sem):
    """sem_rk_stage_mixed with caller-owned float32 mirrors, ten SSP-RK3 steps
    on the non-conforming mesh, against the oracle's float64 steps."""
    m, o, X, perm = make_pair(sem, **MESHES["twolevel-N4"])
    q_o = vortex_state(o.XG, o.Lz)
    q_ref = q_o.copy()
    for _ in range(10):
        q_ref = ork.rk_step(o, PRM, q_ref, 1.0)
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    w1, w2 = torch.empty_like(q), torch.empty_like(q)
    q32, w132, w232 = (torch.empty(q.shape, dtype=torch.float32, device="cuda") for _ in range(3))
    sem.sem_mirror(m, q, q32)
    np.testing.assert_allclose(host(q32), host(q), rtol=2.4e-7)
    for _ in range(10):
        sem.sem_rk_stage_mixed(m, p, 0, q, q, q32, w1, w132, 1.0)
        sem.sem_rk_stage_mixed(m, p, 1, q, w1, w132, w2, w232, 1.0)
        sem.sem_rk_stage_mixed(m, p, 2, q, w2, w232, w1, w132, 1.0)
        q, w1, q32, w132 = w1, q, w132, q32
    got = host(q)
    z = X[:, 2]
    err = group_rel_l2(full_fields(got, z), full_fields(q_ref[:, perm], z))
    assert np.all(err <= 1e-4), err
    inc = increment_err(got, q_o[:, perm], q_ref[:, perm])
    assert np.all(inc <= 1e-4), inc
    np.testing.assert_allclose(host(q32), got, rtol=2.4e-7, atol=1e-30)
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("name", ["uniform-6x6x4-N4", "twolevel-N4", "uniform-3x3x2-N2", "uniform-5x4x3-N6",
                                  "stretched-twolevel-N4", "twolevel-N5"])
def test_step_mixed_increment_form_matches_oracle(sem, name):
    """sem_step_mixed (float32 stage increments, one float64 accumulation per
    step) against ten float64 oracle steps."""
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = vortex_state(o.XG, o.Lz)
    dt = 0.5 if name in ("uniform-5x4x3-N6", "stretched-twolevel-N4", "twolevel-N5") else 1.0
    q_ref = q_o.copy()
    for _ in range(10):
        q_ref = ork.rk_step(o, PRM, q_ref, dt)
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    for _ in range(10):
        sem.sem_step_mixed(m, p, q, q32, work, dt)
    got = host(q)
    z = X[:, 2]
    err = group_rel_l2(full_fields(got, z), full_fields(q_ref[:, perm], z))
    assert np.all(err <= 1e-4), err
    pert = group_rel_l2(got, q_ref[:, perm])
    assert np.all(pert <= 1e-3), pert
    inc = increment_err(got, q_o[:, perm], q_ref[:, perm])
    assert np.all(inc <= 1e-4), inc
    np.testing.assert_allclose(host(q32), got, rtol=2.4e-7, atol=1e-30)
    assert sem.sem_status(m) == 0


def test_autotune_then_step_parity(sem):
    """Every element-kernel variant the autotuner times gives the same
    (correct) step: tune, then check the increment-form step again."""
    m, o, X, perm = make_pair(sem, **MESHES["twolevel-N4"])
    q_o = vortex_state(o.XG, o.Lz)
    q_ref = ork.rk_step(o, PRM, q_o, 1.0)
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    rows, chosen = sem.sem_autotune(m, p, q32, 2)
    assert len(rows) >= 2 and 0 <= chosen < len(rows)
    assert all(r[2] > 0 for r in rows)
    sem.sem_step_mixed(m, p, q, q32, work, 1.0)
    z = X[:, 2]
    err = group_rel_l2(full_fields(host(q), z), full_fields(q_ref[:, perm], z))
    assert np.all(err <= 1e-4), err


@pytest.mark.parametrize("name", ["twolevel-N4", "twolevel-17-layers-N4", "stretched-twolevel-N4", "twolevel-N5"])
def test_every_variant_step_matches_oracle(sem, name):
    """The increment-form step through each element-kernel variant (z-pencil
    and line exchange, every layers-per-CTA count): two steps within 1e-4 of
    the oracle, the mirror equal to the state rounded to float32, and the
    line-exchange variants (the same arithmetic per node) within 1e-5 of each
    other in the state's change."""
    spec = dict(MESHES.get(name, {}))
    if name == "twolevel-17-layers-N4":
        spec = dict(L=300e3, Lz=24e3, nx=4, nz=17, N=4, leaves=two_level_leaves())
    m, o, X, perm = make_pair(sem, **spec)
    q_o = vortex_state(o.XG, o.Lz)
    q_ref = q_o.copy()
    for _ in range(2):
        q_ref = ork.rk_step(o, PRM, q_ref, 0.5)
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q0 = dev(q_o[:, perm])
    q32 = torch.empty(q0.shape, dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q0, q32)
    rows, _ = sem.sem_autotune(m, p, q32, 1)
    z = X[:, 2]
    lines = []
    for row in range(len(rows)):
        sem.sem_autotune_select(m, row)
        q = q0.clone()
        sem.sem_mirror(m, q, q32)
        work = torch.full((10, m.NG), float("nan"), dtype=torch.float32, device="cuda")
        for _ in range(2):
            sem.sem_step_mixed(m, p, q, q32, work, 0.5)
        got = host(q)
        err = group_rel_l2(full_fields(got, z), full_fields(q_ref[:, perm], z))
        assert np.all(err <= 1e-4), (row, rows[row], err)
        inc = increment_err(got, q_o[:, perm], q_ref[:, perm])
        assert np.all(inc <= 1e-4), (row, rows[row], inc)
        np.testing.assert_allclose(host(q32), got, rtol=2.4e-7, atol=1e-30)
        if rows[row][3] == 1:
            lines.append(got)
    assert len(lines) >= 2
    for got in lines[1:]:
        assert np.all(group_rel_l2(got - q_o[:, perm], lines[0] - q_o[:, perm]) <= 1e-5)
    assert sem.sem_status(m) == 0


def _instance_mesh(sem, nx, nz, N, L, levels, radius):
    from synth.workloads import geometric_flags
    m = sem.sem_mesh_create(L, L, 24e3, nx, nx, nz, N, lvl_max=max(levels, 1))
    for _ in range(levels):
        lv = [tuple(x) for x in sem.sem_mesh_leaves_host(m)]
        m = sem.sem_transfer_plan(m, geometric_flags(lv, nx, nz, L, radius, levels))
    return m


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("with_big", [False, True])
def test_batched_steps_equal_single_mesh_steps(sem, use_graph, with_big):
    """One persistent launch per stage over five meshes of different order,
    size and refinement gives the same states as stepping each mesh alone.
    With with_big, two meshes large enough to fill the GPU (at least 2 x SMs
    columns) join them: they keep their own tuned launches, on branch streams
    that run beside the shared queue."""
    specs = [(4, 2, 3, 300e3, 0), (4, 3, 4, 300e3, 1), (3, 2, 5, 300e3, 0),
             (3, 2, 6, 300e3, 1), (5, 17, 2, 300e3, 0)]
    dts = [0.5, 0.25, 0.4, 0.2, 1.0]
    if with_big:
        specs += [(18, 1, 2, 300e3, 0), (20, 2, 3, 300e3, 0)]
        dts += [0.5, 0.5]
    meshes = [_instance_mesh(sem, nx, nz, N, L, lev, 120e3) for nx, nz, N, L, lev in specs]
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    init = [dev(random_state(sem.sem_mesh_coords_host(m).T, 24e3, 30 + k)) for k, m in enumerate(meshes)]

    def fresh():
        qs = [q.clone() for q in init]
        q32 = [torch.empty(q.shape, dtype=torch.float32, device="cuda") for q in qs]
        work = [torch.empty((10, q.shape[1]), dtype=torch.float32, device="cuda") for q in qs]
        for m, q, a in zip(meshes, qs, q32):
            sem.sem_mirror(m, q, a)
        return qs, q32, work

    # the batch first: it tunes the large meshes' element kernels, which the
    # single-mesh steps then use as well
    qb, b32, wb = fresh()
    batch = sem.sem_batch_create(meshes)
    for _ in range(2):
        sem.sem_batch_step_mixed(batch, p, qb, b32, wb, dts, use_graph=use_graph)
    qa, a32, wa = fresh()
    for _ in range(2):
        for k, m in enumerate(meshes):
            sem.sem_step_mixed(m, p, qa[k], a32[k], wa[k], dts[k])
    torch.cuda.synchronize()
    if with_big:
        assert min(m.Ncol for m in meshes[-2:]) >= 2 * torch.cuda.get_device_properties(0).multi_processor_count
    for k in range(len(meshes)):
        d = (qa[k] - qb[k]).abs().max().item()
        scale = qa[k].abs().max().item()
        assert d <= 1e-13 * scale, (k, d)
        assert torch.equal(a32[k], b32[k]) or (a32[k] - b32[k]).abs().max().item() <= 1e-6
    assert sem.sem_batch_status(batch) == 0


@pytest.mark.parametrize("use_graph", [False, True])
@pytest.mark.parametrize("with_big", [False, True])
def test_batched_steps_match_oracle(sem, use_graph, with_big):
    """The batched step against the oracle: meshes of orders 3, 4, 5 and 6,
    each refined by one level inside 120 km (2:1 faces), plus an unrefined
    order-4 mesh, run together by sem_batch_step_mixed (the persistent
    column-queue element kernel and the concatenated increment kernel, with
    or without graph replay); with with_big, two meshes large enough for their
    own launches join them.  After two steps every instance's state is within
    1e-4 (relative L2 per field group) of two float64 oracle steps on its own
    mesh, in the full fields and in the change of the state."""
    specs = [(4, 2, 3, 300e3, 1), (4, 2, 4, 300e3, 1), (3, 2, 5, 300e3, 1),
             (3, 2, 6, 300e3, 1), (5, 3, 4, 300e3, 0)]
    dts = [0.5, 0.5, 0.4, 0.25, 0.5]
    if with_big:
        specs += [(18, 1, 2, 300e3, 0), (20, 2, 3, 300e3, 0)]
        dts += [0.5, 0.5]
    meshes = [_instance_mesh(sem, nx, nz, N, L, lev, 120e3) for nx, nz, N, L, lev in specs]
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    oracles, perms, init = [], [], []
    for k, (m, (nx, nz, N, L, lev)) in enumerate(zip(meshes, specs)):
        o = om.OracleMesh(L, L, 24e3, nx, nx, nz, N, leaves=[tuple(x) for x in sem.sem_mesh_leaves_host(m)])
        perm = node_perm(sem.sem_mesh_coords_host(m), o.XG)
        q_o = random_state(o.XG, 24e3, 40 + k)
        oracles.append((o, q_o))
        perms.append(perm)
        init.append(dev(q_o[:, perm]))
    if with_big:
        assert min(m.Ncol for m in meshes[-2:]) >= 2 * torch.cuda.get_device_properties(0).multi_processor_count
    assert sum(1 for m, s in zip(meshes, specs) if s[4] and m.Ncol > s[0] ** 2) == 4
    qs = [q.clone() for q in init]
    q32 = [torch.empty(q.shape, dtype=torch.float32, device="cuda") for q in qs]
    work = [torch.empty((10, q.shape[1]), dtype=torch.float32, device="cuda") for q in qs]
    for m, q, a in zip(meshes, qs, q32):
        sem.sem_mirror(m, q, a)
    batch = sem.sem_batch_create(meshes)
    for _ in range(2):
        sem.sem_batch_step_mixed(batch, p, qs, q32, work, dts, use_graph=use_graph)
    assert sem.sem_batch_status(batch) == 0
    for k, ((o, q_o), perm, m) in enumerate(zip(oracles, perms, meshes)):
        q_ref = q_o
        for _ in range(2):
            q_ref = ork.rk_step(o, PRM, q_ref, dts[k])
        got = host(qs[k])
        z = o.XG[perm, 2]
        err = group_rel_l2(full_fields(got, z), full_fields(q_ref[:, perm], z))
        assert np.all(err <= 1e-4), (k, specs[k], err)
        inc = increment_err(got, q_o[:, perm], q_ref[:, perm])
        assert np.all(inc <= 1e-4), (k, specs[k], inc)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_paper_set_matches_oracle_and_single_mesh_steps(sem, use_graph):
    """The batched step with the paper's equation set (the persistent queue
    over that set's line-exchange body): meshes of orders 3 to 6, refined by
    one level (2:1 faces), an unrefined one with 17 layers, and two meshes
    large enough for their own launches.  After two steps every instance is
    within 1e-4 of two float64 oracle steps (full fields and change) and
    within 1e-13 of stepping each mesh alone; a conservative-set step of the
    same batch afterwards still matches its single-mesh steps (the tables,
    tuning and graph follow the set)."""
    specs = [(4, 2, 3, 300e3, 1), (4, 2, 4, 300e3, 1), (3, 2, 5, 300e3, 1),
             (3, 2, 6, 300e3, 1), (5, 17, 4, 300e3, 0), (18, 1, 2, 300e3, 0), (20, 2, 3, 300e3, 0)]
    dts = [0.5, 0.5, 0.4, 0.25, 0.5, 0.5, 0.5]
    meshes = [_instance_mesh(sem, nx, nz, N, L, lev, 120e3) for nx, nz, N, L, lev in specs]
    assert min(m.Ncol for m in meshes[-2:]) >= 2 * torch.cuda.get_device_properties(0).multi_processor_count
    p = sem.sem_params_default(eqset=1, precision=sem.SEM_PREC_MIXED)
    oracles, perms, init = [], [], []
    for k, (m, (nx, nz, N, L, lev)) in enumerate(zip(meshes, specs)):
        o = om.OracleMesh(L, L, 24e3, nx, nx, nz, N, leaves=[tuple(x) for x in sem.sem_mesh_leaves_host(m)])
        perm = node_perm(sem.sem_mesh_coords_host(m), o.XG)
        q_o = random_state(o.XG, 24e3, 60 + k, "NC")
        oracles.append((o, q_o))
        perms.append(perm)
        init.append(dev(q_o[:, perm]))

    def fresh(states):
        qs = [q.clone() for q in states]
        q32 = [torch.empty(q.shape, dtype=torch.float32, device="cuda") for q in qs]
        work = [torch.empty((10, q.shape[1]), dtype=torch.float32, device="cuda") for q in qs]
        for m, q, a in zip(meshes, qs, q32):
            sem.sem_mirror(m, q, a)
        return qs, q32, work

    qb, b32, wb = fresh(init)
    batch = sem.sem_batch_create(meshes)
    for _ in range(2):
        sem.sem_batch_step_mixed(batch, p, qb, b32, wb, dts, use_graph=use_graph)
    assert sem.sem_batch_status(batch) == 0
    qa, a32, wa = fresh(init)
    for _ in range(2):
        for k, m in enumerate(meshes):
            sem.sem_step_mixed(m, p, qa[k], a32[k], wa[k], dts[k])
    torch.cuda.synchronize()
    for k, ((o, q_o), perm) in enumerate(zip(oracles, perms)):
        q_ref = q_o
        for _ in range(2):
            q_ref = ork.rk_step(o, PRM, q_ref, dts[k], "NC")
        got = host(qb[k])
        z = o.XG[perm, 2]
        err = group_rel_l2(full_fields(got, z, "NC"), full_fields(q_ref[:, perm], z, "NC"))
        assert np.all(err <= 1e-4), (k, specs[k], err)
        inc = increment_err(got, q_o[:, perm], q_ref[:, perm])
        assert np.all(inc <= 1e-4), (k, specs[k], inc)
        d = (qa[k] - qb[k]).abs().max().item()
        assert d <= 1e-13 * qa[k].abs().max().item(), (k, d)
    # the same batch with the conservative set
    pc = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    initc = [dev(random_state(sem.sem_mesh_coords_host(m).T, 24e3, 80 + k)) for k, m in enumerate(meshes)]
    qb, b32, wb = fresh(initc)
    sem.sem_batch_step_mixed(batch, pc, qb, b32, wb, dts, use_graph=use_graph)
    qa, a32, wa = fresh(initc)
    for k, m in enumerate(meshes):
        sem.sem_step_mixed(m, pc, qa[k], a32[k], wa[k], dts[k])
    torch.cuda.synchronize()
    for k in range(len(meshes)):
        d = (qa[k] - qb[k]).abs().max().item()
        assert d <= 1e-13 * qa[k].abs().max().item(), (k, d)
    assert sem.sem_batch_status(batch) == 0


def test_mixed_pressure_both_branches(sem):
    """The mixed form evaluates (1 + x)^gamma - 1, x = (rho theta)'/(rho theta)0,
    by its binomial series for |x| <= 1/8 and by expm1/log1p beyond: a state
    with |x| up to about 0.3 exercises both against the oracle."""
    m, o, X, perm = make_pair(sem, **MESHES["uniform-6x6x4-N4"])
    q_o = random_state(o.XG, o.Lz, 13)
    rng = np.random.default_rng(0)
    ref = refstate.reference_state(o.XG[:, 2], PRM)
    q_o[4] = ref["rhotheta0"] * rng.uniform(-0.3, 0.3, size=o.NG)
    q_o[3, o.z_bottom | o.z_top] = 0.0
    T_o = orhs.rhs(o, q_o, PRM, "C")
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    out = torch.empty_like(q)
    sem.sem_rhs(m, p, q, out)
    err = group_rel_l2(host(out), T_o[:, perm])
    assert np.all(err <= 1e-4), err


@pytest.mark.parametrize("name", ["twolevel-N4", "stretched-twolevel-N4"])
@pytest.mark.parametrize("prec", [0, 1])
def test_checkpoint_resume_is_bitwise(sem, prec, tmp_path, name):
    """Six steps straight through equal three steps, checkpoint, a fresh mesh
    and state read back from the file, and three more steps, bit for bit."""
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q0 = dev(vortex_state(o.XG, o.Lz)[:, perm])
    p = sem.sem_params_default(precision=prec)
    dt = 0.5 if "stretched" in name else 1.0

    def steps(mesh, q, n):
        if prec == 0:
            w1, w2 = torch.empty_like(q), torch.empty_like(q)
            for _ in range(n):
                sem.sem_step(mesh, p, q, w1, w2, dt)
        else:
            q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
            work = torch.empty((10, mesh.NG), dtype=torch.float32, device="cuda")
            sem.sem_mirror(mesh, q, q32)
            for _ in range(n):
                sem.sem_step_mixed(mesh, p, q, q32, work, dt)
        return q

    a = steps(m, q0.clone(), 6)
    b = steps(m, q0.clone(), 3)
    path = tmp_path / "state.ckpt"
    sem.sem_checkpoint_write(m, b, path, time=3.0, step=3)
    m2, t, s = sem.sem_checkpoint_read_mesh(path)
    assert (t, s) == (3.0, 3)
    c = torch.empty((5, m2.NG), dtype=torch.float64, device="cuda")
    sem.sem_checkpoint_read_state(path, m2, c)
    c = steps(m2, c, 3)
    torch.cuda.synchronize()
    assert torch.equal(a, c)


@pytest.mark.parametrize("name", ["twolevel-N4", "uniform-5x4x3-N6"])
def test_adapt_flags_at_given_levels_match_oracle(sem, name):
    """sem_adapt_flags_levels: the rule evaluated at per-element levels (random
    levels 0..3) and at one level for all, against the oracle's rule at the
    same levels; flags equal away from ties, maxima within 1e-14."""
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = vortex_state(o.XG, o.Lz)
    lv = sem.sem_mesh_leaves_host(m)
    oleaf = {tuple(l): c for c, l in enumerate(o.leaves)}
    emap = np.array([oleaf[tuple(l)] * o.nz + k for l in lv for k in range(o.nz)])
    thr = [2.0, 5.0, 7.5]
    p = sem.sem_params_default(thresholds=thr, lvl_max=3)
    q = dev(q_o[:, perm])
    rng = np.random.default_rng(3)
    lev_lib = rng.integers(0, 4, size=m.Ne).astype(np.int8)
    lev_o = np.zeros(o.Ne, dtype=np.int64)
    lev_o[emap] = lev_lib
    cases = [(dev(lev_lib), -1, lev_o)] + [(None, L, np.full(o.Ne, L)) for L in range(4)]
    for lev_dev, L, lev_oracle in cases:
        fl_o, cmax_o = adapt.criterion_flags(o, q_o, PRM, thr, 3, levels=lev_oracle)
        flags = torch.empty(m.Ne, dtype=torch.int8, device="cuda")
        cmax = torch.empty(m.Ne, dtype=torch.float64, device="cuda")
        sem.sem_adapt_flags_levels(m, p, q, flags, level=lev_dev, level_all=L, cmax=cmax)
        fl, cm = host(flags), host(cmax)
        np.testing.assert_allclose(cm, cmax_o[emap], rtol=1e-14)
        tie = np.min(np.abs(cmax_o[emap][:, None] - np.array(thr)[None]), axis=1) <= 1e-12 * max(thr)
        assert np.array_equal(fl[~tie], fl_o[emap][~tie]), L
        if lev_dev is not None:
            assert len(set(fl.tolist())) >= 2
    with pytest.raises(sem.SemError):
        sem.sem_adapt_flags_levels(m, p, q, flags, level_all=4)


def test_merge_flags_every_combination(sem):
    """sem_merge_flags on every (criterion, prediction, level) combination:
    refine if either asks, coarsen only if both do, requests the level
    cannot take (refine at lvl_max, coarsen at 0) count as keep."""
    lvl_max = 2
    c, pr, lv = np.meshgrid([-1, 0, 1], [-1, 0, 1], range(lvl_max + 1), indexing="ij")
    c, pr, lv = c.ravel(), pr.ravel(), lv.ravel()
    want = np.empty_like(c)
    for k in range(len(c)):
        cc, pp = c[k], pr[k]
        if lv[k] >= lvl_max:
            cc, pp = min(cc, 0), min(pp, 0)
        if lv[k] <= 0:
            cc, pp = max(cc, 0), max(pp, 0)
        want[k] = 1 if (cc > 0 or pp > 0) else (-1 if (cc < 0 and pp < 0) else 0)
    t = lambda a: dev(a.astype(np.int8))
    got = host(sem.sem_merge_flags(t(c), t(pr), t(lv), lvl_max))
    assert np.array_equal(got, want.astype(np.int8))


@pytest.mark.parametrize("name", ["twolevel-17-layers-N4", "uniform-6x6x4-N4"])
def test_tma_staged_variant_equals_plain_variant(sem, name):
    """The line-exchange variant that stages the state with bulk copies (TMA,
    kind 4) reads the same values as the plain one with the same layers and
    CTAs per SM: the stage's outputs are equal bit for bit, with a 16-byte
    aligned mirror (staged) and with one offset by 4 bytes (the plain loads);
    17 layers give three chunks and the prefetch between them, the two-level
    mesh hanging lines that are not staged."""
    spec = dict(MESHES.get(name, {}))
    if name == "twolevel-17-layers-N4":
        spec = dict(L=300e3, Lz=24e3, nx=4, nz=17, N=4, leaves=two_level_leaves())
    m, o, X, perm = make_pair(sem, **spec)
    q = dev(random_state(o.XG, o.Lz, 14)[:, perm])
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    rows, _ = sem.sem_autotune(m, p, q32, 1)
    row = {(r[0], r[1], r[3]): k for k, r in enumerate(rows)}
    big = torch.empty(q.numel() + 4, dtype=torch.float32, device="cuda")
    shifted = big[1:1 + q.numel()].view(q.shape)      # 4 bytes past a 16-byte boundary
    shifted.copy_(q32)
    assert q32.data_ptr() % 16 == 0 and shifted.data_ptr() % 16 == 4
    for mb in (3, 2):
        for mirror in (q32, shifted):
            outs = []
            for kind in (1, 4):
                sem.sem_autotune_select(m, row[(8, mb, kind)])
                out, out32 = torch.empty_like(q), torch.empty_like(q32)
                sem.sem_rk_stage_mixed(m, p, 0, q, q, mirror, out, out32, 0.5)
                outs.append((out, out32))
            torch.cuda.synchronize()
            assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1]), (mb, mirror.data_ptr() % 16)
    assert sem.sem_status(m) == 0


@pytest.mark.parametrize("name", ["uniform-6x6x4-N4", "twolevel-N4", "twolevel-N3-open", "uniform-5x4x3-N6",
                                  "stretched-twolevel-N4"])
def test_step_mixed_paper_set_matches_oracle(sem, name):
    """sem_step_mixed with the paper's set (rho', u, v, w, theta'): the column
    element kernel feeds the same increment-form stages; ten steps against
    the oracle's, 1e-4 in the full fields and in the change, and against the
    mixed stage-by-stage form (sem_rk_stage_mixed) at 1e-5 of the change."""
    m, o, X, perm = make_pair(sem, **MESHES[name])
    q_o = vortex_state(o.XG, o.Lz, eqset="NC")
    dt = 0.5 if name in ("uniform-5x4x3-N6", "stretched-twolevel-N4") else 1.0
    q_ref = q_o.copy()
    for _ in range(10):
        q_ref = ork.rk_step(o, PRM, q_ref, dt, eqset="NC")
    p = sem.sem_params_default(eqset=1, precision=sem.SEM_PREC_MIXED)
    q = dev(q_o[:, perm])
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32)
    for _ in range(10):
        sem.sem_step_mixed(m, p, q, q32, work, dt)
    got = host(q)
    z = X[:, 2]
    assert np.all(group_rel_l2(full_fields(got, z, "NC"), full_fields(q_ref[:, perm], z, "NC")) <= 1e-4)
    assert np.all(increment_err(got, q_o[:, perm], q_ref[:, perm]) <= 1e-4)
    # the stage-by-stage mixed form (float64 stage states) on the same steps
    qs = dev(q_o[:, perm])
    w1, w2 = torch.empty_like(qs), torch.empty_like(qs)
    m1, m2 = torch.empty(q32.shape, dtype=torch.float32, device="cuda"), torch.empty_like(q32)
    m0 = torch.empty_like(q32)
    for _ in range(10):
        sem.sem_mirror(m, qs, m0)
        sem.sem_rk_stage_mixed(m, p, 0, qs, qs, m0, w1, m1, dt)
        sem.sem_rk_stage_mixed(m, p, 1, qs, w1, m1, w2, m2, dt)
        sem.sem_rk_stage_mixed(m, p, 2, qs, w2, m2, w1, m1, dt)
        qs.copy_(w1)
    assert np.all(increment_err(got, q_o[:, perm], host(qs)) <= 1e-5)
    assert sem.sem_status(m) == 0
