"""Pins of the oracle's criterion, mesh update, transfer and diagnostics
(Sec. 3.1-3.2, Algorithm 3, Sec. 4.2)."""
import itertools

import numpy as np
import pytest

from oracle import adapt, diag, mesh, refstate, transfer
from synth.vortex import vortex_state, random_state
from tests.test_oracle_mesh import two_level_leaves

PRM = refstate.Params()


def _state_with_speed(m, speed_per_col):
    """EqSet C state whose velocity magnitude is constant per column."""
    ref = refstate.reference_state(m.XG[:, 2], PRM)
    q = np.zeros((5, m.NG))
    # assign every global node the speed of the (first) column owning it
    sp = np.zeros(m.NG)
    for e in range(m.Ne):
        g = m.gid[e * m.P:(e + 1) * m.P]
        g = g[g >= 0]
        sp[g] = speed_per_col[m.col[e]]
    q[1] = sp * ref["rho0"]
    return q


def test_criterion_hand_example():
    """Constant speed everywhere on a mesh with levels 0, 1 and 2; thresholds
    [5, 10], lvl_max = 2 (text rule of Sec. 3.1)."""
    m = mesh.OracleMesh(300e3, 300e3, 12e3, 4, 4, 1, 4, leaves=two_level_leaves())
    ref = refstate.reference_state(m.XG[:, 2], PRM)
    expect = {  # speed -> flag per level (0, 1, 2)
        1.0: (0, -1, -1),    # <= thr(1)=5: coarsen where possible
        7.0: (1, 0, -1),     # 5 < 7 <= 10
        12.0: (1, 1, 0),     # > 10; level 2 is lvl_max
    }
    for speed, per_level in expect.items():
        q = np.zeros((5, m.NG))
        q[2] = speed * ref["rho0"]
        fl, cmax = adapt.criterion_flags(m, q, PRM, [5.0, 10.0], lvl_max=2)
        np.testing.assert_allclose(cmax, speed, rtol=1e-14)
        for e in range(m.Ne):
            assert fl[e] == per_level[m.level[e]]


def test_criterion_rule_brute_force():
    m = mesh.OracleMesh(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=two_level_leaves())
    q = vortex_state(m.XG, 12e3)
    for thr in ([5.0, 10.0], [2.0, 5.0], [7.5, 15.0, 22.5]):
        lvl_max = len(thr)
        fl, cmax = adapt.criterion_flags(m, q, PRM, thr, lvl_max)
        s = adapt.criterion_speed(m, q, PRM)
        for e in range(m.Ne):
            lv = m.level[e]
            up = lv < lvl_max and np.any(s[e] > thr[lv])
            down = lv > 0 and np.all(s[e] <= thr[lv - 1])
            assert fl[e] == (1 if up else (-1 if down else 0))
        assert set(np.unique(fl)) <= {-1, 0, 1}


def test_criterion_monotone_in_thresholds():
    m = mesh.OracleMesh(600e3, 600e3, 24e3, 6, 6, 2, 4)
    q = vortex_state(m.XG, 24e3)
    f1, _ = adapt.criterion_flags(m, q, PRM, [5.0, 10.0], 2)
    f2, _ = adapt.criterion_flags(m, q, PRM, [8.0, 16.0], 2)
    assert np.all(f2 <= f1)           # stricter thresholds never refine more


def _random_balanced_leaves(rng, nx, ny, lmax, steps=6):
    leaves = [(0, i, j) for j in range(ny) for i in range(nx)]
    for _ in range(steps):
        fl = rng.integers(-1, 2, size=len(leaves)).astype(np.int8)
        leaves, _ = adapt.update_leaves(leaves, fl, 1, nx, ny, lmax)
    return leaves


@pytest.mark.parametrize("seed", range(6))
def test_update_invariants(seed):
    rng = np.random.default_rng(seed)
    nx = ny = 4
    nz = 2
    leaves = _random_balanced_leaves(rng, nx, ny, 3)
    assert adapt.is_balanced(leaves, nx, ny)
    fl = rng.integers(-1, 2, size=len(leaves) * nz).astype(np.int8)
    new, origin = adapt.update_leaves(leaves, fl, nz, nx, ny, 3)
    mesh.OracleMesh(80e3, 80e3, 10e3, nx, ny, 1, 2, leaves=new)   # tiles the domain
    assert adapt.is_balanced(new, nx, ny)
    colflag = fl.reshape(-1, nz).max(axis=1)
    refined = {o[1] for o in origin if o[0] == "refine"}
    for c, (l, i, j) in enumerate(leaves):
        if colflag[c] == 1 and l < 3:
            assert c in refined                       # a flagged column refines
    for o, lf in zip(origin, new):
        if o[0] == "coarsen":
            assert all(colflag[s] == -1 for s in o[1])  # only fully flagged groups
            assert all(leaves[s][0] == lf[0] + 1 for s in o[1])
        elif o[0] == "refine":
            assert lf[0] == leaves[o[1]][0] + 1         # one level at most
        else:
            assert lf == leaves[o[1]]


def test_update_balance_propagation_example():
    """Refining a level-1 column next to a level-0 column forces the level-0
    neighbour to refine once (2:1 balance), and nothing else."""
    leaves = [(0, 0, 0), (0, 1, 0), (0, 0, 1)] + [(1, 2 + a, 2 + b) for b in (0, 1) for a in (0, 1)]
    fl = np.zeros(len(leaves), dtype=np.int8)
    fl[leaves.index((1, 2, 2))] = 1
    new, origin = adapt.update_leaves(leaves, fl, 1, 2, 2, 3)
    assert adapt.is_balanced(new, 2, 2)
    got = sorted(new)
    assert (2, 4, 4) in got and (1, 2, 2) not in got
    # every level-0 column touches (1,2,2) through faces/corners (periodic): all refine
    assert all(l >= 1 for l, _, _ in got)


def test_coarsening_cancelled_by_balance():
    """3x3 base, all level 1 except level-1 cell (1, 1) refined to level 2.
    A sibling group far from the level-2 cells coarsens; the group next to
    them would put level 0 beside level 2 and is cancelled."""
    leaves = [(1, i, j) for j in range(6) for i in range(6) if (i, j) != (1, 1)]
    leaves += [(2, 2 + a, 2 + b) for b in (0, 1) for a in (0, 1)]
    assert adapt.is_balanced(leaves, 3, 3)
    far = [(1, 4 + a, 4 + b) for b in (0, 1) for a in (0, 1)]
    near = [(1, 2 + a, 0 + b) for b in (0, 1) for a in (0, 1)]
    fl = np.array([-1 if lf in far + near else 0 for lf in leaves], dtype=np.int8)
    new, origin = adapt.update_leaves(leaves, fl, 1, 3, 3, 3)
    assert (0, 2, 2) in new and not any(lf in new for lf in far)
    assert all(lf in new for lf in near) and (0, 1, 0) not in new
    assert adapt.is_balanced(new, 3, 3)


def test_transfer_refine_then_coarsen_is_identity_and_conservative():
    m = mesh.OracleMesh(600e3, 600e3, 24e3, 4, 4, 2, 4)
    q = vortex_state(m.XG, 24e3)
    fl, _ = adapt.criterion_flags(m, q, PRM, [5.0, 10.0], 2)
    new, org = adapt.update_leaves(m.leaves, fl, 2, 4, 4, 2)
    assert len(new) > 16
    m2, q2 = transfer.transfer(m, new, org, q)
    assert m2.n_hanging > 0
    np.testing.assert_allclose((m2.M * q2).sum(1), (m.M * q).sum(1),
                               rtol=1e-13, atol=1e-13 * np.abs(m.M * q).sum())
    new3, org3 = adapt.update_leaves(m2.leaves, -np.ones(m2.Ne, np.int8), 2, 4, 4, 2)
    m3, q3 = transfer.transfer(m2, new3, org3, q2)
    assert np.array_equal(m3.XG, m.XG)
    np.testing.assert_allclose(q3, q, rtol=0, atol=1e-13 * np.abs(q).max())


def test_transfer_coarsen_conserves_and_projects_linear_fields_exactly():
    leaves = two_level_leaves()
    m = mesh.OracleMesh(80e3, 80e3, 10e3, 4, 4, 2, 4, leaves=leaves, periodic=(False, False))
    X = m.XG
    lin = np.stack([1 + X[:, 0] / 4e4, X[:, 1] / 4e4 - X[:, 2] / 1e4, 2 + 0 * X[:, 0],
                    X[:, 0] * X[:, 1] / 1.6e9, 3 * X[:, 2] / 1e4])
    rnd = random_state(np.where(True, X, X), 10e3, 3)
    fl = np.array([-1 if m.level[e] == 2 else 0 for e in range(m.Ne)], dtype=np.int8)
    new, org = adapt.update_leaves(m.leaves, fl, 2, 4, 4, 2, periodic=(False, False))
    assert any(o[0] == "coarsen" for o in org)
    m2, l2 = transfer.transfer(m, new, org, lin)
    X2 = m2.XG
    ex = np.stack([1 + X2[:, 0] / 4e4, X2[:, 1] / 4e4 - X2[:, 2] / 1e4, 2 + 0 * X2[:, 0],
                   X2[:, 0] * X2[:, 1] / 1.6e9, 3 * X2[:, 2] / 1e4])
    np.testing.assert_allclose(l2, ex, atol=1e-12)
    m2, r2 = transfer.transfer(m, new, org, rnd)
    np.testing.assert_allclose((m2.M * r2).sum(1), (m.M * rnd).sum(1),
                               rtol=1e-12, atol=1e-12 * np.abs(m.M * rnd).sum())


def test_wind_diagnostics_on_analytic_fields():
    m = mesh.OracleMesh(200e3, 200e3, 10e3, 4, 4, 2, 4)
    ref = refstate.reference_state(m.XG[:, 2], PRM)
    q = np.zeros((5, m.NG))
    q[1] = 3.0 * ref["rho0"]
    q[2] = 4.0 * ref["rho0"]
    d = diag.wind_diagnostics(m, q, PRM)
    assert abs(d["max_wind"] - 5.0) < 1e-13 and abs(d["max_mean_wind"] - 5.0) < 1e-13
    # speed growing with height: the mean is largest at the top
    q[1] = ref["rho0"] * (1.0 + m.XG[:, 2] / 1e4)
    q[2] = 0.0
    d = diag.wind_diagnostics(m, q, PRM)
    assert abs(d["max_mean_wind"] - 2.0) < 1e-13
    # a single spike outside [-50, 50] km is ignored, one inside is found
    s = np.argmax(np.abs(m.XG[:, 0]) > 60e3)
    q2 = q.copy()
    q2[1, s] = 100.0 * ref["rho0"][s]
    assert diag.wind_diagnostics(m, q2, PRM)["max_wind"] == pytest.approx(2.0)


def test_criterion_at_given_levels_equals_the_rule_at_those_levels():
    """criterion_flags with levels=L gives, element by element, what the rule
    gives on a mesh whose elements are at L: checked against a mesh whose
    elements all have level 0 (levels=0 must equal the default there) and
    against the three-level hand example's flags shifted by hand."""
    from synth.vortex import vortex_state
    m = mesh.OracleMesh(600e3, 600e3, 24e3, 4, 4, 2, 4)
    q = vortex_state(m.XG, 24e3)
    thr = [5.0, 10.0, 15.0]
    f0, c0 = adapt.criterion_flags(m, q, PRM, thr, 3)
    g0, d0 = adapt.criterion_flags(m, q, PRM, thr, 3, levels=np.zeros(m.Ne, dtype=int))
    assert np.array_equal(f0, g0) and np.array_equal(c0, d0)
    speed = adapt.CRITERIA["speed"](m, q, PRM, "C").max(axis=1)
    for L in range(4):
        fl, _ = adapt.criterion_flags(m, q, PRM, thr, 3, levels=np.full(m.Ne, L))
        T = (speed[:, None] > np.array(thr)[None]).sum(axis=1)     # thresholds exceeded
        want = np.where(T > L, 1, np.where(T < L, -1, 0))
        assert np.array_equal(fl, want), L
