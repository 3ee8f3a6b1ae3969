"""Refinement criterion and mesh update (Sec. 3.1-3.2, Algorithm 3).

Criterion (Sec. 3.1, "The refinement/coarsening criterion"): with C_{k,e} the
criterion variable at node k of element e and threshold(1..lvl_max) one value
per refinement level,
    refine  (adapt = +1) if some k has C_{k,e} > threshold(lvl(e)+1) and lvl(e) < lvl_max,
    coarsen (adapt = -1) if every k has C_{k,e} <= threshold(lvl(e)) and lvl(e) > 0,
    otherwise adapt = 0.
The criterion variable of the paper's runs is the velocity magnitude
(Sec. 4.1).  Sec. 3.1 lets the variable depend on the level (C^l), and the
paper names vorticity and potential vorticity, alone or combined, as the
candidates for further criteria (Sec. 1, Sec. 5); `variables[l]` picks the
variable whose element maximum is compared with threshold(l+1):
  "speed"      |u| (3-D velocity magnitude),
  "vorticity"  |dv/dx - du/dy| (vertical relative vorticity),
  "pv"         |(curl u + f e_z) . grad theta| / rho (dry Ertel potential
               vorticity, theta the full potential temperature),
with element-local derivatives of the element polynomials (hanging nodes
take the interpolated values, as everywhere).  Algorithm 3's
loop writes adapt(e) once per (node, level) pair, so a later pair can
overwrite an earlier refine decision with 0; the rule above is the statement
in the text, which the loop is meant to implement, and it does not depend on
the visiting order.  Refinement wins if both conditions hold (only possible
with non-increasing thresholds).

Mesh update (Sec. 3.1, "Refining/Coarsening an element", Remark 3.1):
* refinement is horizontal; a column refines into 4 children when any of its
  elements is flagged +1 (the whole column is refined);
* 4 sibling columns that share a corner coarsen into their parent only when
  every element of all 4 is flagged -1;
* levels change by at most one per pass;
* the result is 2:1 balanced across faces and corners (the balance P4est
  keeps); refinement is propagated to neighbours to restore balance and a
  coarsening that would break it is cancelled.

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np

from .refstate import reference_state


def criterion_speed(mesh, qG, prm, eqset="C"):
    """C_{k,e} = |u| at every local node, shape (Ne, P)."""
    qL = mesh.to_local(qG)
    if eqset == "C":
        rho = reference_state(mesh.X[:, :, 2], prm)["rho0"] + qL[0]
        s = np.sqrt(qL[1] * qL[1] + qL[2] * qL[2] + qL[3] * qL[3]) / rho
    else:
        s = np.sqrt(qL[1] * qL[1] + qL[2] * qL[2] + qL[3] * qL[3])
    return s


def _velocity_theta(mesh, qL, prm, eqset):
    """u, v, w, full theta and rho at every local node, each (Ne, P)."""
    ref = reference_state(mesh.X[:, :, 2], prm)
    if eqset == "C":
        rho = ref["rho0"] + qL[0]
        u, v, w = qL[1] / rho, qL[2] / rho, qL[3] / rho
        theta = (ref["rhotheta0"] + qL[4]) / rho
    else:
        rho = ref["rho0"] + qL[0]
        u, v, w = qL[1], qL[2], qL[3]
        theta = ref["theta0"] + qL[4]
    return u, v, w, theta, rho


def _element_gradient(mesh, phi):
    """Element-local x, y, z derivatives of nodal values phi (Ne, P)."""
    out = [np.zeros_like(phi) for _ in range(3)]
    for lev, es, G in mesh.op_groups():
        for d in range(3):
            out[d][es] = phi[es] @ G[d].T
    return out


def criterion_vorticity(mesh, qG, prm, eqset="C"):
    """C_{k,e} = |dv/dx - du/dy| at every local node, shape (Ne, P)."""
    u, v, w, _, _ = _velocity_theta(mesh, mesh.to_local(qG), prm, eqset)
    gu, gv = _element_gradient(mesh, u), _element_gradient(mesh, v)
    return np.abs(gv[0] - gu[1])


def criterion_pv(mesh, qG, prm, eqset="C"):
    """C_{k,e} = |(curl u + f e_z) . grad theta| / rho, shape (Ne, P)."""
    u, v, w, th, rho = _velocity_theta(mesh, mesh.to_local(qG), prm, eqset)
    gu, gv, gw, gt = (_element_gradient(mesh, a) for a in (u, v, w, th))
    wx = gw[1] - gv[2]
    wy = gu[2] - gw[0]
    wz = gv[0] - gu[1] + prm.f
    return np.abs(wx * gt[0] + wy * gt[1] + wz * gt[2]) / rho


CRITERIA = {"speed": criterion_speed, "vorticity": criterion_vorticity, "pv": criterion_pv}


def criterion_flags(mesh, qG, prm, thresholds, lvl_max, eqset="C", variables=None, levels=None):
    """adapt(e) in {-1, 0, 1} for every element; also returns max_k C_{k,e}
    of the variable of the element's refinement test (threshold(lvl+1), or
    threshold(lvl) at lvl_max).  variables[l] names the variable compared
    with threshold(l+1) (default: speed at every level).  levels (one per
    element, default the mesh's own) are the levels lvl the rule is applied
    with; the variables are always evaluated on the mesh itself."""
    thr = np.asarray(thresholds, dtype=np.float64)
    if variables is None:
        variables = ["speed"] * len(thr)
    lvls = mesh.level if levels is None else np.asarray(levels)
    cm = {name: CRITERIA[name](mesh, qG, prm, eqset).max(axis=1) for name in set(variables)}
    flags = np.zeros(mesh.Ne, dtype=np.int8)
    cmax = np.zeros(mesh.Ne)
    for e in range(mesh.Ne):
        lv = int(lvls[e])
        refine = lv < lvl_max and cm[variables[lv]][e] > thr[lv]
        coarsen = lv > 0 and cm[variables[lv - 1]][e] <= thr[lv - 1]
        flags[e] = 1 if refine else (-1 if coarsen else 0)
        test = lv if lv < lvl_max else lv - 1
        cmax[e] = cm[variables[test]][e] if 0 <= test < len(variables) else cm[variables[0]][e]
    return flags, cmax


def _cells(leaf, lmax):
    l, i, j = leaf
    f = 1 << (lmax - l)
    return i * f, (i + 1) * f, j * f, (j + 1) * f


def _neighbours(region, owner, periodic):
    """Leaves owning a cell in the one-cell ring around region (faces+corners)."""
    x0, x1, y0, y1 = region
    NX, NY = owner.shape
    out = set()
    for X in range(x0 - 1, x1 + 1):
        for Y in range(y0 - 1, y1 + 1):
            if x0 <= X < x1 and y0 <= Y < y1:
                continue
            if not (0 <= X < NX):
                if not periodic[0]:
                    continue
                X %= NX
            if not (0 <= Y < NY):
                if not periodic[1]:
                    continue
                Y %= NY
            out.add(int(owner[X, Y]))
    return out


def owner_grid(leaves, nx, ny, lmax):
    owner = -np.ones((nx << lmax, ny << lmax), dtype=np.int64)
    for c, lf in enumerate(leaves):
        x0, x1, y0, y1 = _cells(lf, lmax)
        owner[x0:x1, y0:y1] = c
    return owner


def is_balanced(leaves, nx, ny, periodic=(True, True)):
    lmax = max(l for l, _, _ in leaves)
    owner = owner_grid(leaves, nx, ny, lmax)
    for c, lf in enumerate(leaves):
        for d in _neighbours(_cells(lf, lmax), owner, periodic):
            if abs(leaves[d][0] - lf[0]) > 1:
                return False
    return True


def update_leaves(leaves, elem_flags, nz, nx, ny, lvl_max, periodic=(True, True)):
    """New leaf list after one AMR pass, and where every new leaf comes from.

    origin[n] = ("same", c) | ("refine", c, a, b) | ("coarsen", (c00, c10, c01, c11))
    where (a, b) is the child position and c.. index the old leaves.
    """
    leaves = [tuple(t) for t in leaves]
    ncol = len(leaves)
    fl = np.asarray(elem_flags).reshape(ncol, nz)
    colflag = fl.max(axis=1)
    lmax = max(max(l for l, _, _ in leaves), 0) + 1
    owner = owner_grid(leaves, nx, ny, lmax)
    lvl = np.array([l for l, _, _ in leaves], dtype=np.int64)
    target = lvl + ((colflag > 0) & (lvl < lvl_max)).astype(np.int64)
    nbr = [_neighbours(_cells(lf, lmax), owner, periodic) for lf in leaves]
    changed = True
    while changed:                      # refinement propagation for balance
        changed = False
        for c in range(ncol):
            need = max((target[d] for d in nbr[c]), default=0) - 1
            if target[c] < need:
                target[c] = need
                changed = True
    # coarsening candidates: complete sibling groups, all flagged -1, not refined
    index = {lf: c for c, lf in enumerate(leaves)}
    groups = {}
    for c, (l, i, j) in enumerate(leaves):
        if l == 0 or colflag[c] != -1 or target[c] != l:
            continue
        key = (l - 1, i >> 1, j >> 1)
        sib = [index.get((l, 2 * key[1] + a, 2 * key[2] + b)) for b in (0, 1) for a in (0, 1)]
        if all(s is not None for s in sib) and all(colflag[s] == -1 and target[s] == l for s in sib):
            groups[key] = tuple(sib)
    ok = {k: True for k in groups}
    member = {}
    for k, sib in groups.items():
        for s in sib:
            member[s] = k
    changed = True
    while changed:
        changed = False
        for k, sib in groups.items():
            if not ok[k]:
                continue
            l = k[0] + 1
            ring = set()
            for s in sib:
                ring |= nbr[s]
            ring -= set(sib)
            for d in ring:
                final = target[d] - 1 if (d in member and ok[member[d]]) else target[d]
                if final > l:
                    ok[k] = False
                    changed = True
                    break
    new, origin = [], []
    done = set()
    for c, (l, i, j) in enumerate(leaves):
        if c in member and ok[member[c]]:
            k = member[c]
            if k not in done:
                done.add(k)
                new.append(k)
                origin.append(("coarsen", groups[k]))
            continue
        if target[c] > l:
            for b in (0, 1):
                for a in (0, 1):
                    new.append((l + 1, 2 * i + a, 2 * j + b))
                    origin.append(("refine", c, a, b))
        else:
            new.append((l, i, j))
            origin.append(("same", c))
    return new, origin
