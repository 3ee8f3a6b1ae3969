"""Learned adaptation schedule: training data from solver trajectories, training
and the missed-refinement comparison against the paper's criterion.

Every field operation runs in libsem.so (steps, criterion, features, network
forward/backward/Adam); this module only sequences the calls and does the
integer bookkeeping of element levels with torch tensor ops.

Protocol.  The solver runs trajectories; every `every` steps it records each
element's features (sem_mlp_features) and the criterion's flag for every
level L in 0..lvl_max (sem_adapt_flags_levels: the Sec. 3.1 rule evaluated
as if the element were at level L).  A training row pairs the features at
step t, with the element's level set to L, with that flag at step t + ahead.
The rule itself, and the merge of the criterion's and the network's flags
(sem_merge_flags), run in the library; this module only selects and counts.

Scheduling (element levels kept as a virtual level per element on the fixed
solver mesh, so that the comparison isolates the scheduling): every `ahead`
steps the levels move by the flags (one level at most, Remark 3.1); at the
checks in between, an element is a missed refinement when the criterion wants
a higher level than it has.  Schedules compared at the same remesh count:
the criterion alone, and the criterion with the network, where an element is
refined when either the current criterion or the network's prediction for
`ahead` steps later asks for it, and coarsened only when both do (the
criterion stays the fallback).

Real adaptive runs (adaptive_run, adaptive_comparison): the same two
schedules drive actual remeshes with solution transfer every `ahead`
seconds, from a mesh refined by the criterion on the initial vortex, and are
compared with the base mesh refined uniformly to lvl_max (the reference):
final maximum wind, remesh count, missed-refinement rate between remeshes,
element count and throughput.
"""
import numpy as np


def level_flags(sem, torch, mesh, p_crit, q, lvl_max):
    """The criterion's flag for every element at each level 0..lvl_max
    ([lvl_max + 1, Ne] int8, on the device)."""
    out = torch.empty((lvl_max + 1, mesh.Ne), dtype=torch.int8, device=q.device)
    for L in range(lvl_max + 1):
        sem.sem_adapt_flags_levels(mesh, p_crit, q, out[L], level_all=L)
    return out


def trajectory(sem, torch, mesh, p_step, p_crits, q0, dt, steps, every, scales):
    """Every `every` steps of a mixed-form run from q0: (features, [per-level
    criterion flags for each parameter set in p_crits])."""
    q = q0.clone()
    q32 = torch.empty(q.shape, dtype=torch.float32, device=q.device)
    work = torch.empty((10, mesh.NG), dtype=torch.float32, device=q.device)
    sem.sem_mirror(mesh, q, q32)
    out = []
    for s in range(steps + 1):
        if s % every == 0:
            fls = [level_flags(sem, torch, mesh, pc, q, pc.lvl_max) for pc in p_crits]
            F = torch.empty((mesh.Ne, 136), dtype=torch.float32, device=q.device)
            sem.sem_mlp_features(mesh, q, scales, F)
            out.append((F, fls))
        if s < steps:
            sem.sem_step_mixed(mesh, p_step, q, q32, work, dt)
    return out


def window_label(torch, snaps, i, k, L, which=0):
    """Label for level L at snapshot i: what the criterion asks of an element
    at level L over the next k checks (i+1 .. i+k): refine (2) if it asks for
    refinement at any of them, coarsen (0) if it asks for coarsening at all
    of them, keep (1) otherwise.  A schedule that remeshes every k checks
    needs exactly this to miss no refinement before its next remesh."""
    fl = torch.stack([snaps[i + j][1][which][L] for j in range(1, k + 1)])
    up = (fl > 0).any(dim=0)
    down = (fl < 0).all(dim=0)
    return torch.where(up, 2, torch.where(down, 0, 1)).to(torch.int8)


def training_rows(torch, snaps, ahead, every, lvl_max):
    """Features at t with the level set to L, labelled by window_label over
    the `ahead` steps after t (classes 0, 1, 2 = coarsen, keep, refine)."""
    k = ahead // every
    Fs, Ys = [], []
    for i in range(len(snaps) - k):
        F = snaps[i][0]
        for L in range(lvl_max + 1):
            G = F.clone()
            G[:, 135] = float(L)
            Fs.append(G)
            Ys.append(window_label(torch, snaps, i, k, L))
    return torch.cat(Fs), torch.cat(Ys)


def train(sem, torch, F, Y, iters=1500, batch=65536, seed=1, lr=1e-3):
    counts = torch.bincount(Y.long(), minlength=3).cpu().numpy()
    cw = (counts.sum() / np.maximum(counts, 1) / 3.0).astype(np.float32)
    batch = min(batch, F.shape[0])
    net = sem.sem_mlp_create(seed, batch)
    g = torch.Generator(device=F.device).manual_seed(seed)
    first = last = None
    for it in range(iters):
        idx = torch.randint(0, F.shape[0], (batch,), device=F.device, generator=g)
        want = it == 0 or it == iters - 1
        loss = sem.sem_mlp_backward(net, F[idx].contiguous(), Y[idx].contiguous(), cw, want_loss=want)
        if it == 0:
            first = loss
        if it == iters - 1:
            last = loss
        sem.sem_mlp_adam(net, lr if it < 2 * iters // 3 else lr / 3)
    return net, first, last


def schedule(sem, torch, snaps, ahead, every, lvl_max, net=None, which=0):
    """Missed-refinement rate, mean refined levels and remesh count of the
    schedule that remeshes every `ahead` steps by the criterion's flags of
    parameter set `which` (and the network's, if given); missed refinements
    are counted against the flags of parameter set 0 (the paper's criterion)."""
    Ne = snaps[0][0].shape[0]
    dev = snaps[0][0].device
    # start from the levels the criterion gives the initial state (lvl_max
    # passes of one level each), as an adaptive run starts from a mesh
    # refined by the criterion
    L = torch.zeros(Ne, dtype=torch.int8, device=dev)
    for _ in range(lvl_max):
        L = (L + snaps[0][1][which].gather(0, L.long()[None]).squeeze(0)).clamp_(0, lvl_max)
    k = ahead // every
    missed = want = 0
    refined = 0.0
    remesh = 0
    for i, (F, fls) in enumerate(snaps):
        fl_lv = fls[0]
        # the criterion's flag at each element's own (tracked) level
        now = fls[which].gather(0, L.long()[None]).squeeze(0)
        judge = fl_lv.gather(0, L.long()[None]).squeeze(0)
        if i % k == 0:
            remesh += 1
            if net is None:
                fl = now
            else:
                G = F.clone()
                G[:, 135] = L.float()
                pred = torch.empty(Ne, dtype=torch.int8, device=dev)
                sem.sem_mlp_predict_flags(net, G, pred)
                fl = sem.sem_merge_flags(now, pred, L, lvl_max)
            L = (L + fl).clamp_(0, lvl_max)
        else:
            missed += int((judge > 0).sum())
            want += int((fl_lv[0] > 0).sum())
        refined += float(L.float().mean())
    return {"missed_rate": missed / max(want, 1), "mean_level": refined / len(snaps),
            "remeshes": remesh}


def gain_experiment(sem, torch, mesh, states, dt, n_train, steps=400, every=10,
                    intervals=(50, 75, 100), thresholds=(15.0, 25.0),
                    control_scales=(0.95, 0.9, 0.85, 0.8, 0.75, 0.7, 0.65, 0.6),
                    scales=(1e-3, 10.0, 10.0, 1.0, 1.0), iters=1500, seed=1):
    """Train one network per remesh interval K on the first n_train initial
    states' trajectories (labels: window_label over the K steps ahead) and
    compare, on the other trajectories and for every K, the criterion alone
    with the criterion plus the network (missed-refinement rate against the
    paper's criterion, mean level, remesh count).  Control at each K: the
    criterion alone with every threshold scaled by the largest factor of
    control_scales at which it refines at least as much as the learned
    schedule (so that the comparison is at equal refined-element count)."""
    lvl_max = len(thresholds)
    p_step = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    p_crits = [sem.sem_params_default(thresholds=[f * t for t in thresholds], lvl_max=lvl_max)
               for f in (1.0,) + tuple(control_scales)]
    sc = np.asarray(scales, dtype=np.float32)
    trajs = [trajectory(sem, torch, mesh, p_step, p_crits, q0, dt, steps, every, sc) for q0 in states]
    status = sem.sem_status(mesh)
    res = {"status": status, "intervals": list(intervals), "by_interval": []}
    held = trajs[n_train:]
    mean = lambda rs, key: float(np.mean([r[key] for r in rs]))
    for K in intervals:
        parts = [training_rows(torch, t, K, every, lvl_max) for t in trajs[:n_train]]
        F = torch.cat([a for a, _ in parts])
        Y = torch.cat([b for _, b in parts])
        net, loss0, loss1 = train(sem, torch, F, Y, iters=iters, seed=seed)
        cri = [schedule(sem, torch, t, K, every, lvl_max) for t in held]
        lrn = [schedule(sem, torch, t, K, every, lvl_max, net) for t in held]
        row = {"interval": K, "rows": int(F.shape[0]), "loss_first": loss0, "loss_last": loss1,
               "remeshes": cri[0]["remeshes"],
               "missed_criterion": mean(cri, "missed_rate"), "missed_learned": mean(lrn, "missed_rate"),
               "level_criterion": mean(cri, "mean_level"), "level_learned": mean(lrn, "mean_level")}
        # control: lowered thresholds, criterion alone, at least the learned refinement
        row["control"] = None
        for w, f in enumerate(control_scales, start=1):
            ctl = [schedule(sem, torch, t, K, every, lvl_max, which=w) for t in held]
            if mean(ctl, "mean_level") >= row["level_learned"]:
                row["control"] = {"threshold_scale": f, "missed": mean(ctl, "missed_rate"),
                                  "level": mean(ctl, "mean_level")}
                break
        res["by_interval"].append(row)
        if K == intervals[0]:
            res["net"] = net
    return res


def element_levels(sem, torch, mesh, device):
    """Refinement level of every element (column level, repeated over the layers), int8."""
    lv = sem.sem_mesh_leaves_host(mesh)
    return torch.from_numpy(np.repeat(lv[:, 0].astype(np.int8), mesh.nz)).to(device)


def adaptive_run(sem, torch, spec, L, Lz, nx, nz, N, lvl_max, thresholds, dt, t_end,
                 remesh_s=50.0, check_s=10.0, net=None, scales=(1e-3, 10.0, 10.0, 1.0, 1.0),
                 uniform_level=None, physics=None, replay=None, fp64=False):
    """A real adaptive run: the mesh is refined and coarsened every remesh_s
    seconds with the solution transferred (Algorithm 3), by the criterion's
    flags alone (net None) or by the criterion combined with the network's
    prediction for remesh_s later (refine if either asks, coarsen only if
    both do).  The initial mesh is refined by the criterion on the initial
    vortex.  With uniform_level the mesh is the base refined uniformly to that
    level and never adapted (the reference).  Returns the final maximum wind,
    the remesh count, the missed-refinement rate (checks every check_s between
    remeshes), the mean element count and DOF-updates/s including remeshes.
    physics: extra step parameters (for example the Smagorinsky stress).
    The flags of every remesh are returned (flag_log); replay runs the same
    remesh schedule from such a log instead of deciding (same meshes), and
    fp64 steps in the float64 form instead of the mixed one: the two
    together give the float64 run on the mixed run's schedule."""
    import time
    from synth.vortex import vortex_state
    dev = "cuda"
    p_step = sem.sem_params_default(precision=sem.SEM_PREC_FP64 if fp64 else sem.SEM_PREC_MIXED,
                                    **(physics or {}))
    p_crit = sem.sem_params_default(thresholds=list(thresholds), lvl_max=lvl_max)
    sc = np.asarray(scales, dtype=np.float32)
    if uniform_level is not None:
        m = sem.sem_mesh_create(L, L, Lz, nx << uniform_level, nx << uniform_level, nz, N)
    else:
        m = sem.sem_mesh_create(L, L, Lz, nx, nx, nz, N, lvl_max=lvl_max)
        for _ in range(lvl_max):
            q = torch.from_numpy(vortex_state(sem.sem_mesh_coords_host(m).T, Lz, spec)).to(dev)
            fl = np.maximum(sem.sem_adapt_flags_host(m, p_crit, q), 0)
            if not fl.any():
                break
            m = sem.sem_transfer_plan(m, fl)
    q = torch.from_numpy(vortex_state(sem.sem_mesh_coords_host(m).T, Lz, spec)).to(dev)

    def buffers(mesh, q):
        if fp64:
            return torch.empty_like(q), torch.empty_like(q)
        q32 = torch.empty(q.shape, dtype=torch.float32, device=dev)
        work = torch.empty((10, mesh.NG), dtype=torch.float32, device=dev)
        sem.sem_mirror(mesh, q, q32)
        return q32, work

    q32, work = buffers(m, q)
    steps = int(round(t_end / dt))
    k_remesh, k_check = int(round(remesh_s / dt)), int(round(check_s / dt))
    missed = want = remeshes = 0
    dof = 0
    elems = []
    flag_log = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(steps):
        remesh_now = s > 0 and s % k_remesh == 0
        if uniform_level is None and replay is not None:
            if remesh_now:
                fl_host = replay[len(flag_log)]
                flag_log.append(fl_host)
                if fl_host.any():
                    new = sem.sem_transfer_plan(m, fl_host)
                    q2 = torch.empty((5, new.NG), dtype=torch.float64, device=dev)
                    sem.sem_transfer(m, new, q, q2)
                    m, q = new, q2
                    q32, work = buffers(m, q)
                    remeshes += 1
        elif uniform_level is None and (remesh_now or (s > 0 and s % k_check == 0)):
            flags = torch.empty(m.Ne, dtype=torch.int8, device=dev)
            sem.sem_adapt_flags(m, p_crit, q, flags)
            if not remesh_now:
                # a missed refinement: the criterion wants more than the mesh has
                base = torch.empty(m.Ne, dtype=torch.int8, device=dev)
                sem.sem_adapt_flags_levels(m, p_crit, q, base, level_all=0)
                missed += int((flags > 0).sum())
                want += int((base > 0).sum())
            else:
                fl = flags
                if net is not None:
                    lev = element_levels(sem, torch, m, dev)
                    F = torch.empty((m.Ne, 136), dtype=torch.float32, device=dev)
                    sem.sem_mlp_features(m, q, sc, F)
                    F[:, 135] = lev.float()
                    pred = torch.empty(m.Ne, dtype=torch.int8, device=dev)
                    sem.sem_mlp_predict_flags(net, F, pred)
                    fl = sem.sem_merge_flags(flags, pred, lev, lvl_max)
                fl_host = fl.cpu().numpy()
                flag_log.append(fl_host)
                if fl_host.any():
                    new = sem.sem_transfer_plan(m, fl_host)
                    q2 = torch.empty((5, new.NG), dtype=torch.float64, device=dev)
                    sem.sem_transfer(m, new, q, q2)
                    m, q = new, q2
                    q32, work = buffers(m, q)
                    remeshes += 1
        if fp64:
            sem.sem_step(m, p_step, q, q32, work, dt)
        else:
            sem.sem_step_mixed(m, p_step, q, q32, work, dt)
        dof += 15 * m.Ne * (N + 1) ** 3
        elems.append(m.Ne)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    status = sem.sem_status(m)
    wind = sem.sem_diag(m, p_step, q, 0.5 * L)["max_wind"] if status == 0 else float("nan")
    return {"max_wind": wind, "remeshes": remeshes, "missed_rate": missed / max(want, 1),
            "mean_elements": float(np.mean(elems)), "dof_updates_per_s": dof / wall,
            "seconds": wall, "status": status, "flag_log": flag_log}


def adaptive_comparison(sem, torch, specs, net, L=150e3, Lz=24e3, nx=24, nz=2, N=4,
                        thresholds=(15.0, 25.0), dt=0.25, t_end=400.0, physics=None):
    """For each vortex: the uniform finest mesh (reference), the criterion
    schedule and the criterion-plus-network schedule; max-wind errors of the
    two schedules against the reference."""
    lvl_max = len(thresholds)
    out = []
    for spec in specs:
        ref = adaptive_run(sem, torch, spec, L, Lz, nx, nz, N, lvl_max, thresholds, dt, t_end,
                           uniform_level=lvl_max, physics=physics)
        cri = adaptive_run(sem, torch, spec, L, Lz, nx, nz, N, lvl_max, thresholds, dt, t_end,
                           physics=physics)
        lrn = adaptive_run(sem, torch, spec, L, Lz, nx, nz, N, lvl_max, thresholds, dt, t_end, net=net,
                           physics=physics)
        # the float64 form on the learned run's remesh schedule: the max-wind
        # gate of the mixed form
        l64 = adaptive_run(sem, torch, spec, L, Lz, nx, nz, N, lvl_max, thresholds, dt, t_end,
                           physics=physics, replay=lrn["flag_log"], fp64=True)
        w = ref["max_wind"]
        out.append({"reference": ref, "criterion": cri, "learned": lrn, "learned_fp64": l64,
                    "wind_err_criterion": abs(cri["max_wind"] - w) / w,
                    "wind_err_learned": abs(lrn["max_wind"] - w) / w,
                    "gate_max_wind_rel_err": abs(lrn["max_wind"] - l64["max_wind"]) / l64["max_wind"]})
    return out
