"""Benchmark: SSP-RK3 steps of the spectral-element solver on the
64 x 64 x 16, N = 4 uniform workload (65,536 elements, 8,192,000 local nodes,
2048 x 2048 x 24 km, warm-core vortex), one step = 3 stages of
(right-hand side + fused RK update) over the whole mesh.

Metric: DOF-updates/s = 5 fields x local nodes x RK stages / second, for the
mixed-precision form (float32 element and face arithmetic, float64 reference
state and stage accumulation); the plain float64 form is measured beside it,
and the maximum-wind error of the mixed form against the float64 form after
100 steps is reported (gate 1e-3).

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference] [--form fp64]

With N > 1 (torchrun) every rank runs an independent replica (the path has
no exchange step); `value` sums the replicas' throughput.  --impl reference
times the CPU oracle on a bounded sample of the same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "uniform-64x64x16-N4"
METRIC = "DOF-updates/s (RHS+RK stage) vs plain FP64 GPU, at <=1e-3 rel max-wind error"


def max_over_ranks(x, world, device):
    """The largest x over the ranks (a job's step time is its slowest rank's);
    every rank calls it at the same point.  None stays None on every rank."""
    if world == 1 or x is None:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_throughput(units_per_rank_step, world, ms):
    """Units all ranks processed per second at the job's step time ms."""
    return units_per_rank_step * world / (ms * 1e-3)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--gate-steps", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched", default="both", choices=["both", "refined", "unrefined"],
                    help="which instance sets of the batched workload to run (profiler runs keep "
                         "the device footprint small with the unrefined one)")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-amr", action="store_true")
    ap.add_argument("--no-physics", action="store_true")
    ap.add_argument("--no-warped", action="store_true")
    ap.add_argument("--no-paper-set", action="store_true")
    ap.add_argument("--mlp-forward-only", action="store_true",
                    help="time only the flag network's forwards on 2^20 feature rows and print that "
                         "object (a short command for profiling them)")
    ap.add_argument("--kernel-row", type=int, default=None,
                    help="use this row of the element-kernel variant table instead of autotuning "
                         "(for profiler runs, whose per-launch overhead distorts the timings)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample(steps=1, n=32):
    """The CPU oracle on a bounded sample of the workload: an n x n x 16 block
    of the same elements (same element size, order, physics), SSP-RK3 steps.
    Returns (DOF-updates/s, threads, description, seconds, busy threads)."""
    import numpy as np
    from oracle import mesh as om, refstate, rk as ork
    from synth.vortex import vortex_state
    L = 2048e3 * n / 64
    o = om.OracleMesh(L, L, 24e3, n, n, 16, 4)
    q = vortex_state(o.XG, 24e3)
    prm = refstate.Params()
    ork.rk_step(o, prm, q, 0.25)            # warm caches
    c0, t0 = time.process_time(), time.perf_counter()
    for _ in range(steps):
        q = ork.rk_step(o, prm, q, 0.25)
    dt = time.perf_counter() - t0
    busy = (time.process_time() - c0) / dt   # threads kept busy on average
    dofs = 5 * o.Ne * o.P * 3 * steps
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    desc = (f"{steps} SSP-RK3 step(s) of the oracle on a {n}x{n}x16 block of the same "
            f"elements ({o.Ne} of 65,536; N=4), float64 numpy/scipy")
    return dofs / dt, threads, desc, dt, busy


def cpu_model():
    """The host CPU's model name (lscpu; /proc/cpuinfo as a fallback)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


_ONE_THREAD = """
import json, sys, time
sys.path.insert(0, {root!r})
from bench import cpu_oracle_sample, cpu_small_case
v, thr, desc, secs, busy = cpu_oracle_sample(steps=1, n={n})
s = cpu_small_case()
print(json.dumps(dict(value=v, desc=desc, seconds=secs, busy=busy, small=s)))
"""


def cpu_small_case():
    """The oracle on the whole small workload: 10 SSP-RK3 steps of 1 s on the
    6 x 6 x 4, N = 4 mesh (600 x 600 x 24 km, 144 elements)."""
    from oracle import mesh as om, refstate, rk as ork
    from synth.vortex import vortex_state
    o = om.OracleMesh(600e3, 600e3, 24e3, 6, 6, 4, 4)
    q = vortex_state(o.XG, 24e3)
    prm = refstate.Params()
    t0 = time.perf_counter()
    for _ in range(10):
        q = ork.rk_step(o, prm, q, 1.0)
    dt = time.perf_counter() - t0
    return {"workload": "uniform-6x6x4-N4, 10 SSP-RK3 steps of 1 s", "seconds": dt,
            "value": 5 * o.Ne * o.P * 3 * 10 / dt}


def cpu_one_thread(n=16):
    """The oracle with its BLAS held to one thread, in a fresh interpreter
    (the thread count is fixed when numpy loads): an n x n x 16 block, one
    step, and the whole small workload."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", _ONE_THREAD.format(root=ROOT, n=n)], env=env,
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        return {"error": r.stderr[-300:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


def batched_measure(sem, torch, steps=10, warmup=3, refine=True, rates=None, eqset=0):
    """The 16-instance batched workload: one CUDA-graph launch per step over
    all instances (persistent element kernel + gather/increment kernel per
    stage) against stepping the instances one after another; eqset 1: the
    paper's equation set."""
    from synth.vortex import VortexSpec, vortex_state
    from synth.workloads import batched_instances, geometric_flags
    insts = batched_instances()
    if not refine:
        import dataclasses
        insts = [dataclasses.replace(it, levels=0) for it in insts]
    meshes, qs, q32, work, dts, dof, init = [], [], [], [], [], 0, []
    p = sem.sem_params_default(eqset=eqset, precision=sem.SEM_PREC_MIXED)
    for k, it in enumerate(insts):
        m = sem.sem_mesh_create(it.L, it.L, it.Lz, it.nx, it.nx, it.nz, it.N, lvl_max=max(it.levels, 1))
        for _ in range(it.levels):
            lv = [tuple(x) for x in sem.sem_mesh_leaves_host(m)]
            m = sem.sem_transfer_plan(m, geometric_flags(lv, it.nx, it.nz, it.L, 3 * it.rmw, it.levels))
        spec = VortexSpec(vmax=it.vmax, rmw=it.rmw, seed=1000 + k)
        q = torch.from_numpy(vortex_state(sem.sem_mesh_coords_host(m).T, it.Lz, spec,
                                          eqset="NC" if eqset else "C")).cuda()
        meshes.append(m)
        init.append(q.clone())
        qs.append(q)
        q32.append(torch.empty(q.shape, dtype=torch.float32, device="cuda"))
        work.append(torch.empty((10, q.shape[1]), dtype=torch.float32, device="cuda"))
        sem.sem_mirror(m, q, q32[-1])
        dts.append(it.dt)
        dof += 5 * m.Ne * (it.N + 1) ** 3
    batch = sem.sem_batch_create(meshes)
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    def seq():
        for k, m in enumerate(meshes):
            sem.sem_step_mixed(m, p, qs[k], q32[k], work[k], dts[k], stream)

    # sequential reference: every instance with its own autotuned element kernel
    for k, m in enumerate(meshes):
        sem.sem_autotune(m, p, q32[k], 3, stream)
    ms_seq = timed(seq)
    ms_graph = timed(lambda: sem.sem_batch_step_mixed(batch, p, qs, q32, work, dts, True, stream))
    ms_nograph = timed(lambda: sem.sem_batch_step_mixed(batch, p, qs, q32, work, dts, False, stream))
    status = sem.sem_batch_status(batch)
    # max-wind gate: every instance after gate_steps batched (graph) steps
    # against its float64 single-mesh run from the same initial state
    gate_steps = 20
    p64 = sem.sem_params_default(eqset=eqset, precision=sem.SEM_PREC_FP64)
    for k, m in enumerate(meshes):
        qs[k].copy_(init[k])
        sem.sem_mirror(m, qs[k], q32[k], stream)
    for _ in range(gate_steps):
        sem.sem_batch_step_mixed(batch, p, qs, q32, work, dts, True, stream)
    errs = []
    for k, m in enumerate(meshes):
        q64 = init[k].clone()
        w1, w2 = torch.empty_like(q64), torch.empty_like(q64)
        for _ in range(gate_steps):
            sem.sem_step(m, p64, q64, w1, w2, dts[k], stream)
        hw = 0.5 * insts[k].L    # the whole box
        a, b = sem.sem_diag(m, p64, qs[k], hw), sem.sem_diag(m, p64, q64, hw)
        errs.append(abs(a["max_wind"] - b["max_wind"]) / b["max_wind"])
    gate = {"steps": gate_steps, "max_wind_rel_err_max": max(errs), "max_wind_rel_err": errs,
            "how": "each instance, batched mixed steps against its own float64 single-mesh steps",
            "status": sem.sem_batch_status(batch)}
    # the rate the mix of orders predicts from single-mesh rates per order:
    # total DOF-updates over the sum of each instance's DOF-updates at its
    # order's rate
    expected = None
    if rates and not eqset:
        dofs = [15 * m.Ne * (it.N + 1) ** 3 for m, it in zip(meshes, insts)]
        expected = sum(dofs) / sum(d / rates[it.N] for d, it in zip(dofs, insts))
    return {"workload": "16 seeded instances, bases 8..48, N 3..6, "
                        + ("0..3 levels" if refine else "unrefined")
                        + (", the paper's equation set" if eqset else ""),
            "expected_from_order_rates": expected,
            "instances": len(insts), "elements": int(sum(m.Ne for m in meshes)),
            "dof_per_stage": dof, "ms_per_step_graph": ms_graph, "ms_per_step_batched_no_graph": ms_nograph,
            "ms_per_step_sequential": ms_seq,
            "value_graph": dof * 3 / (ms_graph * 1e-3), "value_sequential": dof * 3 / (ms_seq * 1e-3),
            "speedup": ms_seq / ms_graph, "status": status, "gate": gate,
            "launches_per_step_graph": 1, "launches_per_step_sequential": 6 * len(insts)}


def order_rates(sem, torch, steps=10):
    """Mixed-step throughput of a single uniform mesh of each order N = 3..6
    (64 x 64 x 16 elements for N <= 4, 48 x 48 x 16 above), autotuned: the
    per-DOF cost of the orders, against which the batched workload's mix of
    orders is judged."""
    from synth.vortex import vortex_state
    stream = torch.cuda.current_stream()
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    out = {}
    for N in (3, 4, 5, 6):
        n = 48 if N >= 5 else 64
        m = sem.sem_mesh_create(2048e3 * n / 64, 2048e3 * n / 64, 24e3, n, n, 16, N)
        q = torch.from_numpy(vortex_state(sem.sem_mesh_coords_host(m).T, 24e3)).cuda()
        q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
        work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
        sem.sem_mirror(m, q, q32, stream)
        sem.sem_autotune(m, p, q32, 3, stream)
        for _ in range(3):
            sem.sem_step_mixed(m, p, q, q32, work, 0.05, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            sem.sem_step_mixed(m, p, q, q32, work, 0.05, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[N] = 15 * m.Ne * (N + 1) ** 3 / (ms * 1e-3)
    return out


def amr_measure(sem, torch, steps=500, t_amr=50):
    """The adaptive workload: 32x32x8 base, N=4, 600 km box, geometric level-3
    refinement inside r < 150 km (2:1 balanced), criterion thresholds
    [5, 10, 15] m/s, remesh with solution transfer every 50 steps, mixed form,
    dt = 0.4 s.  Reports throughput including the remeshes."""
    from synth.vortex import vortex_state
    from synth.workloads import geometric_flags
    L, Lz, n, nz, N, dt = 600e3, 24e3, 32, 8, 4, 0.4
    thr = [5.0, 10.0, 15.0]
    m = sem.sem_mesh_create(L, L, Lz, n, n, nz, N, lvl_max=3)
    for _ in range(3):
        lv = [tuple(x) for x in sem.sem_mesh_leaves_host(m)]
        m = sem.sem_transfer_plan(m, geometric_flags(lv, n, nz, L, 150e3, 3))
    q = torch.from_numpy(vortex_state(sem.sem_mesh_coords_host(m).T, Lz)).cuda()
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    pc = sem.sem_params_default(thresholds=thr, lvl_max=3)
    stream = torch.cuda.current_stream()
    history = []
    flag_log = []
    dof = 0
    m0, q0 = m, q.clone()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    remesh_s = 0.0
    s = 0
    while s < steps:
        q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
        work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
        sem.sem_mirror(m, q, q32, stream)
        for _ in range(min(t_amr, steps - s)):
            sem.sem_step_mixed(m, p, q, q32, work, dt, stream)
            dof += 3 * 5 * m.Ne * (N + 1) ** 3
            s += 1
        history.append({"step": s, "elements": int(m.Ne),
                        "levels": [int(m.info.level_hist[k]) for k in range(4)]})
        if s < steps:
            torch.cuda.synchronize()
            r0 = time.perf_counter()
            flags = sem.sem_adapt_flags_host(m, pc, q, stream)
            flag_log.append(flags)
            new = sem.sem_transfer_plan(m, flags)
            qn = torch.empty((5, new.NG), dtype=torch.float64, device="cuda")
            sem.sem_transfer(m, new, q, qn, stream)
            torch.cuda.synchronize()
            remesh_s += time.perf_counter() - r0
            m, q = new, qn
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    d = sem.sem_diag(m, pc, q)
    status = sem.sem_status(m)
    # the float64 form on the same remesh schedule (the recorded flags
    # replayed, so the meshes are the same): the max-wind gate
    p64 = sem.sem_params_default(precision=sem.SEM_PREC_FP64)
    m64, q64, s = m0, q0, 0
    for r in range(len(flag_log) + 1):
        w1, w2 = torch.empty_like(q64), torch.empty_like(q64)
        for _ in range(min(t_amr, steps - s)):
            sem.sem_step(m64, p64, q64, w1, w2, dt, stream)
            s += 1
        if r < len(flag_log):
            new = sem.sem_transfer_plan(m64, flag_log[r])
            qn = torch.empty((5, new.NG), dtype=torch.float64, device="cuda")
            sem.sem_transfer(m64, new, q64, qn, stream)
            m64, q64 = new, qn
    d64 = sem.sem_diag(m64, pc, q64)
    return {"workload": "32x32x8 base N=4, level 3 inside 150 km, thresholds [5,10,15], remesh every 50",
            "steps": steps, "wall_s": wall, "remesh_s": remesh_s, "dof_updates_per_s": dof / wall,
            "history": history, "status": status, "max_wind": d["max_wind"],
            "gate": {"max_wind_fp64": d64["max_wind"],
                     "max_wind_rel_err": abs(d["max_wind"] - d64["max_wind"]) / d64["max_wind"],
                     "max_mean_wind_rel_err": abs(d["max_mean_wind"] - d64["max_mean_wind"]) / d64["max_mean_wind"],
                     "how": "float64 form through the same meshes (the mixed run's flags replayed)",
                     "status_fp64": sem.sem_status(m64)}}


def warped_measure(sem, torch, steps=20, warmup=3, gate_steps=100, amplitude=600.0, k=4):
    """The benchmark mesh (64x64x16, N = 4, 2048 km x 24 km) with warped
    layers: every node lifted by amplitude sin(2 pi k x / Lx) sin(2 pi k y / Ly)
    sin(pi zeta / Lz) (flat lids), so every element is non-affine and carries
    float64 metric terms per node.  Mixed increment-form steps, autotuned
    among the line-exchange variants; per-kernel durations; the algorithmic
    bytes of the non-affine pass (the affine bytes plus the float32 metric
    terms, 3 per local node of each column line, and the packed reference
    state per global node); the max-wind gate against the float64 form on
    the same mesh."""
    from synth.vortex import vortex_state
    L, Lz, n, nz, N, dt = 2048e3, 24e3, 64, 16, 4, 0.25
    m = sem.sem_mesh_create(L, L, Lz, n, n, nz, N, warp=(amplitude, k, k))
    q0 = torch.from_numpy(vortex_state(sem.sem_mesh_coords_host(m).T, Lz)).cuda()
    p = sem.sem_params_default(precision=sem.SEM_PREC_MIXED)
    p64 = sem.sem_params_default(precision=sem.SEM_PREC_FP64)
    stream = torch.cuda.current_stream()
    q = q0.clone()
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32, stream)
    rows, chosen = sem.sem_autotune(m, p, q32, 5, stream)
    for _ in range(warmup):
        sem.sem_step_mixed(m, p, q, q32, work, dt, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sem.sem_step_mixed(m, p, q, q32, work, dt, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    sem.sem_profile_begin()
    for _ in range(steps):
        sem.sem_step_mixed(m, p, q, q32, work, dt, stream)
    torch.cuda.synchronize()
    pr = sem.sem_profile_end()
    NG, NL, Ncol, Nq = m.NG, m.Ne * (N + 1) ** 3, m.Ncol, (N + 1) ** 2
    metric_bytes = 12 * Ncol * Nq * nz * (N + 1)
    ref_bytes = 16 * NG
    elem = 20 * NG + 4 * NL + metric_bytes + ref_bytes
    stage = 124 * NG + 4 * NL + metric_bytes + ref_bytes
    hbm, _ = peaks()
    kern = {}
    for name, (nl, tot) in pr.items():
        if name == "mirror":
            continue
        avg = tot / max(nl, 1)
        ab = elem if name.startswith("volume") else stage - elem
        kern[name] = {"launches": nl, "ms_avg": avg, "alg_bytes": ab,
                      "frac": ab / (avg * 1e-3) / 1e9 / hbm}
    # max-wind gate: mixed against float64 steps on the same warped mesh
    gate = None
    if gate_steps > 0:
        qm, qd = q0.clone(), q0.clone()
        sem.sem_mirror(m, qm, q32, stream)
        w1, w2 = torch.empty_like(qd), torch.empty_like(qd)
        for _ in range(gate_steps):
            sem.sem_step_mixed(m, p, qm, q32, work, dt, stream)
            sem.sem_step(m, p64, qd, w1, w2, dt, stream)
        dm, dd = sem.sem_diag(m, p64, qm), sem.sem_diag(m, p64, qd)
        gate = {"steps": gate_steps, "max_wind_fp64": dd["max_wind"],
                "max_wind_rel_err": abs(dm["max_wind"] - dd["max_wind"]) / dd["max_wind"]}
    return {"workload": f"uniform-64x64x16-N4 with warped layers (amplitude {amplitude:g} m, "
                        f"{k} x {k} periods, flat lids)",
            "ms_per_step": ms, "value": 3 * 5 * NL / (ms * 1e-3),
            "autotune": {"variants": [{"layers_per_cta": r[0], "min_ctas_per_sm": r[1], "ms": r[2],
                                       "kind": r[3]} for r in rows], "chosen": chosen},
            "alg_bytes": {"element_pass": elem, "stage": stage, "metric": metric_bytes,
                          "reference_state": ref_bytes},
            "stage_frac": stage / (ms / 3 * 1e-3) / 1e9 / hbm, "kernels": kern,
            "gate": gate, "status": sem.sem_status(m)}


def paper_set_measure(sem, torch, steps=20, warmup=3, gate_steps=100, warp=None):
    """The benchmark mesh (64x64x16, N = 4) with the paper's own equation set
    (mass in flux form, momentum and theta' in advective form, variables
    rho', u, v, w, theta'): mixed increment-form steps, autotuned among that
    set's line-exchange variants; per-kernel durations against the same
    algorithmic bytes as the conservative set (the state and residual arrays
    have the same shapes; on warped layers plus the float32 metric terms and
    the reference state per node, as in warped_measure); the max-wind gate
    against the float64 form.  warp = (amplitude, kx, ky): warped layers."""
    from synth.vortex import vortex_state
    L, Lz, n, nz, N, dt = 2048e3, 24e3, 64, 16, 4, 0.25
    m = sem.sem_mesh_create(L, L, Lz, n, n, nz, N, warp=warp)
    q0 = torch.from_numpy(vortex_state(sem.sem_mesh_coords_host(m).T, Lz, eqset="NC")).cuda()
    p = sem.sem_params_default(eqset=1, precision=sem.SEM_PREC_MIXED)
    p64 = sem.sem_params_default(eqset=1, precision=sem.SEM_PREC_FP64)
    stream = torch.cuda.current_stream()
    q = q0.clone()
    q32 = torch.empty(q.shape, dtype=torch.float32, device="cuda")
    work = torch.empty((10, m.NG), dtype=torch.float32, device="cuda")
    sem.sem_mirror(m, q, q32, stream)
    rows, chosen = sem.sem_autotune(m, p, q32, 5, stream)
    for _ in range(warmup):
        sem.sem_step_mixed(m, p, q, q32, work, dt, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sem.sem_step_mixed(m, p, q, q32, work, dt, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    sem.sem_profile_begin()
    for _ in range(steps):
        sem.sem_step_mixed(m, p, q, q32, work, dt, stream)
    torch.cuda.synchronize()
    pr = sem.sem_profile_end()
    NG, NL, Ncol, Nq = m.NG, m.Ne * (N + 1) ** 3, m.Ncol, (N + 1) ** 2
    extra = 0 if warp is None else 12 * Ncol * Nq * nz * (N + 1) + 16 * NG
    elem, stage = 20 * NG + 4 * NL + extra, 124 * NG + 4 * NL + extra
    hbm, _ = peaks()
    kern = {}
    for name, (nl, tot) in pr.items():
        if name == "mirror":
            continue
        avg = tot / max(nl, 1)
        ab = elem if name.startswith("volume") else stage - elem
        kern[name] = {"launches": nl, "ms_avg": avg, "alg_bytes": ab,
                      "frac": ab / (avg * 1e-3) / 1e9 / hbm}
    gate = None
    if gate_steps > 0:
        qm, qd = q0.clone(), q0.clone()
        sem.sem_mirror(m, qm, q32, stream)
        w1, w2 = torch.empty_like(qd), torch.empty_like(qd)
        for _ in range(gate_steps):
            sem.sem_step_mixed(m, p, qm, q32, work, dt, stream)
            sem.sem_step(m, p64, qd, w1, w2, dt, stream)
        dm, dd = sem.sem_diag(m, p64, qm), sem.sem_diag(m, p64, qd)
        gate = {"steps": gate_steps, "max_wind_fp64": dd["max_wind"],
                "max_wind_rel_err": abs(dm["max_wind"] - dd["max_wind"]) / dd["max_wind"]}
    what = "" if warp is None else (f" on warped layers (amplitude {warp[0]:g} m, {warp[1]} x {warp[2]} "
                                    "periods, flat lids)")
    return {"workload": "uniform-64x64x16-N4, the paper's equation set" + what,
            "ms_per_step": ms, "value": 3 * 5 * NL / (ms * 1e-3),
            "autotune": {"variants": [{"layers_per_cta": r[0], "min_ctas_per_sm": r[1], "ms": r[2],
                                       "kind": r[3]} for r in rows], "chosen": chosen},
            "alg_bytes": {"element_pass": elem, "stage": stage},
            "stage_frac": stage / (ms / 3 * 1e-3) / 1e9 / hbm, "kernels": kern,
            "gate": gate, "status": sem.sem_status(m)}


def mlp_forward_measure(sem, torch, rows=1 << 20, reps=20):
    """Forward throughput of the flag network on `rows` feature rows: the
    tcgen05 forward (default) and the mma.sync one, TFLOP/s of the three GEMMs
    against the measured bfloat16 peak."""
    X = torch.randn((rows, 136), dtype=torch.float32, device="cuda")
    net = sem.sem_mlp_create(3, rows)
    prob = torch.empty((rows, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    flop = 2.0 * (136 * 128 + 128 * 128 + 128 * 3) * rows
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = json.load(f)["bf16_tflops"]
    except Exception:
        bf16 = 1900.0
    out = {"rows": rows, "gflop": flop / 1e9, "bf16_peak_tflops": bf16}
    for tc in (1, 0):
        sem.sem_mlp_select_forward(net, tc)
        for _ in range(3):
            sem.sem_mlp_forward(net, X, prob, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            sem.sem_mlp_forward(net, X, prob, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out["tcgen05" if tc else "mma_sync"] = {"ms": ms, "tflops": flop / (ms * 1e-3) / 1e12,
                                                "frac_bf16_peak": flop / (ms * 1e-3) / 1e12 / bf16}
    out["status"] = sem.sem_mlp_status(net)
    return out


def learned_measure(sem, torch):
    """The learned adaptation schedule against the criterion alone (same
    remesh count): ten seeded translating vortices, train on eight."""
    from paper_2410_21607_gb300 import learned
    from synth.vortex import vortex_state
    from synth.workloads import translating_vortices
    L, Lz = 150e3, 24e3
    m = sem.sem_mesh_create(L, L, Lz, 24, 24, 2, 4, lvl_max=2)
    X = sem.sem_mesh_coords_host(m).T
    states = [torch.from_numpy(vortex_state(X, Lz, s)).cuda() for s in translating_vortices()]
    t0 = time.perf_counter()
    res = learned.gain_experiment(sem, torch, m, states, dt=1.0, n_train=8)
    out = {"status": res["status"], "by_interval": res["by_interval"]}
    out["workload"] = ("24x24x2 N=4, 150 km box, 10 translating vortices x 400 steps of 1 s, "
                       "one network per remesh interval (window labels), criterion checked every 10 steps")
    # the two schedules driving real remeshes on the held-out vortices, against
    # the base mesh refined uniformly to the top level
    # (horizontal Smagorinsky stress C_s = 0.5 on every run: without it the
    # non-conforming interfaces swept by the background wind go unstable)
    runs = learned.adaptive_comparison(sem, torch, translating_vortices()[8:], res["net"],
                                       physics=dict(smag_cs=0.5))
    out["adaptive_runs"] = {
        "workload": "held-out vortices 9, 10: 400 s at dt 0.25 s, remesh every 50 s, levels 0..2, "
                    "Smagorinsky C_s 0.5",
        "wind_err_criterion": [r["wind_err_criterion"] for r in runs],
        "wind_err_learned": [r["wind_err_learned"] for r in runs],
        "missed_criterion": [r["criterion"]["missed_rate"] for r in runs],
        "missed_learned": [r["learned"]["missed_rate"] for r in runs],
        "remeshes": [[r["criterion"]["remeshes"], r["learned"]["remeshes"]] for r in runs],
        "mean_elements": [[r["reference"]["mean_elements"], r["criterion"]["mean_elements"],
                           r["learned"]["mean_elements"]] for r in runs],
        "dof_updates_per_s": [[r["reference"]["dof_updates_per_s"], r["criterion"]["dof_updates_per_s"],
                               r["learned"]["dof_updates_per_s"]] for r in runs],
        "seconds": [[r["reference"]["seconds"], r["criterion"]["seconds"], r["learned"]["seconds"]]
                    for r in runs],
        "gate_max_wind_rel_err": [r["gate_max_wind_rel_err"] for r in runs],
        "gate": "mixed learned run against the float64 form on the same remesh schedule (flags replayed)",
        "status": max(max(r[k]["status"] for k in ("reference", "criterion", "learned", "learned_fp64"))
                      for r in runs)}
    out["forward"] = mlp_forward_measure(sem, torch)
    out["seconds"] = time.perf_counter() - t0
    return out


def run_reference(a):
    import torch.distributed as dist  # noqa: F401
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    # each step: one SSP-RK3 step of the oracle on a 16x16x16 block
    import numpy as np  # noqa: F401
    from oracle import mesh as om, refstate, rk as ork
    from synth.vortex import vortex_state
    n = 16
    L = 2048e3 * n / 64
    o = om.OracleMesh(L, L, 24e3, n, n, 16, 4)
    q = vortex_state(o.XG, 24e3)
    prm = refstate.Params()
    for _ in range(a.warmup):
        q = ork.rk_step(o, prm, q, 0.25)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        q = ork.rk_step(o, prm, q, 0.25)
    dt = time.perf_counter() - t0
    value = 5 * o.Ne * o.P * 3 * a.steps / dt
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-updates/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * dt / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{n}x{n}x16 block", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": threads,
                             "kind": "oracle",
                             "sample": f"SSP-RK3 steps on a {n}x{n}x16 block of the workload's elements"},
            "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2410_21607_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2410_21607_gb300 import sem
    from synth.vortex import vortex_state

    if a.mlp_forward_only:
        if rank == 0:
            print(json.dumps({"mlp_forward": mlp_forward_measure(sem, torch)}), flush=True)
        return 0

    L, Lz, n, nz, N, dt = 2048e3, 24e3, 64, 16, 4, 0.25
    m = sem.sem_mesh_create(L, L, Lz, n, n, nz, N)
    xyz = sem.sem_mesh_coords_host(m).T
    q0_host = vortex_state(xyz, Lz)
    q0 = torch.from_numpy(q0_host).cuda()
    prec = sem.SEM_PREC_MIXED if a.form == "mixed" else sem.SEM_PREC_FP64
    p = sem.sem_params_default(precision=prec)
    p64 = sem.sem_params_default(precision=sem.SEM_PREC_FP64)
    stream = torch.cuda.current_stream()

    def new_bufs():
        b = [q0.clone(), torch.empty_like(q0), torch.empty_like(q0)]
        m32 = [torch.empty(q0.shape, dtype=torch.float32, device="cuda"),
               torch.empty((10, q0.shape[1]), dtype=torch.float32, device="cuda")]
        sem.sem_mirror(m, b[0], m32[0], stream)
        return b + m32

    def step(b, prm):
        qn, w1, w2, q32, work = b
        if prm.precision == sem.SEM_PREC_MIXED:
            # increment form: float32 stage increments, float64 state update
            sem.sem_step_mixed(m, prm, qn, q32, work, dt, stream)
            return b
        # float64 form, ping-pong: q -> w1 -> w2 -> w1, then w1 is the state
        sem.sem_rk_stage(m, prm, 0, qn, qn, w1, dt, stream)
        sem.sem_rk_stage(m, prm, 1, qn, w1, w2, dt, stream)
        sem.sem_rk_stage(m, prm, 2, qn, w2, w1, dt, stream)
        return [w1, qn, w2, q32, work]

    bufs = new_bufs()
    tune = None
    if a.form == "mixed" and a.kernel_row is not None:
        sem.sem_autotune_select(m, a.kernel_row)
        tune = {"variants": None, "chosen": a.kernel_row}
    elif a.form == "mixed":
        rows, chosen = sem.sem_autotune(m, p, bufs[3], 5, stream)
        tune = {"variants": [{"layers_per_cta": r[0], "min_ctas_per_sm": r[1], "ms": r[2],
                              "kind": r[3]} for r in rows], "chosen": chosen}
    dof_stage = 5 * m.Ne * (N + 1) ** 3
    # the arithmetic peaks of this GPU, from the library's FMA probe
    fp32_peak = sem.sem_peak_probe(sem.SEM_PREC_MIXED, stream)
    fp64_peak = sem.sem_peak_probe(sem.SEM_PREC_FP64, stream)
    for _ in range(max(a.warmup, 3)):
        bufs = step(bufs, p)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(a.steps):
        bufs = step(bufs, p)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / a.steps
    # the same K steps again with an event pair around every launch, for the
    # per-kernel durations of the roofline (the events add about 5 % to a step,
    # so the step time above comes from the pass without them)
    sem.sem_profile_begin()
    for _ in range(a.steps):
        bufs = step(bufs, p)
    torch.cuda.synchronize()
    prof = sem.sem_profile_end()
    ck = clocks.stop()
    ms = max_over_ranks(ms, world, "cuda")
    if world > 1:
        dist.barrier()
    value = job_throughput(dof_stage * 3, world, ms)
    status = sem.sem_status(m)

    # per-kernel roofline of the timed region, on the method's algorithmic
    # bytes per RK stage: per global node the float64 stage reads and writes
    # (qn 40 B, qs 40 B or its float32 mirror 20 B, q_out 40 B and its mirror
    # 20 B) and the inverse mass (8 or 4 B), plus 4 B of constraint index per
    # local node.  Mixed: 124 B per global node + 4 B per local node; float64:
    # 128 + 4.  The element kernel's share is its read of the state (the
    # mirror, 20 B, or the float64 state, 40 B) and the index; the gather /
    # stage kernel has the rest.  The column residuals the element kernel
    # writes and the gather kernel reads back are an intermediate of this
    # implementation, not algorithmic bytes: they are reported beside them.
    hbm, peak_kind = peaks()
    Ncol, Nq, NZ, NG, NH = m.Ncol, (N + 1) ** 2, m.NZ, m.NG, m.NH
    NL = m.Ne * (N + 1) ** 3
    rbytes = 4 if a.form == "mixed" else 8
    stage_bytes = (124 if a.form == "mixed" else 128) * NG + 4 * NL
    elem_bytes = 5 * rbytes * NG + 4 * NL
    resid_bytes = 5 * rbytes * Ncol * Nq * NZ
    alg = {"volume": elem_bytes, "dss_rk": stage_bytes - elem_bytes, "dss_inc": stage_bytes - elem_bytes}
    kernels = {}
    for name, (launches, tot) in prof.items():
        if name == "mirror":
            continue
        base = name.rsplit("_", 1)[0]
        avg = tot / max(launches, 1)
        kernels[name] = {"launches": launches, "ms_avg": avg, "share": None,
                         "alg_bytes": alg[base], "gbs": alg[base] / (avg * 1e-3) / 1e9,
                         "frac": alg[base] / (avg * 1e-3) / 1e9 / hbm,
                         "intermediate_bytes": resid_bytes}
    tot_all = sum(v[1] for v in prof.values()) or 1.0
    for name in list(kernels):
        kernels[name]["share"] = prof[name][1] / tot_all
    dom = max(kernels, key=lambda k: prof[k][1])
    # measured DRAM traffic of the dominant kernel (ncu, same kernel and
    # workload, kept under profiles/); null until a capture of the current
    # kernel source exists
    traffic = None
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        with open(os.path.join(ROOT, "paper_2410_21607_gb300", "csrc", "k_stage.cu"), "rb") as f:
            cur = hashlib.sha1(f.read()).hexdigest()
        if tr.get("k_stage_sha1") == cur and dom in tr:
            traffic = tr[dom]["bytes"]
    except Exception:
        traffic = None
    flop_node = 300.0        # float32 flop per local node of the element kernel (estimate of the method)
    dav = kernels[dom]["ms_avg"]
    roof = {"kernel": dom, "bound": "hbm", "achieved": kernels[dom]["gbs"], "peak": hbm,
            "unit": "GB/s", "frac": kernels[dom]["frac"], "traffic": traffic,
            "alg_bytes": alg[dom.rsplit("_", 1)[0]], "intermediate_bytes": resid_bytes,
            "traffic_over_alg": None if traffic is None else traffic / alg[dom.rsplit("_", 1)[0]],
            "peak_source": peak_kind + " (MEASURED_PEAKS.json copy bandwidth)",
            "alu": {"flop_per_local_node": flop_node,
                    "achieved_tflops": flop_node * NL / (dav * 1e-3) / 1e12,
                    "peak_tflops": fp32_peak if a.form == "mixed" else fp64_peak,
                    "peak_source": "sem_peak_probe (this GPU, FMA chains)",
                    "frac": flop_node * NL / (dav * 1e-3) / 1e12 / (fp32_peak if a.form == "mixed" else fp64_peak)},
            "stage": {"alg_bytes": stage_bytes, "ms": ms / 3,
                      "achieved": stage_bytes / (ms / 3 * 1e-3) / 1e9,
                      "frac": stage_bytes / (ms / 3 * 1e-3) / 1e9 / hbm},
            "timing": "CUDA events around each launch on its stream, over a second pass of the K timed steps"}

    # FP64 form beside it, and the max-wind gate after gate_steps steps
    fp64_ms = None
    fp64_kernels = None
    if a.form == "mixed":
        b64 = new_bufs()
        for _ in range(2):
            b64 = step(b64, p64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nfp = 3
        for _ in range(nfp):
            b64 = step(b64, p64)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_ms = max_over_ranks(e0.elapsed_time(e1) / nfp, world, "cuda")
        sem.sem_profile_begin()
        for _ in range(nfp):
            b64 = step(b64, p64)
        torch.cuda.synchronize()
        pr64 = sem.sem_profile_end()
        st64 = 128 * NG + 4 * NL
        fp64_kernels = {}
        for k, (nl, tot) in pr64.items():
            avg = tot / max(nl, 1)
            fp64_kernels[k] = {"launches": nl, "ms_avg": avg}
            if k.startswith("dss_rk"):
                # the whole stage's algorithmic bytes (128 B per global node +
                # 4 B per local node) over the gather / stage kernel alone
                fp64_kernels[k].update(stage_alg_bytes=st64,
                                       frac_stage_bytes=st64 / (avg * 1e-3) / 1e9 / hbm)
            if k.startswith("volume"):
                fp64_kernels[k].update(achieved_tflops=flop_node * NL / (avg * 1e-3) / 1e12,
                                       frac_fp64_peak=flop_node * NL / (avg * 1e-3) / 1e12 / fp64_peak)
    gate = None
    if a.gate_steps > 0:
        bm = new_bufs()
        bd = new_bufs()
        for _ in range(a.gate_steps):
            bm = step(bm, p)
            bd = step(bd, p64)
        dm = sem.sem_diag(m, p64, bm[0])
        dd = sem.sem_diag(m, p64, bd[0])
        gate = {"steps": a.gate_steps, "max_wind_fp64": dd["max_wind"],
                "max_wind_rel_err": abs(dm["max_wind"] - dd["max_wind"]) / dd["max_wind"],
                "max_mean_wind_rel_err": abs(dm["max_mean_wind"] - dd["max_mean_wind"])
                / dd["max_mean_wind"]}

    # the same step with the terms of the paper's runs (Sec. 4): horizontal
    # Smagorinsky stress C_s = 0.21, absorbing layer gamma = 1/s, z_d = 4 km
    physics_res = None
    if not a.no_physics and a.form == "mixed":
        pphys = dict(smag_cs=0.21, sponge_gamma=1.0, sponge_depth=4000.0)
        pp = sem.sem_params_default(precision=sem.SEM_PREC_MIXED, **pphys)
        bp = new_bufs()
        for _ in range(3):
            bp = step(bp, pp)
        torch.cuda.synchronize()
        kp = max(3, min(a.steps, 10))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(kp):
            bp = step(bp, pp)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_p = max_over_ranks(e0.elapsed_time(e1) / kp, world, "cuda")
        sem.sem_profile_begin()
        for _ in range(kp):
            bp = step(bp, pp)
        torch.cuda.synchronize()
        pr = sem.sem_profile_end()
        physics_res = {"params": pphys, "ms_per_step": ms_p, "value": job_throughput(dof_stage * 3, world, ms_p),
                       "step_time_ratio": ms_p / ms,
                       "kernels_ms_avg": {k: v[1] / max(v[0], 1) for k, v in pr.items()},
                       "status": sem.sem_status(m)}

    # end to end through the C ABI with host buffers (pinned), copies timed:
    # every step copies its input state in from pinned host memory and its
    # result out.  Consecutive steps overlap their copies with the computation
    # of their neighbours (copy-in streams, the compute stream, copy-out
    # streams, three buffer sets), as a caller streaming states through the
    # solver would; each copy is split over several streams so that several
    # copy engines share it; the computation stays on one stream (the mesh's
    # residual scratch is shared by its steps).
    # three buffer sets, so that step k's copy in, step k-1's computation and
    # step k-2's copy out each have a set of their own
    nsets = 3
    hq = torch.from_numpy(q0_host).pin_memory()
    houts = [torch.empty_like(hq).pin_memory() for _ in range(nsets)]
    sets = [new_bufs() for _ in range(nsets)]
    ncopy = 4                                  # copy streams per direction (copy engines)
    s_in = [torch.cuda.Stream() for _ in range(ncopy)]
    s_out = [torch.cuda.Stream() for _ in range(ncopy)]
    ev_in = [[torch.cuda.Event() for _ in range(ncopy)] for _ in range(nsets)]
    ev_cmp = [torch.cuda.Event() for _ in range(nsets)]
    ev_out = [[torch.cuda.Event() for _ in range(ncopy)] for _ in range(nsets)]
    flat = hq.numel()
    cuts = [flat * c // ncopy for c in range(ncopy + 1)]
    ke = max(3, a.steps)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for c in range(ncopy):
        s_in[c].wait_event(e0)
    for k in range(ke):
        bi = k % nsets
        dst = sets[bi][0].view(-1)
        for c in range(ncopy):
            if k >= nsets:
                s_in[c].wait_event(ev_out[bi][c])      # the buffer set's previous result is out
            with torch.cuda.stream(s_in[c]):
                dst[cuts[c]:cuts[c + 1]].copy_(hq.view(-1)[cuts[c]:cuts[c + 1]], non_blocking=True)
            ev_in[bi][c].record(s_in[c])
            stream.wait_event(ev_in[bi][c])
        if a.form == "mixed":
            sem.sem_mirror(m, sets[bi][0], sets[bi][3], stream)
        sets[bi] = step(sets[bi], p)
        ev_cmp[bi].record(stream)
        src = sets[bi][0].view(-1)
        for c in range(ncopy):
            s_out[c].wait_event(ev_cmp[bi])
            with torch.cuda.stream(s_out[c]):
                houts[bi].view(-1)[cuts[c]:cuts[c + 1]].copy_(src[cuts[c]:cuts[c + 1]], non_blocking=True)
            ev_out[bi][c].record(s_out[c])
    for bi in range(nsets):
        for c in range(ncopy):
            stream.wait_event(ev_out[bi][c])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / ke, world, "cuda")
    assert all(torch.equal(houts[0], hb) for hb in houts[1:]), "the streamed steps disagree"
    nbytes = 5 * NG * 8

    batched = None
    if not a.no_batched and a.form == "mixed":
        rates = order_rates(sem, torch)
        batched = ([batched_measure(sem, torch, rates=rates)] if a.batched in ("both", "refined") else []) + \
                  ([batched_measure(sem, torch, refine=False, rates=rates)]
                   if a.batched in ("both", "unrefined") else [])
        if a.batched in ("both", "unrefined"):
            batched.append(batched_measure(sem, torch, refine=False, eqset=1))
        batched.append({"order_rates_dof_updates_per_s": {str(k): v for k, v in rates.items()},
                        "how": "single uniform mesh per order, autotuned mixed steps"})

    warped_res = None
    if not a.no_warped and a.form == "mixed":
        warped_res = warped_measure(sem, torch, gate_steps=a.gate_steps)
    paper_res = None
    if not a.no_paper_set and a.form == "mixed":
        paper_res = paper_set_measure(sem, torch, gate_steps=a.gate_steps)
        if not a.no_warped:
            paper_res["warped"] = paper_set_measure(sem, torch, gate_steps=a.gate_steps, warp=(600.0, 4, 4))
    amr_res = None
    if not a.no_amr and a.form == "mixed":
        amr_res = amr_measure(sem, torch)
    learned_res = None
    if not a.no_learned and a.form == "mixed":
        learned_res = learned_measure(sem, torch)

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not a.no_cpu_baseline:
            v, thr, desc, secs, busy = cpu_oracle_sample()
            one = cpu_one_thread()
            cpu = {"value": v, "unit": "DOF-updates/s", "cores": thr, "kind": "oracle",
                   "sample": desc, "seconds": secs, "busy_threads": busy, "cpu_model": cpu_model(),
                   "one_thread": one, "small_workload_all_threads": cpu_small_case()}
        line = {
            "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64acc" if a.form == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": a.form, "elements": m.Ne,
                       "local_nodes": m.Ne * (N + 1) ** 3, "global_nodes": NG, "dt": dt,
                       "l2": "inputs larger than L2 (state 3 x 170 MB + residual scratch)",
                       "parallelism": f"replicas x{world}"},
            "fp64_form": None if fp64_ms is None else {
                "ms_per_step": fp64_ms, "value": job_throughput(dof_stage * 3, world, fp64_ms),
                "speedup_mixed_over_fp64": fp64_ms / ms, "kernels": fp64_kernels,
                "stage_frac": (128 * NG + 4 * NL) / (fp64_ms / 3 * 1e-3) / 1e9 / hbm},
            "peaks": {"hbm_gbs": hbm, "hbm_source": peak_kind, "fp32_tflops": fp32_peak,
                      "fp64_tflops": fp64_peak, "fma_source": "sem_peak_probe"},
            "gate": gate,
            "roofline": roof, "kernels": kernels, "autotune": tune, "batched": batched,
            "learned": learned_res, "amr": amr_res, "physics": physics_res, "warped": warped_res,
            "paper_set": paper_res,
            "cpu_baseline": cpu,
            "e2e": {"value": job_throughput(dof_stage * 3, world, e2e_ms), "unit": "DOF-updates/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                    "ms_per_step": e2e_ms},
            "gpu_launches": sum(v[0] for v in prof.values()),
            "clocks": ck, "status": status,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
