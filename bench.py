"""Benchmark of the stencil hot path on the 3D heat workload.

Workload (one "step"): the 3D 7-point damped-Jacobi / heat solve on a 256^3
interior (1-cell zero halo, RHS f uniform in [-1, 1) from seed 202,
lam = dt*alpha = 1/8), 200 sweeps with ping-pong grids, and every 10 sweeps a
fused sweep + do_reduce returning the L2 residual of the iterate it reads
(20 residuals per step).  Primary arithmetic FP64; the FP32-storage variant
runs in the same invocation and is reported under "variants".

Metric: grid-point updates per second (whole job, all ranks), device-timed
with CUDA events on the launching stream; the working set (three 137 MB FP64
grids) is larger than the 126 MB L2.  "e2e" repeats the step through the
C ABI from pinned host buffers: the H2D copy of u0 and f and the D2H copy of
the final grid and residuals are inside its timed region.

--impl reference times the FP64 CPU oracle (the plain C loop nest) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 256
LAM = 0.125
SWEEPS = 200
EVERY = 10
SEED = 202
TERMS_PLAIN = 8                # FMAs per point of the plain sweep (one per stencil input)
BYTES_PER_PT = {"f64": 24, "f32": 12, "bf16": 6}  # u read, f read, u' written


def load_json(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def measured_peaks():
    return load_json(os.path.join(ROOT, "MEASURED_PEAKS.json"))


def profile_traffic(kernel_key):
    """DRAM bytes per launch from the committed ncu summaries (a line
    'traffic <key> <bytes>' in one of profiles/*.md), else None."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        try:
            for line in open(path):
                parts = line.strip().strip("`").split()
                if len(parts) == 3 and parts[0] == "traffic" and parts[1] == kernel_key:
                    return float(parts[2])
        except OSError:
            pass
    return None


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for name, val in zip(names, p[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def warm(fn, warmup, min_s=0.25):
    """Untimed warm-up: at least `warmup` calls of `fn`, and more until about
    `min_s` seconds of them have run on the device, so that a workload whose
    step lasts well under a millisecond still starts its timed region at the
    GPU's working clocks.  Under --profile only the `warmup` calls run, so
    that profiler launch counts stay fixed."""
    import torch

    if PROFILE:
        min_s = 0.0
    t0, k = time.perf_counter(), 0
    while k < warmup or (time.perf_counter() - t0 < min_s and k < 100000):
        fn()
        k += 1
        if k % 4 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()


# ------------------------------------------------------------------ GPU arm
def run_gpu(dtype, steps, warmup, dist, n=N_SIDE, sweeps=SWEEPS, clocks=None):
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S

    h = (1, 1, 1)
    shape = (n, n, n)
    u0, f = I.heat3d(SEED, n)
    u, v = B.Grid(shape, h, dtype).upload(u0), B.Grid(shape, h, dtype).upload(u0)
    F = B.Grid(shape, h, dtype).upload(f)
    fused, plain = B.Stencil(S.heat7_fused(LAM)), B.Stencil(S.heat7(LAM))
    groups = sweeps // EVERY
    res = torch.zeros(groups, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ev = []

    def step(timed):
        for m in range(groups):
            if timed:
                e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                e[0].record(stream)
            B.do_reduce(B.L2, fused, [u, F], [v], result=res[m:m + 1])
            if timed:
                e[1].record(stream)
            B.swap(u, v)
            if timed:
                e[2].record(stream)
            B.do_all(plain, [u, F], [v], sweeps=EVERY - 1)
            if timed:
                e[3].record(stream)
                ev.append(e)
            B.swap(u, v)

    for _ in range(warmup):
        step(False)
    torch.cuda.synchronize()
    dist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ctx = clocks if clocks is not None else _Null()
    with ctx:
        t0.record(stream)
        for _ in range(steps):
            step(True)
        t1.record(stream)
        torch.cuda.synchronize()
    dist.barrier()
    B.sync()
    ms = t0.elapsed_time(t1)
    fused_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / len(ev)
    plain_ms = sum(e[2].elapsed_time(e[3]) for e in ev) / (len(ev) * (EVERY - 1))
    residuals = res.cpu().tolist()
    return {"ms_total": ms, "ms_per_step": ms / steps, "fused_launch_ms": fused_ms, "plain_launch_ms": plain_ms,
            "launches": steps * sweeps, "points": n ** 3, "residuals": residuals}


def run_temporal(dtype, n=N_SIDE, sweeps=13, reps=5):
    """Temporal blocking on the plain heat sweep (FP32 / BF16 storage): the
    time per sweep of `sweeps`-sweep gscl_do_all calls with K = 1 .. 4 sweeps
    fused per pass over HBM (GSCL_TEMPORAL), then the factor gscl_tune_sweeps
    picks for these grids (remembered, so the variant runs use it).  The last
    launch of a call is a single sweep, so 13 sweeps are 12 fused ones (6, 4
    or 3 passes for K = 2, 3, 4) and one single sweep."""
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S

    h, shape = (1, 1, 1), (n, n, n)
    u0, f = I.heat3d(SEED, n)
    u, v, F = B.Grid(shape, h, dtype).upload(u0), B.Grid(shape, h, dtype).upload(u0), B.Grid(shape, h, dtype).upload(f)
    op = B.Stencil(S.heat7(LAM))
    stream = torch.cuda.current_stream()
    out = {"sweeps_per_call": sweeps}
    old = os.environ.get("GSCL_TEMPORAL")
    try:
        for K in (1, 2, 3, 4):
            os.environ["GSCL_TEMPORAL"] = str(K)
            B.do_all(op, [u, F], [v], sweeps=sweeps)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                B.do_all(op, [u, F], [v], sweeps=sweeps)
            e1.record(stream)
            torch.cuda.synchronize()
            out[f"k{K}_ms_per_sweep"] = round(e0.elapsed_time(e1) / (reps * sweeps), 5)
    finally:
        if old is None:
            os.environ.pop("GSCL_TEMPORAL", None)
        else:
            os.environ["GSCL_TEMPORAL"] = old
    out["tuned_factor"] = B.tune_sweeps(op, [u, F], [v], trial_sweeps=8)
    out["speedup_k2_vs_k1"] = round(out["k1_ms_per_sweep"] / out["k2_ms_per_sweep"], 3)
    B.sync()
    return out


def run_fusion_ablation(dtype, reps=20, n=N_SIDE):
    """Section 5.2's fused diffusion + convergence test against the two-pass
    form on the heat workload: one fused sweep returning the L2 residual of
    the iterate it reads, against a plain sweep plus a separate residual
    reduction over the same iterate (u and f read twice).  Mean per pair of
    operations, CUDA events on the launching stream."""
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S

    h = (1, 1, 1)
    shape = (n, n, n)
    u0, f = I.heat3d(SEED, n)
    u, v = B.Grid(shape, h, dtype).upload(u0), B.Grid(shape, h, dtype).upload(u0)
    F = B.Grid(shape, h, dtype).upload(f)
    fused, plain, resid = B.Stencil(S.heat7_fused(LAM)), B.Stencil(S.heat7(LAM)), B.Stencil(S.residual7())
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def fused_step():
        B.do_reduce(B.L2, fused, [u, F], [v], result=res[0:1])

    def two_pass_step():
        B.do_all(plain, [u, F], [v])
        B.do_reduce(B.L2, resid, [u, F], [], result=res[1:2])

    out = {}
    for name, fn in (("fused_ms", fused_step), ("two_pass_ms", two_pass_step)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = round(e0.elapsed_time(e1) / reps, 4)
    B.sync()
    out["speedup"] = round(out["two_pass_ms"] / out["fused_ms"], 3)
    r = res.cpu().tolist()
    out["residuals_agree_rel"] = abs(r[0] - r[1]) / max(abs(r[1]), 1e-300)
    return out


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def run_e2e(dtype, steps, warmup, n=N_SIDE, sweeps=SWEEPS):
    """The same step through the C ABI from pinned host memory: every step
    copies u0 and f in (gscl_grid_copy_from_host, into u, v and f) and reads
    the final grid and the residual vector back (gscl_grid_copy_to_host), all
    inside the timed region.  Steps are pipelined over two sets of device
    grids: step s + 1's uploads run on a copy stream while step s computes,
    and step s's downloads on another while step s + 1 computes."""
    import numpy as np
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S
    import ctypes

    h = (1, 1, 1)
    shape = (n, n, n)
    u0, f = I.heat3d(SEED, n)
    tdt = {"f64": torch.float64, "f32": torch.float32}[dtype]
    hu0 = torch.from_numpy(u0).to(tdt).pin_memory()
    hf = torch.from_numpy(f).to(tdt).pin_memory()
    hout = [torch.empty_like(hu0).pin_memory() for _ in range(2)]
    groups = sweeps // EVERY
    hres = [torch.empty(groups, dtype=torch.float64).pin_memory() for _ in range(2)]
    sets = [[B.Grid(shape, h, dtype) for _ in range(3)] for _ in range(2)]
    res = [torch.zeros(groups, dtype=torch.float64, device="cuda") for _ in range(2)]
    fused, plain = B.Stencil(S.heat7_fused(LAM)), B.Stencil(S.heat7(LAM))
    comp = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    L = B.lib()
    ev = lambda: torch.cuda.Event()

    def upload(b, after):
        with torch.cuda.stream(up):
            if after is not None:
                up.wait_event(after)
            sp = B.stream_ptr(up)
            u, v, F = sets[b]
            B.check(L.gscl_grid_copy_from_host(u.handle, ctypes.c_void_p(hu0.data_ptr()), sp))
            B.check(L.gscl_grid_copy_from_host(v.handle, ctypes.c_void_p(hu0.data_ptr()), sp))
            B.check(L.gscl_grid_copy_from_host(F.handle, ctypes.c_void_p(hf.data_ptr()), sp))
            e = ev()
            e.record(up)
        return e

    def compute(b, uploaded):
        comp.wait_event(uploaded)
        u, v, F = sets[b]
        for m in range(groups):
            B.do_reduce(B.L2, fused, [u, F], [v], result=res[b][m:m + 1])
            B.swap(u, v)
            B.do_all(plain, [u, F], [v], sweeps=EVERY - 1)
            B.swap(u, v)
        e = ev()
        e.record(comp)
        return e

    def download(b, computed):
        with torch.cuda.stream(down):
            down.wait_event(computed)
            B.check(L.gscl_grid_copy_to_host(sets[b][0].handle, ctypes.c_void_p(hout[b].data_ptr()),
                                             B.stream_ptr(down)))
            hres[b].copy_(res[b], non_blocking=True)
            e = ev()
            e.record(down)
        return e

    def run(k):
        done = [None, None]       # the last download of each set (its grids free again)
        uploaded = upload(0, None)
        for s in range(k):
            b = s % 2
            nxt = upload(1 - b, done[1 - b]) if s + 1 < k else None
            computed = compute(b, uploaded)
            done[b] = download(b, computed)
            uploaded = nxt
        comp.wait_event(done[(k - 1) % 2])
        if k > 1:
            comp.wait_event(done[k % 2])

    run(warmup)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(comp)
    up.wait_event(t0)
    down.wait_event(t0)
    run(steps)
    t1.record(comp)
    torch.cuda.synchronize()
    B.sync()
    ms = t0.elapsed_time(t1) / steps
    ok = bool(all(np.all(np.isfinite(r.numpy())) for r in hres))
    return {"ms_per_step": ms, "h2d": 3 * hu0.numel() * hu0.element_size(),
            "d2h": hout[0].numel() * hout[0].element_size() + hres[0].numel() * 8, "finite": ok,
            "pipelined": "two grid sets; uploads and downloads on copy streams overlap the neighbouring steps"}


# ------------------------------------------------------------------ batched workload
def run_batched(steps, warmup, count=96, sweeps=100, tune=True, compare=True, fixed_temporal=None):
    """96 independent 3D 7-point heat instances (sides uniform on 32..224 per
    axis, FP32 storage, zero 1-cell halo, lam = 1/8), `sweeps` sweeps of all
    of them per step: one launch per sweep from the batch's work-list, the
    whole group replayed as one CUDA graph.  Also times the same sweeps as one
    gscl_do_all call per instance for comparison."""
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S

    h = (1, 1, 1)
    sides = I.batch_sides(4040, count)
    insts = []
    for i, n in enumerate(sides):
        u0 = I.batch_instance(i, n)
        insts.append(([B.Grid(n, h, "f32").upload(u0)], [B.Grid(n, h, "f32").upload(u0)]))
    op = B.Stencil(S.heat7(LAM, with_f=False))
    batch = B.Batch(op, insts)
    cfg = batch.tune(trial_sweeps=10) if tune else None
    if fixed_temporal:  # profiling runs: a given number of sweeps per launch instead of the tuner's
        batch.set_temporal(fixed_temporal)
    info = batch.info()
    tile = batch.tile()
    temporal = batch.temporal()  # sweeps per launch the tuner kept (1 or 2 for 3D batches)
    points = sum(a * b * c for a, b, c in sides)
    stream = torch.cuda.current_stream()

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    ms_batch = timed(lambda: batch.run(sweeps, graph=True), steps, warmup)
    if not compare:  # profiling run: the graph replay only
        B.sync()
        return {"points": points, "ms_per_step": ms_batch, "value": sweeps * points / (ms_batch * 1e-3) / 1e9,
                "sweep_ms": ms_batch / sweeps, "launch_ms": ms_batch / sweeps * temporal[0],
                "hbm_gbs": 8 * points / (ms_batch / sweeps * 1e-3) / 1e9,
                "per_instance_loop_ms": float("nan"), "speedup_vs_loop": float("nan"), "tuned": cfg, "info": info,
                "tile": tile, "temporal": temporal, "launches": batch._launches(sweeps),
                "sides_min_max": [min(min(s) for s in sides), max(max(s) for s in sides)]}
    # the roofline's kernel: one sweep of the batch alone (no graph), or, when
    # the tuner fuses k sweeps per launch, one such pass: run(2k + 1) is two
    # passes and a single sweep (the last launch of a run is single)
    ms_sweep = timed(lambda: batch.run(1), 5 * steps, 2)
    k = temporal[0]
    ms_launch = ms_sweep
    if k > 1:
        ms_two_passes = timed(lambda: batch.run(2 * k + 1), 5 * steps, 2)
        ms_launch = max(1e-6, (ms_two_passes - ms_sweep) / 2)

    def per_instance():
        for ins, outs in insts:
            B.do_all(op, ins, outs, sweeps=sweeps)

    ms_loop = timed(per_instance, max(1, steps // 2), 1)
    B.sync()
    nbytes = 8 * points * k  # FP32: u read, u' written, per point-update; k updates per launch
    return {"points": points, "ms_per_step": ms_batch, "value": sweeps * points / (ms_batch * 1e-3) / 1e9,
            "sweep_ms": ms_sweep, "launch_ms": ms_launch, "hbm_gbs": nbytes / (ms_launch * 1e-3) / 1e9,
            "per_instance_loop_ms": ms_loop, "speedup_vs_loop": ms_loop / ms_batch, "tuned": cfg, "info": info,
            "tile": tile, "temporal": temporal, "launches": batch._launches(sweeps),
            "sides_min_max": [min(min(s) for s in sides), max(max(s) for s in sides)]}


# ------------------------------------------------------------------ 2D Laplace workload
def run_laplace2d(steps, warmup, n=256, sweeps=100, compare=True):
    """2D 5-point Jacobi for Laplace on a 256 x 256 FP64 interior (halo
    sin(pi x), interior uniform [0, 1) from seed 101): one step = 100 sweeps
    with two ping-pong grids, then the max-abs residual |u_100 - u_99|.  The
    grid (0.5 MB) lives in L2 and one sweep is ~0.5 us of work, so single
    sweeps are launch-bound.  The step runs as a batch of one replayed as a
    CUDA graph, with the sweeps fused per launch that the batch tuner picks
    (temporal blocking); one launch per sweep under the graph, and the same
    sweeps as one gscl_do_all call (100 launches, no graph), are timed for
    comparison."""
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S

    u0 = I.laplace2d(101, n)
    shape, h = (n, n, 1), (1, 1, 0)
    u, v = B.Grid(shape, h, "f64", 2).upload(u0), B.Grid(shape, h, "f64", 2).upload(u0)
    op, diff = B.Stencil(S.jacobi5_2d()), B.Stencil(S.difference())
    batch = B.Batch(op, [([u], [v])])
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def step_graph():
        batch.run(sweeps, graph=True)          # even: u holds u_100, v holds u_99
        B.do_reduce(B.MAXABS, diff, [u, v], result=res)

    def step_plain():
        B.do_all(op, [u], [v], sweeps=sweeps)
        B.do_reduce(B.MAXABS, diff, [u, v], result=res)

    def timed(fn, k, w):
        for _ in range(w):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    # single sweeps first (one launch per sweep), then the factor and tile the
    # batch tuner picks (several sweeps per launch, the paper's wide ghost
    # areas on chip; the last launch stays a single sweep, so the pair still
    # holds u_100 and u_99)
    ms_single = timed(step_graph, steps, warmup) if compare else float("nan")
    ms_plain = timed(step_plain, steps, warmup) if compare else float("nan")
    batch.tune(trial_sweeps=16)
    k, tx, ty = batch.temporal()
    launches = batch._launches(sweeps)
    ms_graph = timed(step_graph, steps, warmup)
    B.sync()
    return {"points": n * n, "ms_per_step": ms_graph, "ms_per_step_no_graph": ms_plain,
            "ms_per_step_single_sweeps": ms_single, "sweeps_per_launch": k, "tile": [tx, ty],
            "launches_per_step": launches, "residual": float(res.cpu()[0]), "sweeps": sweeps}


# ------------------------------------------------------------------ climate workload
def run_climate(dtype, steps, warmup, sweeps=50):
    """The multi-grid operator on 256 x 256 x 80 (halo 2, 2, 1): 8 input grids
    (q0..q2, kappa, w, t0..t2; smooth fields from seed 303) -> 3 outputs
    q0'..q2', 50 sweeps per step with the three q grids ping-ponged.  Every
    input is read once per sweep from HBM: 88 B per point in FP64, 44 B in
    FP32."""
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S

    n, h = (256, 256, 80), (2, 2, 1)
    fields = I.climate(303, n, h)
    g = {k: B.Grid(n, h, dtype).upload(a) for k, a in fields.items()}
    cur = [g["q0"], g["q1"], g["q2"]]
    nxt = [B.Grid(n, h, dtype).upload(fields[k]) for k in ("q0", "q1", "q2")]
    fixed = [g["kappa"], g["w"], g["t0"], g["t1"], g["t2"]]
    op = B.Stencil(S.climate())
    stream = torch.cuda.current_stream()
    launch_ms = []

    def step(timed_launches=False):
        nonlocal cur, nxt
        for k in range(sweeps):
            if timed_launches and k == sweeps // 2:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.do_all(op, cur + fixed, nxt)
                e1.record(stream)
                launch_ms.append((e0, e1))
            else:
                B.do_all(op, cur + fixed, nxt)
            cur, nxt = nxt, cur

    warm(step, warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step(True)
    e1.record(stream)
    torch.cuda.synchronize()
    B.sync()
    ms = e0.elapsed_time(e1) / steps
    lms = sum(a.elapsed_time(b) for a, b in launch_ms) / len(launch_ms)
    pts = n[0] * n[1] * n[2]
    return {"points": pts, "ms_per_step": ms, "launch_ms": lms, "sweeps": sweeps,
            "specialization": B.specialization(op, len(cur + fixed), len(nxt))}


# ------------------------------------------------------------------ ordered workload
def run_ordered(dtype, steps, warmup, n=(256, 256, 80), reps=10, interpreted=False, along_x=False):
    """Ordered iteration space (do_k_inc): bidiagonal forward substitution
    x(k) = g(k) - m(k) x(k-1) down every (i, j) column of a 256 x 256 x 80
    grid (g uniform [-1, 1), m uniform [-0.9, 0.9], seeds 606 / 607), `reps`
    solves per step.  Algorithmic bytes per point: g and m read, x written.
    `interpreted`: the runtime term loop instead of the compiled recurrence;
    `along_x`: the same recurrence along x (do_i_inc, rows of 256)."""
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I

    h = (1, 1, 1)
    g = B.Grid(n, h, dtype).upload(I.random_interior(606, n, h, -1.0, 1.0))
    m = B.Grid(n, h, dtype).upload(I.random_interior(607, n, h, -0.9, 0.9))
    x = B.Grid(n, h, dtype).upload(I.random_interior(608, n, h, 0.0, 0.0))
    order = B.I_INC if along_x else B.K_INC
    prev = (-1, 0, 0) if along_x else (0, 0, -1)
    terms = [(0, 0, 0, 1, B.NONE, 0, 1.0), (*prev, 0, 2, 0, -1.0)]
    op = B.Stencil(terms)
    stream = torch.cuda.current_stream()
    saved = os.environ.get("GSCL_GENERIC_ONLY")
    if interpreted:
        os.environ["GSCL_GENERIC_ONLY"] = "1"
    else:
        os.environ.pop("GSCL_GENERIC_ONLY", None)
    path = B.ordered_specialization(order, op, [x, g, m], [x])

    def step():
        for _ in range(reps):
            B.do_ordered(order, op, [x, g, m], [x])

    warm(step, warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    B.sync()
    if saved is None:
        os.environ.pop("GSCL_GENERIC_ONLY", None)
    else:
        os.environ["GSCL_GENERIC_ONLY"] = saved
    ms = e0.elapsed_time(e1) / steps
    pts = n[0] * n[1] * n[2]
    return {"points": pts, "ms_per_step": ms, "solve_ms": ms / reps, "reps": reps, "path": path}


# ------------------------------------------------------------------ red-black workload
def run_redblack(steps, warmup, n=256, iters=10, solve_n=128, solve=True):
    """Red-black SOR (Section 3's colouring) on the 3D Poisson problem
    6u - sum6 = f, zero Dirichlet halo, f uniform [-1, 1) (seed 707), u = 0,
    omega = 2 / (1 + sin(pi / (n + 1))).  (a) Device time of `iters`
    iterations (2 `iters` half-sweeps, in place) on n^3 FP64 per step.
    (b) With `solve`: time to relative L2 residual 1e-6 on solve_n^3 for
    red-black SOR and for Jacobi (u' = (sum6 + f) / 6, ping-pong), the
    residual checked every 20 iterations / 500 sweeps."""
    import numpy as np
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S

    h = (1, 1, 1)

    def problem(m):
        u = B.Grid((m,) * 3, h, "f64").upload(np.zeros(I.padded_shape((m,) * 3, h)))
        f = B.Grid((m,) * 3, h, "f64").upload(I.random_interior(707, (m,) * 3, h, -1.0, 1.0))
        return u, f

    omega = lambda m: 2.0 / (1.0 + math.sin(math.pi / (m + 1)))
    u, f = problem(n)
    op = B.Stencil(S.poisson_sor(omega(n)))
    stream = torch.cuda.current_stream()

    def timed(compact):
        saved = os.environ.get("GSCL_COLOR_COMPACT")
        os.environ["GSCL_COLOR_COMPACT"] = "1" if compact else "0"
        try:
            warm(lambda: B.do_colored(op, [u, f], [u], color=0, half_sweeps=2 * iters), warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                B.do_colored(op, [u, f], [u], color=0, half_sweeps=2 * iters)
            e1.record(stream)
            torch.cuda.synchronize()
        finally:
            if saved is None:
                os.environ.pop("GSCL_COLOR_COMPACT", None)
            else:
                os.environ["GSCL_COLOR_COMPACT"] = saved
        return e0.elapsed_time(e1) / steps

    ms = timed(True)
    out = {"points": n ** 3, "ms_per_step": ms, "iter_ms": ms / iters, "iters": iters}
    if not solve:
        return out
    out["uncompacted_iter_ms"] = timed(False) / iters
    # FP64 grids in FP32-pair arithmetic (opt-in precision mode)
    B.set_fp64_arithmetic("pair")
    try:
        out["pair_iter_ms"] = timed(True) / iters
    finally:
        B.set_fp64_arithmetic("ieee")
    resid = B.Stencil(S.residual7())

    def to_tol(kind):
        u, f = problem(solve_n)
        v = B.Grid((solve_n,) * 3, h, "f64").upload(np.zeros(I.padded_shape((solve_n,) * 3, h)))
        norm_f = B.do_reduce(B.L2, None, [f])
        sor = B.Stencil(S.poisson_sor(omega(solve_n)))
        jac = B.Stencil(S.poisson_jacobi())
        torch.cuda.synchronize()
        t = time.perf_counter()
        done, rel = 0, 1.0
        while rel > 1e-6 and done < 2_000_000:
            if kind == "rbsor":
                B.do_colored(sor, [u, f], [u], color=0, half_sweeps=40)
                done += 20
            else:
                B.do_all(jac, [u, f], [v], sweeps=500)
                u, v = v, u
                done += 500
            rel = B.do_reduce(B.L2, resid, [u, f]) / norm_f
        sec = time.perf_counter() - t
        return {"seconds": round(sec, 4), "iterations": done, "rel_residual": rel}

    out["solve"] = {"side": solve_n, "rbsor": to_tol("rbsor"), "jacobi": to_tol("jacobi")}
    out["solve"]["speedup_rbsor_vs_jacobi"] = round(out["solve"]["jacobi"]["seconds"]
                                                    / out["solve"]["rbsor"]["seconds"], 2)
    return out


# ------------------------------------------------------------------ run-time compiled operators
# (real) casts keep FP32 programs in FP32 arithmetic (a double literal would
# promote the expression to FP64, as C++ does)
HEAT_BODY = ("out0 = (real)0.25 * in0(0,0,0) + (real)0.125 * (in0(1,0,0) + in0(-1,0,0) + in0(0,1,0)"
             " + in0(0,-1,0) + in0(0,0,1) + in0(0,0,-1)) + (real)0.125 * in1(0,0,0);")


def run_program(dtype, steps, warmup, n=256, sweeps=20):
    """The heat sweep of the default workload (lam = 1/8) given as a body of
    CUDA C++ statements and compiled at run time (NVRTC), `sweeps` ping-pong
    sweeps per step on n^3, against the same sweeps through gscl_do_all's
    compiled operator table.  Returns per-sweep device times."""
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S

    h = (1, 1, 1)
    u0, f0 = I.heat3d(SEED, n)
    u, v, f = (B.Grid((n,) * 3, h, dtype).upload(a) for a in (u0, u0, f0))
    t = time.perf_counter()
    prog = B.Program(HEAT_BODY, 2, 1, dtype, (1, 1, 1))
    compile_s = time.perf_counter() - t
    op = B.Stencil(S.heat7(LAM))
    stream = torch.cuda.current_stream()
    out = {"compile_s": compile_s}
    for key, fn in (("program", lambda: prog.run([u, f], [v], sweeps=sweeps)),
                    ("table", lambda: B.do_all(op, [u, f], [v], sweeps=sweeps))):
        warm(fn, warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[key] = e0.elapsed_time(e1) / (steps * sweeps)
    B.sync()
    out["points"] = n ** 3
    return out


# ------------------------------------------------------------------ do_diamond workload
def run_diamond(steps, warmup, n=(512, 512, 64), single=(4096, 4096, 1)):
    """do_diamond (Section 3): one natural-order Gauss-Seidel sweep of the
    2D 5-point Poisson operator u = (u(i-1,j) + u(i,j-1) + u(i+1,j) + u(i,j+1)
    + f) / 4 in place, (a) on `n[2]` independent n[0] x n[1] FP64 planes
    (u uniform [-1, 1) seed 808, f seed 809, halo 0.5) and (b) on one
    4096^2 plane, where the wavefront leaves most of the GPU idle.
    Algorithmic bytes per point: u read and written, f read (24 B in FP64)."""
    import torch

    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I

    terms = [(1, 0, 0, 0, B.NONE, 0, 0.25), (-1, 0, 0, 0, B.NONE, 0, 0.25), (0, 1, 0, 0, B.NONE, 0, 0.25),
             (0, -1, 0, 0, B.NONE, 0, 0.25), (0, 0, 0, 1, B.NONE, 0, 0.25)]
    op = B.Stencil(terms)
    stream = torch.cuda.current_stream()
    out = {}
    for key, m in (("planes", n), ("single", single)):
        h = (1, 1, 1) if m[2] > 1 else (1, 1, 0)
        u = B.Grid(m, h, "f64").upload(I.random_interior(808, m, h, -1.0, 1.0, halo_value=0.5))
        f = B.Grid(m, h, "f64").upload(I.random_interior(809, m, h, -1.0, 1.0))
        warm(lambda: B.do_diamond(op, [u, f], [u]), warmup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            B.do_diamond(op, [u, f], [u])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        tiles = -(-m[0] // 32) + -(-m[1] // 32) - 1
        out[key] = {"shape": list(m), "points": m[0] * m[1] * m[2], "ms_per_sweep": ms, "launches": tiles}
    return out


# ------------------------------------------------------------------ serving workload
def run_serving(sample=8, window_s=10.0, rate=200.0, time_cap=30.0, check_every=200):
    """Poisson solves (side uniform on 64..256, f uniform in [-1, 1), stop at
    ||f - A u|| / ||f|| <= 1e-6).  (a) The first `sample` requests all
    arriving at t = 0, served by every solve mode: Jacobi with continuous
    batching in mixed precision and in FP64, FP64 Jacobi one request at a
    time, red-black SOR in FP64 and as the FP32 inner solver of the mixed
    refinement: solves/s and latency of each, and the speedups.  (b) The
    literal arrival process (Poisson, `rate` per second, seed 5050) over
    `window_s` seconds and (c) a load-scaled one at 70% of the measured
    capacity, both served by the fastest mode of (a), stopped after
    `time_cap` seconds: completed, backlog, p50/p99."""
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import serving as SV

    def reqs(k, arrivals=None):
        out = []
        for r in range(k):
            n, f = I.poisson_request(r)
            out.append(SV.Request(rid=r, n=n, f=f, arrival=0.0 if arrivals is None else arrivals[r]))
        return out

    closed = {}
    for mode in ("mixed", "fp64"):
        srv = SV.PoissonServer(mode=mode, check_every=check_every)
        closed[mode] = srv.run_trace(reqs(sample))
    # the plain FP64 per-request path: one request on the GPU at a time
    srv = SV.PoissonServer(mode="fp64", check_every=check_every, max_active=1)
    closed["fp64_per_request"] = srv.run_trace(reqs(sample))
    # red-black SOR (per-request launches): O(n) iterations instead of O(n^2),
    # in FP64 and as the FP32 inner solver of the mixed refinement
    for mode in ("rbsor", "mixed_rbsor"):
        srv = SV.PoissonServer(mode=mode)
        closed[mode] = srv.run_trace(reqs(sample))
    best = max(closed, key=lambda m: closed[m]["solves_per_s"])

    def traces(mode):
        # literal arrival rate: the offered load is far above capacity, so report the backlog
        arrivals = I.poisson_arrivals(rate, window_s)
        srv = SV.PoissonServer(mode=mode, check_every=check_every, max_active=32)
        trace = srv.run_trace(reqs(len(arrivals), arrivals), time_cap=time_cap)
        trace["rate_per_s"] = rate
        trace["window_s"] = window_s
        # load-scaled: arrivals at 70% of the measured capacity of that mode
        scaled_rate = 0.7 * closed[mode]["solves_per_s"]
        arr2 = I.poisson_arrivals(scaled_rate, 20.0)
        srv = SV.PoissonServer(mode=mode, check_every=check_every, max_active=32)
        scaled = srv.run_trace(reqs(len(arr2), arr2), time_cap=90.0)
        scaled["rate_per_s"] = scaled_rate
        scaled["window_s"] = 20.0
        return trace, scaled

    # the configured method (Jacobi sweeps in FP32 with the FP64 correction), and the fastest mode
    trace, scaled = traces("mixed")
    best_trace, best_scaled = traces(best) if best not in ("mixed", "fp64_per_request") else (None, None)
    sides = [I.poisson_request(r)[0] for r in range(sample)]
    return {"closed": closed, "trace": trace, "scaled": scaled, "sample_sides": sides, "best": best,
            "best_trace": best_trace, "best_scaled": best_scaled,
            "speedup_solves_per_s": closed["mixed"]["solves_per_s"] / max(closed["fp64"]["solves_per_s"], 1e-30),
            "speedup_vs_per_request": closed["mixed"]["solves_per_s"]
            / max(closed["fp64_per_request"]["solves_per_s"], 1e-30),
            "speedup_rbsor_vs_mixed": closed["rbsor"]["solves_per_s"] / max(closed["mixed"]["solves_per_s"], 1e-30),
            "speedup_mixed_rbsor_vs_mixed": closed["mixed_rbsor"]["solves_per_s"]
            / max(closed["mixed"]["solves_per_s"], 1e-30)}


# ------------------------------------------------------------------ CPU oracle
def host_cores():
    """Cores this process may run on (its affinity mask), and the machine's count."""
    try:
        avail = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        avail = os.cpu_count() or 1
    return avail, os.cpu_count() or avail


def oracle_sample(n=N_SIDE, sweeps=10, threads=0):
    """The FP64 oracle on a bounded sample: one fused sweep + residual and
    sweeps-1 plain sweeps of the same 256^3 workload.  threads = 0: the
    checker build (gcc -O2, one thread); threads >= 1: the timing build
    (-O3 -march=native -fopenmp, same results) on that many threads."""
    from oracle import drivers as D
    from oracle import oracle as O
    from paper_1207_1746_b300 import inputs as I

    h = (1, 1, 1)
    u0, f = I.heat3d(SEED, n)
    a, b, F = O.Grid(u0.copy(), h), O.Grid(u0.copy(), h), O.Grid(f, h)
    terms = D.heat_terms(LAM)
    used = 1
    try:
        if threads >= 1:
            O.use_library(O.build(timing=True))
            used = O.threads(threads)
        t = time.perf_counter()
        for s in range(sweeps):
            if s % EVERY == 0:
                O.do_reduce(O.L2, terms, [a, F], [b])
            else:
                O.do_all(terms, [a, F], [b])
            a, b = b, a
        sec = time.perf_counter() - t
    finally:
        if threads >= 1:
            O.use_library(None)
    return {"value": sweeps * n ** 3 / sec / 1e9, "sec": sec, "sweeps": sweeps, "threads": used}


def cpu_baseline_heat(n=N_SIDE):
    """The oracle timed on the host: the timing build on every available core
    (the line's value) and on one thread, and the checker build on one thread,
    each over one fused and nine plain sweeps of the 256^3 workload."""
    avail, total = host_cores()
    allc = oracle_sample(n, EVERY, threads=avail)
    one = oracle_sample(n, EVERY, threads=1)
    chk = oracle_sample(n, EVERY, threads=0)
    sample = f"{EVERY} sweeps (1 fused + {EVERY - 1} plain) of the 256^3 FP64 grid"
    return {"value": round(allc["value"], 6), "unit": "GPoint-updates/s", "cores": allc["threads"],
            "kind": "oracle", "sample": f"{sample}, {allc['sec']:.2f} s",
            "build": "gcc -O3 -march=native -fopenmp -ffp-contract=off (timing build: planes over threads, "
                     "same results as the checker)",
            "nproc": total, "cores_available": avail,
            "single_thread": {"value": round(one["value"], 6), "cores": 1, "sample": f"{sample}, {one['sec']:.2f} s"},
            "checker_single_thread": {"value": round(chk["value"], 6), "cores": 1,
                                      "build": "gcc -O2 -ffp-contract=off (the checker as it stands)",
                                      "sample": f"{sample}, {chk['sec']:.2f} s"}}


def run_error_vs_oracle(n=64, sweeps=SWEEPS):
    """Error after the step's sweeps against the FP64 oracle, per arithmetic:
    the heat step's recipe (seed, lambda, fused L2 residual every 10 sweeps)
    on an n^3 grid, the oracle run in FP64 from the same storage-rounded
    initial data.  ||g - o||_inf / ||o||_inf of the final grid, and the
    largest relative error of the residuals."""
    import numpy as np
    import torch

    from oracle import drivers as D
    from oracle import oracle as O
    from paper_1207_1746_b300 import binding as B
    from paper_1207_1746_b300 import inputs as I
    from paper_1207_1746_b300 import stencils as S

    h, shape = (1, 1, 1), (n, n, n)
    u0, f = I.heat3d(SEED, n)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
    fused, plain = B.Stencil(S.heat7_fused(LAM)), B.Stencil(S.heat7(LAM))
    oracle_runs = {}
    out = {"grid": f"{n}^3", "sweeps": sweeps, "residual_every": EVERY}
    avail, _ = host_cores()
    for name, dt, arith in (("f64", "f64", "ieee"), ("f64_pair", "f64", "pair"), ("f32", "f32", "ieee"),
                            ("bf16", "bf16", "ieee")):
        B.set_fp64_arithmetic(arith)
        try:
            u, v, F = B.Grid(shape, h, dt).upload(u0), B.Grid(shape, h, dt).upload(u0), B.Grid(shape, h, dt).upload(f)
            res = []
            for _ in range(sweeps // EVERY):
                res.append(B.do_reduce(B.L2, fused, [u, F], [v]))
                B.swap(u, v)
                B.do_all(plain, [u, F], [v], sweeps=EVERY - 1)
                B.swap(u, v)
            got = u.download().double().numpy()
        finally:
            B.set_fp64_arithmetic("ieee")
        if dt not in oracle_runs:
            def rnd(a):
                return torch.from_numpy(np.ascontiguousarray(a)).to(tdt[dt]).double().numpy()
            try:
                O.use_library(O.build(timing=True))  # the checker's numbers, on every core
                O.threads(avail)
                oracle_runs[dt] = D.heat_run(O.Grid(rnd(u0), h), O.Grid(rnd(f), h), LAM, sweeps, every=EVERY)
            finally:
                O.use_library(None)
        ou, ores = oracle_runs[dt]
        err = float(np.max(np.abs(got - ou.a)) / np.max(np.abs(ou.a)))
        rerr = max(abs(a - b) / b for a, b in zip(res, ores))
        out[name] = {"rel_inf_error": float(f"{err:.3e}"), "residual_max_rel_error": float(f"{rerr:.3e}")}
    return out


# ------------------------------------------------------------------ roofline
def roofline_fp64(plain_ms, points, peaks, sm_mhz, measured_tflops=None):
    """FP64 sweeps are bound by the FP64 pipe: the method's 8 multiply-adds
    (16 FLOP) per point are the algorithmic count.  `peak` is derived from
    unit counts and the maximum clock; the FMA microbenchmark's measured rate
    is reported beside it.  With equal neighbour weights the kernel sums the
    six neighbours as a tree and runs two of its additions on the integer
    pipe (exact IEEE additions): the FP64 pipe then executes 6 operations
    per point, and the algorithmic rate may exceed the FP64-pipe peak by up
    to 8/6."""
    flops = 2.0 * TERMS_PLAIN * points
    achieved = flops / (plain_ms * 1e-3) / 1e12
    peak = 148 * 2 * 2 * 2032e6 / 1e12  # SMs x DFMA/clk/SM x FLOP/FMA x max SM clock
    traffic = profile_traffic("f64_plain")
    int_add = os.environ.get("GSCL_FP64_INT_ADD", "1")[:1] != "0"
    fp64_ops = TERMS_PLAIN - 2 if int_add else TERMS_PLAIN
    extra = {"fp64_pipe_ops_per_point": fp64_ops,
             "fp64_pipe_frac": round(achieved * fp64_ops / TERMS_PLAIN / peak, 4)}
    if measured_tflops:
        extra.update({"peak_measured_fma": round(measured_tflops, 4),
                      "frac_of_measured_fma": round(achieved / measured_tflops, 4)})
    return {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, **extra,
            "peak_source": "derived: 148 SMs x 2 DFMA/clk/SM x 2 FLOP x 2032 MHz",
            "hbm_gbs": round(BYTES_PER_PT["f64"] * points / (plain_ms * 1e-3) / 1e9, 1),
            "hbm_frac_of_measured": round(BYTES_PER_PT["f64"] * points / (plain_ms * 1e-3) / 1e9
                                          / peaks.get("hbm_gbs", 6400.0), 4)}


def roofline_hbm(dtype, plain_ms, points, peaks):
    nbytes = BYTES_PER_PT[dtype] * points
    achieved = nbytes / (plain_ms * 1e-3) / 1e9
    peak = peaks.get("hbm_gbs")
    src = "measured" if peak else "fallback"
    peak = peak or 6400.0
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": profile_traffic(f"{dtype}_plain"),
            "peak_source": src}


def variant_roofline(dtype, plain_ms, temporal, points, peaks):
    """HBM roofline of the plain FP32 / BF16 sweeps: with K > 1 sweeps fused
    per pass (the tuner's factor) one launch does K sweeps and moves the
    bytes of one, so the launch time is K times the time per sweep."""
    K = temporal.get("tuned_factor", 1) if temporal else 1
    if K <= 1:
        r = roofline_hbm(dtype, plain_ms, points, peaks)
    else:
        r = roofline_hbm(dtype, temporal[f"k{K}_ms_per_sweep"] * K, points, peaks)
        r["traffic"] = None
        r["note"] = f"{K} sweeps per launch (temporal blocking): the bytes of one sweep per launch"
    grids_mb = 3 * points * {"f64": 8, "f32": 4, "bf16": 2}[dtype] / 1e6
    if grids_mb < 126:  # u, f and v fit in the 126 MB L2 together
        r["l2_note"] = (f"working set 3 x {grids_mb / 3:.1f} MB = {grids_mb:.1f} MB fits in the 126 MB L2: "
                        "consecutive sweeps partly hit L2 (DRAM traffic below the algorithmic bytes), so "
                        "frac bounds the sweep's HBM efficiency from above")
    return r


PROFILE = False  # --profile: short runs for profilers, without the FMA microbenchmark


def B_fma():
    """Measured FP64 FMA rate of this GPU in TFLOP/s (gscl_fma_throughput)."""
    if PROFILE:
        return float("nan")
    from paper_1207_1746_b300 import binding as B
    return B.fma_throughput("f64", 2048) / 1e12


# ------------------------------------------------------------------ main
class _Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as td
            td.init_process_group(backend)
            self.pg = td

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x):
        if self.pg is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gscl", choices=["gscl", "reference"])
    ap.add_argument("--n", "--side", dest="n", type=int, default=N_SIDE,
                    help="grid side of the heat workload (--side also works under torchrun)")
    ap.add_argument("--sweeps", type=int, default=SWEEPS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--batch-temporal", type=int, default=None,
                    help="batched workload: sweeps per launch to use instead of the tuner's (profiling runs)")
    ap.add_argument("--profile", action="store_true",
                    help="one short step for profilers: no warm-up, tuner, comparison runs, e2e, CPU leg or "
                         "FMA microbenchmark (the printed numbers are not benchmark values)")
    ap.add_argument("--workload", default="heat3d",
                    choices=["heat3d", "batched", "serving", "laplace2d", "climate", "ordered", "redblack",
                             "diamond", "program", "temporal"],
                    help="heat3d: the 256^3 heat solve (default line); batched: 96 uneven FP32 instances; "
                         "serving: Poisson solve requests; laplace2d: 256^2 FP64 Jacobi, 100 sweeps; "
                         "climate: 8 -> 3 grid operator on 256 x 256 x 80, FP64 and FP32, 50 sweeps; "
                         "ordered: do_k_inc bidiagonal solve down 256 x 256 columns of 80; "
                         "redblack: red-black SOR on the 256^3 FP64 Poisson problem; "
                         "diamond: natural-order Gauss-Seidel (do_diamond) on 64 planes of 512^2 FP64; "
                         "program: the 256^3 heat sweep as a run-time compiled body; "
                         "temporal: K = 1..4 sweeps per pass (temporal blocking) on the 256^3 heat sweep, FP32 / BF16")
    args = ap.parse_args()
    if args.profile:
        global PROFILE
        PROFILE = True
        args.steps, args.warmup, args.no_e2e, args.no_cpu = 1, 0, True, True
    if args.sweeps % EVERY:
        ap.error("--sweeps must be a multiple of 10")
    dist = _Dist()
    workload = (f"heat3d_7pt_{args.n}^3: 3D 7-point damped Jacobi/heat, {args.sweeps} sweeps, "
                f"ping-pong grids + RHS, lam=1/8, fused L2 residual every {EVERY} sweeps")
    config = {"workload": workload, "grid": [args.n] * 3, "halo": 1, "sweeps_per_step": args.sweeps,
              "residual_every": EVERY,
              "l2": "FP64 (the measured line) and FP32 variant: working set (3 grids) larger than the 126 MB "
                    "L2, no flush; BF16 variant: 3 x 33.5 MB fit in L2 (see its roofline's l2_note)",
              "parallelism": f"replicas{args.gpus}" if args.gpus > 1 else "single"}

    if args.impl == "reference":
        dist.init("gloo")
        if dist.rank != 0:
            return
        # a bounded sample per step: one fused and one plain sweep of the 256^3
        # grid, the oracle's timing build on every core this process may use
        avail, total = host_cores()
        t_all = []
        used = 1
        for i in range(args.warmup + args.steps):
            r = oracle_sample(args.n, 2, threads=avail)
            used = r["threads"]
            if i >= args.warmup:
                t_all.append(r["sec"])
        sec = sum(t_all) / len(t_all)
        value = 2 * args.n ** 3 / sec / 1e9
        line = {"impl": "reference", "metric": "GPoint-updates/s", "value": round(value, 6),
                "unit": "GPoint-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(sec * 1e3, 1), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "cpu_baseline": {"value": round(value, 6), "unit": "GPoint-updates/s", "cores": used, "kind": "oracle",
                                 "nproc": total,
                                 "build": "gcc -O3 -march=native -fopenmp -ffp-contract=off (timing build)",
                                 "sample": "per step: 1 fused + 1 plain sweep of the 256^3 grid (of 200)"},
                "e2e": {"value": round(value, 6), "unit": "GPoint-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    torch.cuda.set_device(dist.local)
    dist.init("nccl")
    peaks = measured_peaks()
    if args.workload == "serving":
        r = run_serving()
        best = r["best"]
        line = {"metric": "solves/s", "value": round(r["closed"]["mixed"]["solves_per_s"], 4), "unit": "solves/s",
                "n_gpus": args.gpus, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": "serving: 3D 7-point Poisson Jacobi solves, side U{64..256}, f U[-1,1), "
                                       "stop at relative L2 residual 1e-6 (FP64), FP32 sweeps + FP64 correction, "
                                       "continuous batching, HBM-budget admission", "mode": "mixed",
                           "sample_sides": r["sample_sides"]},
                "closed_sample": r["closed"], "poisson_trace_literal": r["trace"],
                "poisson_trace_load_scaled": r["scaled"],
                "fastest_mode": {"mode": best, "solves_per_s": round(r["closed"][best]["solves_per_s"], 4),
                                 "poisson_trace_literal": r["best_trace"],
                                 "poisson_trace_load_scaled": r["best_scaled"]},
                "speedup_mixed_vs_fp64": round(r["speedup_solves_per_s"], 3),
                "speedup_mixed_vs_fp64_per_request": round(r["speedup_vs_per_request"], 3),
                "speedup_rbsor_vs_mixed": round(r["speedup_rbsor_vs_mixed"], 3),
                "speedup_mixed_rbsor_vs_mixed": round(r["speedup_mixed_rbsor_vs_mixed"], 3)}
        if dist.rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "laplace2d":
        r = run_laplace2d(args.steps, args.warmup, compare=not args.profile)
        t = dist.max(r["ms_per_step"])
        upd = r["sweeps"] * r["points"]
        fma_tflops = B_fma()
        achieved = 2.0 * 4 * upd / (t * 1e-3) / 1e12  # 4 FMA-pipe operations per point
        line = {"metric": "GPoint-updates/s", "value": round(dist.world * upd / (t * 1e-3) / 1e9, 3),
                "unit": "GPoint-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(t, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": "laplace2d: 2D 5-point Jacobi, 256x256 FP64, halo sin(pi x), interior "
                                       "U[0,1) seed 101, 100 sweeps (ping-pong, one CUDA graph, tuned sweeps "
                                       "per launch) + max-abs residual |u_100 - u_99|", "grid": [256, 256],
                           "halo": 1, "l2": "L2-resident (2 x 0.5 MB): launch-bound, not HBM-bound"},
                "roofline": {"bound": "alu", "achieved": round(achieved, 5), "peak": round(fma_tflops, 4),
                             "unit": "TFLOP/s", "frac": round(achieved / fma_tflops, 5), "traffic": None,
                             "peak_source": "measured FP64 FMA rate (gscl_fma_throughput)",
                             "note": "algorithmic FLOPs (one evaluation per point and sweep; fused "
                                     "launches recompute frame points on top); the time includes launch gaps"},
                "sweeps_per_launch": r["sweeps_per_launch"], "temporal_tile": r["tile"],
                "ms_per_step_single_sweeps": round(r["ms_per_step_single_sweeps"], 4),
                "temporal_speedup": round(r["ms_per_step_single_sweeps"] / t, 3),
                "ms_per_step_no_graph": round(r["ms_per_step_no_graph"], 4),
                "graph_speedup": round(r["ms_per_step_no_graph"] / r["ms_per_step_single_sweeps"], 3),
                "residual_maxabs": r["residual"], "gpu_launches": args.steps * (r["launches_per_step"] + 1)}
        if dist.rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "climate":
        out = {}
        for dt in ("f64", "f32"):
            r = run_climate(dt, args.steps, args.warmup)
            t = dist.max(r["ms_per_step"])
            upd = r["sweeps"] * r["points"]
            bpp = {"f64": 88, "f32": 44}[dt]
            out[dt] = {"value": round(dist.world * upd / (t * 1e-3) / 1e9, 3), "ms_per_step": round(t, 3),
                       "launch_ms": round(r["launch_ms"], 4), "specialization": r["specialization"],
                       "hbm_gbs": round(bpp * r["points"] / (r["launch_ms"] * 1e-3) / 1e9, 1)}
        fma_tflops = B_fma()
        f64 = out["f64"]
        # FP64 pipe operations per point of the compile-time climate operator: per output 1 (q) + 13 + 1
        # (biharmonic run, times kappa) + 2 + 1 (advection run, times w) + 1 (tendency) = 19, x 3 outputs
        ops = 57
        ach = 2.0 * ops * 256 * 256 * 80 / (f64["launch_ms"] * 1e-3) / 1e12
        # with the group evaluation each biharmonic ring of four takes one
        # integer-pipe addition and the vertical pair one integer-pipe
        # difference: 4 fewer FP64-pipe operations per output
        pipe_ops = ops - 12 if os.environ.get("GSCL_FP64_INT_ADD", "1")[:1] != "0" else ops
        peak_hbm = measured_peaks().get("hbm_gbs", 6400.0)
        line = {"metric": "GPoint-updates/s", "value": f64["value"], "unit": "GPoint-updates/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": f64["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": "climate: 8 -> 3 grid operator (13-point biharmonic x kappa + centred "
                                       "vertical advection x w + tendency), 256x256x80, halo (2,2,1), smooth "
                                       "fields seed 303, 50 sweeps", "l2": "working set 11 grids > L2"},
                "roofline": {"bound": "alu", "achieved": round(ach, 4), "peak": round(fma_tflops, 4),
                             "unit": "TFLOP/s", "frac": round(ach / fma_tflops, 4), "traffic": profile_traffic("climate_f64"),
                             "peak_source": "measured FP64 FMA rate (gscl_fma_throughput); the operator's 57 "
                                            "operations per point counted as FMAs (algorithmic)",
                             "fp64_pipe_ops_per_point": pipe_ops,
                             "fp64_pipe_frac": round(ach * pipe_ops / ops / fma_tflops, 4)},
                "kernel_ms": f64["launch_ms"], "hbm_gbs": f64["hbm_gbs"],
                "variants": {"f32": {"dtype": "f32", "value": out["f32"]["value"],
                                     "ms_per_step": out["f32"]["ms_per_step"], "kernel_ms": out["f32"]["launch_ms"],
                                     "roofline": {"bound": "hbm", "achieved": out["f32"]["hbm_gbs"],
                                                  "peak": peak_hbm, "unit": "GB/s",
                                                  "frac": round(out["f32"]["hbm_gbs"] / peak_hbm, 4),
                                                  "traffic": profile_traffic("climate_f32"),
                                                  "peak_source": "measured"}}},
                "gpu_launches": 2 * args.steps * 50}
        if dist.rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "program":
        peak_hbm = peaks.get("hbm_gbs", 6400.0)
        fma = B_fma()
        res = {}
        for dt in ("f64", "f32"):
            r = run_program(dt, args.steps, args.warmup)
            t = dist.max(r["program"])
            if dt == "f64":   # 8 FMAs per point on the FP64 pipe
                ach = 2 * 8 * r["points"] / (t * 1e-3) / 1e12
                roof = {"bound": "alu", "achieved": round(ach, 4), "peak": fma, "unit": "TFLOP/s",
                        "frac": round(ach / fma, 4) if fma == fma else None, "traffic": None,
                        "peak_source": "measured FP64 FMA rate (gscl_fma_throughput)"}
            else:
                gbs = BYTES_PER_PT["f32"] * r["points"] / (t * 1e-3) / 1e9
                roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak_hbm, "unit": "GB/s",
                        "frac": round(gbs / peak_hbm, 4), "traffic": None, "peak_source": "measured"}
            res[dt] = {"value": round(dist.world * r["points"] / (t * 1e-3) / 1e9, 3), "sweep_ms": round(t, 4),
                       "table_sweep_ms": round(r["table"], 4), "program_vs_table": round(r["table"] / t, 3),
                       "compile_s": round(r["compile_s"], 3), "roofline": roof}
        line = {"metric": "GPoint-updates/s", "value": res["f64"]["value"], "unit": "GPoint-updates/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(res["f64"]["sweep_ms"] * 20, 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "program: the 256^3 7-point heat sweep (lam 1/8) as a body of CUDA C++ "
                                       "statements compiled at run time, 20 ping-pong sweeps per step",
                           "l2": "working set (3 grids) larger than the 126 MB L2, no flush"},
                "roofline": res["f64"]["roofline"], "f64": res["f64"], "variants": {"f32": res["f32"]},
                "gpu_launches": args.steps * 20}
        if dist.rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "diamond":
        r = run_diamond(args.steps, args.warmup)
        peak_hbm = peaks.get("hbm_gbs", 6400.0)
        res = {}
        for key, v in r.items():
            t = dist.max(v["ms_per_sweep"])
            gbs = 24 * v["points"] / (t * 1e-3) / 1e9
            res[key] = {"shape": v["shape"], "value": round(dist.world * v["points"] / (t * 1e-3) / 1e9, 3),
                        "ms_per_sweep": round(t, 4), "launches_per_sweep": v["launches"],
                        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak_hbm, "unit": "GB/s",
                                     "frac": round(gbs / peak_hbm, 4), "traffic": None, "peak_source": "measured"}}
        line = {"metric": "GPoint-updates/s", "value": res["planes"]["value"], "unit": "GPoint-updates/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": res["planes"]["ms_per_sweep"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "diamond: natural-order Gauss-Seidel sweep (do_diamond, 5-point, in place) "
                                       "on 64 independent 512x512 FP64 planes; one sweep per step",
                           "l2": "working set 2 x 134 MB larger than the 126 MB L2, no flush"},
                "roofline": res["planes"]["roofline"], "variants": {"single_4096": res["single"]},
                "gpu_launches": args.steps * r["planes"]["launches"]}
        # the FP64 pipe: five DFMAs per point, one chain per element
        fma = B_fma() if not args.profile else None
        if fma:
            g_ops = 5 * r["planes"]["points"] / (res["planes"]["ms_per_sweep"] * 1e-3) / 1e9
            peak_ops = fma * 1e3 / 2
            line["fp64_pipe"] = {"achieved_g_dfma": round(g_ops, 1), "peak_g_dfma_measured": round(peak_ops, 1),
                                 "frac": round(g_ops / peak_ops, 4)}
        if dist.rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "redblack":
        r = run_redblack(args.steps, args.warmup, solve=not args.profile)
        t = dist.max(r["iter_ms"])
        pts = r["points"]
        fma = B_fma()
        # a colour-compacted half-sweep evaluates the 8-FMA operator at the
        # elements of its colour: 8 operations per point and iteration (the
        # algorithmic count); with equal neighbour weights two of them are
        # additions on the integer pipe, so the FP64 pipe executes 6
        g_ops = 8 * pts / (t * 1e-3) / 1e9
        fp64_ops = 6 if os.environ.get("GSCL_FP64_INT_ADD", "1")[:1] != "0" else 8
        gbs = 32 * pts / (t * 1e-3) / 1e9   # per half-sweep: u read, f and u' at half the points
        line = {"metric": "GPoint-updates/s", "value": round(dist.world * pts / (t * 1e-3) / 1e9, 3),
                "unit": "GPoint-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(dist.max(r["ms_per_step"]), 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "redblack: red-black SOR (optimal omega) on the 256^3 FP64 Poisson problem, "
                                       "in place, 10 iterations (20 half-sweeps) per step; a point update is one "
                                       "element of one iteration",
                           "l2": "working set (2 grids, 268 MB) larger than the 126 MB L2, no flush"},
                "iteration_ms": round(t, 4),
                "roofline": {"bound": "alu", "achieved": round(g_ops * 2 / 1e3, 4), "peak": fma, "unit": "TFLOP/s",
                             "frac": round(g_ops * 2 / 1e3 / fma, 4) if fma == fma else None,
                             "traffic": (2 * profile_traffic("redblack_half_sweep")
                                         if profile_traffic("redblack_half_sweep") else None),
                             "traffic_note": "DRAM bytes per iteration: two half-sweeps of the ncu capture",
                             "peak_source": "measured FP64 FMA rate (gscl_fma_throughput); 8 FMAs per point "
                                            "and iteration (each colour evaluated once)",
                             "fp64_pipe_ops_per_point": fp64_ops,
                             "fp64_pipe_frac": (round(g_ops * fp64_ops / 8 * 2 / 1e3 / fma, 4)
                                                if fma == fma else None),
                             "hbm_gbs": round(gbs, 1)},
                "uncompacted_iteration_ms": round(r["uncompacted_iter_ms"], 4) if "uncompacted_iter_ms" in r else None,
                "pair_arithmetic_iteration_ms": round(r["pair_iter_ms"], 4) if "pair_iter_ms" in r else None,
                "time_to_solution": r.get("solve"), "gpu_launches": args.steps * 2 * r["iters"]}
        if dist.rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "ordered":
        peak_hbm = peaks.get("hbm_gbs", 6400.0)
        out = {}
        runs = [("f64", False, False), ("f32", False, False)]
        if not args.profile:
            runs += [("f64", True, False), ("f32", True, False)]
        runs += [("f64", False, True), ("f32", False, True)]
        for dt, interp, along_x in runs:
            r = run_ordered(dt, args.steps, args.warmup, interpreted=interp, along_x=along_x)
            t = dist.max(r["ms_per_step"])
            bpp = {"f64": 24, "f32": 12}[dt]
            gbs = bpp * r["points"] / (r["solve_ms"] * 1e-3) / 1e9
            out[dt + ("_interpreted" if interp else "") + ("_along_x" if along_x else "")] = {
                "value": round(dist.world * r["reps"] * r["points"] / (t * 1e-3) / 1e9, 3),
                "ms_per_step": round(t, 3), "solve_ms": round(r["solve_ms"], 4), "path": r["path"],
                "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak_hbm, "unit": "GB/s",
                             "frac": round(gbs / peak_hbm, 4),
                             "traffic": profile_traffic("ordered_f64") if (dt, interp, along_x) == ("f64", False, False)
                             else None,
                             "peak_source": "measured"}}
        # FP64: three FP64-pipe instructions per point (DFMA a g, DMUL m x(k-1),
        # DFMA of the sum), each taking the pipe as long as one DFMA
        fma = B_fma() if not args.profile else None
        if fma:
            f64 = out["f64"]
            g_ops = 3 * r["points"] / (f64["solve_ms"] * 1e-3) / 1e9
            peak_ops = fma * 1e3 / 2          # measured FMA rate in G DFMA/s
            f64["fp64_pipe"] = {"achieved_g_ops": round(g_ops, 1), "peak_g_dfma_measured": round(peak_ops, 1),
                                "frac": round(g_ops / peak_ops, 4)}
        line = {"metric": "GPoint-updates/s", "value": out["f64"]["value"], "unit": "GPoint-updates/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": out["f64"]["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "ordered: do_k_inc bidiagonal forward substitution x(k) = g(k) - m(k) x(k-1) "
                                       "down every column of 256x256x80, 10 solves per step",
                           "l2": "working set 3 grids > L2 in FP64"},
                "roofline": out["f64"]["roofline"], "kernel_ms": out["f64"]["solve_ms"],
                "fp64_pipe": out["f64"].get("fp64_pipe"), "path": out["f64"]["path"],
                "variants": {k: {"dtype": k.split("_")[0], **v} for k, v in out.items() if k != "f64"},
                "gpu_launches": args.steps * 10}
        if dist.rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "temporal":
        t = {dt: run_temporal(dt, args.n, reps=1 if args.profile else 5) for dt in ("f32", "bf16")}
        k1 = dist.max(t["f32"]["k1_ms_per_sweep"])
        best = min((t["f32"][f"k{K}_ms_per_sweep"], K) for K in (1, 2, 3, 4))
        line = {"metric": "GPoint-updates/s", "value": round(dist.world * args.n ** 3 / (best[0] * 1e-3) / 1e9, 3),
                "unit": "GPoint-updates/s", "n_gpus": args.gpus, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"temporal blocking: plain 3D 7-point heat sweep (lam = 1/8, RHS), "
                                       f"{args.n}^3, 13 sweeps per gscl_do_all call (12 fused, the last single), K sweeps per pass over HBM",
                           "grid": [args.n] * 3},
                "roofline": roofline_hbm("f32", best[0] * best[1], args.n ** 3, peaks) if best[1] == 1 else
                variant_roofline("f32", k1, {"tuned_factor": best[1], **t["f32"]}, args.n ** 3, peaks),
                "best_factor": best[1], "f32": t["f32"], "bf16": t["bf16"],
                "gpu_launches": 5 * 8}
        if dist.rank == 0:
            print(json.dumps(line))
        return
    if args.workload == "batched":
        r = run_batched(args.steps, args.warmup, tune=not args.profile, compare=not args.profile,
                        fixed_temporal=args.batch_temporal)
        t = dist.max(r["ms_per_step"])
        line = {"metric": "GPoint-updates/s", "value": round(dist.world * 100 * r["points"] / (t * 1e-3) / 1e9, 3),
                "unit": "GPoint-updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(t, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batched heat3d: 96 instances, sides U{32..224} per axis (seed 4040), "
                                       "FP32, zero halo, lam=1/8, 100 sweeps per step, the tuner's sweeps per "
                                       "launch (1, or 2 in two-sweep passes), CUDA graph",
                           "points": r["points"], "sides": r["sides_min_max"],
                           "l2": "working set 2 x %.2f GB > L2" % (4 * r["points"] / 1e9)},
                "roofline": {"bound": "hbm", "achieved": round(r["hbm_gbs"], 1), "peak": peaks.get("hbm_gbs", 6400.0),
                             "unit": "GB/s", "frac": round(r["hbm_gbs"] / peaks.get("hbm_gbs", 6400.0), 4),
                             "traffic": profile_traffic("batched_sweep" if r["temporal"][0] == 1 else
                                                        f"batched_pass{r['temporal'][0]}"),
                             "note": "algorithmic bytes: 8 B per point-update, the updates of one launch "
                                     f"({r['temporal'][0]} sweep(s)) over its duration ({r['launch_ms']:.4f} ms)"},
                "per_instance_loop_ms": round(r["per_instance_loop_ms"], 3),
                "speedup_vs_per_instance_loop": round(r["speedup_vs_loop"], 3),
                "tuned_warps_prefetch": r["tuned"], "tile": r["tile"], "batch": r["info"],
                "tuned_sweeps_per_launch": r["temporal"][0], "single_sweep_ms": round(r["sweep_ms"], 4),
                "gpu_launches": args.steps * r["launches"]}
        if dist.rank == 0:
            print(json.dumps(line))
        return
    gpu_uuid = torch.cuda.get_device_properties(dist.local).uuid
    sampler = ClockSampler(f"GPU-{gpu_uuid}")
    main_run = run_gpu("f64", args.steps, args.warmup, dist, args.n, args.sweeps, clocks=sampler)
    t_max = dist.max(main_run["ms_total"])
    updates = dist.world * args.steps * args.sweeps * args.n ** 3
    value = updates / (t_max * 1e-3) / 1e9
    clocks = sampler.summary()
    fma_tflops = B_fma()
    roof = roofline_fp64(main_run["plain_launch_ms"], args.n ** 3, peaks, clocks.get("sm_mhz"), fma_tflops)

    variants = {}
    temporal = {}
    if not args.no_variants:
        # FP64 storage in pair arithmetic (FP32 pairs off the FP64 pipe; within the
        # FP64 tolerance, 2^-47 instead of 2^-53 per operation)
        from paper_1207_1746_b300 import binding as B
        B.set_fp64_arithmetic("pair")
        try:
            rp = run_gpu("f64", args.steps, args.warmup, dist, args.n, args.sweeps)
        finally:
            B.set_fp64_arithmetic("ieee")
        tp = dist.max(rp["ms_total"])
        rl = roofline_hbm("f64", rp["plain_launch_ms"], args.n ** 3, peaks)
        rl["traffic"] = None
        rl["note"] = "issue-bound on the FP32 / integer pipes (the FP64-pipe bound of IEEE FP64 is lifted)"
        variants["f64_pair"] = {
            "dtype": "f64 storage, FP32-pair arithmetic", "value": round(updates / (tp * 1e-3) / 1e9, 3),
            "unit": "GPoint-updates/s", "ms_per_step": round(tp / args.steps, 3), "roofline": rl,
            "fused_launch_ms": round(rp["fused_launch_ms"], 4), "plain_launch_ms": round(rp["plain_launch_ms"], 4),
            "final_residual": rp["residuals"][-1],
            "speedup_vs_ieee_fp64": round(t_max / tp, 3)}
        # FP32 storage, and BF16 storage (FP32 arithmetic; a smoothing-grade precision),
        # with the temporal factor the tuner picks for the plain sweeps
        for vdt in ("f32", "bf16"):
            temporal[vdt] = run_temporal(vdt, args.n)
            rv = run_gpu(vdt, args.steps, args.warmup, dist, args.n, args.sweeps)
            tv = dist.max(rv["ms_total"])
            variants[vdt] = {
                "dtype": vdt, "value": round(updates / (tv * 1e-3) / 1e9, 3), "unit": "GPoint-updates/s",
                "ms_per_step": round(tv / args.steps, 3),
                "roofline": variant_roofline(vdt, rv["plain_launch_ms"], temporal[vdt], args.n ** 3, peaks),
                "fused_launch_ms": round(rv["fused_launch_ms"], 4), "plain_launch_ms": round(rv["plain_launch_ms"], 4),
                "temporal_factor": temporal[vdt]["tuned_factor"], "final_residual": rv["residuals"][-1]}

    e2e = None
    if not args.no_e2e:
        e = run_e2e("f64", max(3, args.steps), 1, args.n, args.sweeps)
        e_ms = dist.max(e["ms_per_step"])
        e2e = {"value": round(dist.world * args.sweeps * args.n ** 3 / (e_ms * 1e-3) / 1e9, 3),
               "unit": "GPoint-updates/s", "h2d_bytes_per_step": e["h2d"], "d2h_bytes_per_step": e["d2h"],
               "ms_per_step": round(e_ms, 3), "steps": max(3, args.steps), "pipelined": e["pipelined"]}

    # Section 5.2's fused vs two-pass comparison (outside the timed region)
    ablation = None
    if not args.profile:
        ablation = {dt: run_fusion_ablation(dt, n=args.n) for dt in ("f64", "f32")}

    cpu = None
    if dist.rank == 0 and not args.no_cpu:
        cpu = cpu_baseline_heat(args.n)

    # error after the step's sweeps against the FP64 oracle, every arithmetic (64^3, outside the timed region)
    errors = None
    if dist.rank == 0 and not args.profile and not args.no_cpu:
        errors = run_error_vs_oracle()

    if dist.rank == 0:
        line = {"metric": "GPoint-updates/s", "value": round(value, 3), "unit": "GPoint-updates/s",
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(t_max / args.steps, 3), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "roofline": roof, "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e,
                "gpu_launches": main_run["launches"],
                "kernel_ms": {"plain_sweep": round(main_run["plain_launch_ms"], 4),
                              "fused_sweep_l2": round(main_run["fused_launch_ms"], 4)},
                "final_residual": main_run["residuals"][-1], "variants": variants,
                "fusion_ablation": ablation, "error_vs_oracle": errors, "temporal_blocking": temporal}
        print(json.dumps(line))


if __name__ == "__main__":
    main()
