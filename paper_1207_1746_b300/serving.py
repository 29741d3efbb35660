"""Continuous-batching server for 3D Poisson solves (-Laplace(u) = f, zero
Dirichlet halo) by Jacobi iteration, stopped per request at
||f - A u||_2 / ||f||_2 <= tol with A u = 6u - sum6(u).

Requests arrive over time; each tick the scheduler admits waiting requests
(first come, first served) while the HBM budget and the slot limit allow,
advances every active request by `check_every` sweeps in one batched launch
per sweep (a CUDA graph replays the group), measures each request's residual
with one batched FP64-accumulated reduction, and retires the converged ones,
recording their latency.  A request whose grids alone exceed the budget is
rejected at admission.  All arithmetic runs in the library's kernels; this
module only schedules.

Solve modes:
  "fp64"  - plain FP64 Jacobi: u' = (sum6(u) + f) / 6, the residual fused
            into the sweep that reads u every `check_every` sweeps.
  "mixed" - mixed-precision iterative refinement: u is kept in FP64; each
            outer step hands r = f - A u (FP64, cast to FP32) to FP32 Jacobi
            sweeps on A d = r until ||r - A d|| <= inner_tol ||r||, then
            u += d in FP64 and the FP64 residual decides convergence.
  "rbsor" - red-black SOR in FP64 (the colouring of Section 3's stateful
            stencils), in place on u, with the factor that is optimal for the
            n^3 Dirichlet problem, 2 / (1 + sin(pi / (n + 1))): O(n) iterations
            where Jacobi takes O(n^2).  Every half-sweep of all active
            requests is one launch of a coloured batch, each request with its
            own factor; the residual is measured every `sor_check_every`
            iterations.
  "mixed_rbsor" - the refinement of "mixed" with red-black SOR in FP32 as
            the inner solver: r = f - A u in FP64, FP32 SOR on A d = r until
            ||r - A d|| <= inner_tol ||r||, u += d in FP64.
Each request follows the same sequence of operations whatever else is
active, so its result does not depend on the mix (batched sweeps are
bit-identical to single-grid ones; batched norms agree to rounding).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import binding as B
from . import stencils as S

H = (1, 1, 1)
VALUE, NONE = B.VALUE, B.NONE


def residual_out_terms():
    """Value r = sum6(u) - 6u + f written to the output as well (inputs u, f)."""
    return S.residual7() + [(0, 0, 0, VALUE, NONE, 0, 1.0)]


@dataclass
class Request:
    rid: int
    n: int
    f: np.ndarray              # dense host array with halo (float64)
    arrival: float = 0.0       # seconds after the start of the trace
    t_admit: float = math.nan
    t_done: float = math.nan
    sweeps: int = 0
    outer: int = 0
    rel_residual: float = math.nan
    u: np.ndarray | None = None  # final FP64 solution (when kept)
    admit_tick: int = -1         # scheduler tick that admitted the request
    done_tick: int = -1          # tick that retired it
    rejected: bool = False       # needs more HBM than the whole budget


@dataclass
class _Slot:
    req: Request
    grids: dict
    phase_sweeps: int = 0
    norm_f: float = 0.0
    norm_r: float = 0.0
    bytes: int = 0
    done: bool = False


def _grid_bytes(n, dtype):
    return B.layout((n, n, n), H, dtype)[2]


def request_bytes(n, mode):
    if mode == "rbsor":
        return 2 * _grid_bytes(n, "f64")
    if mode == "mixed_rbsor":
        return 3 * _grid_bytes(n, "f64") + 2 * _grid_bytes(n, "f32")
    if mode == "fp64":
        return 3 * _grid_bytes(n, "f64")
    return 3 * _grid_bytes(n, "f64") + 3 * _grid_bytes(n, "f32")


class PoissonServer:
    def __init__(self, mode="mixed", hbm_budget=64 << 30, max_active=256, check_every=200, tol=1e-6,
                 inner_tol=1e-3, max_sweeps=2_000_000, keep_solution=False, use_graph=True, sor_check_every=20):
        if mode not in ("mixed", "fp64", "rbsor", "mixed_rbsor"):
            raise ValueError("mode is 'mixed', 'fp64', 'rbsor' or 'mixed_rbsor'")
        self.mode = mode
        self.sor_check_every = sor_check_every
        self.budget = hbm_budget
        self.max_active = max_active
        self.check_every = check_every
        self.tol = tol
        self.inner_tol = inner_tol
        self.max_sweeps = max_sweeps
        self.keep = keep_solution
        self.use_graph = use_graph
        self.waiting: list[Request] = []
        self.active: list[_Slot] = []
        self.done: list[Request] = []
        self.rejected: list[Request] = []
        self.in_use = 0
        self.ticks = 0
        self.t0 = time.perf_counter()
        self._batches = {}
        self.fused64 = B.Stencil(S.heat7_fused(1.0 / 6.0))   # u' = u + r/6 with r returned
        self.jacobi32 = B.Stencil(S.poisson_jacobi())         # d' = (sum6 d + r) / 6
        self.resid = B.Stencil(S.residual7())                 # value r - A d
        self.resid_out = B.Stencil(residual_out_terms())      # r64 = f - A u, written and returned
        self._sor = {}                                        # SOR operator per grid side

    # ------------------------------------------------------------ bookkeeping
    def now(self):
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.waiting.append(req)

    def _admit(self):
        while self.waiting and len(self.active) < self.max_active:
            req = self.waiting[0]
            need = request_bytes(req.n, self.mode)
            if need > self.budget:  # could never run: reject instead of blocking the queue
                self.waiting.pop(0)
                req.rejected = True
                self.rejected.append(req)
                continue
            if self.in_use + need > self.budget:
                break
            self.waiting.pop(0)
            req.admit_tick = self.ticks
            self.active.append(self._start(req, need))
            self.in_use += need

    def _start(self, req, need):
        n = (req.n,) * 3
        req.t_admit = self.now()
        # the right-hand side is the request's payload (one host copy); every
        # other grid starts at zero, halo included, set on the device
        g = {"f": B.Grid(n, H, "f64").upload(req.f)}
        zeros = {"rbsor": [("u", "f64")],
                 "mixed_rbsor": [("u", "f64"), ("r", "f64"), ("da", "f32"), ("r32", "f32")],
                 "fp64": [("u", "f64"), ("v", "f64")],
                 "mixed": [("u", "f64"), ("r", "f64"), ("da", "f32"), ("db", "f32"), ("r32", "f32")]}[self.mode]
        for name, dtype in zeros:
            g[name] = B.Grid(n, H, dtype).zero()
        slot = _Slot(req=req, grids=g, bytes=need)
        slot.norm_f = B.do_reduce(B.L2, None, [g["f"]])
        if self.mode in ("mixed", "mixed_rbsor"):
            self._outer_start(slot, first=True)
        return slot

    def _outer_start(self, slot, first=False):
        """r = f - A u in FP64 (with its norm); converged or hand r to the FP32 solve."""
        g = slot.grids
        if first:
            slot.norm_r = slot.norm_f
            B.convert(g["r32"], g["f"])
        else:
            B.convert(g["u"], g["da"], accumulate=True)          # u += d
            slot.norm_r = B.do_reduce(B.L2, self.resid_out, [g["u"], g["f"]], [g["r"]])
            slot.req.outer += 1
            if slot.norm_r <= self.tol * slot.norm_f:
                self._finish(slot, slot.norm_r / slot.norm_f)
                return
            B.convert(g["r32"], g["r"])
        B.convert(g["da"], g["da"], alpha=0.0)                   # d = 0
        slot.phase_sweeps = 0

    def _finish(self, slot, rel):
        req = slot.req
        req.rel_residual = rel
        if self.keep:
            req.u = slot.grids["u"].download().numpy()
        req.t_done = self.now()
        req.done_tick = self.ticks
        slot.done = True

    # ------------------------------------------------------------ one tick
    def _batch(self, key, op, instances):
        handles = tuple(g.handle for ins, outs in instances for g in ins + outs)
        b = self._batches.get((key, handles))
        if b is None:
            if len(self._batches) > 64:
                self._batches.clear()
            b = B.Batch(op, instances)
            self._batches[(key, handles)] = b
        return b

    def _colored_batch(self, key, x, rhs):
        """Coloured batch of the active requests' SOR sweeps on grids x (in place)
        with right-hand sides rhs, each request with its own factor."""
        ops = [self.sor_operator(s.req.n) for s in self.active]
        insts = [([s.grids[x], s.grids[rhs]], [s.grids[x]]) for s in self.active]
        handles = tuple(g.handle for ins, outs in insts for g in ins + outs)
        b = self._batches.get((key, handles))
        if b is None:
            if len(self._batches) > 64:
                self._batches.clear()
            b = B.ColoredBatch(ops, insts)
            self._batches[(key, handles)] = b
        return b

    def sor_operator(self, n):
        op = self._sor.get(n)
        if op is None:
            omega = 2.0 / (1.0 + math.sin(math.pi / (n + 1)))
            op = self._sor[n] = B.Stencil(S.poisson_sor(omega))
        return op

    def tick(self):
        self._admit()
        if not self.active:
            return False
        self.ticks += 1
        k = self.check_every
        res = torch.zeros(len(self.active), dtype=torch.float64, device="cuda")
        if self.mode == "rbsor":
            k = self.sor_check_every
            # 2k half-sweeps of every active request, one launch each, then
            # every request's residual in one batched reduction
            self._colored_batch("sor64", "u", "f").run_colored(0, 2 * k, graph=self.use_graph)
            rinsts = [([s.grids["u"], s.grids["f"]], []) for s in self.active]
            self._batch("resid64", self.resid, rinsts).reduce(B.L2, res)
            r = res.cpu().numpy()
            for s, rv in zip(self.active, r):
                s.req.sweeps += k
                rel = rv / s.norm_f
                if rel <= self.tol or s.req.sweeps >= self.max_sweeps:
                    self._finish(s, rel)
        elif self.mode == "mixed_rbsor":
            k = self.sor_check_every
            self._colored_batch("sor32", "da", "r32").run_colored(0, 2 * k, graph=self.use_graph)
            rinsts = [([s.grids["da"], s.grids["r32"]], []) for s in self.active]
            self._batch("resid32", self.resid, rinsts).reduce(B.L2, res)
            r = res.cpu().numpy()
            for s, rv in zip(self.active, r):
                s.req.sweeps += k
                s.phase_sweeps += k
                if rv <= self.inner_tol * s.norm_r or s.req.sweeps >= self.max_sweeps:
                    self._outer_start(s)
                    if not s.done and s.req.sweeps >= self.max_sweeps:
                        self._finish(s, s.norm_r / s.norm_f)
        elif self.mode == "fp64":
            # k - 1 plain sweeps, then the fused sweep that returns the residual of the iterate it reads
            insts = [([s.grids["u"], s.grids["f"]], [s.grids["v"]]) for s in self.active]
            if k > 1:
                self._batch("sweep64", S.poisson_jacobi(), insts).run(k - 1, graph=self.use_graph)
                for s in self.active:
                    B.swap(s.grids["u"], s.grids["v"])
            self._batch("fused64", self.fused64, insts).reduce(B.L2, res)
            for s in self.active:
                B.swap(s.grids["u"], s.grids["v"])
            r = res.cpu().numpy()
            for s, rv in zip(self.active, r):
                s.req.sweeps += k
                rel = rv / s.norm_f   # residual of the iterate one sweep before the latest
                if rel <= self.tol or s.req.sweeps >= self.max_sweeps:
                    self._finish(s, rel)
        else:
            insts = [([s.grids["da"], s.grids["r32"]], [s.grids["db"]]) for s in self.active]
            self._batch("sweep32", self.jacobi32, insts).run(k, graph=self.use_graph)
            for s in self.active:
                B.swap(s.grids["da"], s.grids["db"])
            rinsts = [([s.grids["da"], s.grids["r32"]], []) for s in self.active]
            self._batch("resid32", self.resid, rinsts).reduce(B.L2, res)
            r = res.cpu().numpy()
            for s, rv in zip(self.active, r):
                s.req.sweeps += k
                s.phase_sweeps += k
                if rv <= self.inner_tol * s.norm_r or s.req.sweeps >= self.max_sweeps:
                    self._outer_start(s)
                    if not s.done and s.req.sweeps >= self.max_sweeps:
                        self._finish(s, s.norm_r / s.norm_f)
        keep = []
        for s in self.active:
            if s.done:
                self.done.append(s.req)
                self.in_use -= s.bytes
            else:
                keep.append(s)
        self.active = keep
        return True

    # ------------------------------------------------------------ traces
    def run_trace(self, requests, time_cap=None):
        """Serves requests whose .arrival times are seconds after the start;
        returns when all are done or time_cap seconds have passed."""
        pending = sorted(requests, key=lambda r: r.arrival)
        self.t0 = time.perf_counter()
        i = 0
        while True:
            t = self.now()
            while i < len(pending) and pending[i].arrival <= t:
                self.submit(pending[i])
                i += 1
            if time_cap is not None and t > time_cap:
                break
            if not self.tick():
                if i >= len(pending):
                    break
                time.sleep(max(0.0, min(0.01, pending[i].arrival - t)))
        return self.stats(len(pending))

    def stats(self, offered):
        lat = sorted(r.t_done - r.arrival for r in self.done)
        elapsed = self.now()

        def pct(p):
            if not lat:
                return None
            return lat[min(len(lat) - 1, int(math.ceil(p / 100.0 * len(lat))) - 1)]

        return {"mode": self.mode, "offered": offered, "completed": len(self.done),
                "rejected": len(self.rejected),
                "backlog": offered - len(self.done) - len(self.rejected), "active_at_end": len(self.active),
                "elapsed_s": elapsed, "solves_per_s": len(self.done) / elapsed if elapsed > 0 else 0.0,
                "p50_s": pct(50), "p99_s": pct(99),
                "max_rel_residual": max((r.rel_residual for r in self.done), default=None),
                "sweeps": sum(r.sweeps for r in self.done)}
