"""Shared helpers of the GPU parity tests: run one operator through the C ABI
and through the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

from oracle import oracle as O
from paper_1207_1746_b300 import binding as B

TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
TOL = {"f64": 1e-13, "f32": 2e-6}


def as_storage(a, dtype):
    """The host array rounded to the storage dtype, widened back to float64."""
    return torch.from_numpy(np.ascontiguousarray(a)).to(TORCH[dtype]).double().numpy()


def run_pair(terms, in_arrays, in_halos, n, out_halos, dtype, rng=None, reduce_op=None):
    """Runs the operator on the GPU and in the oracle.

    Returns (gpu_outs, oracle_outs, gpu_value, oracle_value, abs_stencil_outs):
    dense float64 arrays with halo; output halos and points outside the
    range start as NaN on both sides."""
    ndim = 2 if (n[2] == 1 and all(h[2] == 0 for h in list(in_halos) + list(out_halos))) else 3
    ins = [B.Grid(n, h, dtype, ndim).upload(a) for a, h in zip(in_arrays, in_halos)]
    outs = []
    for h in out_halos:
        g = B.Grid(n, h, dtype, ndim)
        g.upload(np.full(g.padded_shape, np.nan))
        outs.append(g)
    gval = None
    if reduce_op is None:
        B.do_all(terms, ins, outs, rng=rng)
    else:
        gval = B.do_reduce(reduce_op, terms, ins, outs, rng=rng)
    B.sync()
    got = [o.download().double().numpy() for o in outs]

    oin = [O.Grid(as_storage(a, dtype), tuple(h)) for a, h in zip(in_arrays, in_halos)]
    oout = [O.Grid(np.full(g.padded_shape, np.nan), tuple(h)) for g, h in zip(outs, out_halos)]
    sout = [O.Grid(np.full(g.padded_shape, np.nan), tuple(h)) for g, h in zip(outs, out_halos)]
    lo, hi = (rng if rng is not None else (None, None))
    oval = None
    if reduce_op is None:
        O.do_all(terms, oin, oout, lo=lo, hi=hi)
    else:
        oval = O.do_reduce(reduce_op, terms if terms is not None else [], oin, oout, lo=lo, hi=hi)
    if terms:
        O.do_all(terms, oin, sout, lo=lo, hi=hi, abs_mode=True)
    return got, [g.a for g in oout], gval, oval, [g.a for g in sout]


def assert_within(got, ref, S, tol):
    """|got - ref| <= tol * S element by element, NaN (unwritten) where ref is NaN."""
    assert np.array_equal(np.isnan(got), np.isnan(ref)), "written/unwritten cells differ"
    m = ~np.isnan(ref)
    err = np.abs(got[m] - ref[m])
    bound = tol * S[m] + 1e-300
    worst = np.max(err / bound) if err.size else 0.0
    assert np.all(err <= bound), f"max error / bound = {worst}"


# Ordered iteration spaces: the predecessor offset of each order, and the
# recurrences compiled for their structure (gscl_ordered_specialization ids
# 0..4) with the terms in the order that defines each id.
ORDER_STEP = {B.I_INC: (-1, 0, 0), B.I_DEC: (1, 0, 0), B.J_INC: (0, -1, 0), B.J_DEC: (0, 1, 0), B.K_INC: (0, 0, -1),
              B.K_DEC: (0, 0, 1)}


def ordered_shape_terms(shape, order):
    """Input 0 is the output x, read at its predecessor; inputs 1, 2 are f, g
    or g, m."""
    prev = ORDER_STEP[order]
    a, b, c = 0.75, -0.5, 0.25
    if shape == 0:   # x = a x(prev) + b f
        return [(*prev, 0, B.NONE, 0, a), (0, 0, 0, 1, B.NONE, 0, b)]
    if shape == 1:   # x = b f + a x(prev), f read at an offset
        return [(1, 0, -1, 1, B.NONE, 0, b), (*prev, 0, B.NONE, 0, a)]
    if shape == 2:   # x = a g + b m x(prev)
        return [(0, 0, 0, 1, B.NONE, 0, a), (*prev, 0, 2, 0, b)]
    if shape == 3:   # x = b m x(prev) + a g, g read at an offset
        return [(*prev, 0, 2, 0, b), (-1, 1, 0, 1, B.NONE, 0, a)]
    # x = a f + b g + c x(prev)
    return [(0, 0, 0, 1, B.NONE, 0, a), (0, -1, 1, 2, B.NONE, 0, b), (*prev, 0, B.NONE, 0, c)]
