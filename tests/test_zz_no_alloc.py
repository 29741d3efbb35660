"""gscl_do_reduce_noalloc: the reduction for callers that cannot allocate
device memory (a fixed memory plan, or a pool that must not be bypassed)
uses a scratch array built into the library instead of a caller workspace.

These tests call it through the C ABI and compare it with gscl_do_reduce,
the entry point that takes a workspace, on two calls in a row (the scratch
keeps the previous call's contents, so the second call checks that it
starts clean).  The file is named to be collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S

pytestmark = pytest.mark.gpu


def noalloc(reduce_op, terms, ins, outs, result):
    """Calls the entry point directly through ctypes; returns (status, host value)."""
    L = B.lib()
    st = B.Stencil(terms) if terms is not None else None
    on_host = result is None
    host = ctypes.c_double(0.0)
    rptr = ctypes.pointer(host) if on_host else ctypes.cast(ctypes.c_void_p(result.data_ptr()),
                                                              ctypes.POINTER(ctypes.c_double))
    status = L.gscl_do_reduce_noalloc(reduce_op, ctypes.byref(st.c) if st else None, B._handles(ins), len(ins),
                                      B._handles(outs), len(outs), None, rptr, int(on_host),
                                      B.stream_ptr())
    return status, host.value


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_workspace_reduce_twice(dtype):
    n, h = (96, 80, 70), (1, 1, 1)
    lam = 0.125
    u0 = I.random_interior(41, n, h, -1.0, 1.0)
    f = I.random_interior(42, n, h, -1.0, 1.0)
    u, F = B.Grid(n, h, dtype).upload(u0), B.Grid(n, h, dtype).upload(f)
    v_ref, v_new = B.Grid(n, h, dtype), B.Grid(n, h, dtype)
    for g in (v_ref, v_new):
        g.upload(np.zeros(g.padded_shape))
    for call in range(2):
        ref = B.do_reduce(B.L2, S.heat7_fused(lam), [u, F], [v_ref])
        status, got = noalloc(B.L2, S.heat7_fused(lam), [u, F], [v_new], None)
        assert status == 0, B.lib().gscl_last_error()
        # same kernel, same launch configuration, same fixed reduction order
        assert got == ref, (call, got, ref)
        assert torch.equal(v_new.download(), v_ref.download())
        # device-resident result, and a plain reduction of a grid with no operator
        dev = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        status, _ = noalloc(B.SUM, None, [u], [], dev)
        assert status == 0, B.lib().gscl_last_error()
        want = B.do_reduce(B.SUM, None, [u])
        assert float(dev.item()) == want, (call, float(dev.item()), want)
        status, mx = noalloc(B.MAXABS, None, [u], [], None)
        assert status == 0 and mx == B.do_reduce(B.MAXABS, None, [u])
    B.sync()


def test_noalloc_large_grid_fits_its_scratch():
    """Launches use one wave of CTAs (at most SMs x resident CTAs partial sums,
    4736 on a 148-SM part), so even a 2D grid of 8192 x 1024 points fits the
    8192-partial scratch and matches the workspace entry point."""
    n, h = (8192, 1024, 1), (1, 1, 0)
    a = I.random_interior(43, n, h, -1.0, 1.0)
    g = B.Grid(n, h, "f64").upload(a)
    for _ in range(2):
        status, got = noalloc(B.L2, None, [g], [], None)
        assert status == 0, B.lib().gscl_last_error()
        ref = B.do_reduce(B.L2, None, [g])
        assert got == ref, (got, ref)
