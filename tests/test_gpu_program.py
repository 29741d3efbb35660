"""GPU parity of run-time compiled point operators (NVRTC) against the oracle
running the same body compiled with gcc: the heat operator as a body in three
storage dtypes and over sweeps, nonlinear bodies with math functions, the
index query of stateful operators, several outputs, in-place point-wise
updates, and reads beyond the declared reach reported without a fault."""
import numpy as np
import pytest
import torch

from gpu_common import as_storage
from oracle import oracle as O
from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S

pytestmark = pytest.mark.gpu

HEAT = ("out0 = 0.25 * in0(0,0,0) + 0.125 * (in0(1,0,0) + in0(-1,0,0) + in0(0,1,0) + in0(0,-1,0)"
        " + in0(0,0,1) + in0(0,0,-1)) + 0.125 * in1(0,0,0);")
NONLINEAR = ("real a = in0(0,0,0), b = in1(1,0,-1);\n"
             "out0 = sin(a) * exp(-b * b) + sqrt(fabs(in0(0,1,0) - in0(0,-1,0)));\n"
             "out1 = (a > b ? a : b) + 0.001 * (real)(i - 2 * j + 3 * k);")


def run_both(body, arrays, n, h, n_out, dtype, reach=(1, 1, 1), rng=None, sweeps=1):
    ndim = 2 if (n[2] == 1 and h[2] == 0) else 3
    gi = [B.Grid(n, h, dtype, ndim).upload(a) for a in arrays]
    go = [B.Grid(n, h, dtype, ndim).upload(np.full(I.padded_shape(n, h), 3.0)) for _ in range(n_out)]
    prog = B.Program(body, len(arrays), n_out, dtype, reach)
    prog.run(gi, go, rng=rng, sweeps=sweeps)
    B.sync()
    got = [g.download().double().numpy() for g in go]
    oi = [O.Grid(as_storage(a, dtype), h) for a in arrays]
    oo = [O.Grid(np.full(I.padded_shape(n, h), 3.0), h) for _ in range(n_out)]
    op = O.Program(body, len(arrays), n_out, reach)
    lo, hi = rng if rng is not None else (None, None)
    for s in range(sweeps):
        op.run(oi, oo, lo=lo, hi=hi)
        if s + 1 < sweeps:
            oi[0], oo[0] = oo[0], oi[0]
    return got, [g.a for g in oo]


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-14), ("f32", 2e-6), ("bf16", 1e-2)])
@pytest.mark.parametrize("n,rng", [((70, 21, 19), None), ((131, 40, 9), ((3, 5, 1), (128, 37, 8)))])
def test_heat_body_matches_oracle(dtype, tol, n, rng):
    h = (1, 1, 1)
    u = I.random_interior(91, n, h, -1.0, 1.0, halo_value=0.5)
    f = I.random_interior(92, n, h, -1.0, 1.0)
    got, want = run_both(HEAT, [u, f], n, h, 1, dtype, rng=rng)
    assert np.max(np.abs(got[0] - want[0])) <= tol * 2


def test_heat_body_sweeps_ping_pong():
    """Four sweeps ping-pong in[0] and out[0] like gscl_do_all (an even count
    leaves the result in out[0] by exchanging the handles)."""
    n, h = (64, 33, 20), (1, 1, 1)
    u = I.random_interior(93, n, h, -1.0, 1.0)
    f = I.random_interior(94, n, h, -1.0, 1.0)
    gu, gf, gv = B.Grid(n, h).upload(u), B.Grid(n, h).upload(f), B.Grid(n, h).upload(u)
    B.Program(HEAT, 2, 1).run([gu, gf], [gv], sweeps=4)
    ref_u, ref_v = B.Grid(n, h).upload(u), B.Grid(n, h).upload(u)
    B.do_all(S.heat7(0.125), [ref_u, B.Grid(n, h).upload(f)], [ref_v], sweeps=4)
    assert np.max(np.abs(gv.download().numpy() - ref_v.download().numpy())) <= 1e-13


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 3e-6)])
def test_nonlinear_body_two_outputs(dtype, tol):
    n, h = (45, 38, 7), (1, 1, 1)
    a = I.random_interior(95, n, h, -2.0, 2.0, halo_value=0.1)
    b = I.random_interior(96, n, h, -1.0, 1.0, halo_value=-0.3)
    got, want = run_both(NONLINEAR, [a, b], n, h, 2, dtype)
    for g, w in zip(got, want):
        assert np.max(np.abs(g - w)) <= tol * max(1.0, np.max(np.abs(w)))


def test_index_query_exact_and_2d():
    n, h = (100, 37, 1), (1, 1, 0)
    u = I.random_interior(97, n, h, -1.0, 1.0)
    got, want = run_both("out0 = (real)(i + 1000 * j + 100000 * k) + 0.0 * in0(0,0,0);", [u], n, h, 1, "f64",
                         reach=(0, 0, 0))
    assert np.array_equal(got[0], want[0])


def test_in_place_point_wise():
    """Reach 0: an output may be its own input (read, then written, per element)."""
    n, h = (50, 20, 10), (1, 1, 1)
    u = I.random_interior(98, n, h, -1.0, 1.0)
    g = B.Grid(n, h).upload(u)
    B.Program("out0 = in0(0,0,0) * in0(0,0,0) - 1.0;", 1, 1, "f64", (0, 0, 0)).run([g], [g])
    want = u.copy()
    I.interior_view(want, n, h)[...] = I.interior_view(u, n, h) ** 2 - 1.0
    assert np.max(np.abs(g.download().numpy() - want)) <= 1e-15


def test_read_beyond_reach_is_reported_not_performed():
    """in0(2, 0, 0) with reach 1: the read returns 0 and gscl_sync reports
    GSCL_ERR_RANGE; no memory outside the declared reach is touched."""
    n, h = (40, 10, 6), (1, 1, 1)
    u = I.random_interior(99, n, h, 1.0, 2.0)
    gu = B.Grid(n, h).upload(u)
    gv = B.Grid(n, h).upload(np.zeros(I.padded_shape(n, h)))
    B.Program("out0 = in0(2,0,0) + in0(0,0,0);", 1, 1, "f64", (1, 1, 1)).run([gu], [gv])
    with pytest.raises(B.GsclError) as e:
        B.sync()
    assert e.value.status == 2
    assert np.array_equal(I.interior_view(gv.download().numpy(), n, h), I.interior_view(u, n, h))
    B.sync()  # the flag is cleared


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("n,rng,reach", [((200, 45, 21), None, (1, 1, 1)),
                                          ((67, 9, 30), ((3, 1, 2), (60, 9, 29)), (1, 1, 1)),
                                          ((130, 20, 12), None, (2, 1, 2))])
def test_staged_kernel_equals_plain_kernel(dtype, n, rng, reach, monkeypatch):
    """The shared-memory staged kernel and the plain-load kernel evaluate the
    same body on the same values: identical results, on tiles with ragged
    edges, sub-ranges, short runs of planes and reaches of 2."""
    h = (2, 2, 2)
    body = ("out0 = in0(0,0,0) * (real)0.5 + (real)0.125 * (in0(1,0,0) + in0(-1,0,0) + in0(0,1,0) + in0(0,-1,0))"
            " + (real)0.0625 * (in0(0,0,1) + in0(0,0,-1)) + in1(0,0,0) * in1(0,0,0);")
    if reach[0] == 2:
        body += " out0 += (real)0.01 * (in0(2,0,0) - in0(-2,0,-2) + in1(0,1,2));"
    u = I.random_interior(120, n, h, -1.0, 1.0, halo_value=0.3)
    f = I.random_interior(121, n, h, -1.0, 1.0, halo_value=-0.2)
    prog = B.Program(body, 2, 1, dtype, reach)
    got = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("GSCL_PROGRAM_STAGED", flag)
        gi = [B.Grid(n, h, dtype).upload(a) for a in (u, f)]
        go = B.Grid(n, h, dtype).upload(np.zeros(I.padded_shape(n, h)))
        prog.run(gi, [go], rng=rng)
        got[flag] = go.download()
    B.sync()
    assert torch.equal(got["1"], got["0"])
    oi = [O.Grid(as_storage(a, dtype), h) for a in (u, f)]
    oo = O.Grid(np.zeros(I.padded_shape(n, h)), h)
    lo, hi = rng if rng is not None else (None, None)
    O.Program(body, 2, 1, reach).run(oi, [oo], lo=lo, hi=hi)
    tol = {"f64": 1e-14, "f32": 3e-6, "bf16": 2e-2}[dtype]
    assert np.max(np.abs(got["1"].double().numpy() - oo.a)) <= tol * 4


RESID = ("value = in0(1,0,0) + in0(-1,0,0) + in0(0,1,0) + in0(0,-1,0) + in0(0,0,1) + in0(0,0,-1)"
         " - (real)6 * in0(0,0,0) + in1(0,0,0);")


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 1e-5)])
@pytest.mark.parametrize("red", [B.SUM, B.MAXABS, B.L2])
def test_reduce_body_value_matches_oracle(dtype, tol, red):
    """The body's value reduced over a sub-range, against the oracle's values
    reduced with math.fsum (SUM, L2) or max |v|."""
    import math
    n, h = (90, 41, 23), (1, 1, 1)
    u = I.random_interior(130, n, h, -1.0, 1.0, halo_value=0.5)
    f = I.random_interior(131, n, h, -1.0, 1.0)
    rng = ((2, 3, 1), (87, 41, 22))
    gi = [B.Grid(n, h, dtype).upload(a) for a in (u, f)]
    got = B.Program(RESID, 2, 0, dtype).reduce(red, gi, [], rng=rng)
    vals = O.Program(RESID.replace("(real)6", "6.0"), 2, 0).run(
        [O.Grid(as_storage(u, dtype), h), O.Grid(as_storage(f, dtype), h)], [], lo=rng[0], hi=rng[1],
        want_value=True).ravel()
    want = {B.SUM: math.fsum(vals), B.MAXABS: float(np.max(np.abs(vals))),
            B.L2: math.sqrt(math.fsum(vals * vals))}[red]
    scale = np.sum(np.abs(vals)) if red == B.SUM else abs(want)
    assert abs(got - want) <= tol * scale


def test_reduce_body_with_outputs_is_a_fused_sweep():
    """value = the residual r, out0 = u + r / 8: one call gives the sweep and
    its residual norm, as the library's fused heat operator does."""
    n, h = (64, 64, 32), (1, 1, 1)
    u = I.random_interior(132, n, h, -1.0, 1.0)
    f = I.random_interior(133, n, h, -1.0, 1.0)
    body = RESID + " out0 = in0(0,0,0) + (real)0.125 * value;"
    gu, gf, gv = B.Grid(n, h).upload(u), B.Grid(n, h).upload(f), B.Grid(n, h).upload(u)
    got = B.Program(body, 2, 1).reduce(B.L2, [gu, gf], [gv])
    ru, rv = B.Grid(n, h).upload(u), B.Grid(n, h).upload(u)
    want = B.do_reduce(B.L2, S.heat7_fused(0.125), [ru, B.Grid(n, h).upload(f)], [rv])
    assert abs(got - want) <= 1e-13 * want
    assert np.max(np.abs(gv.download().numpy() - rv.download().numpy())) <= 1e-14


def test_reduce_body_empty_range_and_device_result():
    n, h = (40, 10, 6), (1, 1, 1)
    gu = B.Grid(n, h).upload(I.random_interior(134, n, h, 1.0, 2.0))
    p = B.Program("value = in0(0,0,0);", 1, 0, "f64", (0, 0, 0))
    assert p.reduce(B.SUM, [gu], [], rng=((0, 0, 3), (40, 10, 3))) == 0.0
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    p.reduce(B.MAXABS, [gu], [], result=res)
    assert float(res.cpu()[0]) == float(np.max(I.interior_view(I.random_interior(134, n, h, 1.0, 2.0), n, h)))
