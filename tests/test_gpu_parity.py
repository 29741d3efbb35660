"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bit-exact where the arithmetic is exact (integer data, dyadic weights: every
partial sum is representable, so any summation order and FMA give the same
bits), element-wise tolerances otherwise: |gpu - oracle| <= tol * S(p) with
S(p) the absolute stencil, tol = 1e-13 for FP64 and 2e-6 for FP32 storage."""
import math

import numpy as np
import pytest
import torch

from gpu_common import TOL, as_storage, assert_within, run_pair
from oracle import drivers as D
from oracle import oracle as O
from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S

pytestmark = pytest.mark.gpu
VALUE, NONE = B.VALUE, B.NONE


@pytest.fixture(autouse=True, params=["compiled", "generic"])
def kernel_path(request, monkeypatch):
    """Every parity test runs once with operator structures compiled where they
    match and once with the generic term-list kernel only."""
    if request.param == "generic":
        monkeypatch.setenv("GSCL_GENERIC_ONLY", "1")
    else:
        monkeypatch.delenv("GSCL_GENERIC_ONLY", raising=False)
    return request.param


def int_field(rng, shape, lim):
    return rng.integers(-lim, lim + 1, size=shape).astype(np.float64)


def dyadic_terms(rng, n_in, n_out, halos, count, with_value=True, dims=3):
    weights = [1.0, -1.0, 2.0, -2.0, 0.5, -0.5, 0.25, -0.125]
    terms = []
    for _ in range(count):
        a = int(rng.integers(0, n_in))
        hx, hy, hz = halos[a]
        o = [int(rng.integers(-hx, hx + 1)), int(rng.integers(-hy, hy + 1)),
             int(rng.integers(-hz, hz + 1)) if dims == 3 else 0]
        c = int(rng.integers(0, n_in)) if rng.random() < 0.3 else NONE
        m = VALUE if (with_value and rng.random() < 0.3) else int(rng.integers(0, n_out))
        terms.append((o[0], o[1], o[2], a, c, m, float(rng.choice(weights))))
    if with_value:
        terms.append((0, 0, 0, 0, NONE, VALUE, 1.0))
        terms.append((0, 0, 0, VALUE, NONE, n_out - 1, -0.5))
    return terms


SHAPES = [
    ((17, 13, 11), [(1, 1, 1), (2, 2, 1), (0, 0, 0)], [(1, 1, 1), (0, 0, 0)]),
    ((150, 37, 21), [(2, 1, 2), (1, 1, 1), (1, 0, 1)], [(1, 1, 1), (2, 2, 2)]),
    ((5, 3, 2), [(1, 1, 1), (1, 1, 1), (0, 0, 0)], [(0, 0, 0), (1, 1, 1)]),
    ((200, 70, 1), [(1, 1, 0), (2, 2, 0), (0, 0, 0)], [(1, 1, 0), (0, 0, 0)]),
]


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("shape_id", range(len(SHAPES)))
def test_bitexact_random_operator(dtype, shape_id):
    n, in_halos, out_halos = SHAPES[shape_id]
    rng = np.random.default_rng(100 + shape_id)
    dims = 2 if n[2] == 1 else 3
    arrays = [int_field(rng, I.padded_shape(n, h), 64) for h in in_halos]
    arrays[2] = int_field(rng, I.padded_shape(n, in_halos[2]), 8)  # coefficient-sized
    terms = dyadic_terms(rng, 3, 2, in_halos, 14, dims=dims)
    got, ref, _, _, _ = run_pair(terms, arrays, in_halos, n, out_halos, dtype)
    for g, r in zip(got, ref):
        if dtype == "bf16":
            r = as_storage(r, "bf16")
        assert np.array_equal(g, r, equal_nan=True)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_bitexact_subrange_and_ragged_edges(dtype):
    n = (300, 41, 19)
    halos = [(2, 2, 2), (1, 1, 1)]
    rng = np.random.default_rng(7)
    arrays = [int_field(rng, I.padded_shape(n, h), 50) for h in halos]
    terms = dyadic_terms(rng, 2, 1, halos, 10)
    for lo, hi in [((3, 1, 2), (141, 40, 17)), ((129, 0, 0), (130, 41, 19)), ((0, 5, 18), (300, 6, 19))]:
        got, ref, _, _, _ = run_pair(terms, arrays, halos, n, [(1, 1, 1)], dtype, rng=(lo, hi))
        assert np.array_equal(got[0], ref[0], equal_nan=True)


def test_spike_gives_reflected_fig1b_pattern():
    n, h = (40, 20, 12), (1, 1, 1)
    a = np.zeros(I.padded_shape(n, h))
    p0 = (33, 7, 5)
    a[p0[2] + 1, p0[1] + 1, p0[0] + 1] = 36.0
    got, ref, _, _, _ = run_pair(S.fig1b(), [a], [h], n, [h], "f64")
    inner = got[0][1:-1, 1:-1, 1:-1]
    assert np.array_equal(got[0], ref[0], equal_nan=True)
    nz = {tuple(int(v) for v in idx): inner[idx] for idx in zip(*np.nonzero(inner))}
    expect = {(p0[2], p0[1], p0[0]): 6.0}
    for dx, dy, dz in S.X6:
        expect[(p0[2] - dz, p0[1] - dy, p0[0] - dx)] = -1.0
    assert nz == expect


@pytest.mark.parametrize("op", [B.SUM, B.MAXABS, B.L2])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_bitexact_reductions_on_integer_data(op, dtype):
    n = (131, 29, 17)
    halos = [(1, 1, 1), (1, 1, 1)]
    rng = np.random.default_rng(11 + op)
    arrays = [int_field(rng, I.padded_shape(n, h), 40) for h in halos]
    terms = dyadic_terms(rng, 2, 1, halos, 9)
    got, ref, gv, ov, _ = run_pair(terms, arrays, halos, n, [(0, 0, 0)], dtype, reduce_op=op)
    assert np.array_equal(got[0], ref[0], equal_nan=True)
    assert gv == ov
    # identity reduction of in[0] over a sub-range
    _, _, gv, ov, _ = run_pair(None, arrays[:1], halos[:1], n, [], dtype, rng=((5, 2, 1), (120, 29, 16)),
                               reduce_op=op)
    assert gv == ov


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_heat_fused_tolerance_random_data(dtype):
    n, h = (97, 45, 33), (1, 1, 1)
    u = I.random_interior(5, n, h, -1.0, 1.0)
    f = I.random_interior(6, n, h, -1.0, 1.0)
    lam = 0.125
    got, ref, gv, ov, Sab = run_pair(S.heat7_fused(lam), [u, f], [h, h], n, [h], dtype, reduce_op=B.L2)
    assert_within(got[0], ref[0], Sab[0], TOL[dtype])
    assert abs(gv - ov) <= TOL[dtype] * ov
    # the plain 8-term sweep computes the same update within the same bound
    got2, _, _, _, Sab2 = run_pair(S.heat7(lam), [u, f], [h, h], n, [h], dtype)
    assert_within(got2[0], ref[0], Sab[0] + Sab2[0], TOL[dtype])


@pytest.mark.parametrize("op", [B.SUM, B.L2])
def test_reduction_tolerance_random_data(op):
    n, h = (64, 64, 64), (1, 1, 1)
    a = I.random_interior(9, n, h, -1.0, 1.0)
    a += 1e6 * (np.indices(a.shape).sum(axis=0) % 2 - 0.5)  # large cancelling alternation
    _, _, gv, ov, _ = run_pair(None, [a], [h], n, [], "f64", reduce_op=op)
    inner = a[1:-1, 1:-1, 1:-1]
    absum = np.abs(inner).sum() if op == B.SUM else (inner ** 2).sum()
    # compensated at every level above groups of 2 values: a few ulps of sum |x|
    bound = 8 * np.finfo(np.float64).eps * absum
    if op == B.SUM:
        assert abs(gv - ov) <= bound
    else:
        assert abs(gv * gv - ov * ov) <= bound


def test_reduction_nan_and_empty_range():
    n, h = (40, 9, 5), (1, 1, 1)
    a = I.random_interior(3, n, h, -1.0, 1.0)
    a[3, 4, 17] = np.nan
    for op in (B.SUM, B.MAXABS, B.L2):
        _, _, gv, _, _ = run_pair(None, [a], [h], n, [], "f64", reduce_op=op)
        assert math.isnan(gv)
        _, _, gv, ov, _ = run_pair(None, [a], [h], n, [], "f64", rng=((0, 0, 2), (40, 9, 2)), reduce_op=op)
        assert gv == 0.0 == ov


def test_reduction_is_deterministic():
    n, h = (128, 128, 64), (1, 1, 1)
    a = I.random_interior(21, n, h, -1.0, 1.0)
    g = B.Grid(n, h).upload(a)
    vals = {B.do_reduce(B.SUM, None, [g]) for _ in range(4)}
    assert len(vals) == 1


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_multisweep_equals_single_sweeps_and_swaps(dtype):
    n, h = (70, 33, 26), (1, 1, 1)
    u0 = I.random_interior(31, n, h, -1.0, 1.0, halo_value=0.25)
    f = I.random_interior(32, n, h, -1.0, 1.0)
    op = B.Stencil(S.heat7(0.125))
    F = B.Grid(n, h, dtype).upload(f)
    for k in (1, 2, 5):
        a, b = B.Grid(n, h, dtype).upload(u0), B.Grid(n, h, dtype).upload(u0)
        B.do_all(op, [a, F], [b], sweeps=k)
        multi = b.download()
        c, d = B.Grid(n, h, dtype).upload(u0), B.Grid(n, h, dtype).upload(u0)
        for _ in range(k):
            B.do_all(op, [c, F], [d])
            B.swap(c, d)
        assert torch.equal(multi, c.download())


def test_laplace2d_100_sweeps_full_size():
    """The 2D Laplace workload at its full size (256 x 256, 100 sweeps)."""
    u0 = I.laplace2d(101, 256)
    n, h = (256, 256, 1), (1, 1, 0)
    a, b = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(u0)
    B.do_all(S.jacobi5_2d(), [a], [b], sweeps=99)       # b = u_99
    B.do_all(S.jacobi5_2d(), [b], [a])                  # a = u_100
    res = B.do_reduce(B.MAXABS, S.difference(), [a, b])
    ou, op, ores = D.jacobi2d_run(O.Grid(u0.copy(), h), 100)
    scale = np.max(np.abs(ou.a))
    assert np.max(np.abs(a.download().numpy() - ou.a)) <= 1e-13 * scale
    assert np.max(np.abs(b.download().numpy() - op.a)) <= 1e-13 * scale
    assert abs(res - ores) <= 1e-13 * scale


def run_heat(u0, f, n, dtype, lam, sweeps, every):
    """Heat/damped-Jacobi loop: every `every` sweeps a fused do_reduce returns the
    residual of the iterate it reads; plain multi-sweep do_all in between."""
    h = (1, 1, 1)
    u, v = B.Grid(n, h, dtype).upload(u0), B.Grid(n, h, dtype).upload(u0)
    F = B.Grid(n, h, dtype).upload(f)
    fused, plain = B.Stencil(S.heat7_fused(lam)), B.Stencil(S.heat7(lam))
    res = torch.zeros(sweeps // every, dtype=torch.float64, device="cuda")
    for m in range(sweeps // every):
        B.do_reduce(B.L2, fused, [u, F], [v], result=res[m:m + 1])
        B.swap(u, v)
        B.do_all(plain, [u, F], [v], sweeps=every - 1)
        B.swap(u, v)
    B.sync()
    return u.download().double().numpy(), res.cpu().numpy()


def test_heat3d_multisweep_small_with_residuals():
    n, h = (32, 32, 32), (1, 1, 1)
    u0, f = I.heat3d(202, 32)
    lam = 0.125
    res = run_heat(u0, f, n, "f64", lam, 40, 10)
    ou, ores = D.heat_run(O.Grid(u0.copy(), h), O.Grid(f.copy(), h), lam, 40, every=10)
    assert np.max(np.abs(res[0] - ou.a)) <= 1e-13 * np.max(np.abs(ou.a))
    assert np.allclose(res[1], ores, rtol=1e-13, atol=0)
    r32 = run_heat(u0, f, n, "f32", lam, 40, 10)
    assert np.max(np.abs(r32[0] - ou.a)) <= 1e-5 * np.max(np.abs(ou.a))
    assert np.allclose(r32[1], ores, rtol=1e-5, atol=0)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_heat3d_full_size_one_fused_sweep_after_nine(dtype):
    """256^3 at the benchmark's launch configuration: nine sweeps, then the
    fused sweep + residual checked point by point against the oracle run from
    the GPU's own ninth iterate."""
    n, h = (256, 256, 256), (1, 1, 1)
    u0, f = I.heat3d(202, 256)
    lam = 0.125
    u, v = B.Grid(n, h, dtype).upload(u0), B.Grid(n, h, dtype).upload(u0)
    F = B.Grid(n, h, dtype).upload(f)
    r0 = B.do_reduce(B.L2, S.heat7_fused(lam), [u, F], [v])
    B.swap(u, v)
    B.do_all(S.heat7(lam), [u, F], [v], sweeps=8)
    B.swap(u, v)
    r9 = B.do_reduce(B.L2, S.heat7_fused(lam), [u, F], [v])
    u9 = u.download().double().numpy()
    u10 = v.download().double().numpy()
    fo = O.Grid(as_storage(f, dtype), h)
    exact_f = math.sqrt(math.fsum((fo.a ** 2).ravel()))
    assert abs(r0 - exact_f) <= TOL[dtype] * exact_f
    out, Sab = O.zeros(n, h), O.zeros(n, h)
    ores = O.do_reduce(O.L2, D.heat_terms(lam), [O.Grid(u9, h), fo], [out])
    O.do_all(D.heat_terms(lam), [O.Grid(u9, h), fo], [Sab], abs_mode=True)
    assert abs(r9 - ores) <= TOL[dtype] * ores
    m = (slice(1, -1),) * 3
    assert np.all(np.abs(u10[m] - out.a[m]) <= TOL[dtype] * Sab.a[m])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_climate_multigrid_operator(dtype):
    n, h = (72, 40, 12), (2, 2, 1)
    fields = I.climate(303, n, h)
    arrays = [fields[k] for k in I.CLIMATE_FIELDS]
    got, ref, _, _, Sab = run_pair(S.climate(), arrays, [h] * 8, n, [h] * 3, dtype)
    for g, r, s in zip(got, ref, Sab):
        assert_within(g, r, s, TOL[dtype])


def test_climate_full_size_one_sweep():
    n, h = (256, 256, 80), (2, 2, 1)
    fields = I.climate(303, n, h)
    arrays = [fields[k] for k in I.CLIMATE_FIELDS]
    got, ref, _, _, Sab = run_pair(S.climate(), arrays, [h] * 8, n, [h] * 3, "f64")
    for g, r, s in zip(got, ref, Sab):
        assert_within(g, r, s, TOL["f64"])


def test_degenerate_single_point_and_zero_halo():
    n, h = (1, 1, 1), (0, 0, 0)
    a = np.array([[[3.0]]])
    got, ref, gv, ov, _ = run_pair([(0, 0, 0, 0, NONE, 0, 2.0), (0, 0, 0, 0, NONE, VALUE, -1.0)], [a], [h], n,
                                   [h], "f64", reduce_op=B.SUM)
    assert got[0][0, 0, 0] == 6.0 == ref[0][0, 0, 0]
    assert gv == -3.0 == ov


def test_sync_reports_clean_status():
    B.sync()


@pytest.mark.parametrize("dst_t,src_t", [("f32", "f64"), ("f64", "f32"), ("f64", "f64"), ("bf16", "f32")])
def test_convert_cast_and_accumulate(dst_t, src_t):
    n, h = (70, 21, 9), (1, 1, 1)
    a = I.random_interior(51, n, h, -3.0, 3.0, halo_value=7.0)
    b = I.random_interior(52, n, h, -1.0, 1.0, halo_value=9.0)
    src = B.Grid(n, h, src_t).upload(a)
    dst = B.Grid(n, h, dst_t).upload(b)
    B.convert(dst, src, alpha=0.5, accumulate=True, rng=((3, 1, 2), (66, 21, 8)))
    got = dst.download().double().numpy()
    sa = as_storage(a, src_t)
    sb = as_storage(b, dst_t)
    want = sb.copy()
    sl = (slice(1 + 2, 1 + 8), slice(1 + 1, 1 + 21), slice(1 + 3, 1 + 66))
    want[sl] = as_storage(0.5 * sa[sl] + sb[sl], dst_t)  # FP64 arithmetic, one rounding
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("which", ["heat_rhs", "heat", "poisson"])
@pytest.mark.parametrize("n,hu", [((150, 37, 21), (1, 1, 1)), ((5, 3, 2), (2, 2, 2)), ((256, 40, 9), (1, 2, 1)),
                                  ((130, 90, 40), (1, 1, 1))])
def test_temporal_blocking_bitexact_with_single_sweeps(monkeypatch, dtype, which, n, hu):
    """K sweeps fused per pass (K = 2, 3, 4) give the bits of K single sweeps;
    on the 130 x 90 x 40 grid the CTAs stream several runs of planes each."""
    op = {"heat_rhs": S.heat7(0.125), "heat": S.heat7(0.125, with_f=False), "poisson": S.poisson_jacobi()}[which]
    rhs = which != "heat"
    u0 = I.random_interior(61, n, hu, -1.0, 1.0, halo_value=0.375)
    f = I.random_interior(62, n, (0, 0, 0), -1.0, 1.0) if rhs else None
    results = {}
    for K in ("1", "2", "3", "4"):
        monkeypatch.setenv("GSCL_TEMPORAL", K)
        a, b = B.Grid(n, hu, dtype).upload(u0), B.Grid(n, hu, dtype).upload(u0)
        ins = [a] + ([B.Grid(n, (0, 0, 0), dtype).upload(f)] if rhs else [])
        B.do_all(op, ins, [b], sweeps=7)
        results[K] = b.download()
    for K in ("2", "3", "4"):
        d = (results[K].double() - results["1"].double()).abs()
        assert torch.equal(results[K], results["1"]), (K, d.max().item(), int((d > 0).sum()))


TEMPORAL_OPS = {  # library operator, oracle operator (the fused form of the same update), lambda, RHS
    "heat_rhs": (lambda: S.heat7(0.125), 0.125, True),
    "heat": (lambda: S.heat7(0.125, with_f=False), 0.125, False),
    "poisson": (lambda: S.poisson_jacobi(), 1.0 / 6.0, True),
}


@pytest.mark.parametrize("which", ["heat_rhs", "heat"])
@pytest.mark.parametrize("n,hu", [((150, 37, 21), (1, 1, 1)), ((256, 40, 9), (1, 2, 1))])
def test_temporal_blocking_bitexact_with_oracle_on_integer_data(monkeypatch, which, n, hu):
    """K sweeps in one pass (K = 1..4) against the oracle's K sweeps, FP32
    storage, integer data (|u|, |f| <= 64) and lambda = 1/8: after s sweeps
    every value and every partial sum is a multiple of 2^-3s below 2^7, which
    FP32 holds exactly for s <= 4, so the GPU's blocked sweeps and the
    oracle's one-at-a-time FP64 sweeps must agree bit for bit.  K + 1 sweeps
    run (the last launch of a run is a single sweep), so the fused pass's
    result u_K is the one in[0] names on return."""
    mk, lam, rhs = TEMPORAL_OPS[which]
    rng = np.random.default_rng(70 + n[0])
    u0 = int_field(rng, I.padded_shape(n, hu), 64)
    f = int_field(rng, I.padded_shape(n, (0, 0, 0)), 64)
    for K in (1, 2, 3, 4):
        monkeypatch.setenv("GSCL_TEMPORAL", str(K))
        a, b = B.Grid(n, hu, "f32").upload(u0), B.Grid(n, hu, "f32").upload(u0)
        ins = [a] + ([B.Grid(n, (0, 0, 0), "f32").upload(f)] if rhs else [])
        B.do_all(mk(), ins, [b], sweeps=K + 1)
        got = a.download().double().numpy()
        want, _ = D.heat_run(O.Grid(u0.copy(), hu), O.Grid(f.copy(), (0, 0, 0)) if rhs else None, lam, K)
        assert np.array_equal(got, want.a), (K, float(np.max(np.abs(got - want.a))))


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("which", ["heat_rhs", "heat", "poisson"])
@pytest.mark.parametrize("n", [(150, 37, 21), (130, 90, 40)])
def test_temporal_blocking_within_tolerance_of_oracle(monkeypatch, dtype, which, n):
    """K sweeps per pass (K = 1..4), 7 sweeps, against the FP64 oracle's 7
    sweeps from the same storage-rounded data.  Each GPU sweep may differ from
    the exact update of its own input by tol * S(p) (FP32 storage: 2e-6; BF16:
    2^-8, one rounding to 8 fraction bits plus FP32 arithmetic), and these
    updates have non-negative weights summing to 1 with fixed halos, so an
    error never grows from one sweep to the next: after N sweeps
    |g - o| <= tol * sum_i max_p S_i(p), S_i the absolute stencil of sweep i.
    The relative error ||g - o||_inf / ||o||_inf is printed for each K."""
    mk, lam, rhs = TEMPORAL_OPS[which]
    tol = {"f32": 2e-6, "bf16": 2.0 ** -8}[dtype]
    hu, sweeps = (1, 1, 1), 7
    u0 = I.random_interior(63, n, hu, -1.0, 1.0, halo_value=0.375)
    f = I.random_interior(64, n, (0, 0, 0), -1.0, 1.0)
    a_o = O.Grid(as_storage(u0, dtype), hu)
    f_o = O.Grid(as_storage(f, dtype), (0, 0, 0)) if rhs else None
    terms = D.heat_terms(lam, rhs)
    bound = 0.0
    cur = a_o.copy()
    for _ in range(sweeps):
        Sab = O.zeros(n, hu)
        O.do_all(terms, [cur] + ([f_o] if rhs else []), [Sab], abs_mode=True)
        bound += tol * float(np.max(Sab.interior()))
        nxt = cur.copy()
        O.do_all(terms, [cur] + ([f_o] if rhs else []), [nxt])
        cur = nxt
    want = cur.a
    for K in (1, 2, 3, 4):
        monkeypatch.setenv("GSCL_TEMPORAL", str(K))
        a, b = B.Grid(n, hu, dtype).upload(u0), B.Grid(n, hu, dtype).upload(u0)
        ins = [a] + ([B.Grid(n, (0, 0, 0), dtype).upload(f)] if rhs else [])
        B.do_all(mk(), ins, [b], sweeps=sweeps)
        got = b.download().double().numpy()
        err = float(np.max(np.abs(got - want)))
        print(f"temporal K={K} {which} {dtype}: ||g - o||_inf / ||o||_inf after {sweeps} sweeps = "
              f"{err / float(np.max(np.abs(want))):.3e} (bound {bound:.3e})")
        assert err <= bound, (K, err, bound)


def test_temporal_tuner_picks_a_factor_and_keeps_bits(monkeypatch):
    monkeypatch.delenv("GSCL_TEMPORAL", raising=False)
    n, h = (128, 64, 48), (1, 1, 1)
    u0 = I.random_interior(71, n, h, -1.0, 1.0)
    f = I.random_interior(72, n, h, -1.0, 1.0)
    a, b, F = B.Grid(n, h, "f32").upload(u0), B.Grid(n, h, "f32").upload(u0), B.Grid(n, h, "f32").upload(f)
    k = B.tune_sweeps(S.heat7(0.125), [a, F], [b], trial_sweeps=4)
    assert 1 <= k <= 4
    assert torch.equal(a.download(), torch.from_numpy(u0).float())   # in[0] untouched
    B.do_all(S.heat7(0.125), [a, F], [b], sweeps=6)
    tuned = b.download()
    monkeypatch.setenv("GSCL_TEMPORAL", "1")
    c, d = B.Grid(n, h, "f32").upload(u0), B.Grid(n, h, "f32").upload(u0)
    B.do_all(S.heat7(0.125), [c, F], [d], sweeps=6)
    assert torch.equal(tuned, d.download())
    # FP64 never fuses
    e, g = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(u0)
    assert B.tune_sweeps(S.heat7(0.125, with_f=False), [e], [g]) == 1


def test_fma_throughput_is_plausible():
    """The measured FP64 / FP32 FMA rates are positive and no faster than the
    SM count x FMA lanes x maximum clock allows (FP64: 2 per SM per clock on
    B300-class parts, FP32: 128)."""
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    f64 = B.fma_throughput("f64", 512)
    f32 = B.fma_throughput("f32", 8192)
    clock_hz = 2.2e9  # above any B300 SM clock
    assert 0 < f32 <= sms * 128 * 2 * clock_hz
    assert 0 < f64 <= f32


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_heat3d_error_after_200_sweeps_reported(dtype):
    """Error after N sweeps against the FP64 oracle run from the same initial
    data (reported, gated only loosely): the heat workload's recipe (seed 202,
    lam = 1/8, fused L2 residual every 10 sweeps) on a 64^3 interior, 200
    sweeps, FP64 and FP32 storage.  The FP32 figure is the accumulated
    storage rounding of 200 sweeps; the FP64 one is rounding-order noise."""
    n = 64
    u0, f = I.heat3d(202, n)
    shape, h = (n, n, n), (1, 1, 1)
    u, v = B.Grid(shape, h, dtype).upload(u0), B.Grid(shape, h, dtype).upload(u0)
    F = B.Grid(shape, h, dtype).upload(f)
    fused, plain = B.Stencil(S.heat7_fused(0.125)), B.Stencil(S.heat7(0.125))
    res = []
    for _ in range(20):
        res.append(B.do_reduce(B.L2, fused, [u, F], [v]))
        B.swap(u, v)
        B.do_all(plain, [u, F], [v], sweeps=9)
        B.swap(u, v)
    got = u.download().double().numpy()
    ou, ores = D.heat_run(O.Grid(as_storage(u0, dtype), h), O.Grid(as_storage(f, dtype), h), 0.125, 200, every=10)
    err = np.max(np.abs(got - ou.a)) / np.max(np.abs(ou.a))
    rerr = max(abs(a - b) / b for a, b in zip(res, ores))
    print(f"heat3d 64^3 {dtype}: |u_200 - oracle|_inf / |oracle|_inf = {err:.3e}; "
          f"max relative residual error = {rerr:.3e}")
    bound = 1e-12 if dtype == "f64" else 1e-4
    assert err <= bound and rerr <= bound, (err, rerr)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_reduce_within_matches_oracle(dtype):
    """gscl_do_reduce_within (logical_and of |value| <= eps) against the
    oracle: eps below and above the largest difference (and exactly at it in
    FP64, where both sides form a - b in the same precision), a planted NaN,
    an empty range, and the device-resident result."""
    n, h = (70, 33, 21), (1, 1, 1)
    a = I.random_interior(81, n, h, -1.0, 1.0)
    b = a + I.random_interior(82, n, h, -1e-3, 1e-3)
    A, Bg = as_storage(a, dtype), as_storage(b, dtype)
    oa, ob = O.Grid(A, h), O.Grid(Bg, h)
    dmax = O.do_reduce(O.MAXABS, D.difference_terms(), [oa, ob])
    ga, gb = B.Grid(n, h, dtype).upload(a), B.Grid(n, h, dtype).upload(b)
    op = S.difference()
    eps_list = [0.5 * dmax, 2.0 * dmax] + ([dmax] if dtype == "f64" else [])
    for eps in eps_list:
        want = O.do_reduce_within(eps, D.difference_terms(), [oa, ob])
        assert B.do_reduce_within(eps, op, [ga, gb]) == want, eps
    res = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
    B.do_reduce_within(2.0 * dmax, op, [ga, gb], result=res)
    assert float(res.cpu()[0]) == 1.0
    assert B.do_reduce_within(0.0, op, [ga, gb], rng=((3, 3, 3), (3, 9, 9))) == 1.0
    a2 = a.copy()
    a2[5, 6, 7] = np.nan
    gn = B.Grid(n, h, dtype).upload(a2)
    assert B.do_reduce_within(1e9, op, [gn, gb]) == 0.0
    with pytest.raises(B.GsclError):
        B.do_reduce_within(-1.0, op, [ga, gb])


def test_reduce_clears_a_stale_ticket_and_reports_a_timeout():
    """A workspace whose arrival ticket an interrupted call left non-zero (here
    planted by hand) still gives the oracle's value: each call clears the
    ticket first.  A bounded wait that gave up (the self-test sets the same
    device flag a timed-out reduction sets) is reported by the next reduction
    that returns its value to the host, as GSCL_ERR_TIMEOUT, once."""
    n, h = (70, 33, 21), (1, 1, 1)
    u0 = I.random_interior(171, n, h, -1.0, 1.0)
    f0 = I.random_interior(172, n, h, -1.0, 1.0)
    u, F, v = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(f0), B.Grid(n, h).zero()
    want = O.do_reduce(O.L2, D.heat_terms(0.125), [O.Grid(u0.copy(), h), O.Grid(f0.copy(), h)], [O.zeros(n, h)])
    ws = B.workspace()
    ws[:256].fill_(0x5a)
    B.sync()
    got = B.do_reduce(B.L2, S.heat7_fused(0.125), [u, F], [v])
    assert abs(got - want) <= TOL["f64"] * want, (got, want)
    B.check(B.lib().gscl_selftest_bounded_wait(None))
    with pytest.raises(B.GsclError) as e:
        B.do_reduce(B.L2, S.heat7_fused(0.125), [u, F], [v])
    assert e.value.status == 9
    got = B.do_reduce(B.L2, S.heat7_fused(0.125), [u, F], [v])  # the flag was cleared
    assert abs(got - want) <= TOL["f64"] * want, (got, want)
    B.sync()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """A wait on a barrier nothing arrives on gives up after its cycle limit;
    gscl_sync reports GSCL_ERR_TIMEOUT once, and the next sweeps run normally."""
    B.check(B.lib().gscl_selftest_bounded_wait(None))
    with pytest.raises(B.GsclError) as e:
        B.sync()
    assert e.value.status == 9
    B.sync()  # the flag was cleared
    n, h = (40, 12, 9), (1, 1, 1)
    u0 = I.random_interior(160, n, h, -1.0, 1.0)
    f0 = I.random_interior(161, n, h, -1.0, 1.0)
    got, want, _, _, S_ = run_pair(S.heat7(0.125), [u0, f0], [h, h], n, [h], "f64")
    assert_within(got[0], want[0], S_[0], TOL["f64"])
