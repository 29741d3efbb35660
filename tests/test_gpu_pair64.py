"""FP64 grids in pair arithmetic (gscl_set_fp64_arithmetic(GSCL_FP64_PAIR)):
parity against the FP64 oracle at the FP64 tolerance |gpu - oracle| <=
1e-13 S(p), bit-exactness where every partial result is representable in
24 + 24 bits (integer data, dyadic weights), and the split of special
values."""
import numpy as np
import pytest
import torch

from gpu_common import assert_within, run_pair
from oracle import drivers as D
from oracle import oracle as O
from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S
from test_gpu_parity import SHAPES, dyadic_terms, int_field

pytestmark = pytest.mark.gpu
TOL = 1e-13


@pytest.fixture(autouse=True)
def pair_mode():
    B.set_fp64_arithmetic("pair")
    yield
    B.set_fp64_arithmetic("ieee")


@pytest.fixture(params=["compiled", "generic"])
def kernel_path(request, monkeypatch):
    if request.param == "generic":
        monkeypatch.setenv("GSCL_GENERIC_ONLY", "1")
    else:
        monkeypatch.delenv("GSCL_GENERIC_ONLY", raising=False)
    return request.param


def test_mode_switch():
    assert B.get_fp64_arithmetic() == "pair"
    assert B.lib().gscl_set_fp64_arithmetic(7) != 0  # GSCL_ERR_INVALID


def test_heat_fused_and_plain_within_fp64_tolerance(kernel_path):
    n, h = (97, 45, 33), (1, 1, 1)
    u = I.random_interior(5, n, h, -1.0, 1.0)
    f = I.random_interior(6, n, h, -1.0, 1.0)
    got, ref, gv, ov, Sab = run_pair(S.heat7_fused(0.125), [u, f], [h, h], n, [h], "f64", reduce_op=B.L2)
    assert_within(got[0], ref[0], Sab[0], TOL)
    assert abs(gv - ov) <= TOL * ov
    got2, ref2, _, _, Sab2 = run_pair(S.heat7(0.125), [u, f], [h, h], n, [h], "f64")
    assert_within(got2[0], ref2[0], Sab2[0], TOL)


def test_weights_not_representable_in_fp32(kernel_path):
    """Weights with a non-zero low part (1/3, 1/7, pi/10) exercise the pair
    weights: still within the FP64 tolerance, far inside FP32's."""
    n, h = (70, 30, 20), (1, 1, 1)
    u = I.random_interior(15, n, h, -3.0, 3.0)
    terms = [(0, 0, 0, 0, B.NONE, 0, 1.0 / 3.0)] + [(dx, dy, dz, 0, B.NONE, 0, w)
                                                   for (dx, dy, dz), w in zip(S.X6, [1 / 7, np.pi / 10] * 3)]
    got, ref, _, _, Sab = run_pair(terms, [u], [h], n, [h], "f64")
    assert_within(got[0], ref[0], Sab[0], TOL)


def test_jacobi2d_and_climate_within_fp64_tolerance(kernel_path):
    n2, h2 = (200, 70, 1), (1, 1, 0)
    a = I.random_interior(21, n2, h2, 0.0, 1.0, halo_value=0.5)
    got, ref, _, _, Sab = run_pair(S.jacobi5_2d(), [a], [h2], n2, [h2], "f64")
    assert_within(got[0], ref[0], Sab[0], TOL)
    n3, h3 = (70, 40, 12), (2, 2, 1)
    fields = I.climate(303, n3, h3)
    ins = [fields[k] for k in I.CLIMATE_FIELDS]
    got, ref, _, _, Sab = run_pair(S.climate(), ins, [h3] * 8, n3, [h3] * 3, "f64")
    for g, r, s in zip(got, ref, Sab):
        assert_within(g, r, s, TOL)


@pytest.mark.parametrize("shape_id", range(len(SHAPES)))
def test_bitexact_integer_data(shape_id):
    """Integers below 2^10 and dyadic weights: every split is exact (lo = 0),
    every product and partial sum is representable, so the pair arithmetic
    gives the oracle's bits."""
    n, in_halos, out_halos = SHAPES[shape_id]
    rng = np.random.default_rng(100 + shape_id)
    dims = 2 if n[2] == 1 else 3
    arrays = [int_field(rng, I.padded_shape(n, h), 64) for h in in_halos]
    arrays[2] = int_field(rng, I.padded_shape(n, in_halos[2]), 8)
    terms = dyadic_terms(rng, 3, 2, in_halos, 14, dims=dims)
    got, ref, _, _, _ = run_pair(terms, arrays, in_halos, n, out_halos, "f64")
    for g, r in zip(got, ref):
        assert np.array_equal(g, r, equal_nan=True)


def test_special_values_through_the_split():
    """Zeros of both signs, values between 2^-100 and 2^-74 (the hardware
    conversion path of the split), values up to 2^100, an infinity and a NaN
    copied by the identity operator (value 1 x): the finite values keep 47 of
    their 53 bits, zeros come out as the oracle's, inf and NaN stay non-finite (the
    exact-product correction of an infinite product is NaN, so an infinity
    comes out as NaN).  (The pair holds magnitudes from about 2^-100 to below
    2^128 only; see the header.)"""
    n, h = (64, 4, 3), (0, 0, 0)
    a = np.full(I.padded_shape(n, h), 1.0)
    v = a.reshape(-1)
    v[:6] = [0.0, -0.0, 3e-30, -2.5e-27, np.inf, np.nan]
    v[8:40] = np.random.default_rng(3).uniform(-1, 1, 32) * 2.0 ** np.arange(-60, 100, 5)
    terms = [(0, 0, 0, 0, B.NONE, 0, 1.0)]
    got, ref, _, _, _ = run_pair(terms, [a], [h], n, [h], "f64")
    g, r = got[0].reshape(-1), ref[0].reshape(-1)
    assert np.isnan(g[5]) and not np.isfinite(g[4])
    # the accumulation starts from +0, so -0 comes out +0 (as in the oracle)
    assert np.array_equal(np.signbit(g[:2]), np.signbit(r[:2])) and np.all(g[:2] == 0)
    m = np.isfinite(r)
    assert np.all(np.abs(g[m] - r[m]) <= 2.0 ** -46 * np.abs(r[m]))


def test_error_after_200_heat_sweeps_reported():
    """Pair arithmetic over the heat workload's 200 sweeps (64^3, seed 202,
    fused L2 residual every 10) against the FP64 oracle, gated by the bound the
    arithmetic gives: each sweep errs by at most c 2^-47 S(p) (the split loses
    below 2^-47 |x| per term, the two-sums and the final rounding add a few
    such units; c = 16), S(p) the absolute stencil of that sweep; the updates
    (lambda = 1/8) have non-negative weights on u summing to 1, so an error
    never grows from one sweep to the next, and after N sweeps
    |g - o| <= c 2^-47 sum_i max_p S_i(p).  The fused sweeps' form
    u + lambda r has S at most the plain form's plus 12 lambda |u|."""
    n = 64
    u0, f = I.heat3d(202, n)
    shape, h = (n, n, n), (1, 1, 1)
    u, v = B.Grid(shape, h).upload(u0), B.Grid(shape, h).upload(u0)
    F = B.Grid(shape, h).upload(f)
    fused, plain = B.Stencil(S.heat7_fused(0.125)), B.Stencil(S.heat7(0.125))
    res = []
    for _ in range(20):
        res.append(B.do_reduce(B.L2, fused, [u, F], [v]))
        B.swap(u, v)
        B.do_all(plain, [u, F], [v], sweeps=9)
        B.swap(u, v)
    got = u.download().numpy()
    ou, ores = D.heat_run(O.Grid(u0.copy(), h), O.Grid(f.copy(), h), 0.125, 200, every=10)
    # the bound: the oracle's absolute stencil of every sweep along the way
    terms = D.heat_terms(0.125, True)
    f_o = O.Grid(f.copy(), h)
    cur, bound = O.Grid(u0.copy(), h), 0.0
    for _ in range(200):
        Sab = O.zeros(shape, h)
        O.do_all(terms, [cur, f_o], [Sab], abs_mode=True)
        bound += 16 * 2.0 ** -47 * (float(np.max(Sab.interior())) + 1.5 * float(np.max(np.abs(cur.interior()))))
        nxt = cur.copy()
        O.do_all(terms, [cur, f_o], [nxt])
        cur = nxt
    abs_err = float(np.max(np.abs(got - ou.a)))
    err = abs_err / np.max(np.abs(ou.a))
    rerr = max(abs(a - b) / b for a, b in zip(res, ores))
    print(f"heat3d 64^3 f64 pair: |u_200 - oracle|_inf / |oracle|_inf = {err:.3e} "
          f"(absolute {abs_err:.3e}, bound {bound:.3e}); max relative residual error = {rerr:.3e}")
    assert abs_err <= bound
    assert rerr <= 1e-11


def test_batch_in_pair_mode_matches_single_grids():
    """A batch planned in pair mode sweeps each instance exactly like
    gscl_do_all on that instance alone in pair mode (same kernel
    arithmetic), and its per-instance L2 norms agree to rounding."""
    shapes = [(33, 40, 35), (64, 17, 50), (90, 90, 20)]
    h = (1, 1, 1)
    op = S.heat7(0.125, with_f=False)
    insts, hosts = [], []
    for k, n in enumerate(shapes):
        u0 = I.random_interior(60 + k, n, h, -1.0, 1.0)
        hosts.append(u0)
        insts.append(([B.Grid(n, h).upload(u0)], [B.Grid(n, h).upload(u0)]))
    batch = B.Batch(op, insts)
    batch.run(4)  # like gscl_do_all, out[0] names the result after the run
    res = torch.zeros(len(shapes), dtype=torch.float64, device="cuda")
    fused = B.Batch(S.heat7_fused(0.125, with_f=False), [([outs[0]], [ins[0]]) for ins, outs in insts])
    fused.reduce(B.L2, res)
    for (ins, outs), u0, n, r in zip(insts, hosts, shapes, res.cpu().tolist()):
        u, v = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(u0)
        B.do_all(op, [u], [v], sweeps=4)
        assert torch.equal(outs[0].download(), v.download())
        ref = B.do_reduce(B.L2, S.heat7_fused(0.125, with_f=False), [v], [u])
        assert abs(r - ref) <= 1e-13 * ref


@pytest.mark.parametrize("omega", [1.0, 1.6])
@pytest.mark.parametrize("n", [(130, 21, 9), (256, 8, 5)])
def test_redblack_in_pair_arithmetic(omega, n, monkeypatch):
    """Red-black SOR in place in pair arithmetic: the colour-compacted and the
    predicated kernels agree bit for bit, and both stay within the FP64
    tolerance of the oracle over three half-sweeps."""
    h = (1, 1, 1)
    u0 = I.random_interior(170, n, h, -1.0, 1.0, halo_value=0.25)
    f0 = I.random_interior(171, n, h, -1.0, 1.0)
    terms = S.poisson_sor(omega)
    got = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("GSCL_COLOR_COMPACT", flag)
        gu, gf = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(f0)
        B.do_colored(terms, [gu, gf], [gu], color=1, half_sweeps=3)
        got[flag] = gu.download()
    assert torch.equal(got["1"], got["0"])
    ou, of = O.Grid(u0.copy(), h), O.Grid(f0.copy(), h)
    for s in range(3):
        O.do_colored((1 + s) % 2, terms, [ou, of], [ou])
    assert np.max(np.abs(got["1"].numpy() - ou.a)) <= TOL * 8 * max(1.0, np.max(np.abs(ou.a)))
