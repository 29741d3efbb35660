"""GPU parity of the ordered iteration spaces (Section 3: do_j_inc/dec,
do_k_inc/dec) against the oracle: integer running sums are bit-exact in
FP64 and FP32 (every partial sum is an integer below 2^24), random
bidiagonal substitutions match within tolerance, and the alias rules are
enforced."""
import numpy as np
import pytest
import torch

from gpu_common import as_storage, ordered_shape_terms
from oracle import oracle as O
from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I

pytestmark = pytest.mark.gpu

NONE, VALUE = B.NONE, B.VALUE
STEP = {B.I_INC: (-1, 0, 0), B.I_DEC: (1, 0, 0), B.J_INC: (0, -1, 0), B.J_DEC: (0, 1, 0), B.K_INC: (0, 0, -1),
        B.K_DEC: (0, 0, 1)}


def integer_grid(seed, n, h, lo=-50, hi=50):
    a = np.zeros(I.padded_shape(n, h))
    rng = np.random.default_rng(seed)
    I.interior_view(a, n, h)[...] = rng.integers(lo, hi, size=(n[2], n[1], n[0]))
    return a


def run_both(order, terms, arrays, h, n, dtype, n_out=1, alias=(0,), rng=None):
    """arrays[0 .. n_out-1] are the outputs (also bound as inputs 0 .. n_out-1);
    the rest are read-only inputs.  Returns (gpu outputs, oracle outputs)."""
    gg = [B.Grid(n, h, dtype).upload(a) for a in arrays]
    B.do_ordered(order, terms, gg, gg[:n_out], rng=rng)
    got = [g.download().double().numpy() for g in gg[:n_out]]
    og = [O.Grid(as_storage(a, dtype), h) for a in arrays]
    lo, hi = (rng if rng is not None else (None, None))
    O.do_ordered(order, terms, og, og[:n_out], lo=lo, hi=hi)
    return got, [g.a for g in og[:n_out]]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("order", [B.K_INC, B.K_DEC, B.J_INC, B.J_DEC, B.I_INC, B.I_DEC])
def test_running_sum_bitexact(order, dtype):
    n, h = (131, 37, 29), (1, 1, 1)
    x0 = integer_grid(1, n, h, -3, 3)       # the halo seeds the recurrence (interior overwritten)
    f = integer_grid(2, n, h)
    d = STEP[order]
    terms = [(d[0], d[1], d[2], 0, NONE, 0, 1.0), (0, 0, 0, 1, NONE, 0, 1.0)]
    got, want = run_both(order, terms, [x0, f], h, n, dtype)
    assert np.array_equal(got[0], want[0])


@pytest.mark.parametrize("order", [B.K_INC, B.K_DEC, B.J_INC, B.I_INC, B.I_DEC])
def test_subrange_reads_untouched_interior_first(order):
    """A range not starting at the boundary: the first element reads the
    grid's existing value just outside the range."""
    n, h = (70, 20, 24), (1, 1, 1)
    x0 = integer_grid(3, n, h)
    f = integer_grid(4, n, h)
    d = STEP[order]
    terms = [(d[0], d[1], d[2], 0, NONE, 0, 1.0), (0, 0, 0, 1, NONE, 0, 2.0)]
    got, want = run_both(order, terms, [x0, f], h, n, "f64", rng=((3, 2, 5), (61, 17, 19)))
    assert np.array_equal(got[0], want[0])


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 1e-5)])
def test_bidiagonal_substitution(dtype, tol):
    """Two recurrences in one call: x(k) = g(k) - m(k) x(k-1) (coefficient
    grid m) and y(k) = g(k) / 2 + y(k-1) / 4; random data, tolerance relative
    to the largest magnitude (FP32 storage rounds every stored element)."""
    n, h = (96, 40, 33), (1, 1, 1)
    g = I.random_interior(5, n, h, -1.0, 1.0)
    m = I.random_interior(6, n, h, -0.9, 0.9)
    x, y = np.zeros_like(g), np.zeros_like(g)
    terms = [(0, 0, 0, 2, NONE, 0, 1.0), (0, 0, -1, 0, 3, 0, -1.0),
             (0, 0, 0, 2, NONE, 1, 0.5), (0, 0, -1, 1, NONE, 1, 0.25)]
    got, want = run_both(B.K_INC, terms, [x, y, g, m], h, n, dtype, n_out=2)
    for a, b in zip(got, want):
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b))


def test_value_terms_feed_outputs():
    """The returned value computed per element and read by the output terms:
    x(k) = v, v = x(k-1) + f(k) (a running sum through the value)."""
    n, h = (64, 9, 17), (1, 1, 1)
    f = integer_grid(7, n, h)
    x = np.zeros_like(f)
    terms = [(0, 0, -1, 0, NONE, VALUE, 1.0), (0, 0, 0, 1, NONE, VALUE, 1.0), (0, 0, 0, VALUE, NONE, 0, 1.0)]
    gx, gf = B.Grid(n, h).upload(x), B.Grid(n, h).upload(f)
    B.do_ordered(B.K_INC, terms, [gx, gf], [gx])
    want = np.cumsum(I.interior_view(f, n, h), axis=0)
    assert np.array_equal(I.interior_view(gx.download().numpy(), n, h), want)


def test_alias_rules_and_unsupported_axis():
    n, h = (32, 8, 8), (1, 1, 1)
    gx = B.Grid(n, h).upload(np.zeros(I.padded_shape(n, h)))
    gf = B.Grid(n, h).upload(integer_grid(8, n, h))
    with pytest.raises(B.GsclError) as e:   # K_DEC's predecessor is (0, 0, +1), not (0, 0, -1)
        B.do_ordered(B.K_DEC, [(0, 0, -1, 0, NONE, 0, 1.0), (0, 0, 0, 1, NONE, 0, 1.0)], [gx, gf], [gx])
    assert e.value.status == 3  # GSCL_ERR_ALIAS
    with pytest.raises(B.GsclError) as e:   # a neighbouring column is not ordered
        B.do_ordered(B.K_INC, [(1, 0, -1, 0, NONE, 0, 1.0)], [gx, gf], [gx])
    assert e.value.status == 3
    with pytest.raises(B.GsclError) as e:   # along x: at most 8 distinct loads per element
        B.do_ordered(B.I_INC, [(dx, dy, 0, 1, NONE, 0, 1.0) for dx in (-1, 0, 1) for dy in (-1, 0, 1)], [gx, gf],
                     [gx])
    assert e.value.status == 10  # GSCL_ERR_UNSUPPORTED
    # reading the output at offset 0 (its old value) is allowed
    B.do_ordered(B.K_INC, [(0, 0, 0, 0, NONE, 0, 2.0), (0, 0, 0, 1, NONE, 0, 1.0)], [gx, gf], [gx])
    B.sync()



@pytest.mark.parametrize("n", [(67, 13, 37), (40, 16, 32), (33, 5, 1)])
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("order", [B.K_INC, B.K_DEC, B.J_INC, B.J_DEC])
@pytest.mark.parametrize("shape", range(5))
def test_compiled_recurrence_matches_interpreted_and_oracle(shape, order, dtype, n, monkeypatch):
    """The compiled recurrences run the interpreted loop's operations in the
    same order: bit-identical results, on columns shorter than, equal to and
    longer than the look-ahead (with a ragged tail), and close to the FP64
    oracle (FP32 / BF16 storage rounds every stored element)."""
    h = (1, 1, 1)
    terms = ordered_shape_terms(shape, order)
    arrays = [I.random_interior(40 + shape, n, h, -1.0, 1.0, halo_value=0.5),
              I.random_interior(50 + shape, n, h, -1.0, 1.0)]
    if shape >= 2:
        arrays.append(I.random_interior(60 + shape, n, h, -0.9, 0.9))

    def run():
        gg = [B.Grid(n, h, dtype).upload(a) for a in arrays]
        path = B.ordered_specialization(order, terms, gg, gg[:1])
        B.do_ordered(order, terms, gg, gg[:1])
        return path, gg[0].download()

    monkeypatch.delenv("GSCL_GENERIC_ONLY", raising=False)
    path, got = run()
    assert path == shape
    monkeypatch.setenv("GSCL_GENERIC_ONLY", "1")
    path_i, got_i = run()
    assert path_i == (-2 if dtype == "bf16" else -1)
    assert torch.equal(got, got_i)

    og = [O.Grid(as_storage(a, dtype), h) for a in arrays]
    O.do_ordered(order, terms, og, og[:1])
    want = I.interior_view(og[0].a, n, h)
    mine = I.interior_view(got.double().numpy(), n, h)
    tol = {"f64": 1e-13, "f32": 1e-5, "bf16": 5e-2}[dtype]
    assert np.max(np.abs(mine - want)) <= tol * max(1.0, np.max(np.abs(want)))



@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 1e-5), ("bf16", 5e-2)])
@pytest.mark.parametrize("order", [B.I_INC, B.I_DEC])
@pytest.mark.parametrize("n", [(100, 37, 5), (32, 40, 3), (70, 1, 33), (1, 9, 4), (150, 5, 2)])
def test_rows_along_x_match_oracle(order, dtype, tol, n):
    """do_i_inc / do_i_dec: rows staged through shared memory in chunks of 16
    steps by a second warp (FP64) or of 64 steps (row lengths 1, 32, 70, 100,
    150: partial, single, and up to ten chunks; row counts not a multiple of
    32), the five
    compiled recurrence structures and an interpreted two-output bidiagonal
    pair, against the oracle."""
    h = (1, 1, 1)
    d = STEP[order]
    x0 = I.random_interior(140, n, h, -1.0, 1.0, halo_value=0.5)
    f = I.random_interior(141, n, h, -1.0, 1.0)
    m = I.random_interior(142, n, h, -0.9, 0.9)
    cases = [ordered_shape_terms(k, order) for k in range(5)]
    cases.append([(0, 0, 0, 2, NONE, 0, 1.0), (*d, 0, 3, 0, -1.0), (0, 0, 0, 2, NONE, 1, 0.5), (*d, 1, NONE, 1, 0.25)])
    for k, terms in enumerate(cases):
        if k < 5:
            arrays = [x0, f] + ([m] if k >= 2 else [])
            got, want = run_both(order, terms, arrays, h, n, dtype)
        else:
            got, want = run_both(order, terms, [x0, x0.copy(), f, m], h, n, dtype, n_out=2)
        for a, b in zip(got, want):
            assert np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b))), (k, order, dtype, n)
        gg = [B.Grid(n, h, dtype).upload(a) for a in ([x0, f, m] if k != 5 else [x0, x0, f, m])]
        assert B.ordered_specialization(order, terms, gg, gg[:1] if k != 5 else gg[:2]) == (k if k < 5 else -3)



@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 1e-5), ("bf16", 5e-2)])
@pytest.mark.parametrize("order", [B.I_INC, B.I_DEC])
@pytest.mark.parametrize("n", [(150, 5, 3), (33, 40, 2)])
def test_rows_along_x_eight_loads_three_outputs(order, dtype, tol, n):
    """Rows along x at the largest staging: 8 distinct loads (one grid at five
    offsets across rows and planes, one at two offsets along x, one behind)
    and 3 outputs, two of them recurrences; against the oracle."""
    h = (2, 1, 1)
    d = STEP[order]
    arrays = [I.random_interior(160 + k, n, h, -1.0, 1.0, halo_value=0.5) for k in range(6)]
    x, y, z, a, b, c = range(6)
    terms = [(0, 0, 0, a, NONE, 0, 1.0), (0, 1, 0, a, NONE, 0, 0.1), (0, -1, 0, a, NONE, 0, 0.1),
             (0, 0, 1, a, NONE, 0, 0.1), (0, 0, -1, a, NONE, 0, 0.1), (*d, x, NONE, 0, -0.5),
             (0, 0, 0, b, NONE, 1, 0.5), (2, 0, 0, b, NONE, 1, 0.25), (*d, y, NONE, 1, 0.3),
             (-1, 0, 0, c, NONE, 2, 1.0), (0, 0, 0, a, NONE, 2, 0.5)]
    got, want = run_both(order, terms, arrays, h, n, dtype, n_out=3)
    for g, w in zip(got, want):
        assert np.max(np.abs(g - w)) <= tol * max(1.0, np.max(np.abs(w))), (order, dtype, n)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("order", [B.I_INC, B.I_DEC])
def test_rows_along_x_compiled_equal_interpreted(order, dtype, monkeypatch):
    n, h = (77, 33, 3), (1, 1, 1)
    arrays = [I.random_interior(150, n, h, -1.0, 1.0, halo_value=0.5), I.random_interior(151, n, h, -1.0, 1.0),
              I.random_interior(152, n, h, -0.9, 0.9)]
    for shape in range(5):
        terms = ordered_shape_terms(shape, order)
        got = {}
        for flag in ("0", "1"):
            monkeypatch.setenv("GSCL_GENERIC_ONLY", flag)
            gg = [B.Grid(n, h, dtype).upload(a) for a in arrays[:3 if shape >= 2 else 2]]
            B.do_ordered(order, terms, gg, gg[:1])
            got[flag] = gg[0].download()
        assert torch.equal(got["0"], got["1"]), shape
