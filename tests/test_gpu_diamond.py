"""GPU parity of do_diamond (Section 3: (i-1, j) and (i, j-1) before (i, j))
against the oracle: summed-area tables bit-exact on integer data, random
operators reading the output on both sides of the wavefront, natural-order
Gauss-Seidel, several tiles with ragged edges, 2D and 3D grids, sub-ranges."""
import numpy as np
import pytest
import torch

from gpu_common import as_storage
from oracle import oracle as O
from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I

pytestmark = pytest.mark.gpu

NONE = B.NONE
SAT = [(0, 0, 0, 1, NONE, 0, 1.0), (-1, 0, 0, 0, NONE, 0, 1.0), (0, -1, 0, 0, NONE, 0, 1.0),
       (-1, -1, 0, 0, NONE, 0, -1.0)]
GS5 = [(1, 0, 0, 0, NONE, 0, 0.25), (-1, 0, 0, 0, NONE, 0, 0.25), (0, 1, 0, 0, NONE, 0, 0.25),
       (0, -1, 0, 0, NONE, 0, 0.25), (0, 0, 0, 1, NONE, 0, 0.25)]
MIXED = [(-1, 0, 0, 0, NONE, 0, 0.3), (0, -1, 0, 0, NONE, 0, 0.2), (-1, -1, 0, 0, NONE, 0, -0.1),
         (1, 0, 0, 0, NONE, 0, 0.15), (0, 1, 0, 0, NONE, 0, 0.25), (1, 1, 0, 0, 1, 0, 0.05),
         (0, 0, 0, 0, NONE, 0, -0.4), (1, -1, 0, 1, NONE, 0, 0.5)]


def integer_grid(seed, n, h, lo, hi):
    a = np.zeros(I.padded_shape(n, h))
    I.interior_view(a, n, h)[...] = np.random.default_rng(seed).integers(lo, hi, size=n[::-1])
    return a


def run_both(terms, arrays, n, h, dtype, rng=None):
    ndim = 2 if (n[2] == 1 and h[2] == 0) else 3
    gg = [B.Grid(n, h, dtype, ndim).upload(a) for a in arrays]
    B.do_diamond(terms, gg, gg[:1], rng=rng)
    got = gg[0].download().double().numpy()
    og = [O.Grid(as_storage(a, dtype), h) for a in arrays]
    lo, hi = rng if rng is not None else (None, None)
    O.do_diamond(terms, og, og[:1], lo=lo, hi=hi)
    return got, og[0].a


@pytest.fixture(params=["compiled", "interpreted"])
def kernel_path(request, monkeypatch):
    """compiled: the summed-area table and natural-order Gauss-Seidel shapes
    with constant offsets; interpreted: the runtime term loop."""
    monkeypatch.delenv("GSCL_GENERIC_ONLY", raising=False)
    if request.param == "interpreted":
        monkeypatch.setenv("GSCL_GENERIC_ONLY", "1")
    return request.param


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,h,rng", [((100, 70, 1), (1, 1, 0), None), ((40, 37, 5), (1, 1, 1), None),
                                     ((129, 65, 3), (1, 1, 1), ((5, 3, 1), (120, 64, 3)))])
def test_summed_area_table_bitexact(kernel_path, dtype, n, h, rng):
    x0 = integer_grid(1, n, h, -3, 3)   # the halo rows/columns seed the sums (interior overwritten)
    f = integer_grid(2, n, h, -20, 20)
    got, want = run_both(SAT, [x0, f], n, h, dtype, rng)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 2e-5), ("bf16", 5e-2)])
@pytest.mark.parametrize("n,h", [((75, 66, 1), (1, 1, 0)), ((33, 40, 4), (1, 1, 1))])
def test_operator_reading_both_sides_of_the_wavefront(dtype, tol, n, h):
    x0 = I.random_interior(3, n, h, -1.0, 1.0, halo_value=0.5)
    f = I.random_interior(4, n, h, -1.0, 1.0)
    terms = MIXED
    if n[2] > 1:   # reads of another plane (not the output's): global memory
        terms = MIXED + [(0, 0, 1, 1, NONE, 0, 0.1), (1, 0, -1, 1, NONE, 0, -0.2)]
    got, want = run_both(terms, [x0, f], n, h, dtype)
    assert np.max(np.abs(got - want)) <= tol * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("terms", ["gs5", "gs5f", "sor5f", "sat"])
def test_compiled_shapes_equal_interpreted_bit_for_bit(terms, dtype, monkeypatch):
    n, h = (77, 70, 2), (1, 1, 1)
    ops = {"gs5": GS5[:4], "gs5f": GS5,
           "sor5f": [(0, 0, 0, 0, NONE, 0, -0.6)] + [(dx, dy, dz, a, c, o, 0.4) for dx, dy, dz, a, c, o, _ in GS5],
           "sat": SAT}
    op = ops[terms]
    arrays = [I.random_interior(9, n, h, -1.0, 1.0, halo_value=0.25), I.random_interior(10, n, h, -1.0, 1.0)]
    if terms == "gs5":
        arrays = arrays[:1]
    got = {}
    for flag in ("0", "1"):
        monkeypatch.setenv("GSCL_GENERIC_ONLY", flag)
        gg = [B.Grid(n, h, dtype).upload(a) for a in arrays]
        B.do_diamond(op, gg, gg[:1], rng=((2, 1, 0), (77, 70, 2)))
        got[flag] = gg[0].download()
    assert torch.equal(got["0"], got["1"])


def test_natural_order_gauss_seidel_sweeps(kernel_path):
    n, h = (96, 80, 1), (1, 1, 0)
    u0 = I.random_interior(5, n, h, -1.0, 1.0, halo_value=1.0)
    f = I.random_interior(6, n, h, -1.0, 1.0)
    gu, gf = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(f)
    ou, of = O.Grid(u0.copy(), h), O.Grid(f.copy(), h)
    for _ in range(5):
        B.do_diamond(GS5, [gu, gf], [gu])
        O.do_diamond(GS5, [ou, of], [ou])
    assert np.max(np.abs(gu.download().numpy() - ou.a)) <= 1e-13


def test_out_of_place_and_two_outputs():
    """Output 0 is the recurrence (in place), output 1 a separate grid written
    from the same element's inputs."""
    n, h = (70, 45, 2), (1, 1, 1)
    x0 = integer_grid(7, n, h, -2, 2)
    f = integer_grid(8, n, h, -9, 9)
    terms = SAT + [(0, 0, 0, 1, NONE, 1, 2.0), (-1, 0, 0, 0, NONE, 1, 1.0)]
    gx, gf = B.Grid(n, h).upload(x0), B.Grid(n, h).upload(f)
    gy = B.Grid(n, h).upload(np.full(I.padded_shape(n, h), 7.0))
    B.do_diamond(terms, [gx, gf], [gx, gy])
    ox, of = O.Grid(x0.copy(), h), O.Grid(f.copy(), h)
    oy = O.Grid(np.full(I.padded_shape(n, h), 7.0), h)
    O.do_diamond(terms, [ox, of], [ox, oy])
    assert np.array_equal(gx.download().numpy(), ox.a)
    assert np.array_equal(gy.download().numpy(), oy.a)
