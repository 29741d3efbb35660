"""GPU parity of red-black colouring (Section 3, stateful stencils) against
the oracle: Gauss-Seidel and SOR half-sweeps in place on 3D and 2D grids,
sub-ranges whose colour follows the interior index, the compiled and the
generic kernels, and the alias rules."""
import numpy as np
import pytest
import torch

from gpu_common import as_storage
from oracle import oracle as O
from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-13, "f32": 3e-6, "bf16": 2e-2}


@pytest.fixture(params=["compiled", "generic", "uncompacted"])
def kernel_path(request, monkeypatch):
    """compiled: the operator tables (FP64 star operators: colour-compacted,
    each thread computing only the colour's elements); generic: the runtime
    term loop; uncompacted: the tables evaluating both colours and storing one."""
    monkeypatch.delenv("GSCL_GENERIC_ONLY", raising=False)
    monkeypatch.delenv("GSCL_COLOR_COMPACT", raising=False)
    if request.param == "generic":
        monkeypatch.setenv("GSCL_GENERIC_ONLY", "1")
    elif request.param == "uncompacted":
        monkeypatch.setenv("GSCL_COLOR_COMPACT", "0")
    return request.param


def run_colored(terms, u0, f0, n, h, dtype, color, half_sweeps, rng=None, ndim=3):
    gu = B.Grid(n, h, dtype, ndim).upload(u0)
    gf = B.Grid(n, h, dtype, ndim).upload(f0)
    B.do_colored(terms, [gu, gf], [gu], color=color, half_sweeps=half_sweeps, rng=rng)
    got = gu.download().double().numpy()
    ou = O.Grid(as_storage(u0, dtype), h)
    of = O.Grid(as_storage(f0, dtype), h)
    lo, hi = rng if rng is not None else (None, None)
    for s in range(half_sweeps):
        O.do_colored((color + s) % 2, terms, [ou, of], [ou], lo=lo, hi=hi)
    return got, ou.a


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("omega", [1.0, 1.4])
@pytest.mark.parametrize("n,rng", [((70, 21, 19), None), ((131, 40, 9), ((3, 5, 1), (128, 37, 8)))])
def test_redblack_in_place_matches_oracle(kernel_path, dtype, omega, n, rng):
    """Three half-sweeps (colour 1, 0, 1) in place; the range's odd start
    checks that the colour follows the interior index, not the range."""
    h = (1, 1, 1)
    u0 = I.random_interior(71, n, h, -1.0, 1.0, halo_value=0.25)
    f0 = I.random_interior(72, n, h, -1.0, 1.0)
    got, want = run_colored(S.poisson_sor(omega), u0, f0, n, h, dtype, 1, 3, rng)
    scale = max(1.0, np.max(np.abs(want)))
    assert np.max(np.abs(got - want)) <= TOL[dtype] * 4 * scale


def test_redblack_2d_jacobi_operator(kernel_path):
    n, h = (150, 77, 1), (1, 1, 0)
    u0 = I.random_interior(73, n, h, -1.0, 1.0, halo_value=1.0)
    gu = B.Grid(n, h, "f64", 2).upload(u0)
    B.do_colored(S.jacobi5_2d(), [gu], [gu], color=0, half_sweeps=4)
    ou = O.Grid(u0.copy(), h)
    for s in range(4):
        O.do_colored(s % 2, S.jacobi5_2d(), [ou], [ou])
    assert np.max(np.abs(gu.download().numpy() - ou.a)) <= 1e-14


@pytest.mark.parametrize("n", [(256, 9, 6), (130, 17, 5), (37, 4, 3)])
def test_compacted_equals_uncompacted_bit_for_bit(n, monkeypatch):
    """The colour-compacted FP64 kernel and the one evaluating both colours
    run the same operations per element: identical results, on widths that
    fill whole 128-column tiles, leave a ragged tile, or fit in one."""
    h = (1, 1, 1)
    u0 = I.random_interior(77, n, h, -1.0, 1.0, halo_value=0.5)
    f0 = I.random_interior(78, n, h, -1.0, 1.0)
    got = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("GSCL_COLOR_COMPACT", flag)
        for omega in (1.0, 1.7):
            gu, gf = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(f0)
            B.do_colored(S.poisson_sor(omega), [gu, gf], [gu], color=1, half_sweeps=5, rng=((1, 0, 1), n))
            got[flag, omega] = gu.download()
    for omega in (1.0, 1.7):
        assert torch.equal(got["1", omega], got["0", omega])


def test_redblack_converges_like_the_oracle():
    """Twenty Gauss-Seidel iterations: the same iterate, and a residual far
    below Jacobi's after as many sweeps."""
    n, h = (64, 64, 64), (1, 1, 1)
    u0 = np.zeros(I.padded_shape(n, h))
    f0 = I.random_interior(74, n, h, -1.0, 1.0)
    got, want = run_colored(S.poisson_sor(1.0), u0, f0, n, h, "f64", 0, 40)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_colored_leaves_the_other_colour_untouched():
    """Out of place: the output keeps its content at the other colour."""
    n, h = (40, 12, 7), (1, 1, 1)
    u0 = I.random_interior(75, n, h, -1.0, 1.0)
    f0 = I.random_interior(76, n, h, -1.0, 1.0)
    gu, gf = B.Grid(n, h).upload(u0), B.Grid(n, h).upload(f0)
    gv = B.Grid(n, h).upload(np.full(I.padded_shape(n, h), 7.0))
    B.do_colored(S.poisson_jacobi(), [gu, gf], [gv], color=1)
    got = I.interior_view(gv.download().numpy(), n, h)
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    other = (i + j + k) % 2 == 0
    assert np.all(got[other] == 7.0)
    ov = O.Grid(np.full(I.padded_shape(n, h), 7.0), h)
    O.do_colored(1, S.poisson_jacobi(), [O.Grid(u0, h), O.Grid(f0, h)], [ov])
    assert np.max(np.abs(got - I.interior_view(ov.a, n, h))) <= 1e-15


def test_colored_alias_and_argument_errors():
    n, h = (32, 8, 8), (1, 1, 1)
    gu = B.Grid(n, h).upload(np.zeros(I.padded_shape(n, h)))
    gf = B.Grid(n, h).upload(np.zeros(I.padded_shape(n, h)))
    with pytest.raises(B.GsclError) as e:       # (1, 1, 0) is the same colour
        B.do_colored([(1, 1, 0, 0, B.NONE, 0, 1.0)], [gu], [gu])
    assert e.value.status == 3
    with pytest.raises(B.GsclError) as e:
        B.do_colored(S.poisson_jacobi(), [gu, gf], [gu], color=2)
    assert e.value.status == 1
    with pytest.raises(B.GsclError) as e:
        B.do_colored(S.poisson_jacobi(), [gu, gf], [gu], half_sweeps=0)
    assert e.value.status == 1
    # odd offsets (1, 1, 1) and (-1, 0, 0) read the other colour: allowed in place
    B.do_colored([(1, 1, 1, 0, B.NONE, 0, 0.5), (-1, 0, 0, 0, B.NONE, 0, 0.5)], [gu], [gu])
    B.sync()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("graph", [False, True])
def test_colored_batch_equals_each_instance_alone(kernel_path, dtype, graph):
    """A coloured batch of uneven instances, each with its own SOR factor:
    five half-sweeps of all of them (one launch per half-sweep) give, bit for
    bit, what gscl_do_colored gives on each instance alone, and stay within
    tolerance of the oracle."""
    h = (1, 1, 1)
    sides = [(70, 21, 19), (33, 64, 12), (130, 9, 25), (5, 3, 2), (256, 17, 6)]
    omegas = [1.05, 1.3, 1.7, 1.9, 1.55]
    u0s = [I.random_interior(80 + k, n, h, -1.0, 1.0, halo_value=0.25) for k, n in enumerate(sides)]
    f0s = [I.random_interior(90 + k, n, h, -1.0, 1.0) for k, n in enumerate(sides)]
    alone = []
    for n, w, u0, f0 in zip(sides, omegas, u0s, f0s):
        gu, gf = B.Grid(n, h, dtype).upload(u0), B.Grid(n, h, dtype).upload(f0)
        B.do_colored(S.poisson_sor(w), [gu, gf], [gu], color=1, half_sweeps=5)
        alone.append(gu.download())
    grids = [(B.Grid(n, h, dtype).upload(u0), B.Grid(n, h, dtype).upload(f0))
             for n, u0, f0 in zip(sides, u0s, f0s)]
    batch = B.ColoredBatch([S.poisson_sor(w) for w in omegas], [([gu, gf], [gu]) for gu, gf in grids])
    batch.run_colored(1, 5, graph=graph)
    for k, ((gu, _), want) in enumerate(zip(grids, alone)):
        assert torch.equal(gu.download(), want), k
    # the oracle, on the instance with the largest factor
    k = 3
    ou, of = O.Grid(as_storage(u0s[k], dtype), h), O.Grid(as_storage(f0s[k], dtype), h)
    for s in range(5):
        O.do_colored((1 + s) % 2, S.poisson_sor(omegas[k]), [ou, of], [ou])
    got = grids[k][0].download().double().numpy()
    assert np.max(np.abs(got - ou.a)) <= TOL[dtype] * 4 * max(1.0, np.max(np.abs(ou.a)))
    # a second group continues from where the first left the grids
    batch.run_colored(0, 2, graph=graph)
    gu, gf = B.Grid(sides[0], h, dtype).upload(u0s[0]), B.Grid(sides[0], h, dtype).upload(f0s[0])
    B.do_colored(S.poisson_sor(omegas[0]), [gu, gf], [gu], color=1, half_sweeps=5)
    B.do_colored(S.poisson_sor(omegas[0]), [gu, gf], [gu], color=0, half_sweeps=2)
    assert torch.equal(grids[0][0].download(), gu.download())


def test_colored_batch_2d_instances():
    """2D instances of the 5-point Jacobi operator, in place by colour."""
    h = (1, 1, 0)
    sides = [(150, 77, 1), (64, 300, 1), (9, 5, 1)]
    u0s = [I.random_interior(100 + k, n, h, -1.0, 1.0, halo_value=1.0) for k, n in enumerate(sides)]
    grids = [B.Grid(n, h, "f64", 2).upload(u0) for n, u0 in zip(sides, u0s)]
    B.ColoredBatch([S.jacobi5_2d()] * 3, [([g], [g]) for g in grids]).run_colored(0, 4)
    for g, n, u0 in zip(grids, sides, u0s):
        ou = O.Grid(u0.copy(), h)
        for s in range(4):
            O.do_colored(s % 2, S.jacobi5_2d(), [ou], [ou])
        assert np.max(np.abs(g.download().numpy() - ou.a)) <= 1e-14


def test_colored_batch_argument_errors():
    n, h = (32, 8, 8), (1, 1, 1)
    gu, gf = B.Grid(n, h).zero(), B.Grid(n, h).zero()
    gv, gw = B.Grid(n, h).zero(), B.Grid(n, h).zero()
    with pytest.raises(B.GsclError) as e:          # the second operator has another structure
        B.ColoredBatch([S.poisson_sor(1.5), S.poisson_jacobi()[:-1]], [([gu, gf], [gu]), ([gv, gw], [gv])])
    assert e.value.status == 1
    with pytest.raises(B.GsclError) as e:          # same-colour read of the output in place
        B.ColoredBatch([[(1, 1, 0, 0, B.NONE, 0, 1.0)]], [([gu], [gu])])
    assert e.value.status == 3
    b = B.ColoredBatch([S.poisson_sor(1.5), S.poisson_sor(1.2)], [([gu, gf], [gu]), ([gv, gw], [gv])])
    with pytest.raises(B.GsclError):
        b.run(1)                                   # a coloured batch runs by colour only
    with pytest.raises(B.GsclError):
        b.run_colored(2, 1)
    with pytest.raises(B.GsclError):
        b.run_colored(0, 0)
    B.sync()
