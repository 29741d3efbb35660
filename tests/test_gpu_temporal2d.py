"""GPU parity of temporal blocking on 2D grids (tb2d_kernel.cuh): K sweeps of
the 5-point Jacobi operator per launch, single grids (gscl_do_all with a
forced or tuned factor) and batches (gscl_batch_set_temporal / tune).

Fused passes evaluate every point with the single sweep's terms, order and
FMAs and take each intermediate sweep's halo from the grid single sweeps
would have written, so both grids of the ping-pong pair must hold, bit for
bit, what single sweeps leave: out[0] the last iterate, in[0] the one before
(the last launch of a run is a single sweep)."""
import numpy as np
import pytest
import torch

from oracle import drivers as D
from oracle import oracle as O
from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S

pytestmark = pytest.mark.gpu

H2 = (1, 1, 0)
SHAPES = [(256, 256), (300, 77), (17, 5), (33, 129)]


def fields(n, seed, dtype):
    """Random interiors; in[0]'s halo 0.375, out[0]'s -0.625 (different on purpose)."""
    shape = (n[0], n[1], 1)
    u0 = I.random_interior(seed, shape, H2, -1.0, 1.0, halo_value=0.375)
    v0 = I.random_interior(seed + 1, shape, H2, -1.0, 1.0, halo_value=-0.625)
    return shape, u0, v0


def single_grid_run(shape, u0, v0, dtype, sweeps, K, tile, monkeypatch):
    monkeypatch.setenv("GSCL_TEMPORAL", str(K))
    monkeypatch.setenv("GSCL_TEMPORAL_TILE", str(tile))
    a, b = B.Grid(shape, H2, dtype, 2).upload(u0), B.Grid(shape, H2, dtype, 2).upload(v0)
    B.do_all(S.jacobi5_2d(), [a], [b], sweeps=sweeps)
    return a.interior().clone(), b.interior().clone()


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("n", SHAPES)
def test_fused_2d_sweeps_bitexact_with_single_sweeps(monkeypatch, dtype, n):
    """21 sweeps: K = 2, 3, 4, 8, 16 over the four tile shapes against K = 1;
    both grids compared (u_21 and u_20)."""
    shape, u0, v0 = fields(n, 81, dtype)
    ref = single_grid_run(shape, u0, v0, dtype, 21, 1, 0, monkeypatch)
    for K in (2, 3, 4, 8, 16):
        for tile in range(4):
            got = single_grid_run(shape, u0, v0, dtype, 21, K, tile, monkeypatch)
            for g, r, name in zip(got, ref, ("in[0] (u_20)", "out[0] (u_21)")):
                d = (g.double() - r.double()).abs()
                assert torch.equal(g, r), (K, tile, name, d.max().item(), int((d > 0).sum()))


@pytest.mark.parametrize("K", [2, 5, 8, 16])
def test_fused_2d_sweeps_bitexact_with_oracle_on_integer_data(monkeypatch, K):
    """Integer data (|u| <= 64) and weights 1/4: after s sweeps every value and
    partial sum is a multiple of 2^-2s of magnitude at most 256, exact in
    FP64 for s <= 22, so the fused passes and the oracle's one-at-a-time
    sweeps agree bit for bit, for u_S and u_{S-1}."""
    rng = np.random.default_rng(90 + K)
    n = (130, 70, 1)
    u0 = rng.integers(-64, 65, size=I.padded_shape(n, H2)).astype(np.float64)
    sweeps = K + 3
    monkeypatch.setenv("GSCL_TEMPORAL", str(K))
    a, b = B.Grid(n, H2, "f64", 2).upload(u0), B.Grid(n, H2, "f64", 2).upload(u0)
    B.do_all(S.jacobi5_2d(), [a], [b], sweeps=sweeps)
    ou, op, _ = D.jacobi2d_run(O.Grid(u0.copy(), H2), sweeps)
    assert np.array_equal(b.download().numpy(), ou.a)
    assert np.array_equal(a.download().numpy(), op.a)


def test_fused_2d_laplace_workload_within_tolerance_of_oracle(monkeypatch):
    """The 2D Laplace workload (256 x 256 FP64, halo sin(pi x)) with 8 sweeps
    fused per launch: u_100, u_99 and their max-abs difference within 1e-13
    of the oracle, relative to max |u|."""
    u0 = I.laplace2d(101, 256)
    n = (256, 256, 1)
    monkeypatch.setenv("GSCL_TEMPORAL", "8")
    a, b = B.Grid(n, H2, "f64", 2).upload(u0), B.Grid(n, H2, "f64", 2).upload(u0)
    B.do_all(S.jacobi5_2d(), [a], [b], sweeps=100)
    res = B.do_reduce(B.MAXABS, S.difference(), [b, a])
    ou, op, ores = D.jacobi2d_run(O.Grid(u0.copy(), H2), 100)
    scale = np.max(np.abs(ou.a))
    assert np.max(np.abs(b.download().numpy() - ou.a)) <= 1e-13 * scale
    assert np.max(np.abs(a.download().numpy() - op.a)) <= 1e-13 * scale
    assert abs(res - ores) <= 1e-13 * scale


def make_batch(sides, dtype, seed):
    """One 2D Jacobi batch over grids of the given sides (different halos in
    in[0] and out[0]); returns the batch and its (a, b) grid pairs."""
    pairs = []
    for i, n in enumerate(sides):
        shape, u0, v0 = fields(n, seed + 2 * i, dtype)
        pairs.append((B.Grid(shape, H2, dtype, 2).upload(u0), B.Grid(shape, H2, dtype, 2).upload(v0)))
    return B.Batch(S.jacobi5_2d(), [([a], [b]) for a, b in pairs]), pairs


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("graph", [False, True])
def test_fused_2d_batch_bitexact_with_single_sweeps(dtype, graph):
    """A batch of uneven 2D grids, K = 3 and 8 per launch over two tile
    shapes, runs of 1, 7 and 20 sweeps in a row: every grid of every instance
    equals the unfused batch's, and out[0] / in[0] hold u_S / u_{S-1}."""
    sides = [(256, 256), (300, 77), (17, 5), (33, 129), (64, 64)]
    ref, rp = make_batch(sides, dtype, 300)
    for sweeps in (1, 7, 20):
        ref.run(sweeps, graph=graph)
    want = [(a.interior().clone(), b.interior().clone()) for a, b in rp]
    for K, tile in ((3, 0), (8, 3)):
        bt, pairs = make_batch(sides, dtype, 300)
        bt.set_temporal(K, tile)
        assert bt.temporal()[0] == K
        for sweeps in (1, 7, 20):
            bt.run(sweeps, graph=graph)
        for (a, b), (wa, wb) in zip(pairs, want):
            assert torch.equal(a.interior(), wa), (K, tile)
            assert torch.equal(b.interior(), wb), (K, tile)


def test_fused_2d_batch_tuner_keeps_bits():
    """gscl_batch_tune on a 2D batch picks a factor and a tile; the tuned batch
    gives the bits of single sweeps (tuning leaves in[0] as it was)."""
    sides = [(256, 256), (100, 37)]
    bt, pairs = make_batch(sides, "f64", 400)
    before = [a.interior().clone() for a, _ in pairs]
    bt.tune(trial_sweeps=8)
    for (a, _), w in zip(pairs, before):
        assert torch.equal(a.interior(), w)
    K, tx, ty = bt.temporal()
    assert 1 <= K <= 16 and (K == 1) == (tx == 0)
    bt.run(30, graph=True)
    ref, rp = make_batch(sides, "f64", 400)
    ref.run(30, graph=True)
    for (a, b), (c, d) in zip(pairs, rp):
        assert torch.equal(a.interior(), c.interior())
        assert torch.equal(b.interior(), d.interior())


def test_tune_sweeps_on_a_2d_grid_keeps_bits(monkeypatch):
    monkeypatch.delenv("GSCL_TEMPORAL", raising=False)
    monkeypatch.delenv("GSCL_TEMPORAL_TILE", raising=False)
    shape, u0, v0 = fields((200, 90), 500, "f64")
    a, b = B.Grid(shape, H2, "f64", 2).upload(u0), B.Grid(shape, H2, "f64", 2).upload(v0)
    k = B.tune_sweeps(S.jacobi5_2d(), [a], [b], trial_sweeps=8)
    assert 1 <= k <= 16
    assert torch.equal(a.download(), torch.from_numpy(u0))  # in[0] untouched
    B.do_all(S.jacobi5_2d(), [a], [b], sweeps=40)
    got = (a.interior().clone(), b.interior().clone())
    ref = single_grid_run(shape, u0, v0, "f64", 40, 1, 0, monkeypatch)
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])


def test_set_temporal_argument_errors():
    bt, _ = make_batch([(40, 30)], "f64", 600)
    for k, t in ((0, 0), (17, 0), (2, -1), (2, 4)):
        with pytest.raises(RuntimeError):
            bt.set_temporal(k, t)
    # a 3D batch does not fuse
    n, h = (20, 20, 20), (1, 1, 1)
    u0 = I.random_interior(601, n, h, -1.0, 1.0)
    g3 = (B.Grid(n, h).upload(u0), B.Grid(n, h).upload(u0))
    b3 = B.Batch(S.heat7(0.125, with_f=False), [([g3[0]], [g3[1]])])
    with pytest.raises(RuntimeError):
        b3.set_temporal(2, 0)
    b3.set_temporal(1, 0)  # K = 1 is always accepted
    assert b3.temporal() == (1, 0, 0)


def test_pair_arithmetic_grids_do_not_fuse(monkeypatch):
    """FP64 grids in FP32-pair arithmetic round differently from the fused
    kernel's IEEE FP64: they never fuse."""
    monkeypatch.delenv("GSCL_TEMPORAL", raising=False)
    shape, u0, v0 = fields((64, 64), 700, "f64")
    a, b = B.Grid(shape, H2, "f64", 2).upload(u0), B.Grid(shape, H2, "f64", 2).upload(v0)
    old = B.get_fp64_arithmetic()
    try:
        B.set_fp64_arithmetic("pair")
        assert B.tune_sweeps(S.jacobi5_2d(), [a], [b], trial_sweeps=8) == 1
    finally:
        B.set_fp64_arithmetic(old)
