"""GPU parity of two-sweep passes in batches of 3D grids (tb2_kernel.cuh in its
work-list form): 3D FP32 / BF16 instances under the 7-point star operators,
two sweeps per launch from the batch's own descriptor tables, bit-identical
to the batch's single sweeps (the pass evaluates every point with the single
sweep's terms and FMAs; the ping-pong grids of an instance carry identical
halos, the precondition of fused 3D passes)."""
import pytest
import torch

from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S

pytestmark = pytest.mark.gpu

H = (1, 1, 1)
# uneven instances: ragged tiles, a grid smaller than one tile, and long z
# columns that split into several runs per CTA
SIDES = [(150, 37, 21), (33, 20, 9), (130, 90, 40), (5, 3, 2), (256, 30, 64)]


def make_batch(op, sides, dtype, seed, rhs):
    insts, grids = [], []
    for i, n in enumerate(sides):
        u0 = I.random_interior(seed + 3 * i, n, H, -1.0, 1.0, halo_value=0.375)
        a, b = B.Grid(n, H, dtype).upload(u0), B.Grid(n, H, dtype).upload(u0)
        ins = [a]
        if rhs:
            ins.append(B.Grid(n, (0, 0, 0), dtype).upload(I.random_interior(seed + 3 * i + 1, n, (0, 0, 0),
                                                                             -1.0, 1.0)))
        insts.append((ins, [b]))
        grids.append((a, b))
    return B.Batch(op, insts), grids


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("which", ["heat", "heat_rhs"])
@pytest.mark.parametrize("graph", [False, True])
def test_two_sweep_batch_bitexact_with_single_sweeps(dtype, which, graph):
    op = {"heat": S.heat7(0.125, with_f=False), "heat_rhs": S.heat7(0.125)}[which]
    rhs = which == "heat_rhs"
    ref, rg = make_batch(op, SIDES, dtype, 900, rhs)
    for sweeps in (1, 5, 8):
        ref.run(sweeps, graph=graph)
    bt, g = make_batch(op, SIDES, dtype, 900, rhs)
    bt.set_temporal(2)
    assert bt.temporal() == (2, 128, 14)
    for sweeps in (1, 5, 8):
        bt.run(sweeps, graph=graph)
    for (a, b), (c, d) in zip(g, rg):
        assert torch.equal(a.interior(), c.interior())
        assert torch.equal(b.interior(), d.interior())


def test_two_sweep_batch_tuner_keeps_bits():
    """gscl_batch_tune times single sweeps against two-sweep passes on a 3D
    batch and keeps the faster; either way the results are those of single
    sweeps, and tuning leaves in[0] as it was."""
    op = S.heat7(0.125, with_f=False)
    bt, g = make_batch(op, SIDES, "f32", 950, False)
    before = [a.interior().clone() for a, _ in g]
    bt.tune(trial_sweeps=6)
    for (a, _), w in zip(g, before):
        assert torch.equal(a.interior(), w)
    K, tx, ty = bt.temporal()
    assert K in (1, 2) and (K == 1) == (tx == 0)
    bt.run(9, graph=True)
    ref, rg = make_batch(op, SIDES, "f32", 950, False)
    ref.run(9, graph=True)
    for (a, b), (c, d) in zip(g, rg):
        assert torch.equal(a.interior(), c.interior())
        assert torch.equal(b.interior(), d.interior())


def test_two_sweep_batch_refuses_other_factors():
    op = S.heat7(0.125, with_f=False)
    bt, _ = make_batch(op, SIDES[:2], "f32", 990, False)
    with pytest.raises(RuntimeError):
        bt.set_temporal(3)
    bt.set_temporal(2)
    bt.set_temporal(1)
    assert bt.temporal() == (1, 0, 0)
