"""Batched sweeps: many uneven instances in one launch per sweep.

A batch must give each instance exactly what gscl_do_all gives it alone
(bit-identical: same point arithmetic, only the schedule differs), with and
without CUDA-graph replay and across ping-pong parities; per-instance
reductions must agree with gscl_do_reduce alone and with the oracle."""
import math

import numpy as np
import pytest
import torch

from gpu_common import TOL
from oracle import drivers as D
from oracle import oracle as O
from paper_1207_1746_b300 import binding as B
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import stencils as S

pytestmark = pytest.mark.gpu

SHAPES = [(33, 40, 35), (64, 17, 50), (90, 90, 20), (31, 64, 64), (130, 10, 40), (7, 5, 3)]
H = (1, 1, 1)


@pytest.fixture(params=["compiled", "generic", "narrow"])
def kernel_path(request, monkeypatch):
    """compiled: the operator tables; generic: the runtime term loop; narrow:
    the tables on 64-column tiles with 4 rows per warp (FP32 / BF16 batches)."""
    monkeypatch.delenv("GSCL_GENERIC_ONLY", raising=False)
    monkeypatch.delenv("GSCL_BATCH_NARROW", raising=False)
    if request.param == "generic":
        monkeypatch.setenv("GSCL_GENERIC_ONLY", "1")
    elif request.param == "narrow":
        monkeypatch.setenv("GSCL_BATCH_NARROW", "1")
    return request.param


def make_instances(dtype, with_f, seed=0, halo_value=0.0):
    insts, host = [], []
    for k, n in enumerate(SHAPES):
        u0 = I.random_interior(seed + 10 * k, n, H, -1.0, 1.0, halo_value=halo_value)
        u, v = B.Grid(n, H, dtype).upload(u0), B.Grid(n, H, dtype).upload(u0)
        ins = [u]
        f = None
        if with_f:
            f = I.random_interior(seed + 10 * k + 1, n, H, -1.0, 1.0)
            ins.append(B.Grid(n, H, dtype).upload(f))
        insts.append((ins, [v]))
        host.append((u0, f))
    return insts, host


def assert_same(got, ref, what):
    if not torch.equal(got, ref):
        d = (got.double() - ref.double()).abs()
        bad = (d > 0).nonzero()
        raise AssertionError(f"{what}: max diff {d.max().item()} at {bad.shape[0]} cells, first {bad[:3].tolist()}")


def alone(dtype, op, u0, f, n, sweeps):
    u, v = B.Grid(n, H, dtype).upload(u0), B.Grid(n, H, dtype).upload(u0)
    ins = [u] + ([B.Grid(n, H, dtype).upload(f)] if f is not None else [])
    B.do_all(op, ins, [v], sweeps=sweeps)
    return v.download()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("with_f", [False, True])
@pytest.mark.parametrize("graph", [False, True])
def test_batch_sweeps_bitexact_with_single_grid(kernel_path, dtype, with_f, graph):
    op = S.heat7(0.125, with_f=with_f)
    insts, host = make_instances(dtype, with_f, seed=7, halo_value=0.5)
    batch = B.Batch(op, insts)
    info = batch.info()
    assert info["ctas"] >= 1 and info["segments"] >= info["ctas"]
    if kernel_path in ("compiled", "narrow"):
        assert info["specialization"] == (0 if with_f else 1)
    else:
        assert info["specialization"] == -1
    # like gscl_do_all, each run starts from in[0]: continuing the iteration
    # swaps in[0] and out[0] between runs (Section 5.2's swap_grids)
    total = 0
    for sweeps in (3, 4, 3):               # odd, even, odd: both starting buffers, cached graphs reused
        batch.run(sweeps, graph=graph)
        total += sweeps
        for k, ((ins, outs), (u0, f), n) in enumerate(zip(insts, host, SHAPES)):
            ref = alone(dtype, op, u0, f, n, total)
            assert_same(outs[0].download(), ref, f"instance {k} {n} after {total} sweeps")
            B.swap(ins[0], outs[0])


def test_batch_matches_oracle():
    insts, host = make_instances("f64", True, seed=3)
    batch = B.Batch(S.heat7(0.125), insts)
    batch.run(6, graph=True)
    for (ins, outs), (u0, f), n in zip(insts, host, SHAPES):
        ou, _ = D.heat_run(O.Grid(u0.copy(), H), O.Grid(f.copy(), H), 0.125, 6)
        got = outs[0].download().numpy()
        assert np.max(np.abs(got - ou.a)) <= 1e-13 * max(1.0, np.max(np.abs(ou.a)))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("red", [B.L2, B.SUM, B.MAXABS])
def test_batch_reduce_per_instance(kernel_path, dtype, red):
    insts, host = make_instances(dtype, True, seed=11)
    res_insts = [(ins, []) for ins, _ in insts]    # residual: value only, no output
    batch = B.Batch(S.residual7(), res_insts)
    got = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    batch.reduce(red, got)
    got = got.cpu().numpy()
    for k, ((ins, _), (u0, f), n) in enumerate(zip(insts, host, SHAPES)):
        want = B.do_reduce(red, S.residual7(), ins)
        if red == B.MAXABS:
            assert got[k] == want
        else:
            assert abs(got[k] - want) <= TOL[dtype] * max(1.0, abs(want)) * (10 if red == B.SUM else 1)
        if dtype == "f64":
            ov = O.do_reduce(red, D.residual_terms(), [O.Grid(u0.copy(), H), O.Grid(f.copy(), H)])
            scale = abs(ov) if red != B.SUM else float(np.abs(u0).sum() * 6 + np.abs(f).sum())
            assert abs(got[k] - ov) <= 1e-13 * max(scale, 1.0)


def test_batch_fused_reduce_writes_outputs():
    insts, host = make_instances("f64", True, seed=5)
    batch = B.Batch(S.heat7_fused(0.125), insts)
    res = torch.zeros(len(insts), dtype=torch.float64, device="cuda")
    batch.reduce(B.L2, res)
    for k, ((ins, outs), (u0, f), n) in enumerate(zip(insts, host, SHAPES)):
        v = B.Grid(n, H)
        v.upload(np.zeros(v.padded_shape))
        want = B.do_reduce(B.L2, S.heat7_fused(0.125), ins, [v])
        assert abs(res[k].item() - want) <= 1e-13 * want
        assert torch.equal(outs[0].download(), v.download())


def test_batch_tile_reports_the_shape(monkeypatch):
    monkeypatch.setenv("GSCL_BATCH_NARROW", "1")
    insts, _ = make_instances("f32", False, seed=3)
    assert B.Batch(S.heat7(0.125, with_f=False), insts).tile() == (64, 32)
    monkeypatch.delenv("GSCL_BATCH_NARROW")
    insts, _ = make_instances("f32", False, seed=3)
    assert B.Batch(S.heat7(0.125, with_f=False), insts).tile() == (128, 16)


def test_batch_tune_keeps_results():
    insts, host = make_instances("f32", False, seed=9)
    batch = B.Batch(S.heat7(0.125, with_f=False), insts)
    w, p = batch.tune(trial_sweeps=2)
    assert w in (2, 4, 8) and p in (1, 2, 3)
    # tuning leaves in[0] unchanged: sweeps from here match the instances alone
    batch.run(5, graph=True)
    for k, ((ins, outs), (u0, f), n) in enumerate(zip(insts, host, SHAPES)):
        assert_same(outs[0].download(), alone("f32", S.heat7(0.125, with_f=False), u0, None, n, 5), f"instance {k}")


def test_batch_rejects_mismatched_instances():
    a = B.Grid((8, 8, 8), (1, 1, 1))
    b = B.Grid((8, 8, 8), (2, 2, 2))
    with pytest.raises(B.GsclError) as e:
        B.Batch(S.heat7(0.125, with_f=False), [([a], [b])])
    assert e.value.status == 5
    c = B.Grid((8, 8, 8), (1, 1, 1), "f32")
    d = B.Grid((8, 8, 8), (1, 1, 1), "f32")
    e2 = B.Grid((8, 8, 8), (1, 1, 1))
    with pytest.raises(B.GsclError):
        B.Batch(S.heat7(0.125, with_f=False), [([c], [d]), ([a], [e2])])


@pytest.mark.parametrize("red", [B.L2, B.SUM, B.MAXABS])
def test_batch_reduce_of_large_instances_is_deterministic(red):
    """Instances large enough to spread over hundreds of work-list segments
    (one warp per instance folds them: fixed chunks per lane, then a fixed
    shuffle tree): two reductions give the same bits, and each agrees with
    gscl_do_reduce on the instance alone (MAXABS exactly)."""
    sides = [(256, 64, 64), (130, 90, 40), (33, 40, 35)]
    insts = []
    for k, n in enumerate(sides):
        u0 = I.random_interior(1300 + k, n, H, -1.0, 1.0)
        f0 = I.random_interior(1310 + k, n, H, -1.0, 1.0)
        insts.append(([B.Grid(n, H).upload(u0), B.Grid(n, H).upload(f0)], []))
    bt = B.Batch(S.residual7(), insts)
    a = torch.zeros(len(sides), dtype=torch.float64, device="cuda")
    b = torch.zeros(len(sides), dtype=torch.float64, device="cuda")
    bt.reduce(red, a)
    bt.reduce(red, b)
    assert torch.equal(a, b)
    for k, ((ins, _), n) in enumerate(zip(insts, sides)):
        want = B.do_reduce(red, S.residual7(), ins)
        got = a[k].item()
        if red == B.MAXABS:
            assert got == want
        elif red == B.L2:
            assert abs(got - want) <= 1e-12 * abs(want)
        else:  # the sum of |terms| bounds the rounding: 8 terms of at most 6 in size per point
            assert abs(got - want) <= 1e-13 * 13.0 * n[0] * n[1] * n[2]
