"""Admission policy of the serving loop, on the CPU: requests are admitted in
arrival order while the HBM budget and the slot limit allow; a request that
alone exceeds the budget is rejected (no GPU work: the solve start is faked)."""
import numpy as np

from paper_1207_1746_b300 import serving as SV


class FakeServer(SV.PoissonServer):
    def _start(self, req, need):
        return SV._Slot(req=req, grids={}, bytes=need)


def req(rid, n):
    return SV.Request(rid=rid, n=n, f=np.zeros((n + 2,) * 3))


def test_budget_limits_admission_in_fifo_order():
    one = SV.request_bytes(32, "mixed")
    srv = FakeServer(mode="mixed", hbm_budget=int(2.5 * one), max_active=10)
    for r in range(5):
        srv.submit(req(r, 32))
    srv._admit()
    assert [s.req.rid for s in srv.active] == [0, 1]
    assert srv.in_use == 2 * one


def test_oversized_request_is_rejected_and_does_not_block_the_queue():
    """The budget is a hard limit: a request whose grids alone exceed it is
    rejected at admission, and the requests behind it are admitted."""
    srv = FakeServer(mode="fp64", hbm_budget=SV.request_bytes(16, "fp64"), max_active=10)
    srv.submit(req(0, 64))
    srv.submit(req(1, 16))
    srv._admit()
    assert [s.req.rid for s in srv.active] == [1]
    assert [r.rid for r in srv.rejected] == [0] and srv.rejected[0].rejected
    assert srv.in_use <= srv.budget


def test_waiting_request_admitted_only_when_memory_frees():
    """Admission never exceeds the budget: the third request waits until one
    of the two active ones retires, and then goes in the same tick."""
    one = SV.request_bytes(32, "fp64")
    srv = FakeServer(mode="fp64", hbm_budget=2 * one, max_active=10)
    for r in range(3):
        srv.submit(req(r, 32))
    srv._admit()
    assert [s.req.rid for s in srv.active] == [0, 1] and [r.rid for r in srv.waiting] == [2]
    retired = srv.active.pop(0)
    srv.in_use -= retired.bytes
    srv._admit()
    assert [s.req.rid for s in srv.active] == [1, 2] and srv.in_use == 2 * one


def test_slot_limit():
    srv = FakeServer(mode="fp64", hbm_budget=1 << 40, max_active=3)
    for r in range(6):
        srv.submit(req(r, 16))
    srv._admit()
    assert len(srv.active) == 3 and len(srv.waiting) == 3


def test_mixed_needs_more_memory_than_fp64_grids_alone():
    assert SV.request_bytes(64, "mixed") > SV.request_bytes(64, "fp64")


def test_memory_per_mode():
    """Grids held per request: FP64 Jacobi u, v, f; red-black SOR u, f in place;
    the mixed modes add FP32 correction grids (two for red-black, in place)."""
    g64 = SV.request_bytes(64, "rbsor") // 2
    assert SV.request_bytes(64, "fp64") == 3 * g64
    assert SV.request_bytes(64, "mixed_rbsor") < SV.request_bytes(64, "mixed")
    assert SV.request_bytes(64, "mixed_rbsor") > SV.request_bytes(64, "fp64")


def test_unknown_mode_rejected():
    import pytest
    with pytest.raises(ValueError):
        SV.PoissonServer(mode="jacobi32")
