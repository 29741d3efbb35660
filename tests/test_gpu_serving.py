"""Serving loop: continuous batching of Poisson solves with per-request stop
on the FP64 residual.  Each finished request's residual is re-measured by the
FP64 oracle from the downloaded solution; a request's result is the same
alone and in the mix; both solve modes agree with a direct sparse solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import drivers as D
from oracle import oracle as O
from paper_1207_1746_b300 import inputs as I
from paper_1207_1746_b300 import serving as SV

pytestmark = pytest.mark.gpu


def small_requests(count, lo=10, hi=18, base=900):
    reqs = []
    for r in range(count):
        n, f = I.poisson_request(r, base_seed=base, lo=lo, hi=hi)
        reqs.append(SV.Request(rid=r, n=n, f=f))
    return reqs


def poisson_matrix(n):
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    Id = sp.identity(n)
    return (sp.kron(sp.kron(Id, Id), T) + sp.kron(sp.kron(Id, T), Id) + sp.kron(sp.kron(T, Id), Id)).tocsc()


@pytest.mark.parametrize("mode", ["mixed", "fp64", "rbsor", "mixed_rbsor"])
def test_requests_converge_by_oracle_residual(mode):
    reqs = small_requests(4)
    srv = SV.PoissonServer(mode=mode, check_every=20, keep_solution=True)
    st = srv.run_trace(reqs)
    assert st["completed"] == 4 and st["backlog"] == 0
    for r in reqs:
        h = (1, 1, 1)
        res, fn = D.poisson_residual(O.Grid(r.u, h), O.Grid(r.f.copy(), h))
        assert res <= 1e-6 * fn, (r.rid, res / fn)
        exact = spla.spsolve(poisson_matrix(r.n), r.f[1:-1, 1:-1, 1:-1].ravel())
        err = np.max(np.abs(r.u[1:-1, 1:-1, 1:-1].ravel() - exact)) / np.max(np.abs(exact))
        assert err <= 1e-4, (r.rid, err)


@pytest.mark.parametrize("mode", ["mixed", "fp64", "rbsor", "mixed_rbsor"])
def test_result_same_alone_and_in_the_mix(mode):
    target = small_requests(1, base=950)[0]
    alone = SV.PoissonServer(mode=mode, check_every=20, keep_solution=True)
    alone.run_trace([SV.Request(rid=0, n=target.n, f=target.f.copy())])
    u_alone = alone.done[0].u
    others = small_requests(3, base=960)
    mix = [SV.Request(rid=0, n=target.n, f=target.f.copy(), arrival=0.0)]
    mix += [SV.Request(rid=k + 1, n=o.n, f=o.f, arrival=0.0) for k, o in enumerate(others)]
    srv = SV.PoissonServer(mode=mode, check_every=20, keep_solution=True)
    srv.run_trace(mix)
    got = [r for r in srv.done if r.rid == 0][0]
    assert got.sweeps == alone.done[0].sweeps
    assert np.max(np.abs(got.u - u_alone)) <= 1e-12 * np.max(np.abs(u_alone))


def test_fp64_and_mixed_agree():
    reqs = small_requests(2, base=970)
    sols = {}
    for mode in ("fp64", "mixed"):
        srv = SV.PoissonServer(mode=mode, check_every=20, keep_solution=True)
        srv.run_trace([SV.Request(rid=r.rid, n=r.n, f=r.f.copy()) for r in reqs])
        sols[mode] = {r.rid: r.u for r in srv.done}
    for r in reqs:
        a, b = sols["fp64"][r.rid], sols["mixed"][r.rid]
        assert np.max(np.abs(a - b)) <= 2e-4 * np.max(np.abs(a))


def test_rbsor_needs_far_fewer_iterations_than_jacobi():
    """Red-black SOR with the optimal factor: O(n) iterations against Jacobi's
    O(n^2), on the same requests and the same stopping rule."""
    reqs = small_requests(2, lo=24, hi=30, base=980)
    sweeps = {}
    for mode in ("fp64", "rbsor"):
        srv = SV.PoissonServer(mode=mode, check_every=10, sor_check_every=5, keep_solution=True)
        st = srv.run_trace([SV.Request(rid=r.rid, n=r.n, f=r.f.copy()) for r in reqs])
        assert st["completed"] == 2 and st["max_rel_residual"] <= 1e-6
        sweeps[mode] = {r.rid: r.sweeps for r in srv.done}
    for r in reqs:
        assert sweeps["rbsor"][r.rid] * 5 < sweeps["fp64"][r.rid], (r.n, sweeps)


def _solo(mode, r, **kw):
    srv = SV.PoissonServer(mode=mode, check_every=20, keep_solution=True, **kw)
    srv.run_trace([SV.Request(rid=r.rid, n=r.n, f=r.f.copy())])
    return srv.done[0]


@pytest.mark.parametrize("mode", ["rbsor", "mixed_rbsor", "mixed", "fp64"])
@pytest.mark.parametrize("limit", ["slots", "budget"])
def test_staggered_arrivals_wait_for_a_retirement(mode, limit):
    """Continuous batching with arrivals in flight: three requests at the
    start and a fourth after two ticks, under a limit that holds two requests
    at a time (max_active = 2, or an HBM budget that fits exactly the first
    two; sides 16..18, so any two need more than the largest one alone).  The
    third waits for a retirement and is admitted in the tick after it; at no
    tick are more than two requests in flight; every request ends with the
    sweeps of its run alone and, within 1e-12 relative, its solution."""
    reqs = small_requests(4, lo=16, hi=18, base=990)
    need = [SV.request_bytes(r.n, mode) for r in reqs]
    if limit == "slots":
        srv = SV.PoissonServer(mode=mode, check_every=20, keep_solution=True, max_active=2)
    else:
        assert need[0] + need[1] >= max(need)
        srv = SV.PoissonServer(mode=mode, check_every=20, keep_solution=True, hbm_budget=need[0] + need[1])
    for r in reqs[:3]:
        srv.submit(SV.Request(rid=r.rid, n=r.n, f=r.f.copy()))
    ticks = 0
    while srv.waiting or srv.active or ticks < 2:
        if ticks == 2:
            srv.submit(SV.Request(rid=reqs[3].rid, n=reqs[3].n, f=reqs[3].f.copy()))
        srv.tick()
        ticks += 1
        assert srv.in_use <= srv.budget and len(srv.active) <= srv.max_active
        assert ticks < 100000
    assert not srv.rejected and len(srv.done) == 4
    done = {r.rid: r for r in srv.done}
    first_retirement = min(done[0].done_tick, done[1].done_tick)
    assert done[2].admit_tick >= first_retirement > 0, (done[2].admit_tick, first_retirement)
    assert done[3].admit_tick >= 2
    # a request is worked on in ticks admit_tick + 1 .. done_tick
    in_flight = [sum(1 for r in done.values() if r.admit_tick < t <= r.done_tick) for t in range(1, srv.ticks + 1)]
    assert max(in_flight) == 2, in_flight
    for r in reqs:
        solo = _solo(mode, r)
        got = done[r.rid]
        assert got.sweeps == solo.sweeps, (r.rid, got.sweeps, solo.sweeps)
        assert np.max(np.abs(got.u - solo.u)) <= 1e-12 * np.max(np.abs(solo.u)), r.rid
        h = (1, 1, 1)
        res, fn = D.poisson_residual(O.Grid(got.u, h), O.Grid(r.f.copy(), h))
        assert res <= 1e-6 * fn, (r.rid, res / fn)


def test_request_larger_than_the_budget_is_rejected():
    reqs = small_requests(2, lo=12, hi=14, base=995)
    big = SV.Request(rid=9, n=40, f=I.poisson_request(0, base_seed=996, lo=40, hi=40)[1])
    budget = SV.request_bytes(14, "mixed_rbsor")
    srv = SV.PoissonServer(mode="mixed_rbsor", check_every=20, hbm_budget=budget)
    st = srv.run_trace([big] + [SV.Request(rid=r.rid, n=r.n, f=r.f.copy()) for r in reqs])
    assert st["rejected"] == 1 and srv.rejected[0].rid == 9
    assert st["completed"] == 2 and st["backlog"] == 0
