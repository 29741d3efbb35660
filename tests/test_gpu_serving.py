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
