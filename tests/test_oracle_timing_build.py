"""The oracle's timing build (-O3 -march=native -fopenmp, several threads),
which bench.py times as the CPU baseline, returns exactly the checker build's
numbers: do_all outputs and values, and every reduction, on 1 and 4 threads."""
import numpy as np

from oracle import drivers as D
from oracle import oracle as O


def _run_all():
    rng = np.random.default_rng(31)
    n, h = (37, 21, 13), (1, 1, 1)
    u = O.Grid(rng.uniform(-1, 1, (n[2] + 2, n[1] + 2, n[0] + 2)), h)
    f = O.Grid(rng.uniform(-1, 1, u.a.shape), h)
    out = O.zeros(n, h)
    val = O.do_all(D.heat_terms(0.125), [u, f], [out], want_value=True)
    res = {"out": out.a.copy(), "val": val}
    for op in (O.SUM, O.MAXABS, O.L2):
        o2 = O.zeros(n, h)
        res[op] = (O.do_reduce(op, D.heat_terms(0.125), [u, f], [o2], lo=(2, 1, 0), hi=(35, 20, 13)), o2.a.copy())
    res["plain"] = O.do_reduce(O.L2, [], [u])
    res["within"] = O.do_reduce_within(0.5, D.heat_terms(0.125), [u, f], [O.zeros(n, h)])
    return res


def test_timing_build_matches_the_checker():
    want = _run_all()
    try:
        O.use_library(O.build(timing=True))
        for nt in (1, 4):
            assert O.threads(nt) == nt
            got = _run_all()
            assert np.array_equal(got["out"], want["out"]) and np.array_equal(got["val"], want["val"])
            for op in (O.SUM, O.MAXABS, O.L2):
                assert got[op][0] == want[op][0], (nt, op)
                assert np.array_equal(got[op][1], want[op][1])
            assert got["plain"] == want["plain"] and got["within"] == want["within"]
    finally:
        O.use_library(None)
    assert O.threads(8) == 1  # the checker has no threads
