"""Host logic of fused-sweep runs, on the CPU: the launch count the Python
binding expects from a batch run (it decides which grid the handles name
afterwards) follows the library's launch plan: fused launches of K sweeps
while more than K sweeps remain, single sweeps after, and one launch more
when the count and the sweep count differ in parity."""
import pytest

from paper_1207_1746_b300 import binding as B


def launches(sweeps, k):
    bt = B.Batch.__new__(B.Batch)  # no device state: only the plan arithmetic
    bt._k = k
    return bt._launches(sweeps)


def plan(sweeps, k):
    """The plan written out from its rule (independent of the binding's loop)."""
    sizes, done = [], 0
    while done < sweeps:
        step = k if (k > 1 and sweeps - done > k) else 1
        sizes.append(step)
        done += step
    if (len(sizes) - sweeps) % 2:
        i = max(j for j, v in enumerate(sizes) if v > 1)
        sizes[i:i + 1] = [sizes[i] - 1, 1]
    return sizes


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8, 12, 16])
def test_launch_count_matches_the_plan_and_keeps_parity(k):
    for sweeps in range(1, 70):
        p = plan(sweeps, k)
        assert sum(p) == sweeps and p[-1] == 1 and max(p) <= max(k, 1)
        n = launches(sweeps, k)
        assert n == len(p), (sweeps, k, n, p)
        assert (n - sweeps) % 2 == 0
        assert 1 <= n <= sweeps


def test_single_sweeps_when_nothing_fuses():
    for sweeps in range(1, 30):
        assert launches(sweeps, 1) == sweeps


def test_laplace_step_plan():
    """The 2D Laplace step: 100 sweeps at 6 per launch are 16 fused launches
    and 4 single sweeps."""
    p = plan(100, 6)
    assert p.count(6) == 16 and p.count(1) == 4 and launches(100, 6) == 20
