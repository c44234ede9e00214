"""The binomial (revolve-style) checkpoint schedule of lbm_adjoint, host arithmetic only:
its recomputation count against the optimum by brute-force dynamic programming over every
split, and against the binomial bound r n (each step advanced at most r times, r the least
with C(c + r, c) >= n for c = s + 1 snapshots, the one holding the segment's start included)."""
import functools
import math

import pytest

from paper_1909_12390_gb300 import lbm


@functools.lru_cache(maxsize=None)
def _optimal(n, s):
    """Fewest forward steps to reverse n steps from a stored start with s free state slots:
    advance m steps into a slot, reverse the last n - m with s - 1 slots, then the first m."""
    if n <= 1:
        return 0
    if s == 0:
        return n * (n - 1) // 2
    return min(m + _optimal(n - m, s - 1) + _optimal(m, s) for m in range(1, n))


def _r(n, s):
    c, r = s + 1, 0
    while math.comb(c + r, c) < n:
        r += 1
    return r


@pytest.mark.parametrize("s", [1, 2, 3, 4, 7])
def test_schedule_is_optimal_on_small_segments(s):
    for n in range(1, 61):
        assert lbm.revolve_steps(n, s) == (n - 1 if s >= n else _optimal(n, s)), (n, s)


@pytest.mark.parametrize("n,s", [(55, 8), (3000, 10), (3000, 55), (500, 3), (10000, 20)])
def test_schedule_respects_the_binomial_bound(n, s):
    assert lbm.revolve_steps(n, s) <= _r(n, s) * n


def test_full_storage_and_arguments():
    assert lbm.revolve_steps(55, 0) == 54 and lbm.revolve_steps(55, 55) == 54
    assert lbm.revolve_steps(0, 3) == -1 and lbm.revolve_steps(10, -1) == -1
