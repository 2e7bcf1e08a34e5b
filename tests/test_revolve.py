"""The binomial checkpointing schedule of the adjoint driver (CPU).

Its recomputation count is pinned to the closed form of binomial
checkpointing (Griewank & Walther, "revolve"): reversing l steps with c
checkpoints (the start state counted) costs r*l - C(c + r, r - 1) forward
steps, r the smallest integer with C(c + r, c) >= l."""
from math import comb

import pytest

from paper_2207_04252_gb300 import adjoint as adj


def _closed_form(l, c):
    if l <= 1:
        return 0
    r = 0
    while comb(c + r, c) < l:
        r += 1
    return r * l - comb(c + r, r - 1)


@pytest.mark.parametrize("l", [1, 2, 3, 7, 20, 41, 100, 200])
@pytest.mark.parametrize("s", [0, 1, 2, 3, 5, 9, 20])
def test_schedule_cost_is_the_binomial_optimum(l, s):
    assert adj.revolve_forward_steps(l, s) == _closed_form(l, s + 1)


def test_limits():
    assert adj.revolve_forward_steps(50, 0) == 50 * 49 // 2  # no snapshot: recompute from the start
    assert adj.revolve_forward_steps(50, 49) == 49           # a snapshot per step: each step once
    costs = [adj.revolve_forward_steps(200, s) for s in range(0, 30)]
    assert all(a >= b for a, b in zip(costs, costs[1:]))     # more snapshots never cost more
