"""Host logic of the gradient window's memory plan (adjoint.plan_window):
the plan fits the budget, takes the fewest recomputed steps, and its peak is
the count of states it holds.  Brute force over every interval and mode on
small cases; the 400M-particle two-species window as a worked case."""
import math

import pytest

pytest.importorskip("torch")
from paper_2208_12795_gb300.adjoint import plan_window  # noqa: E402


def _peak(n, K, every, stash, S, A):
    nck = math.ceil(K / every)
    return nck * (S + 4 * n) + ((every + 1) if stash else 2) * S + 2 * A


def _recompute(K, every, stash):
    if stash:
        return K
    segs = [min(every, K - s * every) for s in range(math.ceil(K / every))]
    return sum(L * (L + 1) // 2 for L in segs)


@pytest.mark.parametrize("K", [1, 7, 20, 50])
@pytest.mark.parametrize("budget_states", [3.5, 6, 9, 14, 1000])
def test_plan_is_the_cheapest_that_fits(K, budget_states):
    n, S, A = 1000, 41_000, 36_000
    budget = int(budget_states * S + 2 * A)
    fits = [(_recompute(K, e, st), _peak(n, K, e, st, S, A), e, st)
            for e in range(1, K + 1) for st in (True, False) if _peak(n, K, e, st, S, A) <= budget]
    if not fits:
        with pytest.raises(MemoryError):
            plan_window(n, K, S, A, budget)
        return
    p = plan_window(n, K, S, A, budget)
    assert p.peak_bytes == _peak(n, K, p.every, p.stash, S, A) <= budget
    assert p.recompute_steps == _recompute(K, p.every, p.stash)
    assert (p.recompute_steps, p.peak_bytes) == min(f[:2] for f in fits)


def test_large_two_species_window_plan():
    """400M particles (FP64 positions, FP32 velocities, tet, status: 41 B;
    adjoint 36 B), K = 20: with 230 GB the reverse sweep stashes (K
    recomputed steps) at the interval of least memory; with 160 GB it
    recomputes each step's pair from the checkpoints."""
    n = 400_000_000
    S, A = 41 * n, 36 * n
    p = plan_window(n, 20, S, A, 230e9)
    assert p.stash and p.recompute_steps == 20 and p.every in (4, 5)
    assert p.peak_bytes <= 230e9
    q = plan_window(n, 20, S, A, 160e9)
    assert not q.stash and q.peak_bytes <= 160e9 and q.recompute_steps > 20
