"""The rule the NMS greedy pass uses to decide a block of 64 rows at once,
modelled on the host: a row is kept once none of its suppressors is kept or
undecided, and suppressed once one of them is kept.  It must give exactly the
sequential greedy decisions, and every round must decide at least one row
(so the loop ends within 64 rounds)."""
import numpy as np
import pytest


def sequential(sup, removed):
    """Greedy in row order: sup[r] = set of rows a < r that suppress r."""
    kept = []
    for r in range(len(sup)):
        if removed[r]:
            continue
        if not any(a in kept for a in sup[r]):
            kept.append(r)
    return set(kept)


def rounds(sup, removed):
    """The ballot-round rule on bitmasks, as the kernel's warp 0 runs it."""
    n = len(sup)
    sb = [sum(1 << a for a in sup[r]) for r in range(n)]
    und = sum(1 << r for r in range(n) if not removed[r])
    kept = 0
    count = 0
    while und:
        live = und | kept
        k = sum(1 << r for r in range(n) if (und >> r) & 1 and not (sb[r] & live))
        x = sum(1 << r for r in range(n) if (und >> r) & 1 and (sb[r] & kept))
        assert k | x, "a round decided no row"
        assert not (k & x)
        kept |= k
        und &= ~(k | x)
        count += 1
    return {r for r in range(n) if (kept >> r) & 1}, count


@pytest.mark.parametrize("density", [0.0, 0.02, 0.1, 0.3, 0.9])
def test_rounds_equal_sequential_greedy(density):
    rng = np.random.default_rng(int(density * 1000) + 1)
    for _ in range(60):
        n = int(rng.integers(1, 65))
        sup = [{a for a in range(r) if rng.uniform() < density} for r in range(n)]
        removed = rng.uniform(size=n) < 0.2
        got, count = rounds(sup, removed)
        assert got == sequential(sup, removed)
        assert count <= n


def test_chain_takes_one_round_per_link():
    # row r suppressed only by row r - 1: kept rows alternate, and each round
    # can settle only the next link of the chain
    n = 64
    sup = [set() if r == 0 else {r - 1} for r in range(n)]
    got, count = rounds(sup, np.zeros(n, bool))
    assert got == set(range(0, n, 2))
    assert count == n
