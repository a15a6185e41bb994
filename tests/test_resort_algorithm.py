"""The near-sorted re-sort's placement rule (k_sort.cu), restated on the host.

The state is in the stable order of its old keys (bucket starts bprev).  A stayer keeps
its key; a mover's new key differs.  New bucket B is [movers from lower old keys |
B's stayers | movers from higher old keys], each part in index order; a stayer's rank
inside B's stayers is (i - bprev[B]) minus the movers of old key B before it, a mover's
rank is its place among the movers of new key B in the movers' stable order.  These
tests check that the rule reproduces the stable sort of the new keys, including empty
buckets, no movers and all movers.
"""
import numpy as np
import pytest


def place(old_keys, new_keys, nbuckets):
    """Destination of every particle by the placement rule (old_keys sorted)."""
    n = len(old_keys)
    counts = np.bincount(new_keys, minlength=nbuckets)
    bstart = np.concatenate([[0], np.cumsum(counts)])
    bprev = np.concatenate([[0], np.cumsum(np.bincount(old_keys, minlength=nbuckets))])
    mover = new_keys != old_keys
    stay = np.bincount(new_keys[~mover], minlength=nbuckets)
    low = np.bincount(new_keys[mover & (old_keys < new_keys)], minlength=nbuckets)
    # movers of each old key before i (the per-old-tile block scan)
    mrank = np.zeros(n, np.int64)
    seen = {}
    for i in range(n):
        if mover[i]:
            mrank[i] = seen.get(old_keys[i], 0)
            seen[old_keys[i]] = mrank[i] + 1
        else:
            mrank[i] = seen.get(old_keys[i], 0)
    dst = np.empty(n, np.int64)
    for i in np.flatnonzero(~mover):
        B = new_keys[i]
        dst[i] = bstart[B] + low[B] + (i - bprev[B]) - mrank[i]
    # movers: compacted in index order, stably sorted by new key
    mi = np.flatnonzero(mover)
    order = mi[np.argsort(new_keys[mi], kind="stable")]
    sstart = np.concatenate([[0], np.cumsum(stay)])
    for j, i in enumerate(order):
        B = new_keys[i]
        r = j - (bstart[B] - sstart[B])
        dst[i] = bstart[B] + r + (stay[B] if r >= low[B] else 0)
    return dst


def check(old_keys, new_keys, nbuckets):
    dst = place(old_keys, new_keys, nbuckets)
    assert np.array_equal(np.sort(dst), np.arange(len(dst)))  # a permutation
    expected = np.argsort(new_keys, kind="stable")  # particle at each sorted position
    got = np.empty_like(dst)
    got[dst] = np.arange(len(dst))
    assert np.array_equal(got, expected)


@pytest.mark.parametrize("seed,move_frac,span", [(0, 0.03, 1), (1, 0.2, 3), (2, 0.6, 8), (3, 0.0, 1),
                                                 (4, 1.0, 5)])
def test_placement_rule_is_the_stable_sort(seed, move_frac, span):
    rng = np.random.default_rng(seed)
    nb = 64
    old = np.sort(rng.integers(0, nb, size=3000))
    new = old.copy()
    m = rng.random(old.size) < move_frac
    new[m] = np.clip(old[m] + rng.integers(-span, span + 1, size=m.sum()), 0, nb - 1)
    if move_frac == 1.0:  # every particle a mover
        new = np.where(new == old, (old + 1) % nb, new)
    check(old, new, nb)


def test_placement_rule_with_empty_buckets_and_everything_moving_up():
    old = np.sort(np.repeat([0, 5, 9], [10, 3, 7]))
    new = np.where(old == 0, 9, np.where(old == 5, 2, old))
    check(old, new, 12)
