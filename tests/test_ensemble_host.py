"""Host logic of the concurrent ensemble solve (no GPU): the placement of members on streams."""
import numpy as np

import paper_2506_04157_gb300 as mfs


def test_place_members_balances_work():
    """The 64-member ensemble (levels drawn from {3, 4, 5} as in the bench) on 8 streams: every
    member placed, all streams used, and the largest-first greedy placement within one
    largest member of a perfect split (the classic bound of list scheduling)."""
    rng = np.random.default_rng(3)
    levels = rng.integers(3, 6, size=64)
    stream_of, load = mfs.place_members(levels, 8)
    assert len(stream_of) == 64 and set(stream_of) == set(range(8))
    work = [0] * 8
    for l, k in zip(levels, stream_of):
        work[k] += 8 ** int(l)
    assert work == load
    total = sum(8 ** int(l) for l in levels)
    assert max(load) <= total / 8 + 8 ** int(max(levels))
    assert sum(load) == total


def test_place_members_small_cases():
    assert mfs.place_members([], 4) == ([], [0])
    s, load = mfs.place_members([2, 2], 8)        # never more streams than members
    assert sorted(s) == [0, 1] and load == [64, 64]
    s, _ = mfs.place_members([5, 3, 3, 3], 2)     # the big member alone, the small ones together
    assert s[0] != s[1] and s[1] == s[2] == s[3]
    s, _ = mfs.place_members([4, 4, 4], 1)
    assert s == [0, 0, 0]
