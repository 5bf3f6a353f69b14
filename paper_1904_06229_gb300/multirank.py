"""Splitting one permanent's Gray range across ranks, and combining the
ranks' partials (the one exchange step of a split sum).

The sum over codes [0, 2^(n-1)) is cut into equal consecutive ranges by the
paper's `distribute` (App. A); each rank computes its ranges' double-double
partials with `perm_c128_range` on its own GPU, and the partials are gathered
to one rank and added in fixed rank order (Sec. 2.B: keep the partial sums in
an array and add them in a fixed order rather than with a plain reduction).
The addition is double-double (Knuth TwoSum), so the combined value carries
the same precision as a single-GPU run.  No collective touches the data path.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple


def distribute(total: int, parts: int, i: int) -> Tuple[int, int]:
    """App. A distribute: piece i of `parts` nearly equal consecutive pieces."""
    q, r = divmod(total, parts)
    return i * q + min(i, r), q + (1 if i < r else 0)


def rank_ranges(n: int, world: int, rank: int, pieces_per_rank: int = 1) -> List[Tuple[int, int]]:
    """Code ranges [first, first+count) of `rank` when the 2^(n-1)-code sum is
    cut into world * pieces_per_rank pieces, dealt round-robin."""
    total = 1 << (n - 1)
    parts = world * pieces_per_rank
    return [distribute(total, parts, p) for p in range(rank, parts, world)]


def _two_sum(a: float, b: float):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def dd_add(a: Tuple[float, float], b: Tuple[float, float]) -> Tuple[float, float]:
    s1, s2 = _two_sum(a[0], b[0])
    t1, t2 = _two_sum(a[1], b[1])
    s2 += t1
    s1, s2 = s1 + s2, s2 - ((s1 + s2) - s1)
    s2 += t2
    return s1 + s2, s2 - ((s1 + s2) - s1)


def combine_partials(partials: Sequence[Sequence[Sequence[float]]], n: int) -> complex:
    """partials[rank][k] = [re_hi, re_lo, im_hi, im_lo] for that rank's k-th
    range.  Adds them in rank order, then range order, and applies
    2 (-1)^(n-1)."""
    re, im = (0.0, 0.0), (0.0, 0.0)
    for per_rank in partials:
        for p in per_rank:
            re = dd_add(re, (float(p[0]), float(p[1])))
            im = dd_add(im, (float(p[2]), float(p[3])))
    s = 2.0 if (n - 1) % 2 == 0 else -2.0
    return complex(s * (re[0] + re[1]), s * (im[0] + im[1]))


def shard_batch(ns: Sequence[int], world: int) -> List[List[int]]:
    """Deal the matrices of a batch to `world` ranks so that each rank's work,
    the sum of 2^(n-1) Gray codes over its matrices, is as even as a greedy
    deal makes it: matrices in decreasing order of cost (ties by index), each
    to the rank with the least work so far (ties to the lowest rank).  Batch
    items share nothing, so the ranks run their shards with no exchange at
    all; returns the matrix indices of each rank, in increasing order."""
    import heapq

    if world < 1:
        raise ValueError("world >= 1")
    order = sorted(range(len(ns)), key=lambda k: (-int(ns[k]), k))
    heap = [(0, r) for r in range(world)]
    shards: List[List[int]] = [[] for _ in range(world)]
    for k in order:
        load, r = heapq.heappop(heap)
        shards[r].append(k)
        heapq.heappush(heap, (load + (1 << (int(ns[k]) - 1)), r))
    return [sorted(s) for s in shards]
