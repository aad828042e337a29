"""Subset positions of the library's sharded subset loop, enumerated here in
plain Python (test infrastructure; no code shared with the library).

The library numbers the (p-2)-subsets c[0] < ... < c[k-1] of the nonzero
centred points (taken in data order) by their colex rank
r = sum_i C(c[i], i + 1), and shard s of S handles the ranks
[floor(N s / S), floor(N (s + 1) / S)) with N = C(nnz, k) (include/tukey_depth.h).
"""
from math import comb


def shard_range(nnz, k, s, S):
    N = comb(nnz, k)
    return N * s // S, N * (s + 1) // S


def colex_unrank(r, k):
    """The k-combination of colex rank r (greedy on the combinatorial number system)."""
    c = [0] * k
    for i in range(k, 0, -1):
        x = i - 1
        while comb(x + 1, i) <= r:
            x += 1
        c[i - 1] = x
        r -= comb(x, i)
    return c


def colex_range(k, lo, hi):
    """The combinations of colex ranks lo .. hi-1, in order."""
    if hi <= lo:
        return []
    c = colex_unrank(lo, k)
    out = [tuple(c)]
    for _ in range(hi - lo - 1):
        i = 0
        while i < k - 1 and c[i] + 1 == c[i + 1]:
            c[i] = i
            i += 1
        c[i] += 1
        out.append(tuple(c))
    return out
