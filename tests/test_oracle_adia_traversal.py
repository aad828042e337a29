"""Algorithm 3's traversal (readings A3-A6) pinned by a second transcription.

tests/adia_transcription.py restates Steps 2-5 of Algorithm 3 (Section 4)
from the paper and the readings, with its own V(S), G(S) (cells of the line
arrangement listed directly), critical points and open depths.  On small
full-rank inputs -- random, with duplicated rows, and in general position --
the oracle's count and every traversal counter (pops, subsets of Step 4,
nodes pushed, the deepest stack, the union of Step 5(a), the subsets of
Step 5(b), d0 after the search) must equal the transcription's.  A slip in
the oracle's order of subsets or critical points, the break of Step 4(a)(iv),
the deletions of Step 4(b), the side chosen in Step 5(a) or the start subset
of Step 2 moves at least one of these counters."""
import numpy as np
import pytest

import oracle
from adia_transcription import adia as adia_py


def _symmetric_cases(p, seed, count):
    """Clouds symmetric about z = 0 plus up to two extra points: many
    hyperplanes of Step 5(a) split the points evenly (the tie of A6)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        Y = rng.integers(-6, 7, size=(int(rng.integers(p + 1, 7)), p))
        extra = rng.integers(-6, 7, size=(int(rng.integers(0, 3)), p))
        X = np.vstack([Y, -Y, extra]).astype(np.int32)
        z = np.zeros(p, np.int32)
        if oracle.rank(X, z)[0] == p and len(X) > 2 * p:
            out.append((X, z))
    return out


def _cases(p, seed, count):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = int(rng.integers(2 * p + 2, {3: 17, 4: 14, 5: 13}[p]))
        lim = int(rng.choice([3, 6, 40]))
        X = rng.integers(-lim, lim + 1, size=(n, p)).astype(np.int32)
        if rng.random() < 0.4:
            X[-2:] = X[:2]                      # duplicated rows
        z = X[int(rng.integers(0, n))] if rng.random() < 0.5 else rng.integers(-lim // 2, lim // 2 + 1, size=p)
        z = np.asarray(z, dtype=np.int32)
        if oracle.rank(X, z)[0] == p:
            out.append((X, z))
    return out


@pytest.mark.parametrize("p,seed", [(3, 1), (3, 2), (4, 3), (4, 4), (5, 5)])
def test_traversal_matches_second_transcription(p, seed):
    checked = searched = 0
    for X, z in _cases(p, seed, 10 if p < 5 else 6) + _symmetric_cases(p, seed + 50, 6 if p < 5 else 4):
        T, st = oracle.adia(X, z)
        T2, st2 = adia_py(X, z)
        assert T == T2, (X.tolist(), z.tolist(), T, T2)
        for k in st2:
            assert st[k] == st2[k], (k, st, st2, X.tolist(), z.tolist())
        checked += 1
        searched += st["pops"] > 0
    assert checked > 0 and searched > 0
