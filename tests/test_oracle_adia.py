"""Pins of the oracle's Algorithm 3 (ADIA, Section 4).

* Critical points (Step 2(c), Step 4(a)(ii)) against an independent brute
  force on tie-heavy 2-D point sets: a point is critical when one of the two
  cells of the line arrangement beside its line has the least count.  Each
  cell is evaluated exactly at a direction turned from the point's line by
  less than the angle between any two distinct lines.
* In general position, against the paper's own condition: the line through
  0 and y_h has a normal u0 with #{u0'y <= 0} - 1 = the closed depth.
* ADIA is never below the exact count (every value it takes is some V(S)),
  on random tie-heavy data; on data in general position it equals the exact
  count, as the paper reports for all its experiments.
* The branches that return without a search: n <= 2p, rank < 3, z outside
  the hull (T = Z).
"""
import numpy as np
import pytest

import oracle
from paper_literal import in_general_position


def _cells_beside(Y, h, L=10 ** 9):
    """min(#left, #right) of the two cells beside the line of h (exact ints)."""
    h = (int(h[0]), int(h[1]))
    rot = (-h[1], h[0])
    out = []
    for s in (1, -1):
        v = (L * h[0] + s * rot[0], L * h[1] + s * rot[1])
        left = right = 0
        for y in Y:
            cr = v[0] * int(y[1]) - v[1] * int(y[0])
            if y[0] == 0 and y[1] == 0:
                continue
            assert cr != 0
            left += cr > 0
            right += cr < 0
        out.append(min(left, right))
    return out


def _critical_bruteforce(Y):
    nz = [i for i, y in enumerate(Y) if y[0] != 0 or y[1] != 0]
    if not nz:
        return 0, np.zeros(len(Y), dtype=np.uint8)
    cells = {i: _cells_beside(Y, Y[i]) for i in nz}
    G = min(min(c) for c in cells.values())
    crit = np.zeros(len(Y), dtype=np.uint8)
    for i, c in cells.items():
        crit[i] = 1 if min(c) == G else 0
    return G, crit


def _tie_heavy_2d(rng, n, lim):
    Y = rng.integers(-lim, lim + 1, size=(n, 2))
    for j in range(n):
        r = rng.random()
        if r < 0.2 and j > 0:
            Y[j] = Y[rng.integers(0, j)] * int(rng.integers(1, 3))     # same line, same side
        elif r < 0.3 and j > 0:
            Y[j] = -Y[rng.integers(0, j)]                              # same line, opposite side
        elif r < 0.35:
            Y[j] = 0                                                   # zero point
    return Y


@pytest.mark.parametrize("seed", range(8))
def test_critical_points_match_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(60):
        n = int(rng.integers(1, 14))
        Y = _tie_heavy_2d(rng, n, int(rng.choice([1, 2, 5, 30])))
        G, crit = oracle.critical(Y)
        Gb, critb = _critical_bruteforce(Y)
        assert G == Gb, (Y.tolist(), G, Gb)
        assert crit.tolist() == critb.tolist(), (Y.tolist(), crit, critb)


def test_critical_points_general_position_paper_condition():
    """The paper's condition of Step 4(a)(ii) on the 2-D quotient: h is
    critical when a normal u0 of the line through 0 and y_h has
    #{u0'y <= 0} - 1 == the closed depth count of the origin."""
    rng = np.random.default_rng(7)
    done = 0
    while done < 150:
        n = int(rng.integers(2, 12))
        Y = rng.integers(-50, 51, size=(n, 2))
        if any((y == 0).all() for y in Y):
            continue
        if any(Y[a, 0] * Y[b, 1] - Y[a, 1] * Y[b, 0] == 0 for a in range(n) for b in range(a + 1, n)):
            continue
        N = oracle.bivariate_closed(Y)
        G, crit = oracle.critical(Y)
        assert G == N  # no zero points: closed and open minimum agree
        for h in range(n):
            u0 = np.array([-Y[h, 1], Y[h, 0]])
            c_plus = int(np.sum(Y @ u0 <= 0))
            c_minus = int(np.sum(Y @ (-u0) <= 0))
            paper = (c_plus - 1 == N) or (c_minus - 1 == N)
            assert bool(crit[h]) == paper, (Y.tolist(), h)
        done += 1


def _nd_cases(seed, count):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        p = int(rng.integers(3, 6))
        n = int(rng.integers(2 * p + 1, 40))
        lim = int(rng.choice([2, 3, 10, 1000]))
        X = rng.integers(-lim, lim + 1, size=(n, p)).astype(np.int32)
        if rng.random() < 0.4:
            k = int(rng.integers(1, n // 3 + 1))
            X[-k:] = X[rng.integers(0, n - k, size=k)]           # duplicates
        if rng.random() < 0.5:
            z = X[int(rng.integers(0, n))].copy()
        else:                                                      # inside the hull, mostly
            z = np.rint(X[rng.integers(0, n, size=3)].mean(axis=0)).astype(np.int32)
        yield X, z


@pytest.mark.parametrize("seed", range(4))
def test_adia_never_below_exact(seed):
    searched = 0
    for X, z in _nd_cases(200 + seed, 40):
        T = oracle.depth(X, z)
        A, st = oracle.adia(X, z)
        assert A >= T, (X.tolist(), z.tolist(), A, T)
        searched += st["algorithm1"] == 0
    assert searched >= 10


@pytest.mark.parametrize("seed", range(3))
def test_adia_exact_in_general_position(seed):
    rng = np.random.default_rng(300 + seed)
    done = 0
    while done < 25:
        p = int(rng.integers(3, 6))
        n = int(rng.integers(2 * p + 2, 16))
        X = rng.integers(-1000, 1001, size=(n, p)).astype(np.int32)
        z = rng.integers(-300, 301, size=p).astype(np.int32)
        if not in_general_position(X, z):
            continue
        T = oracle.depth(X, z)
        A, st = oracle.adia(X, z)
        assert A == T, (X.tolist(), z.tolist(), A, T, st)
        done += 1


def test_adia_branches_without_search():
    rng = np.random.default_rng(9)
    # n <= 2p: Algorithm 1 directly
    X = rng.integers(-5, 6, size=(7, 4)).astype(np.int32)
    z = np.zeros(4, np.int32)
    A, st = oracle.adia(X, z)
    assert st["algorithm1"] == 1 and A == oracle.depth(X, z)
    # rank 2 data in p = 4: Algorithm 2 after the rank reduction
    B = rng.integers(-3, 4, size=(2, 4))
    X = (rng.integers(-4, 5, size=(20, 2)) @ B).astype(np.int32)
    A, st = oracle.adia(X, np.zeros(4, np.int32))
    assert st["algorithm1"] == 1 and A == oracle.depth(X, np.zeros(4, np.int32))
    # z outside the hull: the best data direction already has no point on its closed side
    X = rng.integers(1, 20, size=(30, 3)).astype(np.int32)
    z = np.array([-5, -5, -5], np.int32)
    A, st = oracle.adia(X, z)
    assert A == 0 and st["algorithm1"] == 1 and oracle.depth(X, z) == 0
    # the same with z at a data point outside the others' hull: T = Z
    X2 = np.vstack([X, z[None, :], z[None, :]])
    A, st = oracle.adia(X2, z)
    assert A == 2 == oracle.depth(X2, z)


def test_adia_search_counters():
    rng = np.random.default_rng(11)
    X = np.clip(np.rint(40 * rng.standard_normal((120, 4))), -127, 127).astype(np.int32)
    z = np.zeros(4, np.int32)
    A, st = oracle.adia(X, z)
    assert st["algorithm1"] == 0
    assert st["pops"] >= 1 and st["nodes"] >= 1 and st["step4_subsets"] >= st["pops"]
    assert st["d0_after_search"] >= A
    assert 4 - 2 <= st["union_points"] <= 120
    assert st["step5_subsets"] == st["union_points"] * (st["union_points"] - 1) // 2
    assert A == oracle.depth(X, z)


@pytest.mark.parametrize("req,query,n,T", [(20, 27, 343, 32), (376, 3, 426, 51)])
def test_adia_is_an_upper_bound_not_the_depth(req, query, n, T):
    """Queries of the seeded request stream where Algorithm 3 stops one above
    the exact count; in the first the optimal subsets are free of ties: the
    paper's observation that Algorithm 3 finds the depth does not hold for
    every input."""
    from paper_1409_3901_gb300 import workloads as W
    d = W.w5_request(4, req)
    z = d.Zq[query]
    assert d.n == n and d.p == 4
    A, st = oracle.adia(d.X, z)
    assert st["algorithm1"] == 0
    assert oracle.depth(d.X, z) == T
    assert A == T + 1
