"""Pins of the CPU oracle against what the paper and the mathematics fix.

* exact brute force on tiny inputs (sign-vector enumeration, tests/bruteforce.py),
  on random, tie-heavy, duplicated, antipodal, rank-deficient and deep cases;
* a second brute force through the critical directions (Proposition 1 with
  r = p - 1, the points on each hyperplane tilted to their best signs);
* the closed forms: p = 1 (Section 3) and an O(n^2) halfplane count for p = 2;
* invariances of Eq. (1): row permutation, integer translation, integer
  unimodular maps, positive integer scaling of X - z;
* bounds: 0 outside the bounding box, >= 1 at data points, Z <= T <= (n+Z)/2;
* T = 0 exactly when z lies outside conv(X) (an exact Caratheodory hull test);
* the paper's literal Algorithm 1 in float64 on data in general position
  (Proposition 1 holds there), and the two tie cases where it is wrong;
* the range form: a partition of the subset positions gives the full result.
"""
import numpy as np
import pytest

import oracle
from bruteforce import depth_bruteforce, depth_critical_normals, depth_p1, depth_p2_halfplanes, in_convex_hull
from paper_literal import in_general_position, literal_alg2, literal_rcom


def _cases(seed, count, pmax=6, nmax=9, lims=(1, 2, 3, 40)):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        p = int(rng.integers(1, pmax + 1))
        n = int(rng.integers(1, (nmax if p <= 4 else min(nmax, 7)) + 1))
        lim = int(rng.choice(lims))
        X = rng.integers(-lim, lim + 1, size=(n, p))
        if n > 1 and rng.random() < 0.35:
            X[-1] = X[int(rng.integers(0, n - 1))]            # duplicate row
        if n > 2 and rng.random() < 0.25:
            X[-2] = -X[0]                                      # antipodal through 0
        if rng.random() < 0.35:
            z = X[int(rng.integers(0, n))].copy()              # query at a data point
        else:
            z = rng.integers(-lim, lim + 1, size=p)
        yield X, z


@pytest.mark.parametrize("seed", range(6))
def test_oracle_matches_bruteforce_ties(seed):
    for X, z in _cases(1000 + seed, 250):
        assert oracle.depth(X, z) == depth_bruteforce(X, z), (X.tolist(), z.tolist())


@pytest.mark.parametrize("seed", range(3))
def test_oracle_matches_critical_normals(seed):
    """A second brute force through the critical directions (Proposition 1
    with r = p - 1), on the same tie-heavy families, wherever the nonzero
    centred points span at least a hyperplane."""
    checked = 0
    for X, z in _cases(3000 + seed, 150, pmax=6):
        xs = (X - z)[np.any(X != z, axis=1)]
        p = X.shape[1]
        if p == 1 or len(xs) == 0 or np.linalg.matrix_rank(xs.astype(float)) < p - 1:
            continue
        assert oracle.depth(X, z) == depth_critical_normals(X, z), (X.tolist(), z.tolist())
        checked += 1
    assert checked > 60


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_oracle_matches_bruteforce_deep(p):
    """Symmetric clouds around z give deep points (T well above 0)."""
    rng = np.random.default_rng(77 + p)
    n = 9 if p <= 4 else 7
    seen = set()
    for _ in range(40):
        half = rng.integers(-4, 5, size=((n + 1) // 2, p))
        X = np.vstack([half, -half[: n - len(half)]])
        X += rng.integers(-1, 2, size=X.shape) * (rng.random(X.shape) < 0.3)
        z = np.zeros(p, dtype=np.int64)
        t = oracle.depth(X, z)
        assert t == depth_bruteforce(X, z), (X.tolist(), z.tolist())
        seen.add(t)
    assert max(seen) >= 2


def _tight_case(rng, p):
    """Points concentrated on a few (p-2)-dimensional subspaces through z, with
    repeated coordinates so that the subset minor on the last rows can vanish,
    plus duplicates and positive multiples: many subsets whose span holds
    extra points (reading R6)."""
    k = p - 2
    pts = []
    for _ in range(2):
        B = rng.integers(-1, 2, size=(k, p))
        if rng.random() < 0.6:
            B[:, -1] = B[:, -2]                       # equal last two rows
        if rng.random() < 0.4:
            B[:, 0] = 0
        for _ in range(int(rng.integers(k, k + 3))):
            c = rng.integers(-2, 3, size=k)
            pts.append(c @ B)
    n = 8 if p <= 4 else 7
    while len(pts) < n:
        pts.append(rng.integers(-2, 3, size=p))
    X = np.array(pts[:n])
    if rng.random() < 0.5:
        X[-1] = 2 * X[0]
    return X, np.zeros(p, dtype=np.int64)


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_oracle_matches_bruteforce_tight_sets(p):
    rng = np.random.default_rng(1500 + p)
    for _ in range(120 if p <= 4 else 60):
        X, z = _tight_case(rng, p)
        sh = rng.integers(-5, 6, size=p)
        assert oracle.depth(X + sh, z + sh) == depth_bruteforce(X, z), (X.tolist(), z.tolist())


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_oracle_matches_bruteforce_twins(p):
    """Every point has a twin on its line through z (a copy, a positive
    multiple or a mirror image), so every subset's span holds extra points and
    the correction of reading R6 decides the result."""
    rng = np.random.default_rng(1700 + p)
    half = 4 if p <= 4 else 3
    for _ in range(80 if p <= 4 else 40):
        B = rng.integers(-2, 3, size=(half, p))
        B[rng.random(B.shape) < 0.3] = 0
        B[np.all(B == 0, axis=1), 0] = 1
        s = rng.choice([1, 1, 2, -1, -2], size=(half, 1))
        X = np.vstack([B, s * B])
        z = rng.integers(-4, 5, size=p)
        assert oracle.depth(X + z, z) == depth_bruteforce(X + z, z), (X.tolist(), z.tolist())


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_critical_normals_on_tight_sets_and_twins(p):
    """The critical-direction brute force on the two families where the
    tight-set correction decides the result (subsets whose span holds extra
    points)."""
    rng = np.random.default_rng(2500 + p)
    checked = 0
    for trial in range(60 if p <= 4 else 30):
        if trial % 2 == 0:
            X, z = _tight_case(rng, p)
        else:
            half = 4 if p <= 4 else 3
            B = rng.integers(-2, 3, size=(half, p))
            B[rng.random(B.shape) < 0.3] = 0
            B[np.all(B == 0, axis=1), 0] = 1
            X = np.vstack([B, rng.choice([1, 1, 2, -1, -2], size=(half, 1)) * B])
            z = np.zeros(p, dtype=np.int64)
        xs = X[np.any(X != 0, axis=1)]
        if len(xs) == 0 or np.linalg.matrix_rank(xs.astype(float)) < p - 1:
            continue
        assert oracle.depth(X, z) == depth_critical_normals(X, z), (X.tolist(), z.tolist())
        checked += 1
    assert checked >= (20 if p <= 4 else 10)


@pytest.mark.parametrize("seed", range(2))
def test_zero_depth_exactly_outside_the_hull(seed):
    """T = 0 iff z lies outside conv(X) (a closed halfspace through z misses
    every data point iff z can be separated strictly), checked by an exact
    hull test that shares nothing with either brute force."""
    outside = inside = 0
    for X, z in _cases(4000 + seed, 200, pmax=6, nmax=8):
        t = oracle.depth(X, z)
        hull = in_convex_hull(X, z)
        assert (t == 0) == (not hull), (X.tolist(), z.tolist(), t)
        outside += not hull
        inside += hull
    assert outside > 20 and inside > 20


@pytest.mark.parametrize("p,r", [(3, 1), (3, 2), (4, 1), (4, 2), (4, 3), (5, 2), (5, 3), (6, 3), (6, 4), (6, 5)])
def test_oracle_rank_deficient(p, r):
    """Nonzero x_i spanning r < p dimensions (reading R7)."""
    rng = np.random.default_rng(10 * p + r)
    for _ in range(15):
        B = rng.integers(-2, 3, size=(r, p))
        n = int(rng.integers(r, 8 if p <= 4 else 7))
        C = rng.integers(-2, 3, size=(n, r))
        z = rng.integers(-3, 4, size=p)
        X = C @ B + z
        assert oracle.depth(X, z) == depth_bruteforce(X, z)


def test_bruteforce_closed_forms():
    """The brute force itself agrees with the p=1 and p=2 closed forms."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(1, 10))
        X = rng.integers(-3, 4, size=(n, 1))
        z = rng.integers(-3, 4, size=1)
        assert depth_bruteforce(X, z) == depth_p1(X, z)
        X = rng.integers(-3, 4, size=(n, 2))
        z = rng.integers(-3, 4, size=2)
        assert depth_bruteforce(X, z) == depth_p2_halfplanes(X, z)


@pytest.mark.parametrize("p", [1, 2])
def test_oracle_closed_forms_larger(p):
    rng = np.random.default_rng(31 + p)
    ref = depth_p1 if p == 1 else depth_p2_halfplanes
    for _ in range(60):
        n = int(rng.integers(1, 60))
        lim = int(rng.choice([2, 5, 100]))
        X = rng.integers(-lim, lim + 1, size=(n, p))
        z = X[0].copy() if rng.random() < 0.3 else rng.integers(-lim, lim + 1, size=p)
        assert oracle.depth(X, z) == ref(X, z)


def _unimodular(rng, p, steps=6):
    A = np.eye(p, dtype=np.int64)
    for _ in range(steps):
        i, j = rng.choice(p, 2, replace=False)
        A[i] += int(rng.choice([-1, 1])) * A[j]
    if rng.random() < 0.5:
        A[0] = -A[0]
    return A


@pytest.mark.parametrize("p", [3, 4, 5])
def test_oracle_invariances(p):
    rng = np.random.default_rng(400 + p)
    n = {3: 40, 4: 24, 5: 14}[p]
    for trial in range(4):
        X = rng.integers(-20, 21, size=(n, p))
        if trial % 2:
            X[: n // 4] = X[n // 4: 2 * (n // 4)]
        z = X[3].copy() if trial == 1 else rng.integers(-5, 6, size=p)
        T = oracle.depth(X, z)
        perm = rng.permutation(n)
        assert oracle.depth(X[perm], z) == T
        sh = rng.integers(-30, 31, size=p)
        assert oracle.depth(X + sh, z + sh) == T
        A = _unimodular(rng, p)
        assert oracle.depth(X @ A.T, A @ z) == T
        s = int(rng.integers(2, 4))
        assert oracle.depth(z + s * (X - z), z) == T


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_oracle_bounds(p):
    rng = np.random.default_rng(600 + p)
    n = {3: 30, 4: 18, 5: 12, 6: 9}[p]
    X = rng.integers(-10, 11, size=(n, p))
    X[1] = X[0]
    outside = X.max(axis=0) + 1
    assert oracle.depth(X, outside) == 0
    assert oracle.depth(X, X.min(axis=0) - np.arange(1, p + 1)) == 0
    for i in range(0, n, 3):
        z = X[i]
        Z = int(np.all(X == z, axis=1).sum())
        T = oracle.depth(X, z)
        assert T >= 1 and T >= Z and T <= (n + Z) // 2
    for _ in range(4):
        z = rng.integers(-10, 11, size=p)
        Z = int(np.all(X == z, axis=1).sum())
        T = oracle.depth(X, z)
        assert Z <= T <= (n + Z) // 2


def test_all_points_at_z():
    X = np.tile(np.array([[3, -1, 2, 5]]), (7, 1))
    assert oracle.depth(X, X[0]) == 7


@pytest.mark.parametrize("p", [3, 4, 5])
def test_literal_paper_general_position(p):
    """Proposition 1 / Algorithm 1 as printed, on data in general position."""
    rng = np.random.default_rng(800 + p)
    n = {3: 16, 4: 12, 5: 10}[p]
    done = 0
    while done < 6:
        X = rng.integers(-800, 801, size=(n, p))
        z = rng.integers(-150, 151, size=p) if done % 2 else np.round(X.mean(axis=0)).astype(np.int64)
        if not in_general_position(X, z):
            continue
        assert oracle.depth(X, z) == literal_rcom(X, z)
        done += 1


def test_literal_paper_fails_under_ties():
    """The two tie cases where the printed algorithms are wrong (readings R5, R6)."""
    # Algorithm 2 flips one point at a time: on {(1,1), (-1,-1)} it returns 0,
    # but every closed halfplane through 0 holds at least one of the two points.
    Y = np.array([[1, 1], [-1, -1]])
    assert literal_alg2(Y) == 0
    assert oracle.bivariate_closed(Y) == 1
    assert depth_p2_halfplanes(Y, [0, 0]) == 1
    # Algorithm 1 with a duplicated point set, truth 2: as printed it returns 1
    # (the one-at-a-time flips under-count first); with the bivariate counts
    # made exact its "- (p-2)" over-estimates and returns 3.
    A = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, -1, -1]])
    X = np.vstack([A, A])
    z = np.zeros(3, dtype=np.int64)
    assert literal_rcom(X, z) == 1
    assert literal_rcom(X, z, grouped=True) == 3
    assert oracle.depth(X, z) == 2
    assert depth_bruteforce(X, z) == 2


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_range_partition(p):
    rng = np.random.default_rng(900 + p)
    n = {2: 20, 3: 25, 4: 15, 5: 11}[p]
    X = rng.integers(-6, 7, size=(n, p))
    X[2] = X[5]
    for z in (X[0], rng.integers(-3, 4, size=p)):
        T = oracle.depth(X, z)
        _, npos, _ = oracle.depth_range(X, z, 0, 1)
        cuts = sorted(set([0, npos] + list(rng.integers(0, npos + 1, size=3))))
        parts = [oracle.depth_range(X, z, a, b)[0] for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        assert min(v for v in parts if v is not None) == T


def test_oracle_rejects_bad_input():
    with pytest.raises(oracle.OracleError):
        oracle.depth(np.zeros((3, 7), np.int32), np.zeros(7, np.int32))
    big = np.array([[2_000_000_000, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0]], np.int64)
    with pytest.raises(oracle.OracleError):
        oracle.depth(big.astype(np.int32), np.array([-2_000_000_000, 0, 0, 0, 0, 0], np.int32))


@pytest.mark.parametrize("p", [3, 4, 5, 6])
def test_subset_min_over_colex_partitions(p):
    """oracle.subset_min (Z + min V(S) over listed subsets, the form in which
    sampled ranges of the library's colex subset loop are checked): over all
    subsets it is the depth, which the brute force pins; over any partition
    of the colex ranks into contiguous ranges the minimum of the parts is the
    depth; a listed dependent subset (two equal points) is counted and
    skipped; the order of the list does not matter."""
    from math import comb

    from subsets import colex_range, shard_range
    rng = np.random.default_rng(700 + p)
    n = {3: 30, 4: 18, 5: 13, 6: 11}[p]
    for trial in range(3):
        X = rng.integers(-3, 4, size=(n, p)).astype(np.int32)
        X[-2:] = X[2:4]                                        # duplicates
        z = X[0] if trial == 0 else rng.integers(-1, 2, size=p).astype(np.int32)
        if oracle.rank(X, z)[0] < p:
            continue
        want = oracle.depth(X, z)
        if n <= 13:
            assert want == depth_bruteforce(X, z)
        nnz = int(n - np.all(X == z, axis=1).sum())
        k = p - 2
        allc = colex_range(k, 0, comb(nnz, k))
        v, dep = oracle.subset_min(X, z, allc)
        assert v == want
        v2, dep2 = oracle.subset_min(X, z, allc[::-1])
        assert (v2, dep2) == (v, dep)
        S = int(rng.integers(2, 9))
        parts = [oracle.subset_min(X, z, colex_range(k, *shard_range(nnz, k, s, S)))[0] for s in range(S)]
        assert min(x for x in parts if x is not None) == want
    # two equal nonzero points make a dependent subset (p = 4: S = {i, j})
    X = np.array([[1, 0, 0, 0], [1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1], [-1, -1, -1, -1]],
                 np.int32)
    v, dep = oracle.subset_min(X, np.zeros(4, np.int32), [[0, 1]])
    assert v is None and dep == 1
