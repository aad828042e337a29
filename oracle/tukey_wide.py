"""TEST INFRASTRUCTURE ONLY: the oracle for int32 inputs of any magnitude.

The same computation as tukey_oracle.c -- T = n * D_n(z) of Eq. (1) by the
subset loop of Algorithm 1 (Section 3) with Algorithm 2 as the inner count,
readings R1-R8 of that file -- in Python integers, so that no intermediate
has a bound: centred coordinates reach 2^32 - 1, the functionals f_a, f_b
about 2^170 at p = 6 and the slope comparisons twice that.  The C oracle
rejects such inputs (coord_bound_ok); this one is slow and meant for small
data (tens of points).

Pins (tests/test_oracle_wide.py): agreement with the C oracle on inputs both
accept, the brute force of tests/bruteforce.py at full-range magnitudes,
Eq. (1)'s invariance under positive integer scaling of the centred data
(in-range data scaled up to the int32 range) and under integer unimodular
maps.
"""
from itertools import combinations


def _det(M):
    """Exact determinant of a square integer matrix (Bareiss elimination;
    every intermediate is a minor of M, every division exact)."""
    A = [list(r) for r in M]
    n = len(A)
    if n == 0:
        return 1
    sign, prev = 1, 1
    for k in range(n - 1):
        if A[k][k] == 0:
            sw = next((r for r in range(k + 1, n) if A[r][k] != 0), None)
            if sw is None:
                return 0
            A[k], A[sw] = A[sw], A[k]
            sign = -sign
        for r in range(k + 1, n):
            for c in range(k + 1, n):
                A[r][c] = (A[r][c] * A[k][k] - A[r][k] * A[k][c]) // prev
            A[r][k] = 0
        prev = A[k][k]
    return sign * A[n - 1][n - 1]


def _rank_pivots(pts, d):
    """Rank of the rows of pts and the pivot columns (increasing) of an exact
    elimination: the projection onto them is injective on the row span (R7)."""
    basis, pcols = [], []
    for x in pts:
        v = list(x)
        for b, pc in zip(basis, pcols):
            f = v[pc]
            if f:
                e = b[pc]
                v = [e * vi - f * bi for vi, bi in zip(v, b)]
        lead = next((c for c in range(d) if v[c] != 0), None)
        if lead is None:
            continue
        basis.append(v)
        pcols.append(lead)
        if len(basis) == d:
            break
    return len(basis), sorted(pcols)


def _closed_bivariate(ys):
    """Algorithm 2 (Section 3) on the projected points ys with readings R3-R5:
    (closed count, M) where M is the least number of nonzero points strictly
    on one side over generic directions and the closed count adds the zero
    projections (step 2 as a count)."""
    nz = [y for y in ys if y != (0, 0)]
    m = len(nz)
    if m == 0:
        return len(ys), 0
    # R4: the side of each point at u = (eps, -1); R3: slopes -y1/y2 as fractions
    side = [(y2 < 0) or (y2 == 0 and y1 > 0) for y1, y2 in nz]
    s1 = sum(side)
    best = min(s1, m - s1)
    finite = []
    for j, (y1, y2) in enumerate(nz):
        if y2 != 0:
            num, den = (-y1, y2) if y2 > 0 else (y1, -y2)
            finite.append((num, den, j))
    # sort by exact slope (num/den, den > 0); ties stay together
    from functools import cmp_to_key

    def cmp(a, b):
        l, r = a[0] * b[1], b[0] * a[1]
        return (l > r) - (l < r)
    finite.sort(key=cmp_to_key(cmp))
    g = 0
    while g < len(finite):               # R5: flip a whole tie group, then read
        h = g
        while h < len(finite) and cmp(finite[g], finite[h]) == 0:
            s1 += -1 if side[finite[h][2]] else 1
            h += 1
        best = min(best, s1, m - s1)
        g = h
    return best + (len(ys) - m), best


def _count(pts, d):
    """The depth count of the origin for the integer points pts (rows of
    length d), Algorithm 1 with R2, R6, R7 (the body of tukey_oracle.c's
    depth_count, without the subset-range form)."""
    cnt = len(pts)
    Z = sum(1 for x in pts if not any(x))
    if Z == cnt:
        return cnt
    r, piv = _rank_pivots(pts, d)
    pts = [tuple(x[c] for c in piv) for x in pts]
    d = r
    if d == 1:
        pos = sum(1 for x in pts if x[0] > 0)
        neg = sum(1 for x in pts if x[0] < 0)
        return Z + min(pos, neg)
    if d == 2:
        return _closed_bivariate([tuple(x) for x in pts])[0]
    k = d - 2
    best = None
    for S in combinations(range(cnt), k):
        xs = [pts[i] for i in S]

        def unit(a):
            return [1 if i == a else 0 for i in range(d)]

        def det_cols(cols):
            return _det([[cols[j][i] for j in range(d)] for i in range(d)])
        # R2: the first row pair (a, b) with det[x_S | e_a | e_b] != 0
        ab = next(((a, b) for a in range(d) for b in range(a + 1, d)
                   if det_cols(xs + [unit(a), unit(b)]) != 0), None)
        if ab is None:
            continue                     # dependent subset, skipped
        a, b = ab
        ca = [det_cols(xs + [unit(j), unit(a)]) for j in range(d)]
        cb = [det_cols(xs + [unit(j), unit(b)]) for j in range(d)]
        ys, tight = [], []
        for x in pts:
            y = (sum(c * v for c, v in zip(ca, x)), sum(c * v for c, v in zip(cb, x)))
            ys.append(y)
            if any(x) and y == (0, 0):
                # R6: tight point, kept on the rows other than a and b
                tight.append(tuple(x[j] for j in range(d) if j != a and j != b))
        N, _ = _closed_bivariate(ys)
        t = len(tight)
        mS = _count(tight, k) if t > k else 0
        V = N - t + mS
        best = V if best is None else min(best, V)
    return best


def depth(X, z):
    """T = n * D_n(z) of z w.r.t. the rows of X (int32 values of any size)."""
    z = [int(v) for v in z]
    pts = [tuple(int(a) - b for a, b in zip(row, z)) for row in X]
    return _count(pts, len(z))


def depth_many(X, Z):
    return [depth(X, z) for z in Z]
