"""Exact brute-force Tukey depth for tiny inputs, independent of the oracle.

Eq. (1) (Section 1) defines T = min over unit u of #{i : u'(X_i - z) <= 0}.
The minimum is taken in an open cell of the arrangement of the hyperplanes
u'x_i = 0 (x_i = X_i - z nonzero): a generic direction does at least as well as
any direction on a hyperplane.  Hence

    T = #{x_i = 0} + min over sign vectors s in {+1,-1}^{n'} that are realisable
        (some u has s_i u'x_i > 0 for every nonzero x_i) of #{i : s_i = -1}.

Realisability of a system of strict homogeneous inequalities a_i'u > 0 is
decided exactly by Fourier-Motzkin elimination on Python integers.  Nothing
here shares code or arithmetic with ``oracle/``: it never projects, sorts or
sweeps.

A second, polynomial check for p = 2 enumerates the halfplanes just beside
every critical line through the origin.

A third route takes the critical directions of Proposition 1 with r = p - 1:
the normals of the hyperplanes spanned by p - 1 nonzero points, each tilted
so that the points on the hyperplane take their best signs (found by the
sign-vector enumeration inside the hyperplane).
"""
from fractions import Fraction
from itertools import combinations
from math import gcd


def _normalise(row):
    g = 0
    for v in row:
        g = gcd(g, abs(v))
    if g > 1:
        row = tuple(v // g for v in row)
    return row


def strictly_feasible(rows):
    """True iff some u satisfies a'u > 0 for every a in rows (integer tuples)."""
    rows = {_normalise(tuple(r)) for r in rows}
    if not rows:
        return True
    d = len(next(iter(rows)))
    for var in range(d - 1, -1, -1):
        if any(all(v == 0 for v in r) for r in rows):
            return False  # 0 > 0
        pos = [r for r in rows if r[var] > 0]
        neg = [r for r in rows if r[var] < 0]
        new = {r[:var] for r in rows if r[var] == 0}
        for a in pos:
            for b in neg:
                c = tuple(a[j] * (-b[var]) + b[j] * a[var] for j in range(var))
                new.add(_normalise(c))
        rows = new
        if not rows:
            return True
    # every variable eliminated: each remaining row reads 0 > 0
    return not rows


def depth_bruteforce(X, z):
    """Exact closed-halfspace depth count by sign-vector enumeration (tiny n)."""
    X = [tuple(int(v) for v in row) for row in X]
    z = tuple(int(v) for v in z)
    xs = [tuple(a - b for a, b in zip(row, z)) for row in X]
    Z = sum(1 for x in xs if all(v == 0 for v in x))
    nz = [x for x in xs if any(v != 0 for v in x)]
    m = len(nz)
    for k in range(m + 1):  # fewest negatives first
        for neg in combinations(range(m), k):
            negset = set(neg)
            rows = [tuple(-v for v in x) if i in negset else x for i, x in enumerate(nz)]
            if strictly_feasible(rows):
                return Z + k
    raise AssertionError("unreachable: the all-positive or all-negative side of a cell exists")


def depth_p1(X, z):
    """p = 1 (Section 3): the smaller of #{X <= z} and #{X >= z}."""
    xs = [int(r[0]) - int(z[0]) for r in X]
    return min(sum(1 for v in xs if v <= 0), sum(1 for v in xs if v >= 0))


def depth_p2_halfplanes(X, z):
    """p = 2: count every closed halfplane through z just beside a critical line.

    The count is piecewise constant in the direction u and changes only where u
    is orthogonal to some nonzero x_i.  Each open arc between critical
    directions is sampled by u = d + eps*d_perp for a critical direction d
    (both orientations of both lines), with eps infinitesimal: then the sign of
    u'x is sign(d'x), or sign(d_perp'x) when d'x = 0.  O(n^2) in total.
    """
    xs = [(int(a) - int(z[0]), int(b) - int(z[1])) for a, b in X]
    Z = sum(1 for x in xs if x == (0, 0))
    nz = [x for x in xs if x != (0, 0)]
    if not nz:
        return Z
    best = None
    for (a, b) in nz:
        for d in ((-b, a), (b, -a)):           # directions orthogonal to x_i
            for side in (1, -1):
                dp = (-d[1] * side, d[0] * side)  # the two tilts
                cnt = 0
                for x in nz:
                    s = d[0] * x[0] + d[1] * x[1]
                    if s == 0:
                        s = dp[0] * x[0] + dp[1] * x[1]
                    if s < 0:
                        cnt += 1
                best = cnt if best is None else min(best, cnt)
    return Z + best


def _det(M):
    """Exact integer determinant by cofactor expansion along the first row."""
    n = len(M)
    if n == 0:
        return 1
    if n == 1:
        return M[0][0]
    return sum((-1) ** c * M[0][c] * _det([row[:c] + row[c + 1:] for row in M[1:]])
               for c in range(n) if M[0][c] != 0)


def depth_critical_normals(X, z):
    """T by the critical directions (Proposition 1 with r = p - 1), exactly.

    For p - 1 nonzero points J with independent rows, n_J (the cofactors of
    their p x (p-1) matrix, so n_J'x = det[x_J | x]) is normal to H = span J.
    A direction s n_J + eps v with v generic in H keeps the points off H on
    their side and splits the points on H by v alone, so the fewest points
    strictly below is #{s n_J'x < 0} + the open depth of the points on H
    inside H.  Every generic direction lies in an open cell whose closure has
    a ray spanned by some n_J when the nonzero points span R^p (or all lie on
    one hyperplane), hence T = Z + the minimum over J and s.  The open depth
    inside H is the sign-vector enumeration on the points of H with one
    coordinate where n_J is nonzero dropped (injective on H).
    """
    p = len(z)
    xs = [tuple(int(a) - int(b) for a, b in zip(row, z)) for row in X]
    Z = sum(1 for x in xs if all(v == 0 for v in x))
    nz = [x for x in xs if any(v != 0 for v in x)]
    if p == 1:
        return depth_p1(X, z)
    if not nz:
        return Z
    best = None
    for J in combinations(range(len(nz)), p - 1):
        rows = [nz[j] for j in J]
        n = tuple((-1) ** k * _det([list(r[:k] + r[k + 1:]) for r in rows]) for k in range(p))
        if all(v == 0 for v in n):
            continue
        jd = next(k for k in range(p) if n[k] != 0)
        dots = [sum(a * b for a, b in zip(n, x)) for x in nz]
        on_h = [x[:jd] + x[jd + 1:] for x, d in zip(nz, dots) if d == 0]
        od = depth_bruteforce(on_h, (0,) * (p - 1))
        v = min(sum(1 for d in dots if d < 0), sum(1 for d in dots if d > 0)) + od
        best = v if best is None else min(best, v)
    if best is None:
        raise ValueError("the nonzero points span less than a hyperplane")
    return Z + best


def _solve_exact(A, b):
    """The unique solution of the square or tall system A x = b in fractions,
    or None when the columns of A are dependent or the system is inconsistent."""
    rows, cols = len(A), len(A[0])
    M = [[Fraction(v) for v in A[r]] + [Fraction(b[r])] for r in range(rows)]
    piv_row = 0
    for c in range(cols):
        pr = next((r for r in range(piv_row, rows) if M[r][c] != 0), None)
        if pr is None:
            return None
        M[piv_row], M[pr] = M[pr], M[piv_row]
        for r in range(rows):
            if r != piv_row and M[r][c] != 0:
                f = M[r][c] / M[piv_row][c]
                M[r] = [a - f * b2 for a, b2 in zip(M[r], M[piv_row])]
        piv_row += 1
    if any(M[r][cols] != 0 for r in range(piv_row, rows)):
        return None
    return [M[r][cols] / M[r][r] for r in range(cols)]


def in_convex_hull(X, z):
    """z in conv(X), exactly: by Caratheodory, z is then a convex combination
    of at most p + 1 affinely independent rows, whose barycentric coordinates
    solve a system with a unique solution (Gaussian elimination in
    fractions)."""
    X = [tuple(int(v) for v in row) for row in X]
    z = tuple(int(v) for v in z)
    p = len(z)
    for k in range(1, min(p + 1, len(X)) + 1):
        for J in combinations(range(len(X)), k):
            A = [[X[j][c] for j in J] for c in range(p)] + [[1] * k]
            lam = _solve_exact(A, list(z) + [1])
            if lam is not None and all(v >= 0 for v in lam):
                return True
    return False
