"""The paper's Algorithms 1 and 2 taken literally, in float64 (test use only).

Algorithm 1 (Section 3): for every (p-2)-subset, an orthonormal basis e1, e2
of the orthogonal complement of the subset's span; the bivariate depth of the
projected points; N_min the smallest such count; return N_min - (p-2).
Algorithm 2 (Section 3): drop the zero points, slopes theta = -y1/y2, start at
u0 = (0,-1) with L_i = [y_i2 <= 0], S1 = sum L, sort the slopes and flip one
point at a time, tracking min(S1, m - S1); return M_min + n - m.

Exact only for data in general position (Section 2); used to check the oracle
on such data and to document the two failure cases under ties.
"""
from itertools import combinations

import numpy as np


def literal_alg2(y, tol=1e-9, grouped=False):
    """Algorithm 2 as printed; grouped=True flips equal slopes together and
    starts from a generic direction next to u0 (the tie readings), still in
    float64 with a tolerance."""
    y = np.asarray(y, dtype=np.float64)
    n = len(y)
    scale = max(1.0, float(np.abs(y).max())) if n else 1.0
    nz = y[np.abs(y).max(axis=1) > tol * scale] if n else y
    m = len(nz)
    if m == 0:
        return n
    if grouped:
        t = tol * scale
        L = ((nz[:, 1] < -t) | ((np.abs(nz[:, 1]) <= t) & (nz[:, 0] > 0))).astype(int)
        S1 = int(L.sum())
        M = min(S1, m - S1)
        ev = np.nonzero(np.abs(nz[:, 1]) > t)[0]
        theta = -nz[ev, 0] / nz[ev, 1]
        order = ev[np.argsort(theta, kind="stable")]
        th = -nz[order, 0] / nz[order, 1]
        g = 0
        while g < len(order):
            h = g
            while h < len(order) and abs(th[h] - th[g]) <= 1e-9 * (1 + abs(th[g])):
                S1 += 1 if L[order[h]] == 0 else -1
                h += 1
            M = min(M, min(S1, m - S1))
            g = h
        return M + n - m
    with np.errstate(divide="ignore", invalid="ignore"):
        theta = -nz[:, 0] / nz[:, 1]
    L = (nz[:, 1] <= 0).astype(int)
    S1 = int(L.sum())
    M = min(S1, m - S1)
    for j in np.argsort(theta, kind="stable"):
        S1 += 1 if L[j] == 0 else -1
        M = min(M, min(S1, m - S1))
    return M + n - m


def literal_rcom(X, z, grouped=False):
    x = np.asarray(X, dtype=np.float64) - np.asarray(z, dtype=np.float64)
    n, p = x.shape
    Nmin = n
    for I in combinations(range(n), p - 2):
        A = x[list(I)].T
        Q, _ = np.linalg.qr(A, mode="complete")
        e = Q[:, p - 2:]
        Nmin = min(Nmin, literal_alg2(x @ e, grouped=grouped))
    return Nmin - (p - 2)


def int_det(rows):
    """Exact determinant of a square integer matrix (Bareiss on Python ints)."""
    m = [list(map(int, r)) for r in rows]
    d = len(m)
    prev, sign = 1, 1
    for k in range(d - 1):
        if m[k][k] == 0:
            sw = next((r for r in range(k + 1, d) if m[r][k] != 0), None)
            if sw is None:
                return 0
            m[k], m[sw] = m[sw], m[k]
            sign = -sign
        for r in range(k + 1, d):
            for c in range(k + 1, d):
                m[r][c] = (m[r][c] * m[k][k] - m[r][k] * m[k][c]) // prev
            m[r][k] = 0
        prev = m[k][k]
    return sign * m[d - 1][d - 1]


def in_general_position(X, z):
    """No p+1 of the points X_1..X_n, z on a common affine hyperplane."""
    pts = [list(map(int, r)) for r in X] + [list(map(int, z))]
    p = len(pts[0])
    for sub in combinations(range(len(pts)), p + 1):
        rows = [pts[i] + [1] for i in sub]
        if int_det(rows) == 0:
            return False
    return True
