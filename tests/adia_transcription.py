"""A second, independent transcription of Algorithm 3 (ADIA, Section 4) in
plain Python with exact integers -- test infrastructure that pins the
oracle's traversal (oracle.adia) to the paper's steps.

It is written from Algorithm 3 (Steps 1-6) and the readings A1-A7 the oracle
documents, shares no code with oracle/, and computes every ingredient its own
way:

  - V(S) (A1, reading R6) as Z + G(S) + m_S, where G(S) is found by listing
    the cells of the line arrangement of the projected points directly (not
    by Algorithm 2's walk) and m_S, the open depth of the tight points inside
    span(S), by the sign-vector brute force of tests/bruteforce.py;
  - the critical points (A2) as the points whose line bounds a cell of count
    G(S);
  - Steps 2-5 in the paper's order with the choices of A3-A6.

Full-rank data only (the nonzero centred points span R^p; reading R7's
reduction is not transcribed) and small n: it is slow.  The counters follow
oracle.ADIA_STATS: pops (Step 4 pops), step4_subsets (subsets evaluated in
Step 4(a)(i)), nodes (pushes into Q, Step 2 included), max_stack (largest N),
union_points (nonzero points of the Step 5(a) union), step5_subsets
(subsets visited in Step 5(b), dependent ones included), d0_after_search (d0 when Step 4
ends), algorithm1 (1 when the search is skipped: A7 hands the query to
Algorithm 1, or A5 finds the count Z at once), union_hash (the sum of
(i + 1)^3 over the union's nonzero points i in data order: the union itself).
"""
from fractions import Fraction
from functools import cmp_to_key
from itertools import combinations

from bruteforce import depth_bruteforce


def _det(M):
    """Exact determinant of a square integer matrix (fraction-free elimination)."""
    A = [list(r) for r in M]
    n = len(A)
    sign, prev = 1, 1
    for k in range(n - 1):
        piv = next((i for i in range(k, n) if A[i][k] != 0), None)
        if piv is None:
            return 0
        if piv != k:
            A[k], A[piv] = A[piv], A[k]
            sign = -sign
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                A[i][j] = (A[i][j] * A[k][k] - A[i][k] * A[k][j]) // prev
        prev = A[k][k]
    return sign * A[n - 1][n - 1] if n else 1


def _rank(vectors, p):
    rows = [[Fraction(v) for v in x] for x in vectors]
    r = 0
    for c in range(p):
        piv = next((i for i in range(r, len(rows)) if rows[i][c] != 0), None)
        if piv is None:
            continue
        rows[r], rows[piv] = rows[piv], rows[r]
        for i in range(len(rows)):
            if i != r and rows[i][c] != 0:
                f = rows[i][c] / rows[r][c]
                rows[i] = [a - f * b for a, b in zip(rows[i], rows[r])]
        r += 1
    return r


def _unit(p, a):
    return [1 if i == a else 0 for i in range(p)]


def _columns_det(cols):
    """det of the matrix whose columns are cols."""
    p = len(cols)
    return _det([[cols[j][i] for j in range(p)] for i in range(p)])


def _functionals(xs_S, p):
    """R2: the first row pair (a, b) with det[x_S | e_a | e_b] != 0 and the
    functionals f_a(x) = det[x_S | x | e_a], f_b(x) = det[x_S | x | e_b], or
    None when S is dependent."""
    for a in range(p):
        for b in range(a + 1, p):
            if _columns_det(list(xs_S) + [_unit(p, a), _unit(p, b)]) != 0:
                return (lambda x, a=a: _columns_det(list(xs_S) + [list(x), _unit(p, a)]),
                        lambda x, b=b: _columns_det(list(xs_S) + [list(x), _unit(p, b)]))
    return None


def _cross(u, v):
    return u[0] * v[1] - u[1] * v[0]


def _line_key(y):
    """The direction of the line through 0 and y, as a representative with
    y2 > 0, or y2 = 0 and y1 > 0."""
    return y if (y[1] > 0 or (y[1] == 0 and y[0] > 0)) else (-y[0], -y[1])


def _cells(ys):
    """(G, lines, counts): the lines through the nonzero projected points in
    angular order over [0, pi), and the count min(#left, #right) of the
    halfplane whose boundary lies strictly between consecutive lines (cell c
    lies between line c and line c+1, the last one wrapping round)."""
    nz = [y for y in ys if y != (0, 0)]
    if not nz:
        return 0, [], []
    keys = {}
    for y in nz:
        k = _line_key(y)
        keys.setdefault(k, k)

    def cmp(u, v):
        # angle in [0, pi): u before v when v is counter-clockwise of u
        c = _cross(u, v)
        return -1 if c > 0 else (1 if c < 0 else 0)
    lines = []
    for k in sorted(keys.values(), key=cmp_to_key(cmp)):
        if not lines or _cross(lines[-1], k) != 0:
            lines.append(k)
    counts = []
    L = len(lines)
    for c in range(L):
        a, b = lines[c], lines[(c + 1) % L]
        if L == 1:
            d = (-a[1], a[0])            # a normal of the only line: the two sides are the cells
            w = (a[0] + d[0], a[1] + d[1])
        elif c + 1 < L:
            w = (a[0] + b[0], a[1] + b[1])
        else:
            w = (a[0] - b[0], a[1] - b[1])  # between the last line and the first one reversed
        # boundary direction w strictly inside the cell; count both sides
        left = sum(1 for y in nz if _cross(w, y) > 0)
        right = sum(1 for y in nz if _cross(w, y) < 0)
        counts.append(min(left, right))
    return min(counts), lines, counts


def subset_eval(xs, S, p):
    """(V, critical) for the subset S (indices into the centred points xs) or
    None when S is dependent.  V = Z + G(S) + m_S (A1 with reading R6);
    critical = the indices whose projected point lies on a line bounding a
    cell of count G(S) (A2)."""
    xs_S = [xs[i] for i in S]
    fs = _functionals(xs_S, p)
    if fs is None:
        return None
    fa, fb = fs
    Z = sum(1 for x in xs if not any(x))
    ys = [(fa(x), fb(x)) for x in xs]
    G, lines, counts = _cells(ys)
    tight = [i for i, (x, y) in enumerate(zip(xs, ys)) if any(x) and y == (0, 0)]
    m = 0
    if len(tight) > p - 2:
        # open depth of the tight points inside span(S): coordinates in the
        # basis x_S (exact fractions, scaled to integers per point)
        coords = []
        for i in tight:
            lam = _solve_in_span(xs_S, xs[i], p)
            den = 1
            for v in lam:
                den = den * v.denominator // _gcd(den, v.denominator)
            coords.append([int(v * den) for v in lam])
        m = depth_bruteforce(coords, [0] * (p - 2))
    crit = set()
    L = len(lines)
    for c in range(L):
        if counts[c] == G:
            for bound in (lines[c], lines[(c + 1) % L]):
                for i, y in enumerate(ys):
                    if y != (0, 0) and _cross(bound, y) == 0:
                        crit.add(i)
    return Z + G + m, crit


def _gcd(a, b):
    while b:
        a, b = b, a % b
    return a


def _solve_in_span(basis, x, p):
    """lam with sum lam_j basis_j = x (x lies in the span; basis independent)."""
    k = len(basis)
    rows = [[Fraction(basis[j][i]) for j in range(k)] + [Fraction(x[i])] for i in range(p)]
    r, piv_cols = 0, []
    for c in range(k):
        piv = next((i for i in range(r, p) if rows[i][c] != 0), None)
        rows[r], rows[piv] = rows[piv], rows[r]
        for i in range(p):
            if i != r and rows[i][c] != 0:
                f = rows[i][c] / rows[r][c]
                rows[i] = [a - f * b for a, b in zip(rows[i], rows[r])]
        piv_cols.append(c)
        r += 1
    return [rows[j][k] / rows[j][j] for j in range(k)]


def adia(X, z):
    """Algorithm 3 on the rows of X and the query z: (count, counters)."""
    p = len(z)
    xs = [tuple(int(a) - int(b) for a, b in zip(row, z)) for row in X]
    n = len(xs)
    nz = [i for i in range(n) if any(xs[i])]
    Z = n - len(nz)
    st = dict(pops=0, step4_subsets=0, nodes=0, max_stack=0, union_points=0, step5_subsets=0,
              d0_after_search=0, algorithm1=0, union_hash=0)
    assert _rank([xs[i] for i in nz], p) == p, "full-rank data only"
    k = p - 2
    if p < 3 or len(nz) <= 2 * p:
        st["algorithm1"] = 1
        return depth_bruteforce(X, z), st

    dot = lambda u, x: sum(a * b for a, b in zip(u, x))
    # Step 2(a), A4: the data direction with the least closed count
    best = None
    for j in nz:
        for sg in (1, -1):
            u = tuple(sg * v for v in xs[j])
            c = sum(1 for x in xs if dot(u, x) <= 0)
            if best is None or c < best[0]:
                best = (c, u)
    u = best[1]
    # Step 2(b): the nonzero points ordered by u'x, ties by index
    order = sorted(nz, key=lambda i: (dot(u, xs[i]), i))
    kneg = sum(1 for i in nz if dot(u, xs[i]) < 0)
    if not any(dot(u, xs[i]) <= 0 for i in nz):     # A5: "k does not exist"
        st["algorithm1"] = 1
        return Z, st
    # A5: the start subset, greedily from position kneg onward, wrapping round
    S0 = []
    for pos in list(range(kneg, len(order))) + list(range(0, kneg)):
        i = order[pos]
        if _rank([xs[j] for j in S0 + [i]], p) == len(S0) + 1:
            S0.append(i)
        if len(S0) == k:
            break
    S0 = tuple(sorted(S0))
    V0, crit0 = subset_eval(xs, S0, p)
    # Step 2(c): the critical point of least index outside S0
    h = min(i for i in crit0 if i not in S0)
    C = (tuple(sorted(S0 + (h,))), V0)
    # Steps 1 and 3: Q (nodes, not deleted) and the stack N
    Q = {C[0]: C[1]}
    N = [C]
    st["nodes"] = 1
    st["max_stack"] = 1
    d0 = C[1]
    # Step 4
    while N:
        node, _ = N.pop()
        st["pops"] += 1
        for S in combinations(node, k):        # A3: lexicographic order
            st["step4_subsets"] += 1
            ev = subset_eval(xs, S, p)
            if ev is None:
                continue
            dtemp, crit = ev
            for t in sorted(i for i in crit if i not in node):   # (ii), A3: increasing index
                key = tuple(sorted(S + (t,)))
                if key not in Q:                                 # (iii)(B)
                    Q[key] = dtemp
                    N.append((key, dtemp))
                    st["nodes"] += 1
                    st["max_stack"] = max(st["max_stack"], len(N))
            if d0 > dtemp:                                       # (iv)
                d0 = dtemp
                break
        # Step 4(b): delete the nodes deeper than d0
        Q = {key: dep for key, dep in Q.items() if dep <= d0}
        N = [(key, dep) for key, dep in N if dep <= d0]
    st["d0_after_search"] = d0
    # Step 5(a), A6: the smaller closed side of every remaining node's hyperplane
    union = set()
    for F in sorted(Q):
        xs_F = [xs[i] for i in F]
        side = [_columns_det(xs_F + [x]) for x in xs]
        le = [i for i in range(n) if side[i] <= 0]
        ge = [i for i in range(n) if side[i] >= 0]
        if len(le) != len(ge):
            pick = le if len(le) < len(ge) else ge
        else:
            first_off = min(i for i in range(n) if side[i] != 0)
            pick = le if side[first_off] < 0 else ge
        union.update(pick)
    un = sorted(i for i in union if any(xs[i]))
    st["union_points"] = len(un)
    st["union_hash"] = sum((i + 1) ** 3 for i in un)
    # Step 5(b): Algorithm 1 over the (p-2)-subsets of the union
    for S in combinations(un, k):
        st["step5_subsets"] += 1
        ev = subset_eval(xs, S, p)
        if ev is not None:
            d0 = min(d0, ev[0])
    return d0, st
