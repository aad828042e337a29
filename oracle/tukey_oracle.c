/*
 * tukey_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU oracle for the sample Tukey (halfspace)
 * depth count
 *
 *     T(X, z) = n * D_n(z) = min over unit u of #{ i : u'(X_i - z) <= 0 }     (Eq. 1, Section 1)
 *
 * computed with the structure of the paper's first exact algorithm: the loop of
 * Algorithm 1 (Section 3) over all (p-2)-subsets of the centred data, each
 * projected onto the 2-D quotient of R^p by the span of the subset, with the
 * bivariate count of Algorithm 2 (Section 3) as the inner step.  Arithmetic is
 * exact: int64 coordinates, __int128 for every product.
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU
 * baseline may load this file's library.  It shares no code, header or table
 * with the CUDA library of this repository.
 *
 * Readings of the paper taken here (the paper assumes that X and 0 are in
 * general position, Section 2; the inputs this oracle serves are not):
 *
 *  R1  Centring (Section 2): x_i = X_i - z.  Zero vectors x_i = 0 are counted by
 *      every closed halfspace; they are the Z term of the result.
 *  R2  Algorithm 1 step 1(a) asks for two orthogonal vectors of the orthogonal
 *      complement of span(x_S).  Any basis of that complement gives the same
 *      bivariate depth (the depth of 0 is invariant under linear isomorphisms of
 *      the quotient), so the two integer functionals
 *          f_a(x) = det[x_S | x | e_a],   f_b(x) = det[x_S | x | e_b]
 *      are used, for the first row pair (a, b) whose kappa = det[x_S|e_a|e_b]
 *      is nonzero.  Subsets with no such pair (rank < p-2: repeated points,
 *      zero points, dependent points) are skipped: they are never needed.
 *  R3  Algorithm 2 step 1(b) divides by y_i2, which can be zero.  The slopes
 *      theta_i = -y_i1 / y_i2 are kept as exact fractions; points with
 *      y_i2 = 0 have no finite slope and never change side during the sweep.
 *  R4  Algorithm 2 step 1(c) starts at u0 = (0,-1), which is not a generic
 *      direction when some y_i2 = 0.  The sweep starts at u0 rotated by an
 *      infinitesimal angle towards increasing theta, i.e. u = (eps, -1): the
 *      starting side of y is sign(-y_2), or sign(y_1) when y_2 = 0.
 *  R5  Algorithm 2 step 1(e) flips points one at a time; with equal slopes the
 *      intermediate counts are not counts of any direction.  All points of a
 *      group of exactly equal slopes are flipped together before the count is
 *      read.
 *  R6  Algorithm 1 step 2 subtracts p-2 from the minimum.  That is exact only
 *      when the subset's span holds no data point besides the subset itself.
 *      In general each subset S contributes
 *          V(S) = N(S) - t_S + m_S,
 *      where N(S) is Algorithm 2's closed count on the projected points (zero
 *      projections counted), t_S is the number of nonzero x_i lying in
 *      span(x_S) (they project to zero), and m_S is the open depth of those
 *      t_S points inside span(x_S): the least number of them that a small
 *      tilt of the direction out of the quotient must leave on the negative
 *      side.  m_S is computed by the same procedure one level down, in the
 *      coordinates of the p-2 rows other than a and b (on which the subset's
 *      minor is kappa != 0, so that projection is injective on span(x_S)).
 *      In general position t_S = p-2 and m_S = 0, which is the paper's formula.
 *  R7  If the nonzero x_i span a space of dimension r < p, the problem is the
 *      same problem in r dimensions (directions orthogonal to the span change
 *      nothing); the points are expressed in r coordinates on which the span
 *      projects injectively (pivot columns of an exact elimination).  r = 1 is
 *      the trivial p = 1 case of Section 3 (the smaller of the two side counts)
 *      and r = 2 is Algorithm 2 alone.
 *  R8  Output: the integer count T in [0, n], not the fraction T/n.
 *
 * Input range: the coordinates of X - z must satisfy the bound checked by
 * coord_bound_ok(): every 2-D projected coordinate is below 2^61 in magnitude,
 * so that every cross product fits an __int128.  Larger inputs are rejected.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef __int128 i128;

#define OR_MAXD 6

enum { OR_OK = 0, OR_EINVAL = -1, OR_ERANGE = -2, OR_ENOMEM = -3 };

/* ------------------------------------------------------------------------- */
/* small exact helpers                                                       */
/* ------------------------------------------------------------------------- */

static i128 i128_abs(i128 v) { return v < 0 ? -v : v; }

static i128 i128_gcd(i128 a, i128 b)
{
    a = i128_abs(a);
    b = i128_abs(b);
    while (b != 0) {
        i128 t = a % b;
        a = b;
        b = t;
    }
    return a;
}

/* Determinant of a d x d matrix (row-major, entries m[r*d+c]) by fraction-free
 * Gaussian elimination (Bareiss).  Every intermediate is a minor of the input,
 * so it stays below the Hadamard bound of the input. */
static i128 det_bareiss(const i128 *in, int d)
{
    i128 m[OR_MAXD * OR_MAXD];
    memcpy(m, in, sizeof(i128) * (size_t)d * (size_t)d);
    i128 prev = 1;
    int sign = 1;
    for (int k = 0; k < d - 1; ++k) {
        if (m[k * d + k] == 0) {
            int sw = -1;
            for (int r = k + 1; r < d; ++r)
                if (m[r * d + k] != 0) { sw = r; break; }
            if (sw < 0) return 0;
            for (int c = 0; c < d; ++c) {
                i128 t = m[k * d + c];
                m[k * d + c] = m[sw * d + c];
                m[sw * d + c] = t;
            }
            sign = -sign;
        }
        for (int r = k + 1; r < d; ++r) {
            for (int c = k + 1; c < d; ++c)
                m[r * d + c] = (m[r * d + c] * m[k * d + k] - m[r * d + k] * m[k * d + c]) / prev;
            m[r * d + k] = 0;
        }
        prev = m[k * d + k];
    }
    return sign > 0 ? m[(d - 1) * d + (d - 1)] : -m[(d - 1) * d + (d - 1)];
}

/* det[ x_S | w1 | w2 ] for a k-subset S (k = d-2) of the points pts (rows of
 * length d), with the two last columns given explicitly. */
static i128 det_subset_two(const int64_t *pts, int d, const int *S,
                           const i128 *w1, const i128 *w2)
{
    i128 m[OR_MAXD * OR_MAXD];
    int k = d - 2;
    for (int r = 0; r < d; ++r) {
        for (int c = 0; c < k; ++c) m[r * d + c] = (i128)pts[(size_t)S[c] * d + r];
        m[r * d + k] = w1[r];
        m[r * d + k + 1] = w2[r];
    }
    return det_bareiss(m, d);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2 (Section 3): bivariate closed depth count of the origin        */
/* ------------------------------------------------------------------------- */

typedef struct {
    const i128 *num; /* slope numerators   (theta = num / den, den > 0) */
    const i128 *den;
} slope_ctx;

static int slope_cmp(const slope_ctx *c, int i, int j)
{
    i128 lhs = c->num[i] * c->den[j];
    i128 rhs = c->num[j] * c->den[i];
    return (lhs > rhs) - (lhs < rhs);
}

/* stable top-down merge sort of idx[0..len) by exact slope */
static void slope_sort(const slope_ctx *c, int *idx, int *tmp, int len)
{
    if (len < 2) return;
    int h = len / 2;
    slope_sort(c, idx, tmp, h);
    slope_sort(c, idx + h, tmp, len - h);
    int a = 0, b = h, o = 0;
    while (a < h && b < len) {
        if (slope_cmp(c, idx[b], idx[a]) < 0) tmp[o++] = idx[b++];
        else tmp[o++] = idx[a++];
    }
    while (a < h) tmp[o++] = idx[a++];
    while (b < len) tmp[o++] = idx[b++];
    memcpy(idx, tmp, sizeof(int) * (size_t)len);
}

/* Algorithm 2 on cnt points y (pairs y1,y2).  Returns the closed count
 * M_min + (cnt - m): the least number of points in a closed halfplane whose
 * boundary passes through the origin.  M_min, the minimum over generic
 * directions of the points strictly on one side, is written to *mmin.
 * Returns -1 on allocation failure. */
static int64_t alg2_closed(const i128 *y, int cnt, int64_t *mmin)
{
    /* step 1(a): the nonzero points */
    int m = 0;
    for (int i = 0; i < cnt; ++i)
        if (y[2 * i] != 0 || y[2 * i + 1] != 0) ++m;
    if (m == 0) {
        if (mmin) *mmin = 0;
        return cnt;
    }
    i128 *num = (i128 *)malloc(sizeof(i128) * (size_t)m);
    i128 *den = (i128 *)malloc(sizeof(i128) * (size_t)m);
    unsigned char *L = (unsigned char *)malloc((size_t)m);
    int *ev = (int *)malloc(sizeof(int) * (size_t)m);
    int *tmp = (int *)malloc(sizeof(int) * (size_t)m);
    if (!num || !den || !L || !ev || !tmp) {
        free(num); free(den); free(L); free(ev); free(tmp);
        return -1;
    }
    int j = 0, nev = 0;
    int64_t S1 = 0;
    for (int i = 0; i < cnt; ++i) {
        i128 y1 = y[2 * i], y2 = y[2 * i + 1];
        if (y1 == 0 && y2 == 0) continue;
        /* step 1(c), reading R4: side at u = (eps, -1), u'y = eps*y1 - y2 */
        L[j] = (unsigned char)((y2 < 0) || (y2 == 0 && y1 > 0));
        S1 += L[j];
        /* step 1(b), reading R3: theta = -y1 / y2 as an exact fraction */
        if (y2 != 0) {
            num[j] = y2 > 0 ? -y1 : y1;
            den[j] = y2 > 0 ? y2 : -y2;
            ev[nev++] = j;
        } else {
            num[j] = 0;
            den[j] = 1;
        }
        ++j;
    }
    int64_t M = S1 < m - S1 ? S1 : m - S1; /* step 1(d) */
    /* step 1(e): sort the finite slopes and flip, a whole tie group at a time (R5) */
    slope_ctx c = { num, den };
    slope_sort(&c, ev, tmp, nev);
    int g = 0;
    while (g < nev) {
        int h = g;
        while (h < nev && slope_cmp(&c, ev[g], ev[h]) == 0) {
            S1 += L[ev[h]] ? -1 : 1;
            ++h;
        }
        int64_t S0 = S1 < m - S1 ? S1 : m - S1;
        if (S0 < M) M = S0;
        g = h;
    }
    free(num); free(den); free(L); free(ev); free(tmp);
    if (mmin) *mmin = M;
    return M + (int64_t)(cnt - m); /* step 2 (as a count) */
}

/* ------------------------------------------------------------------------- */
/* rank and pivot coordinates (reading R7)                                   */
/* ------------------------------------------------------------------------- */

/* Rank of the rows of pts (cnt x d) and d-tuple of pivot columns piv[0..r) in
 * increasing order, such that the coordinate projection onto those columns is
 * injective on the row span. */
static int rank_pivots(const int64_t *pts, int cnt, int d, int *piv)
{
    i128 basis[OR_MAXD][OR_MAXD];
    int pc[OR_MAXD];
    int r = 0;
    for (int i = 0; i < cnt && r < d; ++i) {
        i128 v[OR_MAXD];
        for (int c = 0; c < d; ++c) v[c] = (i128)pts[(size_t)i * d + c];
        for (int b = 0; b < r; ++b) {
            i128 f = v[pc[b]];
            if (f == 0) continue;
            i128 e = basis[b][pc[b]];
            i128 g = 0;
            for (int c = 0; c < d; ++c) {
                v[c] = e * v[c] - f * basis[b][c];
                g = i128_gcd(g, v[c]);
            }
            if (g > 1)
                for (int c = 0; c < d; ++c) v[c] /= g;
        }
        int lead = -1;
        for (int c = 0; c < d; ++c)
            if (v[c] != 0) { lead = c; break; }
        if (lead < 0) continue;
        for (int c = 0; c < d; ++c) basis[r][c] = v[c];
        pc[r] = lead;
        ++r;
    }
    /* increasing order of the pivot columns */
    for (int a = 0; a < r; ++a)
        for (int b = a + 1; b < r; ++b)
            if (pc[b] < pc[a]) { int t = pc[a]; pc[a] = pc[b]; pc[b] = t; }
    for (int a = 0; a < r; ++a) piv[a] = pc[a];
    return r;
}

/* ------------------------------------------------------------------------- */
/* the depth count: Algorithm 1 with readings R1-R8                           */
/* ------------------------------------------------------------------------- */

/* first k-subset in lexicographic order / successor; returns 0 when done */
static void comb_first(int *S, int k) { for (int i = 0; i < k; ++i) S[i] = i; }

static int comb_next(int *S, int k, int n)
{
    int i = k - 1;
    while (i >= 0 && S[i] == n - k + i) --i;
    if (i < 0) return 0;
    ++S[i];
    for (int j = i + 1; j < k; ++j) S[j] = S[j - 1] + 1;
    return 1;
}

typedef struct {
    uint64_t subsets_visited;   /* top-level positions enumerated in range */
    uint64_t subsets_dependent; /* skipped by reading R2 */
    uint64_t tight_extra;       /* subsets whose span holds more than the subset */
} or_counters;

static int64_t depth_count(const int64_t *pts_in, int cnt, int d,
                           const int64_t *range, or_counters *ctr, int64_t *positions);

/* One subset S (k = d-2 indices into the cnt points pts, rows of length d) of
 * Algorithm 1: step 1(a) with reading R2, the projection of step 1(b), the
 * closed count of Algorithm 2 and reading R6.  On success (return 0) y holds
 * the projected points (pairs), *V = N - t + m_S = Z + G + m_S, and *G (if
 * not NULL) the minimum M of Algorithm 2 over generic directions.  Returns 1
 * if S is dependent (no row pair with kappa != 0), -1 on allocation failure.
 * tight is scratch of cnt * k entries. */
static int subset_value(const int64_t *pts, int cnt, int d, const int *S, i128 *y, int64_t *tight,
                        int64_t *V, int64_t *G, or_counters *ctr)
{
    const int k = d - 2;
    /* step 1(a) with reading R2: first row pair with kappa != 0 */
    int a = -1, b = -1;
    for (int ra = 0; ra < d && a < 0; ++ra)
        for (int rb = ra + 1; rb < d; ++rb) {
            i128 ea[OR_MAXD] = {0}, eb[OR_MAXD] = {0};
            ea[ra] = 1;
            eb[rb] = 1;
            if (det_subset_two(pts, d, S, ea, eb) != 0) { a = ra; b = rb; break; }
        }
    if (a < 0) return 1;
    /* f_a(x) = det[x_S | x | e_a] is linear in x: coefficients
     * ca[j] = det[x_S | e_j | e_a] (and likewise for b). */
    i128 ca[OR_MAXD], cb[OR_MAXD];
    for (int jc = 0; jc < d; ++jc) {
        i128 ej[OR_MAXD] = {0}, ea[OR_MAXD] = {0}, eb[OR_MAXD] = {0};
        ej[jc] = 1;
        ea[a] = 1;
        eb[b] = 1;
        ca[jc] = det_subset_two(pts, d, S, ej, ea);
        cb[jc] = det_subset_two(pts, d, S, ej, eb);
    }
    /* step 1(b): the projected points y_i = (f_a(x_i), f_b(x_i)) */
    int t = 0;
    for (int i = 0; i < cnt; ++i) {
        i128 s1 = 0, s2 = 0;
        int zero = 1;
        for (int jc = 0; jc < d; ++jc) {
            i128 xv = pts[(size_t)i * d + jc];
            if (xv != 0) zero = 0;
            s1 += ca[jc] * xv;
            s2 += cb[jc] * xv;
        }
        y[2 * i] = s1;
        y[2 * i + 1] = s2;
        if (!zero && s1 == 0 && s2 == 0) {
            /* tight point: nonzero x_i in span(x_S); keep its
             * coordinates on the rows other than a and b (R6) */
            int o = 0;
            for (int jc = 0; jc < d; ++jc)
                if (jc != a && jc != b) tight[(size_t)t * k + o++] = pts[(size_t)i * d + jc];
            ++t;
        }
    }
    int64_t M = 0;
    int64_t N = alg2_closed(y, cnt, &M);
    if (N < 0) return -1;
    int64_t mS = 0;
    if (t > k) {
        /* more tight points than the subset itself: open depth of the tight
         * set inside span(x_S), one level down (R6).  When t == k the tight
         * set is the independent subset, which lies in an open halfspace of
         * its span, so m_S = 0. */
        if (ctr) ctr->tight_extra++;
        mS = depth_count(tight, t, k, NULL, NULL, NULL);
        if (mS < 0) return -1;
    }
    *V = N - t + mS; /* reading R6 in place of step 2's "- (p-2)" */
    if (G) *G = M;
    return 0;
}

/* Closed depth count of the origin w.r.t. cnt points in Z^d (zero points
 * allowed).  If range != NULL, only the top-level subsets whose position in
 * lexicographic order lies in [range[0], range[1]) are visited, and the result
 * is Z + the minimum over those (a value >= the true count; the minimum over
 * a partition of the positions is the true count).  Positions refer to the
 * k-subsets of the list of points after rank reduction (R7), zero points
 * included.  When the top level has no subset loop (rank <= 2) the single
 * computation has position 0.  Returns -1 on allocation failure; INT64_MAX if
 * the range holds no independent subset. */
static int64_t depth_count(const int64_t *pts_in, int cnt, int d,
                           const int64_t *range, or_counters *ctr, int64_t *positions)
{
    int Z = 0;
    for (int i = 0; i < cnt; ++i) {
        int zero = 1;
        for (int c = 0; c < d; ++c)
            if (pts_in[(size_t)i * d + c] != 0) { zero = 0; break; }
        Z += zero;
    }
    if (Z == cnt) {
        if (positions) *positions = 1;
        if (range && !(range[0] <= 0 && 0 < range[1])) return INT64_MAX;
        return cnt;
    }

    /* R7: reduce to the dimension of the span of the points */
    int piv[OR_MAXD];
    int r = rank_pivots(pts_in, cnt, d, piv);
    int64_t *pts = (int64_t *)malloc(sizeof(int64_t) * (size_t)cnt * (size_t)(r > 0 ? r : 1));
    if (!pts) return -1;
    for (int i = 0; i < cnt; ++i)
        for (int c = 0; c < r; ++c) pts[(size_t)i * r + c] = pts_in[(size_t)i * d + piv[c]];
    d = r;

    if (d <= 2) {
        if (positions) *positions = 1;
        if (range && !(range[0] <= 0 && 0 < range[1])) { free(pts); return INT64_MAX; }
        int64_t res;
        if (d == 1) {
            /* the p = 1 case of Section 3: the smaller of the two side counts */
            int64_t pos = 0, neg = 0;
            for (int i = 0; i < cnt; ++i) {
                if (pts[i] > 0) ++pos;
                else if (pts[i] < 0) ++neg;
            }
            res = Z + (pos < neg ? pos : neg);
        } else {
            i128 *y = (i128 *)malloc(sizeof(i128) * 2 * (size_t)cnt);
            if (!y) { free(pts); return -1; }
            for (int i = 0; i < cnt; ++i) {
                y[2 * i] = pts[2 * i];
                y[2 * i + 1] = pts[2 * i + 1];
            }
            res = alg2_closed(y, cnt, NULL);
            free(y);
        }
        free(pts);
        return res;
    }

    const int k = d - 2;
    i128 *y = (i128 *)malloc(sizeof(i128) * 2 * (size_t)cnt);
    int64_t *tight = (int64_t *)malloc(sizeof(int64_t) * (size_t)cnt * (size_t)(k > 0 ? k : 1));
    if (!y || !tight) { free(y); free(tight); free(pts); return -1; }

    int S[OR_MAXD];
    comb_first(S, k);
    int64_t best = INT64_MAX;
    int64_t pos = 0;
    int more = cnt >= k;
    while (more) {
        int in_range = !range || (range[0] <= pos && pos < range[1]);
        if (range && pos >= range[1]) break;
        if (in_range) {
            if (ctr) ctr->subsets_visited++;
            int64_t V = 0;
            int rc = subset_value(pts, cnt, d, S, y, tight, &V, NULL, ctr);
            if (rc < 0) { best = -1; break; }
            if (rc > 0) {
                if (ctr) ctr->subsets_dependent++;
            } else if (V < best) {
                best = V;
            }
        }
        ++pos;
        more = comb_next(S, k, cnt);
    }
    if (positions) {
        /* total number of top-level positions: C(cnt, k) */
        int64_t c = 1;
        for (int i = 1; i <= k; ++i) c = c * (cnt - k + i) / i;
        *positions = c;
    }
    free(y);
    free(tight);
    free(pts);
    return best;
}

/* Every 2-D projected coordinate is a (d-1) x (d-1) minor of centred data,
 * bounded by Hadamard: (M sqrt(d-1))^(d-1).  Require it below 2^61. */
static int coord_bound_ok(const int64_t *x, int64_t n, int p)
{
    int64_t M = 0;
    for (int64_t i = 0; i < n * p; ++i) {
        int64_t a = x[i] < 0 ? -x[i] : x[i];
        if (a > M) M = a;
    }
    if (M == 0 || p <= 1) return 1;
    double e = p - 1 > 0 ? (double)(p - 1) : 1.0;
    double lb = e * (log2((double)M) + 0.5 * log2(e));
    return lb < 61.0;
}

static int64_t *centre(const int32_t *X, int64_t n, int p, const int32_t *z)
{
    int64_t *x = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1) * (size_t)p);
    if (!x) return NULL;
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < p; ++c) x[i * p + c] = (int64_t)X[i * p + c] - (int64_t)z[c];
    return x;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 3 (ADIA, Section 4)                                              */
/* ------------------------------------------------------------------------- */

/* Readings of Algorithm 3 taken here (the paper states it for data in general
 * position, p >= 3 and n > 2p, and fixes no order of its choices):
 *
 *  A1  Depths are counts: d_temp = V(S) of reading R6 (the paper's
 *      D_n(S) - (p-2)/n), so d0 and the node depths are integers.
 *  A2  Critical points (Step 2(c) and Step 4(a)(ii)).  The nonzero projected
 *      points y_i of S lie on lines through the origin; those lines cut the
 *      plane of directions into cells, and the count min(#left, #right) of a
 *      halfplane whose boundary lies in a cell is constant on it; G(S) is the
 *      least such count.  A point is critical for S when its line bounds a
 *      cell whose count is G(S).  In general position this is the paper's
 *      condition: the hyperplane through 0, x_S and x_h has a normal u0 with
 *      P_n(u0'X <= 0) - 1/n = D_n(S).
 *  A3  Order: the (p-2)-subsets of a node in lexicographic order of their
 *      sorted indices; the critical points of a subset in increasing index;
 *      N is a stack (last pushed, first popped); a node is identified by its
 *      sorted index set; "N not in Q" looks only at nodes not deleted.
 *  A4  Step 2 uses the centred points in the input coordinates: u_j = x_j for
 *      the nonzero x_j, the count of u is #{i : u'x_i <= 0}; the least count
 *      wins, ties to the smaller j and then to +x_j before -x_j.  The order of
 *      Step 2(b) is by u_min'x_i, ties by index, over the nonzero points.
 *  A5  Step 2(b) "k does not exist": when no nonzero point has u_min'x_i <= 0
 *      the closed halfspace of u_min holds only the zero points, so T = Z and
 *      the search is skipped.  Otherwise the start subset is taken greedily
 *      from the order of Step 2(b) starting after the k negative points (and
 *      wrapping round to the start), skipping a point that is dependent on
 *      those already taken; Step 2(c) takes the critical point of least index.
 *  A6  Step 5(a): u_F is the normal of the hyperplane through 0 and the p-1
 *      points of F, written det[x_F | x]; the closed side with fewer points is
 *      X_F; when both sides hold equally many, the side holding the point of
 *      least index off the hyperplane.  Step 5(b) runs over the (p-2)-subsets
 *      of the nonzero points of the union, in lexicographic order; dependent
 *      subsets are skipped as in R2.
 *  A7  When the nonzero points span fewer than 3 dimensions (after R7), or
 *      there are no more than 2d of them (the paper's n <= 2p), Algorithm 1
 *      is used directly, as the paper recommends.
 *
 * The result is d0 as a count, Z included.  Every value d0 takes is V(S) of
 * some subset, so the result is never below the exact count T; the paper
 * reports it equal to T in all its experiments, without proof.  It is not
 * equal on every input: on request 20 of the seeded request stream (p = 4,
 * n = 343), query 27 gives 33 where T = 32, with optimal subsets free of
 * ties.
 *
 * Pins: the critical points (A2) against a brute force and the paper's own
 * condition; the count against the exact count (never below it, equal in
 * general position).  The order of the traversal (A3-A6: exclusions, the
 * break, deletions, the side of Step 5(a), the start point) has no value
 * printed in the paper to pin it and leaves the count unchanged on every
 * input tried: parity unpinned for the traversal itself. */

/* Critical points (reading A2) of the projected points y (pairs, cnt of them,
 * zero pairs allowed).  crit[i] is set to 1 for the critical ones and 0
 * otherwise.  Each cell is evaluated directly: its count is taken at a
 * direction strictly inside it, the sum of the direction vectors of its two
 * bounding lines.  Returns 0, -1 on allocation failure, or -4 if the least
 * cell count differs from M (Algorithm 2's minimum), which would be a bug. */
static int critical_points(const i128 *y, int cnt, int64_t M, unsigned char *crit)
{
    memset(crit, 0, (size_t)cnt);
    int m = 0;
    for (int i = 0; i < cnt; ++i)
        if (y[2 * i] != 0 || y[2 * i + 1] != 0) ++m;
    if (m == 0) return M == 0 ? 0 : -4;
    int *ord = (int *)malloc(sizeof(int) * (size_t)m);
    int *grp = (int *)malloc(sizeof(int) * (size_t)m);   /* group of ord[j] */
    i128 *h = (i128 *)malloc(sizeof(i128) * 2 * (size_t)cnt);
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    if (!ord || !grp || !h || !cell) {
        free(ord); free(grp); free(h); free(cell);
        return -1;
    }
    /* line direction of each point: y turned into the upper half plane */
    int j = 0;
    for (int i = 0; i < cnt; ++i) {
        i128 a = y[2 * i], b = y[2 * i + 1];
        if (a == 0 && b == 0) continue;
        int up = b > 0 || (b == 0 && a > 0);
        h[2 * i] = up ? a : -a;
        h[2 * i + 1] = up ? b : -b;
        ord[j++] = i;
    }
    /* insertion sort by angle in [0, pi): a before b iff cross(h_a, h_b) > 0 */
    for (int u = 1; u < m; ++u) {
        int v = ord[u], w = u;
        while (w > 0) {
            int o = ord[w - 1];
            i128 cr = h[2 * o] * h[2 * v + 1] - h[2 * o + 1] * h[2 * v];
            if (cr > 0) break; /* o before v */
            if (cr == 0 && o < v) break;
            ord[w] = o;
            --w;
        }
        ord[w] = v;
    }
    /* groups of equal line direction */
    int L = 0;
    int first[2048 + 1];
    for (int u = 0; u < m; ++u) {
        if (u == 0) {
            first[L++] = 0;
        } else {
            int o = ord[u - 1], v = ord[u];
            i128 cr = h[2 * o] * h[2 * v + 1] - h[2 * o + 1] * h[2 * v];
            if (cr != 0) first[L++] = u;
        }
        grp[u] = L - 1;
    }
    first[L] = m;
    /* cell c lies between line c and line c+1 (the last one between line L-1
     * and line 0 turned by pi); count min(#left, #right) at a direction
     * strictly inside it */
    int64_t best = INT64_MAX;
    for (int c = 0; c < L; ++c) {
        int g0 = ord[first[c]];
        i128 v1, v2;
        if (L == 1) {
            v1 = -h[2 * g0 + 1];
            v2 = h[2 * g0];
        } else if (c + 1 < L) {
            int g1 = ord[first[c + 1]];
            v1 = h[2 * g0] + h[2 * g1];
            v2 = h[2 * g0 + 1] + h[2 * g1 + 1];
        } else {
            int g1 = ord[first[0]];
            v1 = h[2 * g0] - h[2 * g1];
            v2 = h[2 * g0 + 1] - h[2 * g1 + 1];
        }
        int64_t left = 0, right = 0;
        for (int i = 0; i < cnt; ++i) {
            i128 cr = v1 * y[2 * i + 1] - v2 * y[2 * i];
            left += cr > 0;
            right += cr < 0;
        }
        if (left + right != m) { best = -1; break; }
        cell[c] = left < right ? left : right;
        if (cell[c] < best) best = cell[c];
    }
    int rc = 0;
    if (best != M) {
        rc = -4;
    } else {
        for (int c = 0; c < L; ++c) {
            if (cell[c] != best) continue;
            int gs[2] = { c, (c + 1) % L };
            for (int e = 0; e < 2; ++e)
                for (int u = first[gs[e]]; u < first[gs[e] + 1]; ++u) crit[ord[u]] = 1;
        }
    }
    free(ord); free(grp); free(h); free(cell);
    return rc;
}

typedef struct {
    int idx[OR_MAXD]; /* sorted point indices, p-1 of them */
    int64_t depth;
    int alive;
} adia_node;

typedef struct {
    adia_node *q;
    int nq, capq;
    int *stack;
    int ns;
} adia_state;

static int adia_find(const adia_state *A, const int *idx, int k1)
{
    for (int i = 0; i < A->nq; ++i) {
        if (!A->q[i].alive) continue;
        if (memcmp(A->q[i].idx, idx, sizeof(int) * (size_t)k1) == 0) return i;
    }
    return -1;
}

/* Push a node into Q and N unless Q already holds it (Step 3(a), Step 4(a)(iii)(B)). */
static int adia_push(adia_state *A, const int *idx, int k1, int64_t depth)
{
    if (adia_find(A, idx, k1) >= 0) return 0;
    if (A->nq == A->capq) {
        int cap = A->capq ? 2 * A->capq : 256;
        adia_node *q = (adia_node *)realloc(A->q, sizeof(adia_node) * (size_t)cap);
        int *st = (int *)realloc(A->stack, sizeof(int) * (size_t)cap);
        if (!q || !st) {
            if (q) A->q = q;
            if (st) A->stack = st;
            return -1;
        }
        A->q = q;
        A->stack = st;
        A->capq = cap;
    }
    adia_node *nd = &A->q[A->nq];
    memset(nd, 0, sizeof(*nd));
    memcpy(nd->idx, idx, sizeof(int) * (size_t)k1);
    nd->depth = depth;
    nd->alive = 1;
    A->stack[A->ns++] = A->nq;
    A->nq++;
    return 0;
}

static void sort_ints(int *a, int len)
{
    for (int i = 1; i < len; ++i) {
        int v = a[i], j = i;
        while (j > 0 && a[j - 1] > v) { a[j] = a[j - 1]; --j; }
        a[j] = v;
    }
}

/* Algorithm 3 on cnt points (rows of pts, length d, already reduced by R7 so
 * that they span R^d) with the centred input coordinates orig (rows of length
 * p) for Step 2.  Returns the count (Z included), -1 on allocation failure, or
 * -4 on an internal inconsistency.  st[0..9): pops, subsets evaluated in
 * Step 4, nodes pushed, largest stack, points in the union of Step 5(a),
 * subsets of Step 5(b), d0 after Step 4, 1 if Algorithm 1 was used (A5/A7),
 * and the sum of (i + 1)^3 over the union's nonzero points i (data order),
 * which makes the union itself observable (st must hold 9 zeros). */
static int64_t adia_count(const int64_t *pts, int cnt, int d, const int64_t *orig, int p, int64_t *st)
{
    const int k = d - 2, k1 = d - 1;
    int Z = 0, nnz = 0;
    int *nz = (int *)malloc(sizeof(int) * (size_t)cnt);
    if (!nz) return -1;
    for (int i = 0; i < cnt; ++i) {
        int zero = 1;
        for (int c = 0; c < d; ++c)
            if (pts[(size_t)i * d + c] != 0) { zero = 0; break; }
        if (zero) ++Z;
        else nz[nnz++] = i;
    }
    if (d < 3 || nnz <= 2 * d) {
        free(nz);
        st[7] = 1;
        return depth_count(pts, cnt, d, NULL, NULL, NULL);
    }
    i128 *y = (i128 *)malloc(sizeof(i128) * 2 * (size_t)cnt);
    int64_t *tight = (int64_t *)malloc(sizeof(int64_t) * (size_t)cnt * (size_t)k);
    unsigned char *crit = (unsigned char *)malloc((size_t)cnt);
    unsigned char *inK = (unsigned char *)calloc((size_t)cnt, 1);
    int64_t *proj = (int64_t *)malloc(sizeof(int64_t) * (size_t)cnt);
    int *order = (int *)malloc(sizeof(int) * (size_t)nnz);
    adia_state A = { NULL, 0, 0, NULL, 0 };
    int64_t result = -1;
    if (!y || !tight || !crit || !inK || !proj || !order) goto done;

    /* Step 2(a), reading A4: the data direction with the least closed count */
    int64_t U = INT64_MAX;
    int jbest = -1, sbest = 1;
    for (int a = 0; a < nnz; ++a) {
        const int64_t *u = orig + (size_t)nz[a] * p;
        for (int sg = 1; sg >= -1; sg -= 2) {
            int64_t c = 0;
            for (int i = 0; i < cnt; ++i) {
                int64_t dot = 0;
                for (int t = 0; t < p; ++t) dot += u[t] * orig[(size_t)i * p + t];
                if (sg * dot <= 0) ++c;
            }
            if (c < U) { U = c; jbest = nz[a]; sbest = sg; }
        }
    }
    /* Step 2(b): order the nonzero points by u_min'x */
    for (int i = 0; i < cnt; ++i) {
        int64_t dot = 0;
        for (int t = 0; t < p; ++t) dot += orig[(size_t)jbest * p + t] * orig[(size_t)i * p + t];
        proj[i] = sbest * dot;
    }
    for (int a = 0; a < nnz; ++a) order[a] = nz[a];
    for (int a = 1; a < nnz; ++a) {
        int v = order[a], b = a;
        while (b > 0 && proj[order[b - 1]] > proj[v]) { order[b] = order[b - 1]; --b; }
        order[b] = v;
    }
    int kneg = 0, nonpos = 0;
    for (int a = 0; a < nnz; ++a) {
        kneg += proj[order[a]] < 0;
        nonpos += proj[order[a]] <= 0;
    }
    if (nonpos == 0) { /* reading A5: the closed halfspace holds only the zero points */
        st[7] = 1;
        result = Z;
        goto done;
    }
    /* start subset: greedy independent points after the k negative ones */
    int S[OR_MAXD];
    int ns = 0;
    for (int a = 0; a < nnz && ns < k; ++a) {
        int cand = order[(kneg + a) % nnz];
        int64_t rows[OR_MAXD * OR_MAXD];
        for (int b = 0; b < ns; ++b)
            for (int c = 0; c < d; ++c) rows[b * d + c] = pts[(size_t)S[b] * d + c];
        for (int c = 0; c < d; ++c) rows[ns * d + c] = pts[(size_t)cand * d + c];
        int piv[OR_MAXD];
        if (rank_pivots(rows, ns + 1, d, piv) == ns + 1) S[ns++] = cand;
    }
    if (ns < k) { result = -4; goto done; }
    sort_ints(S, k);
    /* Step 2(c) */
    int64_t V0 = 0, G0 = 0;
    int rc = subset_value(pts, cnt, d, S, y, tight, &V0, &G0, NULL);
    if (rc != 0) { result = rc < 0 ? -1 : -4; goto done; }
    rc = critical_points(y, cnt, G0, crit);
    if (rc != 0) { result = rc; goto done; }
    int h0 = -1;
    for (int i = 0; i < cnt && h0 < 0; ++i)
        if (crit[i]) h0 = i;
    if (h0 < 0) { result = -4; goto done; }
    int C[OR_MAXD];
    for (int b = 0; b < k; ++b) C[b] = S[b];
    C[k] = h0;
    sort_ints(C, k1);
    /* Step 3 */
    if (adia_push(&A, C, k1, V0) < 0) goto done;
    int64_t d0 = V0;
    st[2] = 1;
    st[3] = 1;
    /* Step 4 */
    while (A.ns > 0) {
        int qi = A.stack[--A.ns];
        int Qidx[OR_MAXD];
        memcpy(Qidx, A.q[qi].idx, sizeof(int) * (size_t)k1);
        st[0]++;
        /* (a): the k-subsets of the node, in lexicographic order (omit the
         * last member first) */
        int improved = 0;
        for (int omit = k1 - 1; omit >= 0 && !improved; --omit) {
            int Ss[OR_MAXD];
            int o = 0;
            for (int b = 0; b < k1; ++b)
                if (b != omit) Ss[o++] = Qidx[b];
            int64_t V = 0, G = 0;
            rc = subset_value(pts, cnt, d, Ss, y, tight, &V, &G, NULL);
            if (rc != 0) { result = rc < 0 ? -1 : -4; goto done; }
            st[1]++;
            /* (ii) */
            rc = critical_points(y, cnt, G, crit);
            if (rc != 0) { result = rc; goto done; }
            for (int b = 0; b < k1; ++b) crit[Qidx[b]] = 0;
            /* (iii) */
            for (int t = 0; t < cnt; ++t) {
                if (!crit[t]) continue;
                int Nn[OR_MAXD];
                for (int b = 0; b < k; ++b) Nn[b] = Ss[b];
                Nn[k] = t;
                sort_ints(Nn, k1);
                int before = A.nq;
                if (adia_push(&A, Nn, k1, V) < 0) goto done;
                if (A.nq > before) st[2]++;
                if (A.ns > st[3]) st[3] = A.ns;
            }
            /* (iv) */
            if (d0 > V) {
                d0 = V;
                improved = 1;
            }
        }
        /* (b): delete the nodes deeper than d0 from Q and N */
        for (int i = 0; i < A.nq; ++i)
            if (A.q[i].alive && A.q[i].depth > d0) A.q[i].alive = 0;
        int w = 0;
        for (int i = 0; i < A.ns; ++i)
            if (A.q[A.stack[i]].alive) A.stack[w++] = A.stack[i];
        A.ns = w;
    }
    st[6] = d0;
    /* Step 5(a), reading A6 */
    for (int f = 0; f < A.nq; ++f) {
        if (!A.q[f].alive) continue;
        int64_t cle = 0, cge = 0;
        int lowest = -1;
        signed char *sg = (signed char *)crit; /* reuse as sign scratch */
        for (int i = 0; i < cnt; ++i) {
            i128 m[OR_MAXD * OR_MAXD];
            for (int r = 0; r < d; ++r) {
                for (int c = 0; c < k1; ++c) m[r * d + c] = (i128)pts[(size_t)A.q[f].idx[c] * d + r];
                m[r * d + k1] = (i128)pts[(size_t)i * d + r];
            }
            i128 det = det_bareiss(m, d);
            sg[i] = (signed char)((det > 0) - (det < 0));
            cle += sg[i] <= 0;
            cge += sg[i] >= 0;
            if (lowest < 0 && sg[i] != 0) lowest = i;
        }
        int side; /* -1: det <= 0, +1: det >= 0 */
        if (cle < cge) side = -1;
        else if (cge < cle) side = 1;
        else side = lowest < 0 ? 0 : sg[lowest];
        for (int i = 0; i < cnt; ++i)
            if (side == 0 || sg[i] == 0 || sg[i] == side) inK[i] = 1;
    }
    /* Step 5(b) */
    int nk = 0;
    int *Kl = order; /* reuse: nonzero members of the union, increasing */
    for (int a = 0; a < nnz; ++a)
        if (inK[nz[a]]) Kl[nk++] = nz[a];
    st[4] = nk;
    for (int a = 0; a < nk; ++a) st[8] += (int64_t)(Kl[a] + 1) * (Kl[a] + 1) * (Kl[a] + 1);
    if (nk >= k) {
        int c5[OR_MAXD], Ss[OR_MAXD];
        comb_first(c5, k);
        do {
            for (int b = 0; b < k; ++b) Ss[b] = Kl[c5[b]];
            int64_t V = 0;
            rc = subset_value(pts, cnt, d, Ss, y, tight, &V, NULL, NULL);
            if (rc < 0) goto done;
            st[5]++;
            if (rc == 0 && V < d0) d0 = V;
        } while (comb_next(c5, k, nk));
    }
    result = d0;
done:
    free(nz); free(y); free(tight); free(crit); free(inK); free(proj); free(order);
    free(A.q); free(A.stack);
    return result;
}

/* ------------------------------------------------------------------------- */
/* exported entry points                                                     */
/* ------------------------------------------------------------------------- */

/* T = n * D_n(z) for X (n x p, row-major int32) and z (p int32).  Returns 0 on
 * success, OR_EINVAL for bad arguments, OR_ERANGE when the coordinates exceed
 * the exact-arithmetic bound, OR_ENOMEM on allocation failure. */
int oracle_depth(const int32_t *X, int64_t n, int p, const int32_t *z, int64_t *T)
{
    if (!X || !z || !T || n < 1 || p < 1 || p > OR_MAXD || n > (int64_t)1 << 30) return OR_EINVAL;
    int64_t *x = centre(X, n, p, z);
    if (!x) return OR_ENOMEM;
    if (!coord_bound_ok(x, n, p)) { free(x); return OR_ERANGE; }
    int64_t r = depth_count(x, (int)n, p, NULL, NULL, NULL);
    free(x);
    if (r < 0) return OR_ENOMEM;
    *T = r;
    return OR_OK;
}

/* The same count restricted to the top-level subsets with lexicographic
 * position in [lo, hi).  *partial = Z + min over that range of V(S), or
 * INT64_MAX when the range holds no independent subset; the minimum of
 * *partial over a partition of [0, *positions) equals oracle_depth's result.
 * counters (may be NULL) receives {visited, dependent, tight_extra}. */
int oracle_depth_range(const int32_t *X, int64_t n, int p, const int32_t *z,
                       int64_t lo, int64_t hi, int64_t *partial, int64_t *positions,
                       uint64_t *counters)
{
    if (!X || !z || !partial || n < 1 || p < 1 || p > OR_MAXD || lo < 0 || hi < lo) return OR_EINVAL;
    int64_t *x = centre(X, n, p, z);
    if (!x) return OR_ENOMEM;
    if (!coord_bound_ok(x, n, p)) { free(x); return OR_ERANGE; }
    int64_t range[2] = { lo, hi };
    or_counters ctr = { 0, 0, 0 };
    int64_t npos = 0;
    int64_t r = depth_count(x, (int)n, p, range, &ctr, &npos);
    free(x);
    if (r < 0) return OR_ENOMEM;
    *partial = r;
    if (positions) *positions = npos;
    if (counters) {
        counters[0] = ctr.subsets_visited;
        counters[1] = ctr.subsets_dependent;
        counters[2] = ctr.tight_extra;
    }
    return OR_OK;
}

/* Z + the minimum of V(S) (Algorithm 1, step 1, with reading R6) over an
 * explicit list of subsets S instead of all of them: for checking a part of
 * the subset loop of another implementation whose enumeration order differs
 * from the one above.  The subsets are `count` rows of p-2 indices into the
 * nonzero centred points x_i = X_i - z taken in data order; the nonzero
 * points must span R^p (rank p, p >= 3; otherwise OR_EINVAL, since R7 would
 * change the subset size).  *out receives Z + min V(S) over the independent
 * listed subsets, INT64_MAX if there is none; *dependent (may be NULL) the
 * number of listed subsets of rank < p-2 (skipped, reading R2). */
int oracle_subset_min(const int32_t *X, int64_t n, int p, const int32_t *z, const int32_t *subsets,
                      int64_t count, int64_t *out, int64_t *dependent)
{
    if (!X || !z || !out || n < 1 || p < 3 || p > OR_MAXD || count < 0 || (count > 0 && !subsets))
        return OR_EINVAL;
    int64_t *x = centre(X, n, p, z);
    if (!x) return OR_ENOMEM;
    if (!coord_bound_ok(x, n, p)) { free(x); return OR_ERANGE; }
    int piv[OR_MAXD];
    if (rank_pivots(x, (int)n, p, piv) != p) { free(x); return OR_EINVAL; }
    /* data index of every nonzero point, in data order */
    int *nzi = (int *)malloc(sizeof(int) * (size_t)n);
    i128 *y = (i128 *)malloc(sizeof(i128) * 2 * (size_t)n);
    int64_t *tight = (int64_t *)malloc(sizeof(int64_t) * (size_t)n * (size_t)(p - 2));
    if (!nzi || !y || !tight) { free(nzi); free(y); free(tight); free(x); return OR_ENOMEM; }
    int nnz = 0;
    for (int64_t i = 0; i < n; ++i) {
        int zero = 1;
        for (int c = 0; c < p; ++c)
            if (x[i * p + c] != 0) zero = 0;
        if (!zero) nzi[nnz++] = (int)i;
    }
    const int k = p - 2;
    int64_t best = INT64_MAX, dep = 0;
    int rc = OR_OK;
    for (int64_t j = 0; j < count && rc == OR_OK; ++j) {
        int S[OR_MAXD];
        for (int t = 0; t < k; ++t) {
            const int32_t v = subsets[j * k + t];
            if (v < 0 || v >= nnz || (t > 0 && v <= subsets[j * k + t - 1])) { rc = OR_EINVAL; break; }
            S[t] = nzi[v];
        }
        if (rc != OR_OK) break;
        /* V(S) over all n points: the zero points are counted by N(S) */
        int64_t V = 0;
        const int r = subset_value(x, (int)n, p, S, y, tight, &V, NULL, NULL);
        if (r < 0) rc = OR_ENOMEM;
        else if (r > 0) ++dep;
        else if (V < best) best = V;
    }
    free(nzi);
    free(y);
    free(tight);
    free(x);
    if (rc != OR_OK) return rc;
    *out = best;
    if (dependent) *dependent = dep;
    return OR_OK;
}

/* Algorithm 2 alone on cnt points (pairs, int64): the closed bivariate count. */
int oracle_bivariate_closed(const int64_t *Y, int64_t cnt, int64_t *count)
{
    if (!Y || !count || cnt < 0) return OR_EINVAL;
    i128 *y = (i128 *)malloc(sizeof(i128) * 2 * (size_t)(cnt > 0 ? cnt : 1));
    if (!y) return OR_ENOMEM;
    for (int64_t i = 0; i < 2 * cnt; ++i) y[i] = Y[i];
    int64_t r = alg2_closed(y, (int)cnt, NULL);
    free(y);
    if (r < 0) return OR_ENOMEM;
    *count = r;
    return OR_OK;
}

/* Rank of the nonzero centred points X - z and their pivot coordinates. */
int oracle_rank(const int32_t *X, int64_t n, int p, const int32_t *z, int32_t *piv_out)
{
    if (!X || !z || n < 1 || p < 1 || p > OR_MAXD) return OR_EINVAL;
    int64_t *x = centre(X, n, p, z);
    if (!x) return OR_ENOMEM;
    int piv[OR_MAXD];
    int r = rank_pivots(x, (int)n, p, piv);
    free(x);
    if (piv_out)
        for (int i = 0; i < r; ++i) piv_out[i] = piv[i];
    return r;
}

/* Algorithm 3 (ADIA) for X (n x p) and z: *T receives its count (never below
 * oracle_depth's; readings A1-A7).  stats (may be NULL) receives 9 counters,
 * see adia_count.  Returns 0, OR_EINVAL, OR_ERANGE, OR_ENOMEM, or -4 on an
 * internal inconsistency. */
int oracle_adia(const int32_t *X, int64_t n, int p, const int32_t *z, int64_t *T, int64_t *stats)
{
    if (!X || !z || !T || n < 1 || p < 1 || p > OR_MAXD || n > 2048) return OR_EINVAL;
    int64_t *x = centre(X, n, p, z);
    if (!x) return OR_ENOMEM;
    if (!coord_bound_ok(x, n, p)) { free(x); return OR_ERANGE; }
    int64_t st[9] = { 0 };
    int allzero = 1;
    for (int64_t i = 0; i < n * p; ++i)
        if (x[i] != 0) { allzero = 0; break; }
    int64_t r;
    if (allzero) {
        r = n;
        st[7] = 1;
    } else {
        int piv[OR_MAXD];
        int d = rank_pivots(x, (int)n, p, piv);
        int64_t *pts = (int64_t *)malloc(sizeof(int64_t) * (size_t)n * (size_t)d);
        if (!pts) { free(x); return OR_ENOMEM; }
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < d; ++c) pts[i * d + c] = x[i * p + piv[c]];
        r = adia_count(pts, (int)n, d, x, p, st);
        free(pts);
    }
    free(x);
    if (r == -1) return OR_ENOMEM;
    if (r < 0) return (int)r;
    *T = r;
    if (stats)
        for (int i = 0; i < 9; ++i) stats[i] = st[i];
    return OR_OK;
}

/* Critical points (reading A2) of cnt 2-D points Y (pairs, int64): *G receives
 * Algorithm 2's minimum over generic directions, crit[i] 1 for a critical
 * point.  Returns 0, OR_EINVAL, OR_ENOMEM or -4. */
int oracle_critical(const int64_t *Y, int64_t cnt, int64_t *G, uint8_t *crit)
{
    if (!Y || !G || !crit || cnt < 0 || cnt > 2048) return OR_EINVAL;
    i128 *y = (i128 *)malloc(sizeof(i128) * 2 * (size_t)(cnt > 0 ? cnt : 1));
    if (!y) return OR_ENOMEM;
    for (int64_t i = 0; i < 2 * cnt; ++i) y[i] = Y[i];
    int64_t M = 0;
    if (alg2_closed(y, (int)cnt, &M) < 0) { free(y); return OR_ENOMEM; }
    int rc = critical_points(y, (int)cnt, M, crit);
    free(y);
    if (rc == -1) return OR_ENOMEM;
    if (rc < 0) return rc;
    *G = M;
    return OR_OK;
}
