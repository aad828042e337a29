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
            /* step 1(a) with reading R2: first row pair with kappa != 0 */
            int a = -1, b = -1;
            for (int ra = 0; ra < d && a < 0; ++ra)
                for (int rb = ra + 1; rb < d; ++rb) {
                    i128 ea[OR_MAXD] = {0}, eb[OR_MAXD] = {0};
                    ea[ra] = 1;
                    eb[rb] = 1;
                    if (det_subset_two(pts, d, S, ea, eb) != 0) { a = ra; b = rb; break; }
                }
            if (a < 0) {
                if (ctr) ctr->subsets_dependent++;
            } else {
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
                int64_t N = alg2_closed(y, cnt, NULL);
                if (N < 0) { best = -1; break; }
                int64_t mS = 0;
                if (t > k) {
                    /* more tight points than the subset itself: open depth of
                     * the tight set inside span(x_S), one level down (R6).  When
                     * t == k the tight set is the independent subset, which lies
                     * in an open halfspace of its span, so m_S = 0. */
                    if (ctr) ctr->tight_extra++;
                    mS = depth_count(tight, t, k, NULL, NULL, NULL);
                    if (mS < 0) { best = -1; break; }
                }
                int64_t V = N - t + mS; /* reading R6 in place of step 2's "- (p-2)" */
                if (V < best) best = V;
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
