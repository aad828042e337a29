/*
 * td_exact.cuh -- exact integer building blocks of the sweep kernels.
 *
 * For a subset S of K = D-2 centred points of Z^D, Algorithm 1 step 1(a)
 * (Section 3) needs two linear functionals that vanish on span(S).  We use
 * f_a(x) = det[x_S | x | e_a] and f_b(x) = det[x_S | x | e_b]: expanding the
 * determinant along its last two columns gives
 *
 *     det[x_S | x | w] = sum_{i<j} P_ij (x_i w_j - x_j w_i),
 *     P_ij = -(-1)^(i+j) M_ij   (0-based rows),
 *
 * where M_ij is the K x K minor of x_S with rows i and j deleted (the Plucker
 * coordinates of span(S)).  With Q the antisymmetric matrix Q_ij = P_ij (i<j),
 * f_a(x) = sum_i Q_ia x_i, and Q_ab = det[x_S | e_a | e_b] = kappa.  For a row
 * pair with kappa != 0 the two functionals are independent (their matrix on
 * e_a, e_b is [[0,-kappa],[kappa,0]]), so y(x) = (f_a(x), f_b(x)) is a linear
 * isomorphism of the quotient R^D / span(S) onto R^2; the bivariate depth of
 * the origin does not depend on which isomorphism is used.  If every minor
 * vanishes, S has rank < K and is skipped.
 *
 * All quantities are exact int64 under the coordinate limits of
 * td_coord_limit(); products of two projected coordinates use __int128.
 */
#pragma once
#include <stdint.h>

typedef __int128 td_i128;

#define TD_FULL 0xffffffffu

/* ---------------------------------------------------------------- warp ops */

__device__ __forceinline__ int td_wsum(int v) { return __reduce_add_sync(TD_FULL, v); }
__device__ __forceinline__ int td_wmin(int v) { return __reduce_min_sync(TD_FULL, v); }
__device__ __forceinline__ int td_wmax(int v) { return __reduce_max_sync(TD_FULL, v); }

__device__ __forceinline__ int td_wscan_incl(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(TD_FULL, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ int td_wscan_max_incl(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(TD_FULL, v, o);
        if (lane >= o) v = max(v, u);
    }
    return v;
}

__device__ __forceinline__ int64_t td_shfl64(int64_t v, int src)
{
    return __shfl_sync(TD_FULL, v, src);
}

/* ------------------------------------------------------- binomials, colex */

__host__ __device__ __forceinline__ uint64_t td_binom(int64_t n, int k)
{
    if (n < k || n < 0) return 0;
    uint64_t u = (uint64_t)n;
    switch (k) {
    case 0: return 1;
    case 1: return u;
    case 2: return u * (u - 1) / 2;
    case 3: return u * (u - 1) / 2 * (u - 2) / 3;
    case 4: return u * (u - 1) / 2 * (u - 2) / 3 * (u - 3) / 4;
    case 5: return u * (u - 1) / 2 * (u - 2) / 3 * (u - 3) / 4 * (u - 4) / 5;
    default: return 0;
    }
}

/* Combination with colex rank r: c[0] < ... < c[K-1], r = sum C(c[i], i+1).
 * (K is a compile-time constant so that c stays in registers.) */
template <int K>
__device__ __forceinline__ void td_unrank_colex(uint64_t r, int n, int (&c)[K > 0 ? K : 1])
{
#pragma unroll
    for (int i = K; i >= 1; --i) {
        int lo = i - 1, hi = n - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (td_binom(mid, i) <= r) lo = mid;
            else hi = mid - 1;
        }
        c[i - 1] = lo;
        r -= td_binom(lo, i);
    }
}

/* Colex successor (the caller guarantees one exists): the first c[i] that can
 * grow grows by one and every c[j], j < i, restarts at j. */
template <int K>
__device__ __forceinline__ void td_next_colex(int (&c)[K > 0 ? K : 1])
{
    bool done = false;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        if (!done) {
            bool can = (i == K - 1) ? true : (c[i] + 1 < c[(i + 1 < K) ? i + 1 : i]);
            if (can) {
                c[i] += 1;
                done = true;
            } else {
                c[i] = i;
            }
        }
    }
}

/* ------------------------------------------------ small exact determinants */

__device__ __forceinline__ int64_t td_det2(int64_t a, int64_t b, int64_t c, int64_t d)
{
    return a * d - b * c;
}

/* K x K determinant of columns s[0..K) restricted to rows r[0..K). */
template <int K, int D>
__device__ __forceinline__ int64_t td_minor(const int64_t (&s)[K > 0 ? K : 1][D], const int *r)
{
    if constexpr (K == 0) {
        return 1;
    } else if constexpr (K == 1) {
        return s[0][r[0]];
    } else if constexpr (K == 2) {
        return td_det2(s[0][r[0]], s[1][r[0]], s[0][r[1]], s[1][r[1]]);
    } else if constexpr (K == 3) {
        /* expansion along column 2 with the 2x2 minors of columns 0,1 */
        int64_t m01 = td_det2(s[0][r[0]], s[1][r[0]], s[0][r[1]], s[1][r[1]]);
        int64_t m02 = td_det2(s[0][r[0]], s[1][r[0]], s[0][r[2]], s[1][r[2]]);
        int64_t m12 = td_det2(s[0][r[1]], s[1][r[1]], s[0][r[2]], s[1][r[2]]);
        return s[2][r[0]] * m12 - s[2][r[1]] * m02 + s[2][r[2]] * m01;
    } else {
        /* Laplace expansion along columns (0,1) versus (2,3) */
        int64_t a[4][4], b[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = i + 1; j < 4; ++j) {
                a[i][j] = td_det2(s[0][r[i]], s[1][r[i]], s[0][r[j]], s[1][r[j]]);
                b[i][j] = td_det2(s[2][r[i]], s[3][r[i]], s[2][r[j]], s[3][r[j]]);
            }
        return a[0][1] * b[2][3] - a[0][2] * b[1][3] + a[0][3] * b[1][2]
             + a[1][2] * b[0][3] - a[1][3] * b[0][2] + a[2][3] * b[0][1];
    }
}

/* Exact subset basis: coefficient columns a and b of Q, kappa = Q_ab. */
template <int D>
struct TdBasis {
    int64_t qa[D], qb[D];
    int a, b;
    int rows[D > 2 ? D - 2 : 1]; /* the K rows other than a and b (intrinsic coordinates) */
};

/* Returns false when every K x K minor of the subset vanishes (rank < K).
 * The row pair (a, b) is the first one, in lexicographic order, of largest
 * |kappa|.  Every array index below is a compile-time constant (selection by
 * predication), so that the whole basis stays in registers. */
template <int D>
__device__ __forceinline__ bool td_make_basis(const int64_t (&s)[D > 2 ? D - 2 : 1][D], TdBasis<D> &B)
{
    constexpr int K = D - 2;
    int64_t Q[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) Q[i][j] = 0;
    int64_t best = 0;
    int ba = -1, bb = -1;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a + 1; b < D; ++b) {
            int r[K > 0 ? K : 1];
            {
                int o = 0;
#pragma unroll
                for (int t = 0; t < D; ++t)
                    if (t != a && t != b) r[o++] = t;
            }
            int64_t M = td_minor<K, D>(s, r);
            int64_t P = ((a + b) & 1) ? M : -M; /* -(-1)^(a+b) M */
            Q[a][b] = P;
            Q[b][a] = -P;
            int64_t ab = P < 0 ? -P : P;
            if (ab > best) {
                best = ab;
                ba = a;
                bb = b;
            }
        }
    if (ba < 0) return false;
    B.a = ba;
    B.b = bb;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = a + 1; b < D; ++b) {
            if (a == ba && b == bb) {
#pragma unroll
                for (int t = 0; t < D; ++t) {
                    B.qa[t] = Q[t][a];
                    B.qb[t] = Q[t][b];
                }
                int o = 0;
#pragma unroll
                for (int t = 0; t < D; ++t)
                    if (t != a && t != b) B.rows[o++] = t;
            }
        }
    return true;
}

/* K x K determinant of m[row][col] (K <= 4; same formulas as td_minor). */
template <int K>
__device__ __forceinline__ int64_t td_detk(const int64_t (&m)[K > 0 ? K : 1][K > 0 ? K : 1])
{
    if constexpr (K == 0) {
        return 1;
    } else if constexpr (K == 1) {
        return m[0][0];
    } else if constexpr (K == 2) {
        return td_det2(m[0][0], m[0][1], m[1][0], m[1][1]);
    } else if constexpr (K == 3) {
        int64_t m01 = td_det2(m[0][0], m[0][1], m[1][0], m[1][1]);
        int64_t m02 = td_det2(m[0][0], m[0][1], m[2][0], m[2][1]);
        int64_t m12 = td_det2(m[1][0], m[1][1], m[2][0], m[2][1]);
        return m[0][2] * m12 - m[1][2] * m02 + m[2][2] * m01;
    } else {
        int64_t a[4][4], b[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = i + 1; j < 4; ++j) {
                a[i][j] = td_det2(m[i][0], m[i][1], m[j][0], m[j][1]);
                b[i][j] = td_det2(m[i][2], m[i][3], m[j][2], m[j][3]);
            }
        return a[0][1] * b[2][3] - a[0][2] * b[1][3] + a[0][3] * b[1][2]
             + a[1][2] * b[0][3] - a[1][3] * b[0][2] + a[2][3] * b[0][1];
    }
}

/* The same determinant in int32, exact when K! max|m|^K < 2^31 (every
 * intermediate, the 2 x 2 minors and the products of the expansion, is
 * bounded by that). */
template <int K>
__device__ __forceinline__ int32_t td_detk32(const int32_t (&m)[K > 0 ? K : 1][K > 0 ? K : 1])
{
    if constexpr (K == 0) {
        return 1;
    } else if constexpr (K == 1) {
        return m[0][0];
    } else if constexpr (K == 2) {
        return m[0][0] * m[1][1] - m[0][1] * m[1][0];
    } else if constexpr (K == 3) {
        const int32_t m01 = m[0][0] * m[1][1] - m[0][1] * m[1][0];
        const int32_t m02 = m[0][0] * m[2][1] - m[0][1] * m[2][0];
        const int32_t m12 = m[1][0] * m[2][1] - m[1][1] * m[2][0];
        return m[0][2] * m12 - m[1][2] * m02 + m[2][2] * m01;
    } else {
        int32_t a[4][4], b[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = i + 1; j < 4; ++j) {
                a[i][j] = m[i][0] * m[j][1] - m[i][1] * m[j][0];
                b[i][j] = m[i][2] * m[j][3] - m[i][3] * m[j][2];
            }
        return a[0][1] * b[2][3] - a[0][2] * b[1][3] + a[0][3] * b[1][2]
             + a[1][2] * b[0][3] - a[1][3] * b[0][2] + a[2][3] * b[0][1];
    }
}

/* Exact integer value of an integer-valued binary32 x with |x| <= 2^22:
 * x + 1.5*2^23 lies in [2^23, 2^24), where binary32 spacing is 1, so the sum
 * is exact and its bit pattern is 0x4B400000 + x. */
__device__ __forceinline__ int32_t td_f2i(float x)
{
    return __float_as_int(x + 12582912.0f) - 0x4B400000;
}

/* Half-plane normalisation of a nonzero projected point: h = y or -y with
 * h2 > 0, or h2 == 0 and h1 > 0.  Returns true when h == y ("orientation +":
 * the point is on the counted side just before its line is crossed). */
__device__ __forceinline__ bool td_normalise(int64_t y1, int64_t y2, int64_t &h1, int64_t &h2)
{
    bool plus = (y2 > 0) || (y2 == 0 && y1 > 0);
    h1 = plus ? y1 : -y1;
    h2 = plus ? y2 : -y2;
    return plus;
}

/* sign of the cross product u x v = u1 v2 - u2 v1 (exact) */
__device__ __forceinline__ int td_cross_sign(int64_t u1, int64_t u2, int64_t v1, int64_t v2)
{
    td_i128 l = (td_i128)u1 * v2;
    td_i128 r = (td_i128)u2 * v1;
    return (l > r) - (l < r);
}

/* The same sign; NARROW: the caller has checked that every coordinate is
 * below 2^31 in magnitude, so both products lie below 2^62 and int64 holds
 * them exactly. */
template <bool NARROW>
__device__ __forceinline__ int td_cross_sign_n(int64_t u1, int64_t u2, int64_t v1, int64_t v2)
{
    if constexpr (NARROW) {
        const int64_t l = u1 * v2, r = u2 * v1;
        return (l > r) - (l < r);
    } else {
        return td_cross_sign(u1, u2, v1, v2);
    }
}
