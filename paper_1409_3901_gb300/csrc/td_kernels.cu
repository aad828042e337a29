/*
 * td_kernels.cu -- the sweep kernels of libtukeydepth.so (sm_103a).
 *
 * Work: for every query z, the minimum over the subsets S of K = d-2 nonzero
 * centred points of V(S) = G(S) + m_S (Algorithm 1, Section 3, with the tie
 * readings of the library header), where
 *   G(S)  = min over generic directions v of the quotient of #{ y_i : v.y_i < 0 }
 *           for the projected points y_i = (f_a(x_i), f_b(x_i)) that are nonzero
 *           (Algorithm 2, Section 3), and
 *   m_S   = the open depth of the points of span(S) inside span(S) (0 unless
 *           the span holds more data points than S).
 * T(z) = Z + min_S V(S), Z = number of x_i = 0.
 *
 * Kernels (one CUDA stream, in this order):
 *   td_k_setup      one CTA per query: centring, Z, rank and pivot
 *                   coordinates (exact), per-coordinate maxima, subset count
 *   td_k_tiles      one CTA: tiles per query and their prefix sums
 *   td_k_filtered   persistent CTAs popping (query, subset-tile) work from a
 *                   counter; one warp per subset sweep; FP32 projection with
 *                   a forward error bound, angular bucket histogram in shared
 *                   memory, exact int64/__int128 fallback
 *   td_k_plain      the plain exact form: one launch per query, exact int64
 *                   projections, comparison sort with an exact comparator
 *   td_k_finalize   out[q] = Z + min
 *
 * The bivariate walk.  Parametrise the boundary line of the halfplane by its
 * direction angle phi in [0, pi).  A nonzero y with line direction psi in
 * [0, pi) lies on the counted (left) side for phi just below psi iff y points
 * into the upper half plane (y2 > 0, or y2 = 0 and y1 > 0; "orientation +"),
 * and changes side at phi = psi.  Hence, starting from A = #{orientation +}
 * (the count just below phi = 0), the count at every generic direction is A
 * plus the running sum of -1 (orientation +) / +1 (orientation -) events in
 * increasing psi, read only between groups of equal psi (reading of
 * Algorithm 2 step 1(e) under ties); the opposite direction has the
 * complementary count.  So G = min over those walk values w of min(w, m - w),
 * m the number of nonzero projected points.  This is Algorithm 2's sweep
 * (steps 1(c)-1(e)) with the start direction u0 = (0,-1) and its slopes
 * replaced by exact line directions.
 *
 * The filtered kernel never sorts.  Directions are binned by a pseudo-angle
 * key in [0,2) into B angular buckets whose boundaries are exact integer
 * directions D_j; a point whose FP32 key is not certified to lie inside one
 * bucket is placed exactly by integer cross products with D_j and D_{j+1}.
 * Per bucket only the counts of +1 and -1 events are kept (one shared-memory
 * atomic per point); the walk value at every bucket boundary is then exact,
 * and inside a bucket whose events all have one sign the extremes are at the
 * boundaries.  Only buckets holding both signs whose in-bucket range could
 * pass the extremes seen at the boundaries are resolved, by gathering their
 * events and ordering them exactly.  The result is the exact G.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <limits.h>

#include <map>
#include <mutex>
#include <type_traits>
#include <utility>

#include "td_internal.h"
#include "td_exact.cuh"

#define TD_WARPS_MAX 8
/* points per round of the sweep loop (four per lane, two staged pairs);
 * the staged points are padded to a multiple of it */
#define TD_ROUND 128
#define TD_SENT 0xFFFFu

/* unit roundoff of binary32 */
#define TD_U (1.0f / 16777216.0f)

/* Reciprocal by the hardware approximation (rcp.approx.ftz.f32: at most 1 ulp
 * from 1/x over the normal range, per the PTX ISA). */
__device__ __forceinline__ float td_rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

/* Shared-memory accesses of the point loop with 32-bit shared-window
 * addresses (no 64-bit generic address arithmetic per point). */
__device__ __forceinline__ unsigned td_saddr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float4 td_lds128(unsigned a)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

__device__ __forceinline__ void td_reds_add(unsigned a, unsigned v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

/* Two binary32 values in one 64-bit register pair (low, high), operated on by
 * the packed f32x2 instructions: each half is rounded exactly as the scalar
 * operation would round it. */
typedef unsigned long long td_f2x;

__device__ __forceinline__ td_f2x td_pk(float lo, float hi)
{
    td_f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void td_upk(td_f2x v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ td_f2x td_mul2(td_f2x a, td_f2x b)
{
    td_f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ td_f2x td_fma2(td_f2x a, td_f2x b, td_f2x c)
{
    td_f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ td_f2x td_add2(td_f2x a, td_f2x b)
{
    td_f2x d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ td_f2x td_sub2(td_f2x a, td_f2x b)
{
    td_f2x d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

/* addition rounded toward +infinity */
__device__ __forceinline__ td_f2x td_add2_rp(td_f2x a, td_f2x b)
{
    td_f2x d;
    asm("add.rp.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

/* ---- staged point layout of the filtered kernel --------------------------
 * Points are staged in pairs: pair j holds points p = 64 (j / 32) + j % 32
 * and q = p + 32 (the two points one lane takes in consecutive quarters of a
 * 128-point round).  Plane c (c < ceil(D/2)) of pair j is one float4
 * (x_2c(p), x_2c(q), x_2c+1(p), x_2c+1(q)), so one 128-bit load yields two
 * packed operand pairs.  Planes are npc pairs apart. */
__device__ __forceinline__ int td_pair_of(int i) { return ((i >> 6) << 5) | (i & 31); }

/* Pairs between planes for rows of up to nmax points: nmax rounded up to a
 * round of 128 points, halved, plus two pairs of padding.  Plane c of a
 * point then starts 8c words (mod 32) after plane 0, so the coordinates of
 * one point occupy banks {0, 2, 8, 10, 16, 18} + b and those of the next
 * point (4 words on) {4, 6, 12, 14, 20, 22} + b: the lanes that form the
 * minors of one subset, or of two consecutive subsets at once, never
 * collide. */
__host__ __device__ inline int td_plane_pairs(int nmax) { return (((nmax + 127) & ~127) >> 1) + 2; }

/* Bytes of `planes` staging planes, rounded up to 128 so that the warp
 * regions after them stay 128-byte aligned. */
__host__ __device__ inline size_t td_staging_bytes(int nmax, int planes)
{
    return ((size_t)planes * td_plane_pairs(nmax) * 16 + 127) & ~(size_t)127;
}

__device__ __forceinline__ int td_xidx(int npc, int i, int r)
{
    return (((r >> 1) * npc + td_pair_of(i)) << 2) + ((r & 1) << 1) + ((i >> 5) & 1);
}

/* int64 -> binary32 off the FP64 pipe: exact-to-nearest when the value fits
 * 32 bits, else hi * 2^32 + lo with two roundings (relative error <= 2u,
 * covered by the error bounds below). */
__device__ __forceinline__ float td_i64_to_f32(int64_t v)
{
    int32_t lo32 = (int32_t)v;
    if ((int64_t)lo32 == v) return __int2float_rn(lo32);
    int32_t hi = (int32_t)(v >> 32);
    uint32_t lo = (uint32_t)v;
    return __fadd_rn(__int2float_rn(hi) * 4294967296.0f, __uint2float_rn(lo));
}

/* The same conversion without a branch: |v| as hi * 2^32 + lo, one rounding
 * of hi and one of the fma (lo below 2^32 is rounded once when hi == 0), so
 * the relative error stays within 2u; the sign is copied back. */
__device__ __forceinline__ float td_i64_to_f32_bf(int64_t v)
{
    const uint64_t a = (uint64_t)(v < 0 ? -v : v);
    const float m = __fmaf_rn(__uint2float_rn((uint32_t)(a >> 32)), 4294967296.0f, __uint2float_rn((uint32_t)a));
    return v < 0 ? -m : m;
}

/* ====================================================================== */
/* per-warp global scratch for the exact tight-set path                    */
/* ====================================================================== */

struct TdScratch {
    int32_t *c0;  /* level-0 intrinsic coordinates [NP][4] */
    int64_t *y0;  /* level-0 normalised projections [NP][2] */
    uint16_t *i0; /* level-0 sort list [NP] */
    int32_t *c1;  /* level-1 coordinates [NP][4] */
    int64_t *y1;  /* level-1 projections [NP][2] */
    uint16_t *i1; /* level-1 sort list [NP] */
    uint16_t *bid;   /* filtered sweep: bucket id per point (rare path) [NP] */
    uint16_t *glist; /* filtered sweep: uncertain / gathered points (rare path) [NP] */
};

__host__ __device__ inline int64_t td_scratch_bytes(int np)
{
    return (int64_t)np * (16 + 16 + 2 + 16 + 16 + 2 + 2 + 2) + 256;
}

__device__ inline TdScratch td_scratch_at(char *base, int np)
{
    TdScratch s;
    char *p = base;
    s.c0 = (int32_t *)p; p += (size_t)np * 16;
    s.y0 = (int64_t *)p; p += (size_t)np * 16;
    s.c1 = (int32_t *)p; p += (size_t)np * 16;
    s.y1 = (int64_t *)p; p += (size_t)np * 16;
    s.i0 = (uint16_t *)p; p += (size_t)np * 2;
    s.i1 = (uint16_t *)p; p += (size_t)np * 2;
    s.bid = (uint16_t *)p; p += (size_t)np * 2;
    s.glist = (uint16_t *)p;
    return s;
}

__host__ __device__ inline int td_pow2_at_least(int v)
{
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}

/* ====================================================================== */
/* exact sort + walk on a list of normalised projections                   */
/* ====================================================================== */

/* Item ids carry the orientation in bit 15 (set = orientation +). */
__device__ __forceinline__ bool td_item_less(uint16_t u, uint16_t v, const int64_t *H)
{
    if (u == TD_SENT) return false;
    if (v == TD_SENT) return true;
    int a = u & 0x7FFF, b = v & 0x7FFF;
    return td_cross_sign(H[2 * a], H[2 * a + 1], H[2 * b], H[2 * b + 1]) > 0;
}

/* Sign of u x v for the exact integer pairs H (u = (u1, u2), ...) with
 * binary32 copies Hf: the FP32 cross product decides when it exceeds its
 * forward error bound, else the exact __int128 one.  Each float is the int64
 * rounded to nearest (relative error <= u = 2^-24, products < 2^125, no
 * overflow); the fma-based cross product then differs from the exact one by
 * less than 6u(|u1 v2| + |u2 v1|), and |u1 v2| <= |p1|(1 + 4u) for the
 * rounded product p1, so |c| > 8u(|p1| + |p2|) fixes the sign. */
__device__ __forceinline__ int td_cross_sign_f(float2 uf, float2 vf, int64_t u1, int64_t u2, int64_t v1, int64_t v2)
{
    const float p2 = uf.y * vf.x;
    const float p1 = uf.x * vf.y;
    const float c = fmaf(uf.x, vf.y, -p2);
    const float b = (8.0f * TD_U) * (fabsf(p1) + fabsf(p2));
    if (c > b) return 1;
    if (c < -b) return -1;
    return td_cross_sign(u1, u2, v1, v2);
}

/* td_item_less with the FP32 filter of td_cross_sign_f (Hf may be null). */
template <bool NARROW = false>
__device__ __forceinline__ bool td_item_less_f(uint16_t u, uint16_t v, const int64_t *H, const float2 *Hf)
{
    if (u == TD_SENT) return false;
    if (v == TD_SENT) return true;
    const int a = u & 0x7FFF, b = v & 0x7FFF;
    if (!Hf) return td_cross_sign_n<NARROW>(H[2 * a], H[2 * a + 1], H[2 * b], H[2 * b + 1]) > 0;
    return td_cross_sign_f(Hf[a], Hf[b], H[2 * a], H[2 * a + 1], H[2 * b], H[2 * b + 1]) > 0;
}

/* Bitonic sort of idx[0..npad) (npad a power of two >= 32; entries beyond the
 * valid ones are TD_SENT) by increasing line direction, one warp. */
__device__ void td_sort_exact(uint16_t *idx, int npad, const int64_t *H, int lane)
{
    for (int size = 2; size <= npad; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < (npad >> 1); t += 32) {
                int i = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
                int j = i + stride;
                bool up = (i & size) == 0;
                uint16_t u = idx[i], v = idx[j];
                bool swap = up ? td_item_less(v, u, H) : td_item_less(u, v, H);
                if (swap) {
                    idx[i] = v;
                    idx[j] = u;
                }
            }
            __syncwarp();
        }
}

/* The same sort for the plain form and the Algorithm 3 search, where
 * registers are not scarce: the pairs of one step are disjoint, so each lane
 * takes four of them at a time (all loads first, then the four comparisons,
 * then the stores; the steps are latency-bound otherwise), and with Hf
 * (binary32 copies of H, may be null) the comparisons are FP32-filtered;
 * they are exact either way.  (The sweep kernel keeps td_sort_exact: this
 * one, inlined there, costs it registers.) */
template <bool NARROW = false>
__device__ void td_sort_exact_fast(uint16_t *idx, int npad, const int64_t *H, int lane, const float2 *Hf)
{
    const int half = npad >> 1;
    for (int size = 2; size <= npad; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            int t = lane;
            for (; t + 96 < half; t += 128) {
                int ii[4], ia[4], ib[4], cr[4];
                uint16_t u[4], v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int tt = t + 32 * k;
                    ii[k] = ((tt & ~(stride - 1)) << 1) | (tt & (stride - 1));
                    u[k] = idx[ii[k]];
                    v[k] = idx[ii[k] + stride];
                    ia[k] = u[k] == TD_SENT ? 0 : (u[k] & 0x7FFF);
                    ib[k] = v[k] == TD_SENT ? 0 : (v[k] & 0x7FFF);
                }
                if (Hf) {
                    float2 fa[4], fb[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        fa[k] = Hf[ia[k]];
                        fb[k] = Hf[ib[k]];
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float p2 = fa[k].y * fb[k].x;
                        const float p1 = fa[k].x * fb[k].y;
                        const float c = fmaf(fa[k].x, fb[k].y, -p2);
                        const float bnd = (8.0f * TD_U) * (fabsf(p1) + fabsf(p2));
                        cr[k] = c > bnd ? 1 : (c < -bnd ? -1 : 2);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (cr[k] == 2)
                            cr[k] = td_cross_sign(H[2 * ia[k]], H[2 * ia[k] + 1], H[2 * ib[k]], H[2 * ib[k] + 1]);
                } else {
                    int64_t a1[4], a2[4], b1[4], b2[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        a1[k] = H[2 * ia[k]];
                        a2[k] = H[2 * ia[k] + 1];
                        b1[k] = H[2 * ib[k]];
                        b2[k] = H[2 * ib[k] + 1];
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) cr[k] = td_cross_sign_n<NARROW>(a1[k], a2[k], b1[k], b2[k]);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    /* u before v iff u is valid and (v is padding or u x v > 0) */
                    const bool uv = u[k] != TD_SENT && (v[k] == TD_SENT || cr[k] > 0);
                    const bool vu = v[k] != TD_SENT && (u[k] == TD_SENT || cr[k] < 0);
                    const bool up = (ii[k] & size) == 0;
                    if (up ? vu : uv) {
                        idx[ii[k]] = v[k];
                        idx[ii[k] + stride] = u[k];
                    }
                }
            }
            for (; t < half; t += 32) {
                int i = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
                int j = i + stride;
                bool up = (i & size) == 0;
                uint16_t u = idx[i], v = idx[j];
                bool swap = up ? td_item_less_f<NARROW>(v, u, H, Hf) : td_item_less_f<NARROW>(u, v, H, Hf);
                if (swap) {
                    idx[i] = v;
                    idx[j] = u;
                }
            }
            __syncwarp();
        }
}

/* Walk over the cnt sorted items: returns min over walk values w of
 * min(w, m - w) where the walk starts at A (orientation + count) and m = cnt. */
template <bool NARROW = false>
__device__ int td_walk_sorted(const uint16_t *idx, int cnt, const int64_t *H, int lane)
{
    int A = 0;
    for (int l = lane; l < cnt; l += 32) A += (idx[l] >> 15) & 1;
    A = td_wsum(A);
    int C = (cnt + 31) >> 5;
    int beg = min(lane * C, cnt), end = min(beg + C, cnt);
    int s = 0;
    for (int l = beg; l < end; ++l) s += (idx[l] & 0x8000) ? -1 : 1;
    int excl = td_wscan_incl(s, lane) - s;
    int v = A + excl;
    int mn = A, mx = A;
    for (int l = beg; l < end; ++l) {
        uint16_t it = idx[l];
        v += (it & 0x8000) ? -1 : 1;
        bool tie = false;
        if (l + 1 < cnt) {
            int a = it & 0x7FFF, b = idx[l + 1] & 0x7FFF;
            tie = td_cross_sign_n<NARROW>(H[2 * a], H[2 * a + 1], H[2 * b], H[2 * b + 1]) == 0;
        }
        if (!tie) {
            mn = min(mn, v);
            mx = max(mx, v);
        }
    }
    mn = td_wmin(mn);
    mx = td_wmax(mx);
    return min(mn, cnt - mx);
}

/* Given normalised projections H[0..cnt) (all nonzero) and orientations,
 * build the item list in idx, sort and walk.  plus(i) from bit list. */
__device__ int td_sweep_list(uint16_t *idx, int cnt, const int64_t *H, int lane)
{
    int npad = td_pow2_at_least(cnt);
    for (int l = cnt + lane; l < npad; l += 32) idx[l] = TD_SENT;
    __syncwarp();
    td_sort_exact(idx, npad, H, lane);
    return td_walk_sorted(idx, cnt, H, lane);
}

/* ====================================================================== */
/* open depth of a small full-rank point set (the tight-set path)         */
/* ====================================================================== */

/* N x N determinant (top-left block of an S x S array) by cofactor expansion
 * (N <= 5, small entries). */
template <int N, int S>
__device__ int64_t td_detn(const int64_t (&m)[S][S])
{
    if constexpr (N == 1) {
        return m[0][0];
    } else {
        int64_t acc = 0;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            int64_t sub[S][S];
#pragma unroll
            for (int r = 1; r < N; ++r) {
                int o = 0;
#pragma unroll
                for (int cc = 0; cc < N; ++cc)
                    if (cc != c) sub[r - 1][o++] = m[r][cc];
            }
            int64_t t = m[0][c] * td_detn<N - 1>(sub);
            acc += (c & 1) ? -t : t;
        }
        return acc;
    }
}

template <int KK>
__device__ int td_open_depth(const int32_t *c, int t, const TdScratch &scr, int lane, int level);
template <int KK, int CS>
__device__ int td_open_depth_s(const int32_t *c, int t, const TdScratch &scr, int lane);

/* 2-D open depth of t nonzero integer points (coordinates 0,1 of c). */
__device__ int td_open_depth2(const int32_t *c, int t, int64_t *Y, uint16_t *I, int lane)
{
    for (int i = lane; i < t; i += 32) {
        int64_t h1, h2;
        bool plus = td_normalise(c[4 * i], c[4 * i + 1], h1, h2);
        Y[2 * i] = h1;
        Y[2 * i + 1] = h2;
        I[i] = (uint16_t)(i | (plus ? 0x8000 : 0));
    }
    __syncwarp();
    return td_sweep_list(I, t, Y, lane);
}

/* Projections of the t points of c (dimension DD) onto the quotient by the
 * subset s (DD-2 points of c); writes nonzero normalised ones to Y/I, and the
 * tight ones' intrinsic coordinates to ct (if DD-2 >= 2) or their sign counts.
 * Returns false if the subset is dependent. */
template <int DD, int CS = 4>
__device__ bool td_project_small(const int32_t *c, int t, const int *sub, int64_t *Y, uint16_t *I,
                                 int32_t *ct, int &nz, int &nt, int &pos, int &neg, int lane)
{
    constexpr int K = DD - 2;
    int64_t s[K > 0 ? K : 1][DD];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int r = 0; r < DD; ++r) s[j][r] = c[CS * sub[j] + r];
    TdBasis<DD> B;
    if (!td_make_basis<DD>(s, B)) return false;
    int *cnt = (int *)nullptr;
    (void)cnt;
    /* lane-parallel projection with warp compaction (stable by ballot) */
    int base_nz = 0, base_t = 0;
    pos = 0;
    neg = 0;
    for (int i0 = 0; i0 < t; i0 += 32) {
        int i = i0 + lane;
        int64_t y1 = 0, y2 = 0;
        bool valid = i < t;
        if (valid) {
#pragma unroll
            for (int r = 0; r < DD; ++r) {
                int64_t x = c[CS * i + r];
                y1 += B.qa[r] * x;
                y2 += B.qb[r] * x;
            }
        }
        bool tight = valid && y1 == 0 && y2 == 0;
        bool nonz = valid && !tight;
        unsigned bn = __ballot_sync(TD_FULL, nonz), bt = __ballot_sync(TD_FULL, tight);
        unsigned below = (1u << lane) - 1u;
        if (nonz) {
            int slot = base_nz + __popc(bn & below);
            int64_t h1, h2;
            bool plus = td_normalise(y1, y2, h1, h2);
            Y[2 * slot] = h1;
            Y[2 * slot + 1] = h2;
            I[slot] = (uint16_t)(slot | (plus ? 0x8000 : 0));
        }
        if (tight) {
            if (K == 1) {
                int32_t v = c[CS * i + B.rows[0]];
                pos += v > 0;
                neg += v < 0;
            } else {
                int slot = base_t + __popc(bt & below);
#pragma unroll
                for (int r = 0; r < K; ++r) ct[4 * slot + r] = c[CS * i + B.rows[r]];
            }
        }
        base_nz += __popc(bn);
        base_t += __popc(bt);
    }
    pos = td_wsum(pos);
    neg = td_wsum(neg);
    nz = base_nz;
    nt = base_t;
    __syncwarp();
    return true;
}

template <int KK>
__device__ int td_open_depth(const int32_t *c, int t, const TdScratch &scr, int lane, int level)
{
    if constexpr (KK == 1) {
        int pos = 0, neg = 0;
        for (int i = lane; i < t; i += 32) {
            pos += c[4 * i] > 0;
            neg += c[4 * i] < 0;
        }
        pos = td_wsum(pos);
        neg = td_wsum(neg);
        return min(pos, neg);
    } else if constexpr (KK == 2) {
        return td_open_depth2(c, t, level == 0 ? scr.y0 : scr.y1, level == 0 ? scr.i0 : scr.i1, lane);
    } else if constexpr (KK == 3) {
        /* subsets of one point; inner tight sets are 1-D (sign counts) */
        int best = INT_MAX;
        for (int s0 = 0; s0 < t; ++s0) {
            int sub[1] = { s0 };
            int nz, nt, pos, neg;
            if (!td_project_small<3>(c, t, sub, scr.y0, scr.i0, nullptr, nz, nt, pos, neg, lane)) continue;
            int G = td_sweep_list(scr.i0, nz, scr.y0, lane);
            best = min(best, G + min(pos, neg));
        }
        return best;
    } else {
        /* subsets of two points; inner tight sets are 2-D */
        int best = INT_MAX;
        for (int s1 = 1; s1 < t; ++s1)
            for (int s0 = 0; s0 < s1; ++s0) {
                int sub[2] = { s0, s1 };
                int nz, nt, pos, neg;
                if (!td_project_small<4>(c, t, sub, scr.y0, scr.i0, scr.c1, nz, nt, pos, neg, lane)) continue;
                int G = td_sweep_list(scr.i0, nz, scr.y0, lane);
                if (G >= best) continue;
                int m = (nt > 2) ? td_open_depth2(scr.c1, nt, scr.y1, scr.i1, lane) : 0;
                best = min(best, G + m);
            }
        return best;
    }
}

/* Open depth of t nonzero points in 5 dimensions with coordinates at stride
 * CS in c (the hyperplanes of the critical-direction form at d = 6): the same
 * subset method with subsets of three points, whose inner tight sets are
 * 3-D (td_open_depth<3>). */
template <int KK, int CS>
__device__ int td_open_depth_s(const int32_t *c, int t, const TdScratch &scr, int lane)
{
    static_assert(KK == 5, "five dimensions only");
    int best = INT_MAX;
    for (int s2 = 2; s2 < t; ++s2)
        for (int s1 = 1; s1 < s2; ++s1)
            for (int s0 = 0; s0 < s1; ++s0) {
                int sub[3] = { s0, s1, s2 };
                int nz, nt, pos, neg;
                if (!td_project_small<5, CS>(c, t, sub, scr.y0, scr.i0, scr.c1, nz, nt, pos, neg, lane)) continue;
                const int G = td_sweep_list(scr.i0, nz, scr.y0, lane);
                if (G >= best) continue;
                const int m = nt > 3 ? td_open_depth<3>(scr.c1, nt, scr, lane, 1) : 0;
                best = min(best, G + m);
            }
    return best;
}

/* m_S for a subset whose span holds t > K data points: the tight points'
 * intrinsic coordinates are in scr.c0[0..t) and the subset's own points are
 * sint[0..K).  A quick test first: if the functional w(x) = sum_j
 * det(S with column j replaced by x) (w(s_j) = det S for every j) has the
 * sign of det S on every tight point, the tight set lies in an open
 * halfspace of span(S) and m_S = 0.  Otherwise the open depth is computed
 * by the same subset method one level down. */
template <int K>
__device__ int td_tight_depth(int t, const int64_t (&sint)[4][4], const TdScratch &scr, int lane)
{
    if constexpr (K <= 1) {
        return 0; /* handled by the caller with sign counts */
    } else {
        int64_t M[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < 4; ++j) M[r][j] = (r < K && j < K) ? sint[j][r] : 0;
        int64_t det = td_detn<K>(M);
        int64_t cw[4] = { 0, 0, 0, 0 };
#pragma unroll
        for (int r = 0; r < K; ++r) {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                int64_t Mr[4][4];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) Mr[rr][jj] = M[rr][jj];
#pragma unroll
                for (int rr = 0; rr < K; ++rr) Mr[rr][j] = (rr == r) ? 1 : 0;
                cw[r] += td_detn<K>(Mr);
            }
        }
        bool ok = true;
        for (int i = lane; i < t; i += 32) {
            int64_t w = 0;
#pragma unroll
            for (int r = 0; r < K; ++r) w += cw[r] * (int64_t)scr.c0[4 * i + r];
            ok &= (det > 0) ? (w > 0) : (w < 0);
        }
        if (__all_sync(TD_FULL, ok)) return 0;
        return td_open_depth<K>(scr.c0, t, scr, lane, 0);
    }
}

/* ====================================================================== */
/* set-up kernel                                                           */
/* ====================================================================== */

__device__ inline td_i128 td_i128_abs(td_i128 v) { return v < 0 ? -v : v; }

/* gcd(|a|, |b|).  When both fit in 63 bits (the usual case) by the binary
 * method (Stein): strip the common power of two, then subtract the smaller
 * odd value from the larger and strip the twos until one is zero; max(x, y)
 * falls every step, so the loop ends within 64 steps per bit pattern.  No
 * division, where Euclid's int128 remainder is a long software sequence.
 * Wider values use Euclid. */
__device__ inline td_i128 td_i128_gcd(td_i128 a, td_i128 b)
{
    a = td_i128_abs(a);
    b = td_i128_abs(b);
    if ((a >> 63) == 0 && (b >> 63) == 0) {
        uint64_t x = (uint64_t)a, y = (uint64_t)b;
        if (x == 0) return (td_i128)y;
        if (y == 0) return (td_i128)x;
        const int sh = __ffsll((long long)(x | y)) - 1;
        x >>= __ffsll((long long)x) - 1;
        do {
            y >>= __ffsll((long long)y) - 1;
            if (x > y) {
                const uint64_t t = x;
                x = y;
                y = t;
            }
            y -= x;
        } while (y != 0);
        return (td_i128)(x << sh);
    }
    while (b != 0) {
        td_i128 r = a % b;
        a = b;
        b = r;
    }
    return a;
}

/* v / g for a divisor g > 0 of v: nothing for g = 1, a 64-bit divide when
 * both are below 2^62, the int128 divide otherwise */
__device__ inline td_i128 td_i128_div_exact(td_i128 v, td_i128 g)
{
    if (g == 1) return v;
    const td_i128 lim = (td_i128)1 << 62;
    if (v < lim && v > -lim && g < lim) return (td_i128)((int64_t)v / (int64_t)g);
    return v / g;
}

__global__ void __launch_bounds__(256) td_k_setup(TdLaunch L)
{
    const int q = blockIdx.x;
    __shared__ int s_z[TD_MAXD];
    __shared__ int s_Z, s_max[TD_MAXD], s_pos, s_neg, s_amax;
    __shared__ int s_d, s_piv[TD_MAXD];
    TdQuery *Q = &L.q[q];
    const int set = Q->set;
    const TdSet S = L.sets[set];
    const int n = S.n, p = S.p;
    const int32_t *X = L.X + S.x_off;
    if (threadIdx.x < TD_MAXD) {
        s_z[threadIdx.x] = threadIdx.x < p ? L.Zq[(int64_t)q * TD_MAXD + threadIdx.x] : 0;
        s_max[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
        s_Z = 0;
        s_pos = 0;
        s_neg = 0;
        s_amax = 0;
    }
    __syncthreads();
    /* Z and the largest centred coordinate (every coordinate) */
    int zc = 0, amx = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        bool zero = true;
        for (int c = 0; c < p; ++c) {
            const int64_t v = (int64_t)X[(int64_t)i * p + c] - s_z[c];
            zero &= v == 0;
            amx = max(amx, (int)min(v < 0 ? -v : v, (int64_t)INT_MAX));
        }
        zc += zero;
    }
    atomicAdd(&s_Z, zc);
    atomicMax(&s_amax, amx);
    __syncthreads();
    /* the range of subset positions of this call: the dataset's time slice
     * if it has one, else the call's shard */
    int64_t sc = L.shard_count > 1 ? L.shard_count : 1;
    int64_t si = L.shard_count > 1 ? L.shard_index : 0;
    if (S.slice_count > 1) {
        sc = S.slice_count;
        si = S.slice_index;
    }
    const bool first_shard = si == 0;
    /* the fast kernels' limit, and for the critical-direction form its own:
     * p! M^p < 2^62, every normal and n.x exact in int64 */
    bool wide = s_amax > td_coord_limit_of(p);
    if (L.critical && !wide) {
        td_i128 v = 1;
        for (int i = 2; i <= p; ++i) v *= i;
        for (int i = 0; i < p && !wide; ++i) {
            v *= s_amax;
            wide = v >= ((td_i128)1 << 62);
        }
    }
    if (wide) {
        /* beyond the limit: no rank, no subset loop, no bound here; the
         * wide kernel (td_wide.cuh) computes the count on the first shard */
        if (threadIdx.x == 0) {
            Q->n = n;
            Q->Z = s_Z;
            Q->nnz = n - s_Z;
            Q->d = 0;
            Q->k = -1;
            Q->direct = first_shard ? TD_DIRECT_WIDE : INT_MAX;
            if (first_shard) atomicAdd(&L.ctr->wide, 1ull);
            Q->amax = s_amax;
            for (int c = 0; c < TD_MAXD; ++c) {
                Q->piv[c] = 0;
                Q->mx[c] = 0;
            }
            Q->nsub = 0;
            Q->lo = Q->hi = 0;
            L.qmin[q] = INT_MAX;
        }
        return;
    }
    /* rank and pivot coordinates, exact: incremental elimination over the
     * nonzero points with primitive (gcd-normalised) basis rows. */
    if (threadIdx.x == 0) {
        td_i128 basis[TD_MAXD][TD_MAXD];
        int pc[TD_MAXD];
        int r = 0;
        for (int i = 0; i < n && r < p; ++i) {
            td_i128 v[TD_MAXD];
            bool nz = false;
            for (int c = 0; c < p; ++c) {
                v[c] = (td_i128)((int64_t)X[(int64_t)i * p + c] - s_z[c]);
                nz |= v[c] != 0;
            }
            if (!nz) continue;
            for (int b = 0; b < r; ++b) {
                td_i128 f = v[pc[b]];
                if (f == 0) continue;
                td_i128 e = basis[b][pc[b]];
                bool big = false;
                for (int c = 0; c < p; ++c) {
                    v[c] = e * v[c] - f * basis[b][c];
                    big |= td_i128_abs(v[c]) > ((td_i128)1 << 60);
                }
                if (big) {
                    td_i128 g = 0;
                    for (int c = 0; c < p; ++c) g = td_i128_gcd(g, v[c]);
                    if (g > 1)
                        for (int c = 0; c < p; ++c) v[c] = td_i128_div_exact(v[c], g);
                }
            }
            int lead = -1;
            for (int c = 0; c < p; ++c)
                if (v[c] != 0) { lead = c; break; }
            if (lead < 0) continue;
            td_i128 g = 0;
            for (int c = 0; c < p; ++c) g = td_i128_gcd(g, v[c]);
            for (int c = 0; c < p; ++c) basis[r][c] = td_i128_div_exact(v[c], g);
            pc[r] = lead;
            ++r;
        }
        for (int a = 0; a < r; ++a)
            for (int b = a + 1; b < r; ++b)
                if (pc[b] < pc[a]) { int t = pc[a]; pc[a] = pc[b]; pc[b] = t; }
        s_d = r;
        for (int a = 0; a < TD_MAXD; ++a) s_piv[a] = a < r ? pc[a] : 0;
    }
    __syncthreads();
    const int d = s_d;
    /* per-coordinate maxima over the projected coordinates, and the sign
     * counts of the single coordinate when d == 1 */
    int lmax[TD_MAXD] = { 0, 0, 0, 0, 0, 0 };
    int pos = 0, neg = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        for (int c = 0; c < d; ++c) {
            int64_t v = (int64_t)X[(int64_t)i * p + s_piv[c]] - s_z[s_piv[c]];
            int64_t a = v < 0 ? -v : v;
            lmax[c] = max(lmax[c], (int)min(a, (int64_t)INT_MAX));
            if (d == 1) {
                pos += v > 0;
                neg += v < 0;
            }
        }
    }
    for (int c = 0; c < d; ++c) atomicMax(&s_max[c], lmax[c]);
    if (d == 1) {
        atomicAdd(&s_pos, pos);
        atomicAdd(&s_neg, neg);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int Z = s_Z;
        Q->n = n;
        Q->Z = Z;
        Q->nnz = n - Z;
        Q->d = d;
        Q->amax = s_amax;
        for (int c = 0; c < TD_MAXD; ++c) {
            Q->piv[c] = s_piv[c];
            Q->mx[c] = c < d ? s_max[c] : 0;
        }
        if (n - Z == 0 || d <= 1) {
            int direct = (n - Z == 0) ? n : Z + min(s_pos, s_neg);
            Q->direct = first_shard ? direct : INT_MAX;
            Q->k = -1;
            Q->nsub = 0;
            Q->lo = Q->hi = 0;
        } else {
            Q->direct = -1;
            Q->k = L.critical ? d - 1 : d - 2;
            int64_t ns = (int64_t)td_binom(n - Z, Q->k);
            Q->nsub = ns;
            Q->lo = (int64_t)((__int128)ns * si / sc);
            Q->hi = (int64_t)((__int128)ns * (si + 1) / sc);
        }
        L.qmin[q] = INT_MAX;
    }
}

/* An upper bound of T from data directions u = +-x_j (Algorithm 3, Step 2):
 * T <= #{i : u'x_i <= 0} for every u, exact in int32 or int64.  qmin starts
 * at that bound minus Z (T = Z + min V, and a sweep reports V exactly
 * whenever it is below qmin), so the coarse bound prunes from the first
 * sweep of every tile on.  No subset is skipped for it.  The bound costs n
 * point evaluations per direction; ndir = min(n, subsets / 64) evenly spaced
 * directions keep it near 1% of the subset loop (none for a loop of fewer
 * than 64 subsets).  Runs after td_k_setup, TD_BOUND_SPLIT CTAs per query
 * (CTA b: query b / split), one direction per warp at a time, the lanes
 * splitting the points; the centred rows staged in shared memory when the
 * dot products fit in int32. */
__global__ void __launch_bounds__(256) td_k_bound(TdLaunch L, int split, int cap)
{
    extern __shared__ __align__(16) int32_t s_xc[]; /* n x p centred rows (int32 form) */
    const int q = blockIdx.x / split, g = blockIdx.x % split;
    const TdQuery &Q = L.q[q];
    if (Q.direct != -1 || L.unseeded) return;
    const int n = Q.n;
    const int ndir = (int)min((int64_t)n, Q.nsub / 64);
    if (ndir <= 0) return;
    const TdSet S = L.sets[Q.set];
    const int p = S.p;
    const int32_t *X = L.X + S.x_off;
    const int32_t *z = L.Zq + (int64_t)q * TD_MAXD;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    /* the dot products in 32 bits when p max|x_c|^2 < 2^31 over every
     * centred coordinate (then every centred entry fits too) */
    const int am = Q.amax;
    const bool n32 = am < 46341 && (int64_t)p * am * am < 2147483648LL && n * p <= cap;
    if (n32) {
        for (int e = threadIdx.x; e < n * p; e += blockDim.x) s_xc[e] = X[e] - z[e % p];
        __syncthreads();
    }
    int ub = INT_MAX;
    for (int kd = g * nw + w; kd < ndir; kd += split * nw) {
        const int j = (int)((int64_t)kd * n / ndir);
        int le = 0, ge = 0;
        bool nz = false;
        if (n32) {
            int xj[TD_MAXD];
#pragma unroll
            for (int c = 0; c < TD_MAXD; ++c) {
                xj[c] = c < p ? s_xc[j * p + c] : 0;
                nz |= xj[c] != 0;
            }
            if (!nz) continue; /* uniform across the warp */
            for (int i = lane; i < n; i += 32) {
                const int32_t *xi = s_xc + i * p;
                int dot = 0;
#pragma unroll
                for (int c = 0; c < TD_MAXD; ++c)
                    if (c < p) dot += xj[c] * xi[c];
                le += dot <= 0;
                ge += dot >= 0;
            }
        } else {
            int64_t xj[TD_MAXD];
#pragma unroll
            for (int c = 0; c < TD_MAXD; ++c) {
                xj[c] = c < p ? (int64_t)X[(int64_t)j * p + c] - z[c] : 0;
                nz |= xj[c] != 0;
            }
            if (!nz) continue;
            for (int i = lane; i < n; i += 32) {
                int64_t dot = 0;
                for (int c = 0; c < p; ++c) dot += xj[c] * ((int64_t)X[(int64_t)i * p + c] - z[c]);
                le += dot <= 0;
                ge += dot >= 0;
            }
        }
        le = td_wsum(le);
        ge = td_wsum(ge);
        ub = min(ub, min(le, ge));
    }
    if (lane == 0 && ub < INT_MAX) atomicMin(&L.qmin[q], ub - Q.Z);
}

/* ====================================================================== */
/* tile prefix kernel                                                      */
/* ====================================================================== */

/* Subsets per warp and tile: about 3 * 2^16 point evaluations per warp and
 * tile (the block barrier at the end of a tile, where the warps wait for
 * the slowest, then costs a few percent), at most 1024, and at most 1/64 of
 * the query's range per CTA tile so that a short subset loop still spreads
 * over many CTAs; at least 4. */
/* a / b for b > 0, by the 32-bit unsigned divide when both operands fit */
__host__ __device__ inline int64_t td_div_nonneg(int64_t a, int64_t b)
{
    if (((uint64_t)a | (uint64_t)b) >> 32 == 0) return (int64_t)((uint32_t)a / (uint32_t)b);
    return a / b;
}

__host__ __device__ inline int td_auto_spw(int nnz, int64_t nrange, int warps)
{
    int64_t s = 196608 / (nnz > 0 ? nnz : 1);
    const int64_t cap = td_div_nonneg(nrange, 64 * (int64_t)(warps > 0 ? warps : 1));
    s = s < cap ? s : cap;
    return s < 4 ? 4 : (s > 1024 ? 1024 : (int)s);
}

/* Tiles of every query, and for each effective dimension D = 2..6 the prefix
 * sums of the tiles of the queries of that dimension in work order
 * (tile_prefix[(D-2)*(nq+1) + j]); resets the work counters. */
__global__ void __launch_bounds__(1024) td_k_tiles(TdLaunch L)
{
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_block, s_total[TD_NDIM];
    const int nq = L.nq;
    const int T = blockDim.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = T >> 5;
    /* the tiles of query q = order[j]: its tile size, stored, and its count */
    auto tiles_of = [&](int j, int &dim) -> int64_t {
        const int q = L.order[j];
        const TdQuery &Q = L.q[q];
        int spw = L.spw;
        if (spw <= 0 && Q.d >= 2 && Q.d <= 6 && Q.nnz > 0) spw = L.spw_tab[Q.d - 2][td_octave(Q.nnz)];
        if (spw <= 0) spw = td_auto_spw(Q.nnz, Q.hi - Q.lo, L.warps);
        const int64_t ts = (int64_t)spw * L.warps;
        L.tile_size[q] = (int)ts;
        dim = (Q.d >= 2 && Q.d <= 6) ? Q.d - 2 : -1;
        return (Q.k >= 0 && Q.hi > Q.lo) ? td_div_nonneg(Q.hi - Q.lo + ts - 1, ts) : 0;
    };
    /* block-wide exclusive scan of v (and the block total) */
    auto block_scan = [&](int64_t v, int64_t &total) -> int64_t {
        int64_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(TD_FULL, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane == 31) s_warp[w] = inc;
        __syncthreads();
        if (w == 0) {
            const int64_t x = lane < nw ? s_warp[lane] : 0;
            int64_t xi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(TD_FULL, xi, o);
                if (lane >= o) xi += u;
            }
            if (lane < nw) s_warp[lane] = xi - x;
            if (lane == 31) s_block = xi; /* nw <= 32: lane 31 holds the total */
        }
        __syncthreads();
        const int64_t ex = s_warp[w] + inc - v;
        total = s_block;
        __syncthreads(); /* s_warp is rewritten by the next scan */
        return ex;
    };
    /* rounds of T consecutive work-order positions (coalesced writes), a
     * running carry per dimension; the block scan only for the dimensions
     * that hold a query in the round (the others' entries are the carry:
     * every dimension's array must be complete, since its sweep kernel maps
     * a ticket to its query by a binary search over all of it) */
    int64_t carry[TD_NDIM] = { 0, 0, 0, 0, 0 };
    for (int base = 0; base < nq; base += T) {
        const int j = base + (int)threadIdx.x;
        int dim = -1;
        const int64_t cnt = j < nq ? tiles_of(j, dim) : 0;
#pragma unroll
        for (int D = 0; D < TD_NDIM; ++D) {
            int64_t ex = 0, tot = 0;
            if (__syncthreads_or(dim == D)) ex = block_scan(dim == D ? cnt : 0, tot);
            if (j < nq) L.tile_prefix[(int64_t)D * (nq + 1) + j] = carry[D] + ex;
            carry[D] += tot;
        }
    }
    if (threadIdx.x < TD_NDIM) s_total[threadIdx.x] = carry[threadIdx.x];
    __syncthreads();
#pragma unroll
    for (int D = 0; D < TD_NDIM; ++D) {
        if (threadIdx.x == 0) {
            L.tile_prefix[(int64_t)D * (nq + 1) + nq] = s_total[D];
            L.ticket[D * TD_TICKET_STRIDE] = 0ull;
        }
    }
}

/* ====================================================================== */
/* shared staging of one query's nonzero centred points                    */
/* ====================================================================== */

/* Bulk copies (the Tensor Memory Accelerator's untiled form) of a dataset
 * into shared memory, completed on an mbarrier.  The source and destination
 * must be 16-byte aligned and the size a multiple of 16 bytes. */
__device__ __forceinline__ void td_mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(td_saddr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void td_bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    /* generic-proxy accesses of dst before this point are ordered before
     * the copy's async-proxy writes */
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(td_saddr(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(td_saddr(dst)), "l"(src), "r"(bytes), "r"(td_saddr(bar))
                 : "memory");
}

/* Wait for the phase `parity` of bar to complete, at most `limit` tries;
 * returns false if it did not. */
__device__ __forceinline__ bool td_mbar_wait(uint64_t *bar, unsigned parity, int limit)
{
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(td_saddr(bar)), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

/* Stage the nonzero projected centred points of query q, in the order of the
 * data (or, under Algorithm 3, in the order L.perm gives), into xs in the
 * pair layout (td_xidx, nplanes planes npc pairs apart) -- exact, the
 * coordinates are integers below 2^24.  The dataset's rows are first copied
 * into raw (shared memory, raw_bytes long) by one bulk copy when they fit
 * and their address is 16-byte aligned (the last size % 16 bytes by plain
 * loads), else read from global memory.  bar / phase: the CTA's mbarrier
 * and the parity its next completion has.  Returns the number staged
 * (== Q.nnz), or -1 if the bulk copy did not complete within its bound
 * (an error the caller reports; the CTA must stop). */
__device__ int td_stage_points(const TdLaunch &L, int q, float *xs, int npc, int nplanes, int *s_tmp,
                               int32_t *raw, size_t raw_bytes, uint64_t *bar, unsigned &phase)
{
    const TdQuery &Q = L.q[q];
    const TdSet S = L.sets[Q.set];
    const int n = S.n, p = S.p, d = Q.d;
    const int32_t *Xg = L.X + S.x_off;
    const int32_t *z = L.Zq + (int64_t)q * TD_MAXD;
    const int T = blockDim.x;
    const unsigned bytes = (unsigned)((size_t)n * p * 4);
    const unsigned bulk = bytes & ~15u;
    const bool tma = bytes <= raw_bytes && bulk > 0 && ((uintptr_t)Xg & 15) == 0;
    const int32_t *X = Xg;
    if (tma) {
        if (threadIdx.x == 0) td_bulk_load(raw, Xg, bulk, bar);
        /* the tail that is not a multiple of 16 bytes */
        for (unsigned b = bulk / 4 + threadIdx.x; b < bytes / 4; b += T) raw[b] = Xg[b];
        const bool ok = td_mbar_wait(bar, phase, 1 << 22);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            /* the copy may still be in flight: give it one more bounded wait */
            td_mbar_wait(bar, phase ^ 1u, 1 << 22);
            return -1;
        }
        X = raw;
    }
    int zc[TD_MAXD];
    int pv[TD_MAXD];
#pragma unroll
    for (int c = 0; c < TD_MAXD; ++c) {
        zc[c] = c < p ? z[c] : 0;
        pv[c] = Q.piv[c];
    }
    /* one pass in rounds of T consecutive rows (lanes on consecutive rows):
     * a ballot per warp, the warps' counts scanned, the nonzero points
     * written in data order */
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = T >> 5;
    const unsigned below = (1u << lane) - 1u;
    int base = 0;
    for (int i0 = 0; i0 < n; i0 += T) {
        const int i = i0 + (int)threadIdx.x;
        bool nz = false;
        if (i < n)
            for (int c = 0; c < p; ++c) nz |= X[(int64_t)i * p + c] != zc[c];
        const unsigned b = __ballot_sync(TD_FULL, nz);
        if (lane == 0) s_tmp[w] = __popc(b);
        __syncthreads();
        int off = base, tot = 0;
        for (int k = 0; k < nw; ++k) {
            const int v = s_tmp[k];
            off += k < w ? v : 0;
            tot += v;
        }
        if (nz) {
            const int o = off + __popc(b & below);
            const int pos = L.perm ? (int)L.perm[(size_t)q * L.perm_stride + o] : o;
            for (int c = 0; c < 2 * nplanes; ++c) {
                float v = 0.f;
                if (c < d) v = (float)((int64_t)X[(int64_t)i * p + pv[c]] - zc[pv[c]]);
                xs[td_xidx(npc, pos, c)] = v;
            }
        }
        base += tot;
        __syncthreads(); /* s_tmp is rewritten by the next round */
    }
    /* zero points up to the next multiple of 128 (the sweep loads them unmasked) */
    const int nnz = Q.nnz, npad = (nnz + TD_ROUND - 1) & ~(TD_ROUND - 1);
    for (int o2 = nnz + (int)threadIdx.x; o2 < npad; o2 += T)
        for (int c = 0; c < 2 * nplanes; ++c) xs[td_xidx(npc, o2, c)] = 0.f;
    __syncthreads();
    return Q.nnz;
}

/* The same staging by one warp into its own area (the D = 2 kernel, where a
 * query has a single subset): nonzero points compacted in data order with
 * ballots, the pivot coordinates of the query, zeros up to a multiple of
 * TD_ROUND.  Returns the number staged. */
__device__ int td_stage_points_warp(const TdLaunch &L, int q, float *xs, int npc, int lane)
{
    const TdQuery &Q = L.q[q];
    const TdSet S = L.sets[Q.set];
    const int n = S.n, p = S.p;
    const int32_t *X = L.X + S.x_off;
    const int32_t *z = L.Zq + (int64_t)q * TD_MAXD;
    const int p0 = Q.piv[0], p1 = Q.piv[1];
    const unsigned below = (1u << lane) - 1u;
    int o = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        bool nz = false;
        float v0 = 0.f, v1 = 0.f;
        if (i < n) {
            for (int c = 0; c < p; ++c) nz |= X[(int64_t)i * p + c] != z[c];
            v0 = (float)((int64_t)X[(int64_t)i * p + p0] - z[p0]);
            v1 = (float)((int64_t)X[(int64_t)i * p + p1] - z[p1]);
        }
        const unsigned b = __ballot_sync(TD_FULL, nz);
        if (nz) {
            const int pos = o + __popc(b & below);
            xs[td_xidx(npc, pos, 0)] = v0;
            xs[td_xidx(npc, pos, 1)] = v1;
        }
        o += __popc(b);
    }
    const int npad = (o + TD_ROUND - 1) & ~(TD_ROUND - 1);
    for (int j = o + lane; j < npad; j += 32) {
        xs[td_xidx(npc, j, 0)] = 0.f;
        xs[td_xidx(npc, j, 1)] = 0.f;
    }
    __syncwarp();
    return o;
}

/* ====================================================================== */
/* filtered sweep (one warp, one subset)                                   */
/* ====================================================================== */

struct TdWarpStats {
    unsigned long long sweeps, dependent, filtered, exact, tight, resolved, errors;
};

template <int D>
__device__ __forceinline__ void td_load_point(const float *xs, int npc, int i, float (&x)[D])
{
    const float *b = xs + td_xidx(npc, i, 0);
#pragma unroll
    for (int r = 0; r < D; ++r) x[r] = b[(((r >> 1) * npc) << 2) + ((r & 1) << 1)];
}

/* Bucket boundary direction D_j for B buckets (pseudo-angle key 2j/B). */
__device__ __forceinline__ void td_bucket_dir(int j, int B, int64_t &d1, int64_t &d2)
{
    if (2 * j <= B) {
        d1 = B - 2 * j;
        d2 = 2 * j;
    } else {
        d1 = B - 2 * j;
        d2 = 2 * B - 2 * j;
    }
}

/* Exact bucket of a normalised direction h, starting from the estimate b. */
__device__ __forceinline__ int td_exact_bucket(int64_t h1, int64_t h2, int b, int B)
{
    for (int it = 0; it < 2 * B && b > 0; ++it) {
        int64_t d1, d2;
        td_bucket_dir(b, B, d1, d2);
        if (td_cross_sign(d1, d2, h1, h2) >= 0) break; /* angle(h) >= angle(D_b) */
        --b;
    }
    for (int it = 0; it < 2 * B && b < B - 1; ++it) {
        int64_t d1, d2;
        td_bucket_dir(b + 1, B, d1, d2);
        if (td_cross_sign(d1, d2, h1, h2) < 0) break; /* angle(h) < angle(D_{b+1}) */
        ++b;
    }
    return b;
}

/* Histogram layout: bucket b at word b.  Lane l owns the per = B/32 buckets
 * [l*per, (l+1)*per).  The scans that run on every sweep (per-lane totals,
 * clearing) visit a lane's chunks of four in the rotated order c = (k + l)
 * mod per/4, so that the lanes of a quarter warp touch distinct bank quads;
 * only the rare in-order pass reads them in order. */
__device__ __forceinline__ int td_phys(int b, int lp, int chm)
{
    (void)lp;
    (void)chm;
    return b;
}

struct TdWarpSmem {
    uint32_t *hist;   /* B packed counters: low 16 bits +1 events, high 16 bits -1 events */
    uint16_t *bid;    /* bucket of each point (TD_SENT = tight) */
    uint16_t *glist;  /* uncertain points, then gathered items */
    int *gcount;
    int64_t *qa, *qb; /* exact basis of the current subset (qb = qa + 8) */
    int *meta;        /* rows[0..3] (intrinsic coordinates), sub[4..7] (subset point ids) */
    td_f2x *fab2;     /* basis rounded to binary32, each value twice (packed f32x2):
                         fa at [0, D), fb at [8, 8 + D) */
    int32_t *q32;     /* basis truncated to int32 (exact when narrow): qa at [0, D), qb at [8, 8 + D) */
};

/* Lane-private coarse histogram of the sweep loop: row c (c < 32 the lane
 * ranges of buckets, 32 the uncertain points) column l at word 32 c + l, so
 * the 32 lanes of one shared reduction always hit 32 different banks.  It
 * shares its storage with the fine histogram, bucket ids and lists, which
 * only the few sweeps that go past the coarse bound build. */
#define TD_COARSE_WORDS (33 * 32)
/* Rows of the two-subset sweep's coarse histograms (the table keeps its
 * 33 x 32 words).  At D >= 5 rows are short, pass 1 weighs more in every
 * sweep and the running minimum is far below almost every bound: 8 rows
 * gave W3 4.83 s (32 rows: 5.08 s, 16: 4.90 s, 4: 4.84 s) and W4 136.9 ms
 * (144.1, 137.2, 142.2) with about as many rescans.  At D = 4, 16 or 8 rows
 * made W2 0.5% slower. */
#ifndef TD_DUAL_ROWS5
#define TD_DUAL_ROWS5 8
#endif
#ifndef TD_DUAL_ROWS4
#define TD_DUAL_ROWS4 32
#endif
#define TD_DUAL_ROWS(D) ((D) >= 5 ? TD_DUAL_ROWS5 : ((D) == 4 ? TD_DUAL_ROWS4 : 32))

/* Histogram words (coarse and fine): the high half counts every event of the
 * bucket, the low half its +1 events (points of orientation -), so that a
 * point adds 0x10000 plus the sign bit of its y2.  Both halves stay below
 * 2^15 (at most nnz events), in single words and in the sums of pass 1. */
__device__ __forceinline__ int td_ev_plus(uint32_t w) { return (int)(w & 0xFFFFu); }
__device__ __forceinline__ int td_ev_minus(uint32_t w) { return (int)(w >> 16) - (int)(w & 0xFFFFu); }

/* q64 (16 int64: qa, qb) at 0, q32 (16 int) at 128, fab2 (32 packed pairs:
 * the columns of subset A at [0, 16), of subset B at [16, 32) when two
 * subsets are swept together) at 192, meta (8 int) at 448 */
#define TD_WARP_META_BYTES 480

/* Coarse histograms per warp: two for D = 3..5, whose warps sweep two
 * subsets at once (td_sweep_dual), one otherwise. */
__host__ __device__ constexpr int td_coarse_tables(int D) { return (D >= 3 && D <= 5) ? 2 : 1; }

/* A warp's shared region: the histogram storage (rbytes), gcount and the
 * basis block, rounded to 128 bytes so that every region -- and every
 * 128-byte row of a coarse histogram -- starts 128-byte aligned (the
 * staging planes before them are multiples of 1024 bytes and the dynamic
 * shared memory is declared 128-byte aligned). */
__host__ __device__ inline size_t td_warp_region_bytes(size_t rbytes)
{
    return (rbytes + 16 + TD_WARP_META_BYTES + 127) & ~(size_t)127;
}

/* the two basis columns from the warp's shared block (32-bit words: qa at
 * [0, D), qb at [8, 8 + D), 16-byte aligned) */
template <int D>
__device__ __forceinline__ void td_load_pair(const void *src, uint32_t (&a)[D], uint32_t (&b)[D])
{
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    const uint4 a4 = s4[0], b4 = s4[2];
    a[0] = a4.x;
    b[0] = b4.x;
    if (D > 1) { a[1] = a4.y; b[1] = b4.y; }
    if (D > 2) { a[2] = a4.z; b[2] = b4.z; }
    if (D > 3) { a[3] = a4.w; b[3] = b4.w; }
    if (D > 4) {
        const uint2 a2 = reinterpret_cast<const uint2 *>(src)[2], b2 = reinterpret_cast<const uint2 *>(src)[6];
        a[4] = a2.x;
        b[4] = b2.x;
        if (D > 5) { a[5] = a2.y; b[5] = b2.y; }
    }
}

/* the two binary32 basis columns as packed pairs (v, v) from the warp's
 * shared block (fa at [0, D), fb at [8, 8 + D), 16-byte aligned) */
template <int D>
__device__ __forceinline__ void td_load_coef2(const td_f2x *src, td_f2x (&A)[D], td_f2x (&Bv)[D])
{
    const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(src);
#pragma unroll
    for (int r = 0; r < D; r += 2) {
        const ulonglong2 u = s2[r >> 1], w = s2[4 + (r >> 1)];
        A[r] = u.x;
        Bv[r] = w.x;
        if (r + 1 < D) {
            A[r + 1] = u.y;
            Bv[r + 1] = w.y;
        }
    }
}

/* Exact placement of the points the FP32 filter could not certify (their ids
 * are in W.glist[0..nu)), one point per lane.  The projection is exact: in
 * int32 when the coefficient bounds A_a, A_b (sums of |q_t| max|x_t|, which
 * bound every partial sum) are below 2^31 (NARROW), else in int64.  A zero
 * projection is a tight point.  Otherwise the bucket of the exact direction
 * h is j = floor(B (s - h1) / (2 s)) with s = |h1| + h2, i.e. floor(key B/2).
 * The binary32 key is within about 11u of the exact one (conversions of h,
 * the sum, the reciprocal, the fma), far less than a bucket, so its floor j0
 * is j, j - 1 or j + 1; one exact comparison of B (s - h1) with 2 s j0 and
 * 2 s (j0 + 1) (64-bit products when NARROW, 128-bit otherwise) settles it.
 * The boundary search td_exact_bucket remains as a guard that never runs
 * while that error bound holds.  Returns the number of tight points. */
template <int D, bool NARROW>
__device__ __forceinline__ int td_exact_pass(const float *xs, int npc, const TdWarpSmem &W, int nu, int blog2,
                                             int lane)
{
    const int B = 1 << blog2;
    const float Mb = __int_as_float(0x4B400000 - ((blog2 - 1) << 23)); /* spacing 2/B, see td_sweep_filtered */
    const int Mbits = __float_as_int(Mb);
    const unsigned hq = td_saddr(W.hist);
    int t = 0;
    for (int l0 = 0; l0 < nu; l0 += 32) {
        const int l = l0 + lane;
        const bool act = l < nu;
        const unsigned i = act ? (unsigned)W.glist[l] : 0u;
        float x[D];
        td_load_point<D>(xs, npc, (int)i, x);
        bool plus, zero, ok;
        float f1, f2;
        int64_t h1, h2;
        int j;
        if constexpr (NARROW) {
            uint32_t qa32[D], qb32[D];
            td_load_pair<D>(W.q32, qa32, qb32);
            int32_t a = 0, b = 0;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                const int32_t xv = td_f2i(x[r]);
                a += (int32_t)qa32[r] * xv;
                b += (int32_t)qb32[r] * xv;
            }
            zero = (a | b) == 0;
            plus = (b > 0) || (b == 0 && a > 0);
            const int32_t g1 = plus ? a : -a, g2 = plus ? b : -b;
            f1 = __int2float_rn(g1);
            f2 = __int2float_rn(g2);
            const float kb = fmaf(-f1, td_rcp(fabsf(f1) + f2), 1.0f);
            j = min(max(__float_as_int(__fadd_rd(kb, Mb)) - Mbits, 0), B - 1);
            /* s < 2^32, s - h1 < 2^33: num < 2^44, den * (j + 1) < 2^45 */
            const int64_t s = (int64_t)(g1 < 0 ? -g1 : g1) + g2;
            const int64_t num = (s - g1) << blog2, den = 2 * s;
            int64_t lo = den * j;
            if (num < lo) {
                --j;
                lo -= den;
            } else if (num >= lo + den) {
                ++j;
                lo += den;
            }
            ok = zero || (lo <= num && num < lo + den);
            h1 = g1;
            h2 = g2;
        } else {
            int64_t Y1 = 0, Y2 = 0;
#pragma unroll
            for (int r = 0; r < D; ++r) {
                const int64_t xv = td_f2i(x[r]);
                Y1 += W.qa[r] * xv;
                Y2 += W.qb[r] * xv;
            }
            zero = (Y1 | Y2) == 0;
            plus = td_normalise(Y1, Y2, h1, h2);
            f1 = td_i64_to_f32(h1);
            f2 = td_i64_to_f32(h2);
            const float kb = fmaf(-f1, td_rcp(fabsf(f1) + f2), 1.0f);
            j = min(max(__float_as_int(__fadd_rd(kb, Mb)) - Mbits, 0), B - 1);
            /* |h| < 2^62: exact in 128 bits */
            const td_i128 s = (td_i128)(h1 < 0 ? -h1 : h1) + h2;
            const td_i128 num = (s - h1) << blog2, den = 2 * s;
            td_i128 lo = den * j;
            if (num < lo) {
                --j;
                lo -= den;
            } else if (num >= lo + den) {
                ++j;
                lo += den;
            }
            ok = zero || (lo <= num && num < lo + den);
        }
        const bool need = act & !ok;
        if (__any_sync(TD_FULL, need)) {
            if (need) j = td_exact_bucket(h1, h2, max(0, min(j, B - 1)), B);
        }
        if (act) {
            W.bid[i] = (uint16_t)(zero ? TD_SENT : (unsigned)j);
            if (!zero) td_reds_add(hq + 4u * (unsigned)j, plus ? 0x10000u : 0x10001u);
            t += zero;
        }
    }
    return td_wsum(t);
}

/* exact normalised projection of point i from the published basis */
template <int D>
__device__ __forceinline__ void td_exact_h(const float *xs, int npc, int i, const int64_t *qa, const int64_t *qb,
                                           int64_t &h1, int64_t &h2, bool &plus)
{
    float xp[D];
    td_load_point<D>(xs, npc, i, xp);
    int64_t Y1 = 0, Y2 = 0;
#pragma unroll
    for (int r = 0; r < D; ++r) {
        const int64_t xv = td_f2i(xp[r]);
        Y1 += qa[r] * xv;
        Y2 += qb[r] * xv;
    }
    plus = td_normalise(Y1, Y2, h1, h2);
}

/* The row pair (pi, pj) of lane l < C(D,2) in lexicographic order, and the
 * other K rows of its minor, as their offsets lr[] in the staged layout (the
 * point part of td_xidx added per point); lanes past C(D,2) get pair (0, 1). */
template <int D>
__device__ __forceinline__ void td_lane_pair(int lane, int npc, int &pi, int &pj, int (&lr)[D > 2 ? D - 2 : 1])
{
    constexpr int NP = D * (D - 1) / 2;
    pi = 0;
    pj = 1;
    int l = lane < NP ? lane : 0;
#pragma unroll
    for (int aa = 0; aa < D - 1; ++aa) {
        const int cnt = D - 1 - aa;
        if (l >= 0 && l < cnt) {
            pi = aa;
            pj = aa + 1 + l;
        }
        l -= cnt;
    }
    lr[0] = 0;
#pragma unroll
    for (int i = 0; i < D - 2; ++i) {
        int r = i;
        r += (r >= pi);
        r += (r >= pj);
        lr[i] = td_xidx(npc, 0, r); /* the point part of td_xidx is zero for point 0 */
    }
}

/* Cofactors of column 0 of a K x K matrix (column 0 unused):
 * cof[i] = (-1)^i det(m without row i and column 0), so that
 * det(m) = sum_i m[i][0] cof[i]. */
template <int K, typename T>
__device__ __forceinline__ void td_cofactors0(const T (&m)[K > 0 ? K : 1][K > 0 ? K : 1], T (&cof)[K > 0 ? K : 1])
{
    if constexpr (K <= 1) {
        cof[0] = 1;
    } else {
        constexpr int J = K - 1;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            T s[J][J];
#pragma unroll
            for (int a = 0; a < J; ++a)
#pragma unroll
                for (int b = 0; b < J; ++b) s[a][b] = m[a + (a >= i)][b + 1];
            T d;
            if constexpr (std::is_same<T, int32_t>::value) d = td_detk32<J>(s);
            else d = td_detk<J>(s);
            cof[i] = (i & 1) ? -d : d;
        }
    }
}

/* Cooperative subset basis.  Lane l < C(D,2) computes the Plucker
 * coordinate P of the l-th row pair (i, j) in lexicographic order: the
 * entries Q_ij = P, Q_ji = -P of the antisymmetric integer matrix whose
 * columns are functionals vanishing on span S.  The warp picks a pair (a, b)
 * with P_ab != 0 and |P_ab| largest up to binary32 rounding (one
 * max-reduction of a 32-bit key; any nonzero P_ab gives a valid basis).
 * Every sweep needs only the two columns a and b rounded to binary32
 * (td_basis_publish); the few sweeps that place points exactly also need
 * them exact, truncated to int32, and the subset's intrinsic rows and point
 * ids (td_basis_publish_exact, which repeats the pick from the cached
 * cofactors and so chooses the same pair). */

/* This lane's Plucker coordinate P (0 for lanes past C(D,2)).  lr[i]: this
 * lane's i-th row of its minor, as the offset of that coordinate within a
 * point's slots (td_xidx less the point part).  The minor is expanded along
 * column 0 (point c[0], the one the colex successor changes most often):
 * the cofactors cof[] of the other columns are recomputed only when refresh
 * is set (c[1..K) changed).  NM: the arithmetic is int32 (the caller has
 * checked K! max|x|^K < 2^31, which bounds every intermediate), else int64. */
template <int D, bool NM>
__device__ __forceinline__ int64_t td_basis_minor(const float *xs, const int (&c)[D > 2 ? D - 2 : 1], int lane,
                                                  int pi, int pj, const int (&lr)[D > 2 ? D - 2 : 1],
                                                  int64_t (&cof)[D > 2 ? D - 2 : 1], bool refresh)
{
    constexpr int K = D - 2;
    constexpr int NP = D * (D - 1) / 2;
    using T = typename std::conditional<NM, int32_t, int64_t>::type;
    if (refresh) {
        T m[K > 0 ? K : 1][K > 0 ? K : 1];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            m[i][0] = 0;
#pragma unroll
            for (int j = 1; j < K; ++j) m[i][j] = td_f2i(xs[lr[i] + ((td_pair_of(c[j]) << 2) | ((c[j] >> 5) & 1))]);
        }
        T cf[K > 0 ? K : 1];
        td_cofactors0<K, T>(m, cf);
#pragma unroll
        for (int i = 0; i < (K > 0 ? K : 1); ++i) cof[i] = cf[i];
    }
    T M = (K > 0) ? 0 : 1;
#pragma unroll
    for (int i = 0; i < K; ++i)
        M += (T)td_f2i(xs[lr[i] + ((td_pair_of(c[0]) << 2) | ((c[0] >> 5) & 1))]) * (T)cof[i];
    int64_t P = ((pi + pj) & 1) ? (int64_t)M : -(int64_t)M; /* -(-1)^(i+j) M */
    return lane < NP ? P : 0;
}

/* The pick: the lane holding the chosen pair, or -1 (uniformly) when every
 * P vanishes (rank < K). */
template <bool NM>
__device__ __forceinline__ int td_basis_pick(int64_t P, int lane)
{
    uint32_t key;
    if constexpr (NM) {
        const int32_t P32 = (int32_t)P;
        key = P32 != 0 ? ((__float_as_uint(__int2float_rn(P32 < 0 ? -P32 : P32)) & ~31u) | (uint32_t)(31 - lane)) : 0u;
    } else {
        key = P != 0 ? ((__float_as_uint(fabsf(td_i64_to_f32_bf(P))) & ~31u) | (uint32_t)(31 - lane)) : 0u;
    }
    const uint32_t kmax = __reduce_max_sync(TD_FULL, key);
    return kmax == 0u ? -1 : 31 - (int)(kmax & 31u);
}

/* Entry t = e % 8 of column a (e < 8) or b (8 <= e < 16) of lane e:
 * Q_t,col = +-P of the pair (min, max), 0 for t == col, fetched with one
 * shuffle; also returns a and b. */
template <int D, bool NM>
__device__ __forceinline__ int64_t td_basis_entry(int64_t P, int wl, int lane, int pi, int pj, int &a, int &b)
{
    a = __shfl_sync(TD_FULL, pi, wl);
    b = __shfl_sync(TD_FULL, pj, wl);
    const int e = lane & 15, t = e & 7, col = (e >> 3) ? b : a;
    const int x = min(t, col), y = max(t, col);
    const int src = x * (2 * D - x - 1) / 2 + (y - x - 1);
    int64_t Pv;
    if constexpr (NM)
        Pv = __shfl_sync(TD_FULL, (int32_t)P, t == col ? 0 : src);
    else
        Pv = __shfl_sync(TD_FULL, P, t == col ? 0 : src);
    return t == col ? 0 : (t < col ? Pv : -Pv);
}

/* Every sweep: the two basis columns rounded to binary32, each value twice
 * (packed pairs), to the warp's shared block.  Returns false (uniformly)
 * when the subset is dependent. */
template <int D, bool NM>
__device__ __forceinline__ bool td_basis_publish(const float *xs, const int (&c)[D > 2 ? D - 2 : 1], int lane,
                                                 int pi, int pj, const int (&lr)[D > 2 ? D - 2 : 1],
                                                 const TdWarpSmem &W, int64_t (&cof)[D > 2 ? D - 2 : 1],
                                                 bool refresh)
{
    const int64_t P = td_basis_minor<D, NM>(xs, c, lane, pi, pj, lr, cof, refresh);
    const int wl = td_basis_pick<NM>(P, lane);
    if (wl < 0) return false;
    int a, b;
    const int64_t v = td_basis_entry<D, NM>(P, wl, lane, pi, pj, a, b);
    __syncwarp();
    const int e = lane & 15;
    if (lane < 16 && (e & 7) < D) {
        const float f = NM ? __int2float_rn((int32_t)v) : td_i64_to_f32_bf(v);
        W.fab2[e] = td_pk(f, f);
    }
    __syncwarp();
    return true;
}

/* The sweeps that go past the coarse bound: the same two columns exact
 * (int64) and truncated to int32, the subset's intrinsic rows (the rows
 * other than a and b) and point ids, to the warp's shared block. */
template <int D, bool NM>
__device__ __forceinline__ void td_basis_publish_exact(const float *xs, const int (&c)[D > 2 ? D - 2 : 1], int lane,
                                                    int pi, int pj, const int (&lr)[D > 2 ? D - 2 : 1],
                                                    const TdWarpSmem &W, int64_t (&cof)[D > 2 ? D - 2 : 1])
{
    constexpr int K = D - 2;
    const int64_t P = td_basis_minor<D, NM>(xs, c, lane, pi, pj, lr, cof, false);
    const int wl = td_basis_pick<NM>(P, lane); /* >= 0: the sweep found the subset independent */
    int a, b;
    const int64_t v = td_basis_entry<D, NM>(P, wl, lane, pi, pj, a, b);
    __syncwarp();
    const int e = lane & 15;
    if (lane < 16 && (e & 7) < D) {
        W.qa[e] = v;
        W.q32[e] = (int32_t)v;
    }
#pragma unroll
    for (int r = 0; r < K; ++r) {
        int rr = r;
        rr += (rr >= a);
        rr += (rr >= b);
        if (lane == 0) {
            W.meta[r] = rr;
            W.meta[4 + r] = c[r];
        }
    }
    __syncwarp();
}

/* Two subsets at once (td_sweep_dual): lanes 0-15 compute the Plucker
 * coordinates of subset A (lane pair e = lane, cH = its points), lanes
 * 16-31 those of subset B (pair e = lane - 16); each half picks its own pair
 * (a, b) as td_basis_pick does, and lane l writes entry l & 15 of the binary32
 * columns of its half's subset to W.fab2[l] (A at [0, 16), B at [16, 32)).
 * The error bound of each subset's projection is formed in the lanes: lane l
 * holds |q_t| max|x_t| for its entry t = l % 8 (mx_lane = max|x_t|, 0 for
 * t >= D), the eight lanes of a column sum them, and E_h = cst * the larger
 * column sum of half h -- the binary32 sum is within (D + 2) u of the exact
 * one in any order, as the bound assumes.  Returns bit 0 when A is
 * dependent, bit 1 when B is.  pi, pj, lr, cof: this lane's pair e. */
template <int D, bool NM>
__device__ __forceinline__ int td_basis_publish_dual(const float *xs, const int (&cH)[D > 2 ? D - 2 : 1], int lane,
                                                     int pi, int pj, const int (&lr)[D > 2 ? D - 2 : 1],
                                                     const TdWarpSmem &W, int64_t (&cof)[D > 2 ? D - 2 : 1],
                                                     bool refresh, float mx_lane, float cst, float &EA, float &EB,
                                                     bool &narrowA, bool &narrowB)
{
    const int e = lane & 15, half = lane & 16;
    const int64_t P = td_basis_minor<D, NM>(xs, cH, e, pi, pj, lr, cof, refresh);
    uint32_t key;
    if constexpr (NM) {
        const int32_t P32 = (int32_t)P;
        key = P32 != 0 ? ((__float_as_uint(__int2float_rn(P32 < 0 ? -P32 : P32)) & ~31u) | (uint32_t)(31 - lane)) : 0u;
    } else {
        key = P != 0 ? ((__float_as_uint(fabsf(td_i64_to_f32_bf(P))) & ~31u) | (uint32_t)(31 - lane)) : 0u;
    }
    const uint32_t kA = __reduce_max_sync(TD_FULL, half ? 0u : key);
    const uint32_t kB = __reduce_max_sync(TD_FULL, half ? key : 0u);
    const int dep = (kA == 0u ? 1 : 0) | (kB == 0u ? 2 : 0);
    const uint32_t kh = half ? kB : kA;
    const int wl = 31 - (int)(kh & 31u); /* a lane of this half (its pair wins) */
    const int a = __shfl_sync(TD_FULL, pi, wl), b = __shfl_sync(TD_FULL, pj, wl);
    const int t = e & 7, col = (e >> 3) ? b : a;
    const int x = min(t, col), y = max(t, col);
    const int src = half + x * (2 * D - x - 1) / 2 + (y - x - 1);
    int64_t Pv;
    if constexpr (NM)
        Pv = __shfl_sync(TD_FULL, (int32_t)P, t == col ? half : src);
    else
        Pv = __shfl_sync(TD_FULL, P, t == col ? half : src);
    const int64_t v = t == col ? 0 : (t < col ? Pv : -Pv);
    const float f = NM ? __int2float_rn((int32_t)v) : td_i64_to_f32_bf(v);
    float sum = fabsf(f) * mx_lane; /* 0 for t >= D (mx_lane = 0, f finite) */
    sum += __shfl_xor_sync(TD_FULL, sum, 4);
    sum += __shfl_xor_sync(TD_FULL, sum, 2);
    sum += __shfl_xor_sync(TD_FULL, sum, 1);
    const float A0 = fmaxf(__shfl_sync(TD_FULL, sum, 0), __shfl_sync(TD_FULL, sum, 8));
    const float A1 = fmaxf(__shfl_sync(TD_FULL, sum, 16), __shfl_sync(TD_FULL, sum, 24));
    EA = A0 * cst;
    EB = A1 * cst;
    narrowA = A0 < 2145386496.0f; /* 2^31 (1 - 2^-10): exact bounds below 2^31 */
    narrowB = A1 < 2145386496.0f;
    __syncwarp();
    if (t < D) W.fab2[lane] = td_pk(f, f);
    __syncwarp();
    return dep;
}

/* Publish the exact basis and the subset to the warp's shared area. */
template <int D>
__device__ __forceinline__ void td_publish_basis(const TdBasis<D> &Bs, const int (&c)[D > 2 ? D - 2 : 1],
                                                 int64_t *qa, int64_t *qb, int *meta, int lane)
{
    constexpr int K = D - 2;
#pragma unroll
    for (int r = 0; r < D; ++r) {
        if (lane == r) qa[r] = Bs.qa[r];
        if (lane == 8 + r) qb[r] = Bs.qb[r];
    }
#pragma unroll
    for (int r = 0; r < K; ++r) {
        if (lane == 16 + r) meta[r] = Bs.rows[r];
        if (lane == 20 + r) meta[4 + r] = c[r];
    }
    __syncwarp();
}

/* Resolution of more than 32 gathered events: exact sort of the list in
 * shared memory by (bucket, direction) and a sequential walk by lane 0. */
template <int D>
__device__ __noinline__ void td_resolve_many(const float *xs, int PS, const int64_t *qa, const int64_t *qb,
                                             const uint32_t *hist, const uint16_t *bid, uint16_t *glist,
                                             int G, int lp, int chm, int lane, int *mn_io, int *mx_io)
{
    int npad = td_pow2_at_least(G);
    for (int l = G + lane; l < npad; l += 32) glist[l] = (uint16_t)TD_SENT;
    __syncwarp();
    for (int size = 2; size <= npad; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int tt = lane; tt < (npad >> 1); tt += 32) {
                int i = ((tt & ~(stride - 1)) << 1) | (tt & (stride - 1));
                int j = i + stride;
                bool up = (i & size) == 0;
                uint16_t u = glist[i], v = glist[j];
                /* (bucket, exact direction) order */
                auto less = [&](uint16_t x, uint16_t y) -> bool {
                    if (x == TD_SENT) return false;
                    if (y == TD_SENT) return true;
                    int bx = bid[x], by = bid[y];
                    if (bx != by) return bx < by;
                    int64_t x1, x2, y1, y2;
                    bool px, py;
                    td_exact_h<D>(xs, PS, x, qa, qb, x1, x2, px);
                    td_exact_h<D>(xs, PS, y, qa, qb, y1, y2, py);
                    return td_cross_sign(x1, x2, y1, y2) > 0;
                };
                bool sw = up ? less(v, u) : less(u, v);
                if (sw) {
                    glist[i] = v;
                    glist[j] = u;
                }
            }
            __syncwarp();
        }
    int lmn = INT_MAX, lmx = INT_MIN;
    if (lane == 0) {
        int j = 0;
        while (j < G) {
            int bk = bid[glist[j]];
            int v = (int)(hist[td_phys(bk, lp, chm)] & 0xFFFFu);
            while (j < G && bid[glist[j]] == bk) {
                int64_t g1, g2;
                bool gp;
                td_exact_h<D>(xs, PS, glist[j], qa, qb, g1, g2, gp);
                while (j < G && bid[glist[j]] == bk) {
                    int64_t c1, c2;
                    bool plus;
                    td_exact_h<D>(xs, PS, glist[j], qa, qb, c1, c2, plus);
                    if (td_cross_sign(g1, g2, c1, c2) != 0) break;
                    v += plus ? -1 : 1;
                    ++j;
                }
                lmn = min(lmn, v);
                lmx = max(lmx, v);
            }
        }
    }
    lmn = __shfl_sync(TD_FULL, lmn, 0);
    lmx = __shfl_sync(TD_FULL, lmx, 0);
    *mn_io = min(*mn_io, lmn);
    *mx_io = max(*mx_io, lmx);
}

/* Per-sweep constants of the FP32 bucket test, packed for f32x2. */
template <int D>
struct TdPairCoef {
    td_f2x fa[D], fb[D]; /* (fa_r, fa_r), (fb_r, fb_r) */
    td_f2x cE, cU;       /* (2E, 2E), (24u, 24u) */
    td_f2x nMb, m1;      /* (-Mb, -Mb), (-1, -1) */
    uint32_t moff;       /* 2^31 - bits(Mb) */
    int B;
    td_f2x nMc;          /* (-Mc, -Mc), Mc = 1.5 * 2^19: binary32 spacing 1/16 */
    uint32_t moffc;      /* 2^31 - bits(Mc) */
};

template <int D>
__device__ __forceinline__ TdPairCoef<D> td_pair_coef(const td_f2x (&FA)[D], const td_f2x (&FB)[D], float E, int blog2)
{
    TdPairCoef<D> C;
#pragma unroll
    for (int r = 0; r < D; ++r) {
        C.fa[r] = FA[r];
        C.fb[r] = FB[r];
    }
    const float cE = 2.0f * E, cU = 24.0f * TD_U;
    /* Mb = 1.5 * 2^23 / (B/2): binary32 spacing 2/B in its binade */
    const float Mb = __int_as_float(0x4B400000 - ((blog2 - 1) << 23));
    C.cE = td_pk(cE, cE);
    C.cU = td_pk(cU, cU);
    C.nMb = td_pk(-Mb, -Mb);
    C.m1 = td_pk(-1.0f, -1.0f);
    C.moff = 0x80000000u - (uint32_t)__float_as_int(Mb);
    C.B = 1 << blog2;
    const float Mc = 786432.0f;
    C.nMc = td_pk(-Mc, -Mc);
    C.moffc = 0x80000000u - (uint32_t)__float_as_int(Mc);
    return C;
}

/* The FP32 buckets of the two points of one staged pair (planes pl[]), see
 * the certification argument below: floor(key B/2) when the interval
 * key +- delta lies in one bucket, else B (uncertain).  inc is the packed
 * event of the point: 0x10001 (+1 event, orientation -) or 0x10000 (-1 event,
 * orientation +).
 *
 * The key is carried negated, kn = y1 rr - 1 = -key with rr = sign(y2) /
 * (|y1| + |y2|), so that every step is one packed f32x2 operation for both
 * points: the floors are round_up(kn -+ delta - Mb) = -round_down(key +- delta
 * + Mb), since rounding to nearest is odd-symmetric and rounding up is
 * rounding down mirrored.  The bucket is then bits(.) + 2^31 - bits(Mb) (the
 * sign flip adds 2^31 to the bit pattern) and the two floors agree iff
 * their bit patterns do.  The sweep loop and td_rescan both use this
 * function, so they take the same decisions. */
template <int D>
__device__ __forceinline__ void td_pair_slots(const float4 (&pl)[(D + 1) / 2], const TdPairCoef<D> &C, int &sp,
                                              int &sq, uint32_t &ip, uint32_t &iq)
{
    td_f2x X[D];
#pragma unroll
    for (int c = 0; c < (D + 1) / 2; ++c) {
        X[2 * c] = td_pk(pl[c].x, pl[c].y);
        if (2 * c + 1 < D) X[2 * c + 1] = td_pk(pl[c].z, pl[c].w);
    }
    td_f2x Y1 = td_mul2(C.fa[0], X[0]), Y2 = td_mul2(C.fb[0], X[0]);
#pragma unroll
    for (int r = 1; r < D; ++r) {
        Y1 = td_fma2(C.fa[r], X[r], Y1);
        Y2 = td_fma2(C.fb[r], X[r], Y2);
    }
    float y1p, y1q, y2p, y2q;
    td_upk(Y1, y1p, y1q);
    td_upk(Y2, y2p, y2q);
    const float rap = td_rcp(__fadd_rn(fabsf(y1p), fabsf(y2p)));
    const float raq = td_rcp(__fadd_rn(fabsf(y1q), fabsf(y2q)));
    const td_f2x RA = td_pk(rap, raq);
    const td_f2x RR = td_pk(copysignf(rap, y2p), copysignf(raq, y2q));
    const td_f2x KN = td_fma2(Y1, RR, C.m1);  /* -key */
    const td_f2x DB = td_fma2(C.cE, RA, C.cU); /* delta */
    /* When |y1|+|y2| <= 4E the interval is at least 1/2 wide, or outside the
     * conversion window, or NaN: it never yields one in-range bucket, so no
     * separate test. */
    const td_f2x FL = td_add2_rp(td_add2(KN, DB), C.nMb); /* -floor((key - delta) B/2) */
    const td_f2x FH = td_add2_rp(td_sub2(KN, DB), C.nMb); /* -floor((key + delta) B/2) */
    float flp, flq, fhp, fhq;
    td_upk(FL, flp, flq);
    td_upk(FH, fhp, fhq);
    const uint32_t blp = (uint32_t)__float_as_int(flp) + C.moff, blq = (uint32_t)__float_as_int(flq) + C.moff;
    sp = ((__float_as_int(flp) == __float_as_int(fhp)) & (blp < (uint32_t)C.B)) ? (int)blp : C.B;
    sq = ((__float_as_int(flq) == __float_as_int(fhq)) & (blq < (uint32_t)C.B)) ? (int)blq : C.B;
    ip = 0x10000u + ((uint32_t)__float_as_int(y2p) >> 31);
    iq = 0x10000u + ((uint32_t)__float_as_int(y2q) >> 31);
}

/* The coarse rows of the two points of one staged pair: floor(key * 16), the
 * lane range of buckets the point's event falls in (row j holds buckets
 * [j B/32, (j + 1) B/32)), when the interval key +- delta lies in one row,
 * else 32 (uncertain at this level).  The same computation as
 * td_pair_slots with the magic constant of spacing 1/16, so the same
 * certification argument holds with 32 buckets. */
template <int D, int ROWS = 32>
__device__ __forceinline__ void td_pair_rows(const float4 (&pl)[(D + 1) / 2], const TdPairCoef<D> &C, int &rp,
                                             int &rq, uint32_t &ip, uint32_t &iq)
{
    td_f2x X[D];
#pragma unroll
    for (int c = 0; c < (D + 1) / 2; ++c) {
        X[2 * c] = td_pk(pl[c].x, pl[c].y);
        if (2 * c + 1 < D) X[2 * c + 1] = td_pk(pl[c].z, pl[c].w);
    }
    td_f2x Y1 = td_mul2(C.fa[0], X[0]), Y2 = td_mul2(C.fb[0], X[0]);
#pragma unroll
    for (int r = 1; r < D; ++r) {
        Y1 = td_fma2(C.fa[r], X[r], Y1);
        Y2 = td_fma2(C.fb[r], X[r], Y2);
    }
    float y1p, y1q, y2p, y2q;
    td_upk(Y1, y1p, y1q);
    td_upk(Y2, y2p, y2q);
    const float rap = td_rcp(__fadd_rn(fabsf(y1p), fabsf(y2p)));
    const float raq = td_rcp(__fadd_rn(fabsf(y1q), fabsf(y2q)));
    const td_f2x RA = td_pk(rap, raq);
    const td_f2x RR = td_pk(copysignf(rap, y2p), copysignf(raq, y2q));
    const td_f2x KN = td_fma2(Y1, RR, C.m1);  /* -key */
    const td_f2x DB = td_fma2(C.cE, RA, C.cU); /* delta */
    /* 32 rows: Mc = 1.5 * 2^19 (spacing 1/16, from C); ROWS = 16, 8 or 4
     * rows: Mc = 1.5 * 2^20, 2^21 or 2^22 (spacing 2/ROWS), floor(key ROWS/2) */
    constexpr int EMC = ROWS == 32 ? 19 : (ROWS == 16 ? 20 : (ROWS == 8 ? 21 : 22));
    static_assert(ROWS == 32 || ROWS == 16 || ROWS == 8 || ROWS == 4, "coarse rows: 32, 16, 8 or 4");
    constexpr uint32_t moffr = 0x80000000u - ((((uint32_t)(127 + EMC)) << 23) | 0x400000u);
    const td_f2x nMr = ROWS == 32 ? C.nMc : td_pk(-1.5f * (float)(1 << EMC), -1.5f * (float)(1 << EMC));
    const uint32_t moff = ROWS == 32 ? C.moffc : moffr;
    const td_f2x FL = td_add2_rp(td_add2(KN, DB), nMr); /* -floor((key - delta) ROWS/2) */
    const td_f2x FH = td_add2_rp(td_sub2(KN, DB), nMr); /* -floor((key + delta) ROWS/2) */
    float flp, flq, fhp, fhq;
    td_upk(FL, flp, flq);
    td_upk(FH, fhp, fhq);
    /* row = bits + 2^31 - bits(Mc), capped at ROWS: one fused add-and-min */
    const uint32_t blp = __viaddmin_u32((uint32_t)__float_as_int(flp), moff, (uint32_t)ROWS);
    const uint32_t blq = __viaddmin_u32((uint32_t)__float_as_int(flq), moff, (uint32_t)ROWS);
    rp = __float_as_int(flp) == __float_as_int(fhp) ? (int)blp : ROWS;
    rq = __float_as_int(flq) == __float_as_int(fhq) ? (int)blq : ROWS;
    ip = 0x10000u + ((uint32_t)__float_as_int(y2p) >> 31);
    iq = 0x10000u + ((uint32_t)__float_as_int(y2q) >> 31);
}

/* Rescan of a sweep's points, for the few sweeps whose bound over the
 * certified points does not reach best: builds the fine histogram of the
 * certified points' events (W.hist, zero on entry) and their bucket ids
 * (the sweep loop keeps only the coarse histogram) and lists the uncertain
 * points in W.glist (the sweep loop only counts them).  The constants are
 * rebuilt from the sweep loop's inputs (the published binary32 basis, E and
 * the bucket count) and td_pair_slots takes the same decisions.  Returns the
 * number of uncertain points listed. */
template <int D>
__device__ __noinline__ int td_rescan(const float *xs, int npc, int nnz, const TdWarpSmem &W, float E, int blog2,
                                      int lane)
{
    constexpr int NPL = (D + 1) / 2;
    td_f2x FA[D], FB[D];
    td_load_coef2<D>(W.fab2, FA, FB);
    const TdPairCoef<D> C = td_pair_coef<D>(FA, FB, E, blog2);
    const int npairs = ((nnz + TD_ROUND - 1) & ~(TD_ROUND - 1)) >> 1; /* a multiple of 32 */
    const unsigned below = (1u << lane) - 1u;
    const float4 *x4 = reinterpret_cast<const float4 *>(xs);
    const unsigned hq = td_saddr(W.hist);
    int cnt = 0;
    for (int j0 = 0; j0 < npairs; j0 += 32) {
        const int j = j0 + lane;
        float4 pl[NPL];
#pragma unroll
        for (int c = 0; c < NPL; ++c) pl[c] = x4[c * npc + j];
        int sp, sq;
        uint32_t ip, iq;
        td_pair_slots<D>(pl, C, sp, sq, ip, iq);
        const int p = ((j >> 5) << 6) | (j & 31), q = p + 32;
        const bool vp = p < nnz, vq = q < nnz;
        if (vp && sp < C.B) {
            W.bid[p] = (uint16_t)sp;
            td_reds_add(hq + 4u * (unsigned)sp, ip);
        }
        if (vq && sq < C.B) {
            W.bid[q] = (uint16_t)sq;
            td_reds_add(hq + 4u * (unsigned)sq, iq);
        }
        const bool up = vp && sp == C.B, uq = vq && sq == C.B;
        const unsigned bp = __ballot_sync(TD_FULL, up), bq = __ballot_sync(TD_FULL, uq);
        if (up) W.glist[cnt + __popc(bp & below)] = (uint16_t)p;
        cnt += __popc(bp);
        if (uq) W.glist[cnt + __popc(bq & below)] = (uint16_t)q;
        cnt += __popc(bq);
    }
    __syncwarp();
    return cnt;
}

/* G(S) for one subset, FP32-filtered (the basis must be published to
 * W.qa/W.qb first).  Returns G(S) exactly whenever G(S) < best; otherwise it
 * may return any value >= best (the subset cannot lower the minimum, so the
 * exact in-bucket order is not resolved).  Also returns the number t of tight
 * points (nonzero points of span S) and the number of nonzero projections.
 *
 * FP32 certification of a point's bucket: with E >= |y_f - y| (both
 * coordinates), for s = |y1_f|+|y2_f| > 4E and a correct orientation the
 * pseudo-angle key = 1 - h1/(|h1|+h2) of the exact point differs from the
 * computed one by at most E/(s-2E) <= 2E/s (the key is 1/s-Lipschitz in the
 * max norm of its argument) plus at most ~10 rounding errors of values <= 2
 * (reciprocal within 2 ulp, products, sums, the +-delta below); delta =
 * 2E/s + 24u covers both.  The bucket floor(key * B/2) is certain when
 * floor((key - delta) B/2) == floor((key + delta) B/2) and lies in [0, B).
 * That test also fixes the orientation: it can be wrong only when
 * |y2_f| <= E, and then the computed key lies within E/s (plus rounding) of
 * 0 or of 2, so key - delta < 0 or key + delta > 2 and the two floors differ
 * (for y1_f = 0 the interval is wider than B; s = 0 gives NaN or an
 * infinite key, which fails the range test). */
/* The coarse histogram is cumulative: the sweep loop adds to it and pass 1
 * reads each row's total and subtracts the total it read at the previous
 * sweep (prev_row, prev_u, kept per lane), instead of clearing the table.
 * A counter word is the integer sum of its packed increments modulo 2^32,
 * and one sweep adds less than 2^31 to a row, so the difference is this
 * sweep's packed count exactly.  clean: the table and the prev_* registers
 * agree (false after a sweep that built its fine histogram in the same
 * storage, and at the start of a tile: the table is then cleared and the
 * prev_* registers reset).  publish_exact() writes the exact basis and the
 * subset's rows and ids before the first exact step of a sweep. */
template <int D, typename PUB>
__device__ __forceinline__ int td_sweep_filtered(const float *xs, int npc, int nnz,
                                                 const td_f2x (&FA)[D], const td_f2x (&FB)[D], float Ea, float Eb,
                                                 bool narrow, const TdWarpSmem &W, int blog2, int lane, int best,
                                                 bool &clean, uint32_t &prev_row, uint32_t &prev_u,
                                                 uint64_t &n_exact, uint32_t &n_resolved, uint32_t &n_rescanned,
                                                 int &t_out,
                                                 int &nzy_out, PUB &&publish_exact)
{
    constexpr int NPL = (D + 1) / 2;        /* planes of the pair layout */
    const int B = 1 << blog2;               /* blog2 >= 7: at least 4 buckets per lane */
    const int lp = blog2 - 5;               /* log2 buckets per lane */
    const int nch = 1 << (lp - 2);          /* chunks of four per lane */
    const int chm = nch - 1;
    /* Bucket floors by the magic-constant addition on the unscaled key: in
     * the binade of Mb = 1.5 * 2^23 / (B/2) the spacing of binary32 is 2/B,
     * so bits(round_down(v + Mb)) - bits(Mb) = floor(v B/2) for v in
     * (-Mb/3, 2 Mb/3).  This is the scaled-by-(B/2) computation with every
     * rounding scaled by the same power of two. */
    const TdPairCoef<D> C = td_pair_coef<D>(FA, FB, fmaxf(Ea, Eb), blog2);
    const unsigned below = (1u << lane) - 1u;
    const unsigned xq = td_saddr(xs) + 16u * (unsigned)lane; /* this lane's pair in the first block */
    const unsigned pstride = 16u * (unsigned)npc;            /* bytes between planes */
    const unsigned cq = td_saddr(W.hist) + 4u * (unsigned)lane; /* this lane's coarse column */
    /* One round places TD_ROUND points, UNR/2 staged pairs per lane: pair
     * i0/2 + 32 h + l holds points i0 + 64 h + l and i0 + 64 h + 32 + l.
     * Each event goes to the lane's column of the coarse histogram, row
     * floor(key * 16) = bucket / (B/32), certified at that level; a point
     * whose row is not certified goes to row 32, whose packed count is then
     * the number of uncertain points plus the number of padding points of
     * the last round (zeros, which project to 0 and so have a NaN key and
     * fail the test).  Neither the fine buckets nor the uncertain points are
     * recorded here: the few sweeps that need them rescan (td_rescan), with
     * the fine test. */
    constexpr int UNR = TD_ROUND / 32;
    constexpr int NPR = UNR / 2; /* pairs per lane and round */
    constexpr bool HALF_TAIL = D >= 5;
    /* the coarse histogram carries the previous sweeps' counts (clean),
     * unless a sweep went past the coarse bound and built its fine
     * histogram in the same storage.  At D = 6 the flag costs spills, and
     * every sweep clears. */
    constexpr bool KEEP_CLEAN = D <= 5;
    if (!clean) {
        uint4 *z4 = reinterpret_cast<uint4 *>(W.hist);
        for (int j = lane; j < (TD_COARSE_WORDS >> 2); j += 32) z4[j] = make_uint4(0u, 0u, 0u, 0u);
        prev_row = 0u;
        prev_u = 0u;
    }
    __syncwarp();
    auto round_full = [&](int i0) {
        int slot[UNR];
        uint32_t inc[UNR];
        float4 pl[NPR][NPL];
        /* all loads of the round first (the accesses keep program order) */
        const unsigned ba = xq + 8u * (unsigned)i0; /* pair i0/2 + l */
#pragma unroll
        for (int h = 0; h < NPR; ++h)
#pragma unroll
            for (int c = 0; c < NPL; ++c) pl[h][c] = td_lds128(ba + 512u * h + c * pstride);
#pragma unroll
        for (int h = 0; h < NPR; ++h) td_pair_rows<D>(pl[h], C, slot[2 * h], slot[2 * h + 1], inc[2 * h], inc[2 * h + 1]);
#pragma unroll
        for (int u = 0; u < UNR; ++u) td_reds_add(cq + ((unsigned)slot[u] << 7), inc[u]);
    };
    /* D >= 5: a round of NH pairs per lane (NPR, or 1 for a last round of at
     * most 64 points) */
    auto round = [&](int i0, auto nh_c) {
        constexpr int NH = decltype(nh_c)::value;
        int slot[2 * NH];
        uint32_t inc[2 * NH];
        float4 pl[NH][NPL];
        /* all loads of the round first (the accesses keep program order) */
        const unsigned ba = xq + 8u * (unsigned)i0; /* pair i0/2 + l */
#pragma unroll
        for (int h = 0; h < NH; ++h)
#pragma unroll
            for (int c = 0; c < NPL; ++c) pl[h][c] = td_lds128(ba + 512u * h + c * pstride);
#pragma unroll
        for (int h = 0; h < NH; ++h) td_pair_rows<D>(pl[h], C, slot[2 * h], slot[2 * h + 1], inc[2 * h], inc[2 * h + 1]);
#pragma unroll
        for (int u = 0; u < 2 * NH; ++u) td_reds_add(cq + ((unsigned)slot[u] << 7), inc[u]);
    };
    /* the last, partial round runs like the others over its padding zeros;
     * at D >= 5 (short rows: up to a fifth of the points are padding) at
     * half width when its points fit in 64 -- at D <= 4 that form of the
     * loop measured slower than the padding it saves */
    int pad;
    if constexpr (HALF_TAIL) {
        const int full = nnz & ~(TD_ROUND - 1), rem = nnz - full;
        for (int i0 = 0; i0 < full; i0 += TD_ROUND) round(i0, std::integral_constant<int, NPR>{});
        if (rem > TD_ROUND / 2) round(full, std::integral_constant<int, NPR>{});
        else if (rem > 0) round(full, std::integral_constant<int, 1>{});
        pad = rem == 0 ? 0 : (rem > TD_ROUND / 2 ? TD_ROUND : TD_ROUND / 2) - rem;
    } else {
        for (int i0 = 0; i0 < nnz; i0 += 32 * UNR) round_full(i0);
        pad = ((nnz + TD_ROUND - 1) & ~(TD_ROUND - 1)) - nnz;
    }
    __syncwarp();
    const uint32_t hUt = W.hist[32 * 32 + lane];
    const uint32_t hU = hUt - prev_u;
    prev_u = hUt;
    /* uncertain points: the padding points of the last round are zeros,
     * whose key is NaN, so each of them added one event to row 32 too */
    const int nu = td_wsum((int)(hU >> 16)) - pad;
    n_exact += (uint64_t)nu;

    /* Pass 1: per-lane totals of the +1/-1 events, i.e. a histogram of 32
     * coarse buckets.  Inside lane l's range the walk stays within
     * [P_l - c-_l, P_l + c+_l], which bounds G from below.  The totals come
     * from row l of the coarse histogram (each lane reads its row's quads in
     * a rotated order, so a quarter warp touches distinct banks) or, after
     * the rescan, from lane l's chunks of the fine histogram. */
    uint4 *h4 = reinterpret_cast<uint4 *>(W.hist) + lane * nch;
    const int rot = lane & chm;
    const int per = B >> 5;
    int Pl, lol, hil;
    auto pass1 = [&](uint32_t acc, int nz) -> int {
        const int cpl = td_ev_plus(acc), cml = td_ev_minus(acc);
        const int A = td_wsum(cml); /* orientation + points: one -1 event each */
        const int netl = cpl - cml;
        const int excl = td_wscan_incl(netl, lane) - netl;
        Pl = A + excl;
        lol = Pl - cml;
        hil = Pl + cpl;
        return min(td_wmin(lol), nz - td_wmax(hil));
    };
    uint32_t acc;
    {
        /* lane l reads row l, its quad k ^ (l mod 8) at step k (the warp
         * region, hence every 128-byte row, is 128-byte aligned) */
        const unsigned rb = (td_saddr(W.hist) + 128u * (unsigned)lane) | ((unsigned)(lane & 7) << 4);
        uint32_t tot = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 v = td_lds128(rb ^ (unsigned)(k << 4));
            tot += __float_as_uint(v.x) + __float_as_uint(v.y) + __float_as_uint(v.z) + __float_as_uint(v.w);
        }
        acc = tot - prev_row;
        prev_row = tot;
    }
    clean = KEEP_CLEAN;
    /* First without the uncertain points (not yet in any histogram): for
     * every direction the walk value w over all nonzero points is w_c + w_u
     * with 0 <= w_u <= (uncertain nonzero points), so min(w, nzy - w) >=
     * min(w_c, n_c - w_c) over the n_c = nnz - nu certified points.  Only
     * when that bound does not reach best are the fine histogram, the bucket
     * ids and the exact placement of the uncertain points (and the tight
     * count) built. */
    int G = pass1(acc, nnz - nu);
    int t = 0;
    if (G < best) {
        ++n_rescanned;
        publish_exact();
        clean = false;
        /* the fine histogram shares the coarse one's storage: clear it */
        uint4 *z4 = reinterpret_cast<uint4 *>(W.hist);
        const int nclr4 = max(B + 4, TD_COARSE_WORDS) >> 2;
        __syncwarp();
        for (int j = lane; j < nclr4; j += 32) z4[j] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        const int nl = td_rescan<D>(xs, npc, nnz, W, fmaxf(Ea, Eb), blog2, lane);
        if (nl > 0)
            t = narrow ? td_exact_pass<D, true>(xs, npc, W, nl, blog2, lane)
                       : td_exact_pass<D, false>(xs, npc, W, nl, blog2, lane);
        __syncwarp();
        acc = 0;
        for (int k = 0; k < nch; ++k) {
            const uint4 v = h4[(k + rot) & chm];
            acc += v.x + v.y + v.z + v.w;
        }
        G = pass1(acc, nnz - t);
    }
    const int nzy = nnz - t;
    t_out = t;
    nzy_out = nzy;
    if (G < best) {
        /* Pass 2, only over the lanes whose range could hold a walk value
         * giving less than best (cooperatively, one bucket per lane, when
         * they are few): the walk value at every bucket boundary, and the
         * in-bucket bounds of buckets holding both event signs.  The values
         * left out are all >= best on the side they could affect. */
        const unsigned cl = __ballot_sync(TD_FULL, lol < best || hil > nzy - best);
        const bool coop = __popc(cl) <= 8;
        int mn = INT_MAX, mx = INT_MIN, lo = INT_MAX, hi = INT_MIN;
        if (coop) {
            unsigned rest = cl;
            while (rest) {
                const int L = __ffs(rest) - 1;
                rest &= rest - 1;
                int carry = __shfl_sync(TD_FULL, Pl, L);
                for (int base = 0; base < per; base += 32) {
                    const int tt = base + lane;
                    const bool v = tt < per;
                    const uint32_t w = v ? W.hist[td_phys(L * per + tt, lp, chm)] : 0u;
                    const int cp = td_ev_plus(w), cm = td_ev_minus(w);
                    const int nt = cp - cm;
                    const int inc = td_wscan_incl(nt, lane);
                    const int Pb = carry + inc - nt;
                    if (v) {
                        mn = min(mn, Pb);
                        mx = max(mx, Pb);
                        if (cp && cm) {
                            lo = min(lo, Pb - cm);
                            hi = max(hi, Pb + cp);
                        }
                    }
                    carry += __shfl_sync(TD_FULL, inc, 31);
                }
                mn = min(mn, carry);
                mx = max(mx, carry);
            }
        } else {
            int P = Pl;
            for (int c = 0; c < nch; ++c) {
                const uint4 v = h4[c];
                const uint32_t w4[4] = { v.x, v.y, v.z, v.w };
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int cp = td_ev_plus(w4[k]), cm = td_ev_minus(w4[k]);
                    mn = min(mn, P);
                    mx = max(mx, P);
                    if (cp && cm) {
                        lo = min(lo, P - cm);
                        hi = max(hi, P + cp);
                    }
                    P += cp - cm;
                }
            }
            mn = min(mn, P);
            mx = max(mx, P);
        }
        mn = td_wmin(mn);
        mx = td_wmax(mx);
        lo = td_wmin(lo);
        hi = td_wmax(hi);
        /* a side is resolved only if its in-bucket range can pass the
         * boundary extremes and could give a value below best; an unresolved
         * side keeps its bound (exact when no bucket can pass the extremes,
         * >= best otherwise) */
        const bool need_lo = lo < mn && lo < best;
        const bool need_hi = hi > mx && hi > nzy - best;
        int mn2 = min(mn, lo), mx2 = max(mx, hi);
        if (need_lo) mn2 = mn;
        if (need_hi) mx2 = mx;
        if (need_lo || need_hi) {
            ++n_resolved;
            /* flag the candidate buckets with their start value (counts stay
             * below 2^15, so bit 31 is free) */
            auto cand = [&](int Pb, int cp, int cm) -> bool {
                return cp && cm && ((need_lo && Pb - cm < mn) || (need_hi && Pb + cp > mx));
            };
            if (coop) {
                unsigned rest = cl;
                while (rest) {
                    const int L = __ffs(rest) - 1;
                    rest &= rest - 1;
                    int carry = __shfl_sync(TD_FULL, Pl, L);
                    for (int base = 0; base < per; base += 32) {
                        const int tt = base + lane;
                        const bool v = tt < per;
                        const int ph = td_phys(L * per + tt, lp, chm);
                        const uint32_t w = v ? W.hist[ph] : 0u;
                        const int cp = td_ev_plus(w), cm = td_ev_minus(w);
                        const int nt = cp - cm;
                        const int inc = td_wscan_incl(nt, lane);
                        const int Pb = carry + inc - nt;
                        if (v && cand(Pb, cp, cm)) W.hist[ph] = 0x80000000u | (uint32_t)Pb;
                        carry += __shfl_sync(TD_FULL, inc, 31);
                    }
                }
            } else {
                int P = Pl;
                for (int c = 0; c < nch; ++c) {
                    const uint4 v = h4[c];
                    uint32_t w4[4] = { v.x, v.y, v.z, v.w };
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int cp = td_ev_plus(w4[k]), cm = td_ev_minus(w4[k]);
                        if (cand(P, cp, cm)) w4[k] = 0x80000000u | (uint32_t)P;
                        P += cp - cm;
                    }
                    h4[c] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
            }
            __syncwarp();
            int Gn = 0;
            for (int i0 = 0; i0 < nnz; i0 += 32) {
                const int i = i0 + lane;
                bool g = false;
                if (i < nnz) {
                    const int b = W.bid[i];
                    g = b < B && (W.hist[td_phys(b, lp, chm)] >> 31);
                }
                const unsigned bg = __ballot_sync(TD_FULL, g);
                if (g) W.glist[Gn + __popc(bg & below)] = (uint16_t)i;
                Gn += __popc(bg);
            }
            __syncwarp();
            if (Gn <= 32) {
                /* one gathered event per lane: exact direction, warp bitonic
                 * sort by (bucket, direction), segmented walk */
                int bk = INT_MAX, e = 0, Pb = 0;
                int64_t h1 = 0, h2 = 0;
                if (lane < Gn) {
                    const int i = W.glist[lane];
                    bool pl;
                    td_exact_h<D>(xs, npc, i, W.qa, W.qb, h1, h2, pl);
                    e = pl ? -1 : 1;
                    bk = W.bid[i];
                    Pb = (int)(W.hist[td_phys(bk, lp, chm)] & 0xFFFFu);
                }
#pragma unroll 1
                for (int size = 2; size <= 32; size <<= 1)
#pragma unroll 1
                    for (int stride = size >> 1; stride > 0; stride >>= 1) {
                        const int obk = __shfl_xor_sync(TD_FULL, bk, stride);
                        const int oe = __shfl_xor_sync(TD_FULL, e, stride);
                        const int oPb = __shfl_xor_sync(TD_FULL, Pb, stride);
                        const int64_t oh1 = __shfl_xor_sync(TD_FULL, h1, stride);
                        const int64_t oh2 = __shfl_xor_sync(TD_FULL, h2, stride);
                        bool o_less, m_less;
                        if (obk != bk) {
                            o_less = obk < bk;
                            m_less = bk < obk;
                        } else if (bk == INT_MAX) {
                            o_less = m_less = false;
                        } else {
                            const int cs = td_cross_sign(h1, h2, oh1, oh2);
                            m_less = cs > 0;
                            o_less = cs < 0;
                        }
                        const bool up = (lane & size) == 0;
                        const bool lower = (lane & stride) == 0;
                        const bool take = (lower == up) ? o_less : m_less;
                        if (take) {
                            bk = obk;
                            e = oe;
                            Pb = oPb;
                            h1 = oh1;
                            h2 = oh2;
                        }
                    }
                const int nbk = __shfl_down_sync(TD_FULL, bk, 1);
                const int64_t nh1 = __shfl_down_sync(TD_FULL, h1, 1);
                const int64_t nh2 = __shfl_down_sync(TD_FULL, h2, 1);
                const int pbk = __shfl_up_sync(TD_FULL, bk, 1);
                const bool valid = lane < Gn;
                const bool tie_next = valid && lane + 1 < Gn && nbk == bk && td_cross_sign(h1, h2, nh1, nh2) == 0;
                const bool head = valid && (lane == 0 || pbk != bk);
                const int S = td_wscan_incl(valid ? e : 0, lane);
                const int hidx = td_wscan_max_incl(head ? lane : 0, lane);
                const int Shead = __shfl_sync(TD_FULL, S, hidx);
                const int ehead = __shfl_sync(TD_FULL, e, hidx);
                const int val = Pb + (S - (Shead - ehead));
                const int vmn = (valid && !tie_next) ? val : INT_MAX;
                const int vmx = (valid && !tie_next) ? val : INT_MIN;
                mn2 = min(mn2, td_wmin(vmn));
                mx2 = max(mx2, td_wmax(vmx));
            } else {
                td_resolve_many<D>(xs, npc, W.qa, W.qb, W.hist, W.bid, W.glist, Gn, lp, chm, lane, &mn2, &mx2);
            }
        }
        G = min(mn2, nzy - mx2);
    }
    __syncwarp();
    return G;
}

/* The coarse bounds of two subsets A and B in one pass over the points
 * (Algorithm 2's walk bounded per lane range, as in td_sweep_filtered,
 * before any exact step): every staged pair is loaded once and projected
 * with both subsets' binary32 bases, and each event goes to its subset's
 * coarse histogram (A at W.hist, B right after it), cumulative as in
 * td_sweep_filtered (prev[0..1]: A's row and uncertain totals, prev[2..3]:
 * B's; clean2: both tables agree with them).  Pass 1 of both subsets shares
 * its warp reductions: the per-lane net counts of A and B are scanned as one
 * 32-bit word (A + 2^16 B, both prefix sums below 2^15 in magnitude, so the
 * two halves are recovered exactly), likewise the counts of -1 events and of
 * uncertain points.  GA, GB: lower bounds of G(A), G(B) over the certified
 * points (the value of td_sweep_filtered's first bound); nuA, nuB: their
 * uncertain points. */
template <int D, int ROWS>
__device__ __forceinline__ void td_sweep_dual(const float *xs, int npc, int nnz, const TdPairCoef<D> &CA,
                                              const TdPairCoef<D> &CB, const TdWarpSmem &W, int lane, bool &clean2,
                                              uint32_t (&prev)[4], int &GA, int &GB, int &nuA, int &nuB)
{
    constexpr int NPL = (D + 1) / 2;
    constexpr int UNR = TD_ROUND / 32;
    constexpr int NPR = UNR / 2;
    constexpr bool HALF_TAIL = D >= 5;
    const unsigned xq = td_saddr(xs) + 16u * (unsigned)lane;
    const unsigned pstride = 16u * (unsigned)npc;
    const unsigned cqA = td_saddr(W.hist) + 4u * (unsigned)lane;
    const unsigned cqB = cqA + 4u * TD_COARSE_WORDS;
    if (!clean2) {
        uint4 *z4 = reinterpret_cast<uint4 *>(W.hist);
        for (int j = lane; j < (2 * TD_COARSE_WORDS >> 2); j += 32) z4[j] = make_uint4(0u, 0u, 0u, 0u);
        prev[0] = prev[1] = prev[2] = prev[3] = 0u;
    }
    __syncwarp();
    auto round_full = [&](int i0) {
        const unsigned ba = xq + 8u * (unsigned)i0;
#pragma unroll
        for (int h = 0; h < NPR; ++h) {
            float4 pl[NPL];
#pragma unroll
            for (int c = 0; c < NPL; ++c) pl[c] = td_lds128(ba + 512u * h + c * pstride);
            int sa0, sa1, sb0, sb1;
            uint32_t ia0, ia1, ib0, ib1;
            td_pair_rows<D, ROWS>(pl, CA, sa0, sa1, ia0, ia1);
            td_pair_rows<D, ROWS>(pl, CB, sb0, sb1, ib0, ib1);
            td_reds_add(cqA + ((unsigned)sa0 << 7), ia0);
            td_reds_add(cqA + ((unsigned)sa1 << 7), ia1);
            td_reds_add(cqB + ((unsigned)sb0 << 7), ib0);
            td_reds_add(cqB + ((unsigned)sb1 << 7), ib1);
        }
    };
    /* D >= 5: a round of NH pairs per lane (NPR, or 1 for a last round of
     * at most 64 points) */
    auto round = [&](int i0, auto nh_c) {
        constexpr int NH = decltype(nh_c)::value;
        const unsigned ba = xq + 8u * (unsigned)i0;
#pragma unroll
        for (int h = 0; h < NH; ++h) {
            float4 pl[NPL];
#pragma unroll
            for (int c = 0; c < NPL; ++c) pl[c] = td_lds128(ba + 512u * h + c * pstride);
            int sa0, sa1, sb0, sb1;
            uint32_t ia0, ia1, ib0, ib1;
            td_pair_rows<D, ROWS>(pl, CA, sa0, sa1, ia0, ia1);
            td_pair_rows<D, ROWS>(pl, CB, sb0, sb1, ib0, ib1);
            td_reds_add(cqA + ((unsigned)sa0 << 7), ia0);
            td_reds_add(cqA + ((unsigned)sa1 << 7), ia1);
            td_reds_add(cqB + ((unsigned)sb0 << 7), ib0);
            td_reds_add(cqB + ((unsigned)sb1 << 7), ib1);
        }
    };
    /* the last round at half width when its points fit in 64, at D >= 5
     * (as in td_sweep_filtered) */
    int pad;
    if constexpr (HALF_TAIL) {
        const int full = nnz & ~(TD_ROUND - 1), rem = nnz - full;
        for (int i0 = 0; i0 < full; i0 += TD_ROUND) round(i0, std::integral_constant<int, NPR>{});
        if (rem > TD_ROUND / 2) round(full, std::integral_constant<int, NPR>{});
        else if (rem > 0) round(full, std::integral_constant<int, 1>{});
        pad = rem == 0 ? 0 : (rem > TD_ROUND / 2 ? TD_ROUND : TD_ROUND / 2) - rem;
    } else {
        for (int i0 = 0; i0 < nnz; i0 += 32 * UNR) round_full(i0);
        pad = ((nnz + TD_ROUND - 1) & ~(TD_ROUND - 1)) - nnz;
    }
    __syncwarp();
    /* uncertain points (row ROWS), padding zeros of the last round included */
    const uint32_t uA = W.hist[ROWS * 32 + lane], uB = W.hist[TD_COARSE_WORDS + ROWS * 32 + lane];
    const uint32_t hA = uA - prev[1], hB = uB - prev[3];
    prev[1] = uA;
    prev[3] = uB;
    const uint32_t usum = (uint32_t)td_wsum((int)((hA >> 16) + ((hB >> 16) << 16)));
    nuA = (int)(usum & 0xFFFFu) - pad;
    nuB = (int)(usum >> 16) - pad;
    uint32_t accA, accB;
    if constexpr (ROWS == 32) {
        /* pass 1: lane l reads row l of both tables (XOR-rotated quads) */
        const unsigned rb = (td_saddr(W.hist) + 128u * (unsigned)lane) | ((unsigned)(lane & 7) << 4);
        uint32_t tA = 0, tB = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 va = td_lds128(rb ^ (unsigned)(k << 4));
            const float4 vb = td_lds128((rb ^ (unsigned)(k << 4)) + 4u * TD_COARSE_WORDS);
            tA += __float_as_uint(va.x) + __float_as_uint(va.y) + __float_as_uint(va.z) + __float_as_uint(va.w);
            tB += __float_as_uint(vb.x) + __float_as_uint(vb.y) + __float_as_uint(vb.z) + __float_as_uint(vb.w);
        }
        accA = tA - prev[0];
        accB = tB - prev[2];
        prev[0] = tA;
        prev[2] = tB;
        clean2 = true;
        const int cpA = td_ev_plus(accA), cmA = td_ev_minus(accA);
        const int cpB = td_ev_plus(accB), cmB = td_ev_minus(accB);
        const uint32_t am = (uint32_t)td_wsum(cmA + (cmB << 16)); /* orientation + points: one -1 event each */
        const int AA = (int)(am & 0xFFFFu), AB = (int)(am >> 16);
        const int netA = cpA - cmA, netB = cpB - cmB;
        const int v = netA + netB * 65536;
        const int ex = td_wscan_incl(v, lane) - v;
        const int exA = (int)(int16_t)(ex & 0xFFFF);
        const int exB = (ex - exA) >> 16;
        const int PA = AA + exA, PB = AB + exB;
        const int ncA = nnz - nuA, ncB = nnz - nuB;
        GA = td_wmin(min(PA - cmA, ncA - (PA + cpA)));
        GB = td_wmin(min(PB - cmB, ncB - (PB + cpB)));
    } else {
        /* pass 1 over ROWS rows: the S = 32/ROWS lanes 2r.. of row r (lane l:
         * row r = l / S, part k = l % S) read 8/S of its quads each, in an
         * order rotated by r so that every quarter warp touches distinct
         * banks, and add their sums with S - 1 XOR-shuffles; the scan over
         * rows steps S lanes at a time */
        constexpr int S = 32 / ROWS, QP = 8 / S;
        const int r = lane / S, k = lane % S;
        const unsigned rb = td_saddr(W.hist) + 128u * (unsigned)r + 16u * (unsigned)(k * QP);
        uint32_t tA = 0, tB = 0;
#pragma unroll
        for (int j = 0; j < QP; ++j) {
            const unsigned a = rb + 16u * (unsigned)(j ^ (r & (QP - 1)));
            const float4 va = td_lds128(a);
            const float4 vb = td_lds128(a + 4u * TD_COARSE_WORDS);
            tA += __float_as_uint(va.x) + __float_as_uint(va.y) + __float_as_uint(va.z) + __float_as_uint(va.w);
            tB += __float_as_uint(vb.x) + __float_as_uint(vb.y) + __float_as_uint(vb.z) + __float_as_uint(vb.w);
        }
#pragma unroll
        for (int o = 1; o < S; o <<= 1) {
            tA += __shfl_xor_sync(TD_FULL, tA, o);
            tB += __shfl_xor_sync(TD_FULL, tB, o);
        }
        accA = tA - prev[0];
        accB = tB - prev[2];
        prev[0] = tA;
        prev[2] = tB;
        clean2 = true;
        const int cpA = td_ev_plus(accA), cmA = td_ev_minus(accA);
        const int cpB = td_ev_plus(accB), cmB = td_ev_minus(accB);
        /* orientation + points: one -1 event each, one lane per row */
        const uint32_t am = (uint32_t)td_wsum(k == 0 ? cmA + (cmB << 16) : 0);
        const int AA = (int)(am & 0xFFFFu), AB = (int)(am >> 16);
        const int netA = cpA - cmA, netB = cpB - cmB;
        const int v = netA + netB * 65536;
        int inc = v;
#pragma unroll
        for (int o = 1; o < ROWS; o <<= 1) {
            const int u = __shfl_up_sync(TD_FULL, inc, o * S);
            if (r >= o) inc += u;
        }
        const int ex = inc - v;
        const int exA = (int)(int16_t)(ex & 0xFFFF);
        const int exB = (ex - exA) >> 16;
        const int PA = AA + exA, PB = AB + exB;
        const int ncA = nnz - nuA, ncB = nnz - nuB;
        GA = td_wmin(min(PA - cmA, ncA - (PA + cpA)));
        GB = td_wmin(min(PB - cmB, ncB - (PB + cpB)));
    }
}

/* Tight-set correction m_S after a sweep.  Tight points are those with bucket
 * id TD_SENT (filtered kernel, bid != NULL) or a zero projection H (plain
 * kernel); coordinates come from xs (float, filtered, pair layout with PS
 * pairs per plane, see td_xidx) or xi (int, plain, stride PSI).
 * The subset's rows and point ids are in meta (published basis). */
template <int D>
__device__ __noinline__ int td_tight_correction(const int *meta, const float *xs, int PS, const int32_t *xi,
                                                int PSI, int nnz, const uint16_t *bid, const int64_t *H,
                                                TdScratch scr, int *gcount, int lane)
{
    constexpr int K = D - 2;
    if constexpr (K <= 0) {
        return 0;
    } else {
        auto is_tight = [&](int i) -> bool {
            if (bid) return bid[i] == TD_SENT;
            return H[2 * i] == 0 && H[2 * i + 1] == 0;
        };
        auto coord = [&](int i, int r) -> int64_t {
            if (xs) return td_f2i(xs[td_xidx(PS, i, r)]);
            return (int64_t)xi[(size_t)i * PSI + r];
        };
        int rows[K];
#pragma unroll
        for (int r = 0; r < K; ++r) rows[r] = meta[r];
        if constexpr (K == 1) {
            int pos = 0, neg = 0;
            for (int i = lane; i < nnz; i += 32)
                if (is_tight(i)) {
                    int64_t v = coord(i, rows[0]);
                    pos += v > 0;
                    neg += v < 0;
                }
            return min(td_wsum(pos), td_wsum(neg));
        } else {
            int t = 0;
            const unsigned below = (1u << lane) - 1u;
            for (int i0 = 0; i0 < nnz; i0 += 32) {
                const int i = i0 + lane;
                const bool g = i < nnz && is_tight(i);
                const unsigned bg = __ballot_sync(TD_FULL, g);
                if (g) {
                    const int slot = t + __popc(bg & below);
#pragma unroll
                    for (int r = 0; r < K; ++r) scr.c0[4 * slot + r] = (int32_t)coord(i, rows[r]);
                }
                t += __popc(bg);
            }
            __syncwarp();
            int64_t sint[4][4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int r = 0; r < 4; ++r) sint[j][r] = (j < K && r < K) ? coord(meta[4 + j], rows[r]) : 0;
            return td_tight_depth<K>(t, sint, scr, lane);
        }
    }
}

/* Process subset positions [r0, r1) of query q with one warp (filtered).
 * The warp's counters ws[] (sweeps, dependent, filtered points, exact
 * points, tight corrections, resolved sweeps, errors, early-exit skips,
 * rescanned sweeps) live in shared memory;
 * the subset loop keeps 32-bit tile counts and lane 0 adds them at the end.
 *
 * For D = 3..5 consecutive subsets are taken two at a time: td_sweep_dual
 * gives both coarse bounds from one pass over the points, and a subset whose
 * bound does not reach best is swept again alone (td_sweep_filtered: the
 * coarse bound, then the exact steps) -- so every value below best is exact
 * and the others are never below best, as in the one-at-a-time form, which
 * D = 2 and D = 6 use throughout.  Each lane computes the minor of its row
 * pair e = lane % 16 for the subset of its half of the warp (both halves
 * the same subset when one is swept alone) and caches the cofactors of the
 * minor's other columns, recomputed when c[1..K) of that subset differs from
 * the one they were made for. */
template <int D>
__device__ void td_warp_filtered(const TdLaunch &L, int q, const float *xs, int npc, int nnz,
                                 uint64_t r0, uint64_t r1, const TdWarpSmem &W, const TdScratch &scr,
                                 int blog2, int lane, int &best, unsigned long long *ws)
{
    constexpr int K = D - 2;
    constexpr int KK = K > 0 ? K : 1;
    constexpr bool DUAL = td_coarse_tables(D) == 2;
    if (r0 >= r1) return;
    const TdQuery &Q = L.q[q];
    int c[KK];
    c[0] = 0;
    td_unrank_colex<K>(r0, nnz, c);
    float mxf[D];
#pragma unroll
    for (int r = 0; r < D; ++r) mxf[r] = (float)Q.mx[r]; /* < 2^22: exact */
    float mx_lane = 0.f; /* max|x_t| of this lane's basis entry t = lane % 8 */
#pragma unroll
    for (int r = 0; r < D; ++r) mx_lane = (lane & 7) == r ? mxf[r] : mx_lane;
    uint32_t n_dep = 0, n_tight = 0, n_res = 0, n_resc = 0;
    uint64_t n_exact = 0;
    bool clean = false;  /* the coarse histogram agrees with prev_row / prev_u */
    bool clean2 = false; /* the two coarse histograms of the dual sweep agree with prev2 */
    uint32_t prev_row = 0u, prev_u = 0u, prev2[4] = { 0u, 0u, 0u, 0u };
    /* forward error bound of the FP32 projection: the fma chain adds at most
     * D u sum |q_i x_i|, the rounded coefficients (at most 2u each, see
     * td_i64_to_f32) 2u more; taken as (D + 3) u, applied to A = sum |q_i|
     * max|x_i| computed in binary32 from the rounded coefficients (relative
     * error below (D + 2) u), the extra factor 1 + 2^-10 covering that and
     * the rounding of the products below */
    const float cst = (float)(D + 3) * TD_U * 1.0009765625f;
    int pi, pj, lr[KK];
    td_lane_pair<D>(lane & 15, npc, pi, pj, lr);
    int64_t cof[KK];  /* cofactors of column 0 of this lane's minor */
    int cmade[KK];    /* the c[1..K) they were made for (-1: none) */
#pragma unroll
    for (int i = 0; i < KK; ++i) cmade[i] = -1;
    /* minors in int32 when K! max|x|^K < 2^31 (max over the coordinates);
     * max|x| < 2^22 and K <= 4, so the product is formed in int64 with an
     * early stop once it reaches 2^31 (each factor is below 2^25) */
    bool nm;
    {
        int64_t mm = 0;
#pragma unroll
        for (int r = 0; r < D; ++r) mm = max(mm, (int64_t)Q.mx[r]);
        int64_t b = 1;
#pragma unroll
        for (int i = 1; i <= K; ++i) b = b < ((int64_t)1 << 31) ? b * (int64_t)i * mm : b;
        nm = b < 2147483647LL;
    }
    constexpr bool REFRESH = D <= 4; /* see the subset loop below */
    /* cofactors stale for this lane's subset cs? (and mark them made) */
    auto stale = [&](const int (&cs)[KK]) -> bool {
        bool st = cmade[0] < 0;
#pragma unroll
        for (int i = 1; i < K; ++i) st |= cs[i] != cmade[i];
#pragma unroll
        for (int i = 0; i < KK; ++i) cmade[i] = i == 0 ? 0 : cs[i];
        return st;
    };
    /* One subset alone: basis, sweep (coarse bound, then the exact steps
     * when it could lower best), tight correction.  Returns false when the
     * subset is dependent. */
    auto single = [&](const int (&cs)[KK]) -> bool {
        const bool refresh = stale(cs);
        if (!(nm ? td_basis_publish<D, true>(xs, cs, lane & 15, pi, pj, lr, W, cof, refresh)
                 : td_basis_publish<D, false>(xs, cs, lane & 15, pi, pj, lr, W, cof, refresh)))
            return false;
        td_f2x FA[D], FB[D];
        td_load_coef2<D>(W.fab2, FA, FB);
        float Aa = 0.0f, Ab = 0.0f;
#pragma unroll
        for (int t = 0; t < D; ++t) {
            float fa, fb, dummy;
            td_upk(FA[t], fa, dummy);
            td_upk(FB[t], fb, dummy);
            Aa = fmaf(fabsf(fa), mxf[t], Aa);
            Ab = fmaf(fabsf(fb), mxf[t], Ab);
        }
        const float Ea = Aa * cst, Eb = Ab * cst;
        /* exact bounds below 2^31 (the binary32 sums are within (D + 2) u) */
        const bool narrow = fmaxf(Aa, Ab) < 2145386496.0f; /* 2^31 (1 - 2^-10) */
        int t, nzy;
        auto publish_exact = [&]() {
            if (nm) td_basis_publish_exact<D, true>(xs, cs, lane & 15, pi, pj, lr, W, cof);
            else td_basis_publish_exact<D, false>(xs, cs, lane & 15, pi, pj, lr, W, cof);
        };
        const int G = td_sweep_filtered<D>(xs, npc, nnz, FA, FB, Ea, Eb, narrow, W, blog2, lane, best, clean,
                                           prev_row, prev_u, n_exact, n_res, n_resc, t, nzy, publish_exact);
        clean2 = false; /* the one-subset sweep used table A's storage */
        int V = G;
        if (t > K && G < best) {
            ++n_tight;
            V = G + td_tight_correction<D>(W.meta, xs, npc, nullptr, 0, nnz, W.bid, nullptr, scr, W.gcount, lane);
        }
        if (REFRESH && V < best && lane == 0) atomicMin(L.qmin + q, V);
        best = min(best, V);
        return true;
    };
    uint32_t nr = (uint32_t)(r1 - r0); /* a tile: below 2^31 */
    uint32_t done = 0;
    /* D <= 4: the query's running minimum in global memory, which other
     * warps lower while this one works, is read again at every step (the
     * load is issued at one step and taken into best at the next, a step's
     * work later), and a subset that lowers best publishes it at once.  Any
     * value it holds is some V(S) or the seeded upper bound, so taking it as
     * best keeps every decision valid.  (At D = 5, 6 the extra live
     * registers cost more than the sweeps they save.) */
    int gbest = best;
    while (done < nr) {
        if constexpr (REFRESH) {
            best = min(best, gbest);
            gbest = *reinterpret_cast<const volatile int32_t *>(L.qmin + q);
        }
        if (DUAL && done + 1 < nr) {
            int cB[KK];
#pragma unroll
            for (int i = 0; i < KK; ++i) cB[i] = c[i];
            td_next_colex<K>(cB);
            int cH[KK];
#pragma unroll
            for (int i = 0; i < KK; ++i) cH[i] = lane < 16 ? c[i] : cB[i];
            const bool refresh = stale(cH);
            float EA, EB;
            bool narA, narB;
            const int dep = nm ? td_basis_publish_dual<D, true>(xs, cH, lane, pi, pj, lr, W, cof, refresh, mx_lane,
                                                                cst, EA, EB, narA, narB)
                               : td_basis_publish_dual<D, false>(xs, cH, lane, pi, pj, lr, W, cof, refresh,
                                                                 mx_lane, cst, EA, EB, narA, narB);
            (void)narA;
            (void)narB;
            if (dep == 0) {
                td_f2x FA[D], FB[D], FA2[D], FB2[D];
                td_load_coef2<D>(W.fab2, FA, FB);
                td_load_coef2<D>(W.fab2 + 16, FA2, FB2);
                const TdPairCoef<D> CA = td_pair_coef<D>(FA, FB, EA, blog2);
                const TdPairCoef<D> CB = td_pair_coef<D>(FA2, FB2, EB, blog2);
                int GA, GB, nuA, nuB;
                td_sweep_dual<D, TD_DUAL_ROWS(D)>(xs, npc, nnz, CA, CB, W, lane, clean2, prev2, GA, GB, nuA, nuB);
                clean = false; /* the dual sweep used table A's storage */
                /* a subset whose bound does not reach best is swept again alone
                 * (repeating the coarse pass there measured faster than a
                 * branch around it in the one-subset sweep) */
                if (GA < best) single(c);
                else n_exact += (uint64_t)nuA;
                if (GB < best) single(cB);
                else n_exact += (uint64_t)nuB;
            } else {
                if (dep & 1) ++n_dep;
                else single(c);
                if (dep & 2) ++n_dep;
                else single(cB);
            }
            done += 2;
            if (L.early_exit && best <= 0) {
                if (lane == 0) ws[7] += nr - done;
                nr = done;
                break;
            }
#pragma unroll
            for (int i = 0; i < KK; ++i) c[i] = cB[i];
            if (done < nr) td_next_colex<K>(c);
        } else {
            if (!single(c)) ++n_dep;
            ++done;
            if (L.early_exit && best <= 0) {
                /* V = 0 is the least value: the rest of the range cannot lower it */
                if (lane == 0) ws[7] += nr - done;
                nr = done;
                break;
            }
            if (done < nr) td_next_colex<K>(c);
        }
    }
    if (lane == 0) {
        const uint64_t sw = (uint64_t)nr - n_dep;
        ws[0] += sw;
        ws[1] += n_dep;
        ws[2] += sw * (uint64_t)nnz - n_exact;
        ws[3] += n_exact;
        ws[4] += n_tight;
        ws[5] += n_res;
        ws[8] += n_resc;
    }
}

/* ====================================================================== */
/* persistent filtered kernel                                              */
/* ====================================================================== */

__device__ __forceinline__ int td_query_of_tile(const int64_t *prefix, int nq, int64_t tile)
{
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

/* Persistent sweep kernel for the queries of effective dimension D: CTAs pop
 * (query, subset-tile) work from the dimension's counter until it runs dry;
 * the points of the current query stay staged in shared memory; every warp
 * sweeps its share of the tile's subsets; one atomicMin per tile. */
template <int D>
__global__ void __launch_bounds__(256, 2) td_k_filtered(TdLaunch L)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int64_t s_tile;
    __shared__ int s_tmp[32];
    __shared__ int s_best[TD_WARPS_MAX];
    __shared__ unsigned long long s_stats[TD_WARPS_MAX][9];
    const int64_t *prefix = L.tile_prefix + (int64_t)(D - 2) * (L.nq + 1);
    unsigned long long *ticket = L.ticket + (D - 2) * TD_TICKET_STRIDE;
    const int64_t total = prefix[L.nq];
    if (total == 0) return;
    if (td_saddr(smem) & 127u) {
        /* the row addressing of pass 1 needs 128-byte aligned warp regions */
        if (threadIdx.x == 0) atomicAdd(&L.ctr->errors, 1ull);
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nmaxp = max(128, td_pow2_at_least(L.nmax));
    /* staging area: ceil(pmax/2) planes of npc pairs (sizing); this
     * dimension uses the first ceil(D/2) */
    const int npc = td_plane_pairs(L.nmax);
    const int nplanes_max = (L.pmax + 1) >> 1;
    const int blog2_cap = L.blog2;
    /* layout: xs (pair planes) | per warp: region { fine hist [Bmax + 4]
     * u32 } or the coarse histogram, whichever is larger | gcount | basis
     * (qa, qb, meta, fab, q32).  The bucket ids and lists of the rare path
     * are in the warp's global scratch. */
    /* D = 2 (one subset a query): every warp takes its own queries, with its
     * own staging area of npc pairs in front of its region, and no block
     * barrier */
    const size_t xs_warp = (D == 2) ? td_staging_bytes(L.nmax, 1) : 0;
    const size_t off = (D == 2) ? 0 : td_staging_bytes(L.nmax, nplanes_max);
    const int Bmax = 1 << blog2_cap;
    const size_t hbytes = (size_t)(Bmax + 4) * 4;
    const size_t rbytes = max((size_t)TD_COARSE_WORDS * 4 * td_coarse_tables(D), hbytes);
    const size_t per_warp = td_warp_region_bytes(rbytes);
    unsigned char *wb = smem + off + (per_warp + xs_warp) * w + xs_warp;
    float *xs = reinterpret_cast<float *>(D == 2 ? wb - xs_warp : smem);
    TdWarpSmem W;
    W.hist = reinterpret_cast<uint32_t *>(wb);
    const int gw = blockIdx.x * (blockDim.x >> 5) + w;
    /* the global scratch keeps the host's sizing (td_scratch_per_warp(nmax)) */
    const TdScratch scr = td_scratch_at(L.scratch + (size_t)gw * L.scratch_per_warp, td_pow2_at_least(L.nmax));
    W.bid = scr.bid;
    W.glist = scr.glist;
    W.gcount = reinterpret_cast<int *>(wb + rbytes);
    W.qa = reinterpret_cast<int64_t *>(wb + rbytes + 16);
    W.qb = W.qa + 8;
    W.q32 = reinterpret_cast<int32_t *>(wb + rbytes + 16 + 128);
    W.fab2 = reinterpret_cast<td_f2x *>(wb + rbytes + 16 + 192);
    W.meta = reinterpret_cast<int *>(wb + rbytes + 16 + 448);
    for (int j = lane; j < max(Bmax + 4, TD_COARSE_WORDS); j += 32) W.hist[j] = 0u;
    unsigned long long *ws = s_stats[w];
    if (lane < 9) ws[lane] = 0ull;
    if constexpr (D == 2) {
        __syncwarp();
        for (;;) {
            unsigned long long tk = 0ull;
            if (lane == 0) tk = atomicAdd(ticket, 1ull);
            const int64_t tile = (int64_t)__shfl_sync(TD_FULL, tk, 0);
            if (tile >= total) break;
            const int j = td_query_of_tile(prefix, L.nq, tile);
            const int q = L.order[j];
            const TdQuery &Q = L.q[q];
            const int nnz = Q.nnz;
            const int64_t ts = L.tile_size[q];
            const int64_t t0 = Q.lo + (tile - prefix[j]) * ts;
            const uint64_t r0 = (uint64_t)t0, r1 = (uint64_t)min(t0 + ts, Q.hi);
            int blog2 = 7;
            while ((2 << blog2) < nnz && blog2 < blog2_cap) ++blog2;
            int best = L.qmin[q];
            if (L.early_exit && best <= 0) {
                if (lane == 0) ws[7] += r1 - r0;
                continue;
            }
            if (Q.d != 2 || blog2 > blog2_cap || nnz > L.nmax) {
                if (lane == 0) ws[6]++; /* inconsistent sizes: the host reports TD_ERR_INTERNAL */
                continue;
            }
            if (td_stage_points_warp(L, q, xs, npc, lane) != nnz) {
                if (lane == 0) ws[6]++;
                continue;
            }
            td_warp_filtered<D>(L, q, xs, npc, nnz, r0, r1, W, scr, blog2, lane, best, ws);
            if (lane == 0 && best < INT_MAX) atomicMin(&L.qmin[q], best);
        }
        __syncwarp();
        if (lane == 0) {
            atomicAdd(&L.ctr->sweeps, ws[0]);
            atomicAdd(&L.ctr->dependent, ws[1]);
            atomicAdd(&L.ctr->filtered_points, ws[2]);
            atomicAdd(&L.ctr->exact_points, ws[3]);
            atomicAdd(&L.ctr->tight, ws[4]);
            atomicAdd(&L.ctr->resolved, ws[5]);
            atomicAdd(&L.ctr->errors, ws[6]);
            if (ws[7]) atomicAdd(&L.ctr->early, ws[7]);
            if (ws[8]) atomicAdd(&L.ctr->rescanned, ws[8]);
        }
        return;
    }
    int staged = -1;
    __shared__ uint64_t s_bar;
    unsigned bar_phase = 0u;
    if (threadIdx.x == 0) td_mbar_init(&s_bar);
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(ticket, 1ull);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= total) break;
        const int j = td_query_of_tile(prefix, L.nq, tile);
        const int q = L.order[j];
        if (q != staged) {
            /* the warp regions are free between tiles (every tile clears its
             * histograms first): the dataset's rows go there */
            if (td_stage_points(L, q, xs, npc, (D + 1) >> 1, s_tmp, reinterpret_cast<int32_t *>(smem + off),
                                per_warp * (blockDim.x >> 5), &s_bar, bar_phase) < 0) {
                if (threadIdx.x == 0) atomicAdd(&L.ctr->errors, 1ull); /* the host reports TD_ERR_INTERNAL */
                break;
            }
            staged = q;
        }
        const TdQuery &Q = L.q[q];
        const int nnz = Q.nnz;
        const int64_t ts = L.tile_size[q];
        const int64_t t0 = Q.lo + (tile - prefix[j]) * ts;
        const int64_t t1 = min(t0 + ts, Q.hi);
        const int64_t spw = ts / (blockDim.x >> 5);
        const uint64_t r0 = (uint64_t)min(t0 + spw * w, t1), r1 = (uint64_t)min(t0 + spw * (w + 1), t1);
        /* buckets: about one per two nonzero points, at least 128 (four per lane) */
        int blog2 = 7;
        while ((2 << blog2) < nnz && blog2 < blog2_cap) ++blog2;
        int best = L.qmin[q];
        if (L.early_exit && best <= 0) {
            /* the query has reached V = 0, the least value (early exit) */
            if (lane == 0) ws[7] += r1 - r0;
        } else if (Q.d == D && blog2 <= blog2_cap && nnz <= L.nmax)
            td_warp_filtered<D>(L, q, xs, npc, nnz, r0, r1, W, scr, blog2, lane, best, ws);
        else if (lane == 0)
            ws[6]++; /* inconsistent sizes: skip, the host reports TD_ERR_INTERNAL */
        if (lane == 0) s_best[w] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            int b = INT_MAX;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) b = min(b, s_best[k]);
            if (b < INT_MAX) atomicMin(&L.qmin[q], b);
        }
    }
    if (lane == 0) {
        atomicAdd(&L.ctr->sweeps, ws[0]);
        atomicAdd(&L.ctr->dependent, ws[1]);
        atomicAdd(&L.ctr->filtered_points, ws[2]);
        atomicAdd(&L.ctr->exact_points, ws[3]);
        atomicAdd(&L.ctr->tight, ws[4]);
        atomicAdd(&L.ctr->resolved, ws[5]);
        atomicAdd(&L.ctr->errors, ws[6]);
        if (ws[7]) atomicAdd(&L.ctr->early, ws[7]);
        if (ws[8]) atomicAdd(&L.ctr->rescanned, ws[8]);
    }
}

/* ====================================================================== */
/* Algorithm 3 (ADIA): search kernel                                        */
/* ====================================================================== */

#include "td_adia.cuh"

/* ====================================================================== */
/* Proposition 1 with r = p-1: critical-direction kernel                    */
/* ====================================================================== */

#include "td_critical.cuh"

/* ====================================================================== */
/* the exact path beyond the fast kernels' coordinate limit                */
/* ====================================================================== */

#include "td_wide.cuh"

/* ====================================================================== */
/* plain exact kernel (one query per launch)                               */
/* ====================================================================== */

template <int D>
__device__ void td_warp_plain(const TdLaunch &L, int q, const int32_t *xi, int PSI, int nnz,
                              uint64_t r0, uint64_t r1, int64_t *H, uint16_t *idx, int *gcount,
                              int64_t *wqa, int64_t *wqb, int *wmeta,
                              const TdScratch &scr, int lane, int &best, TdWarpStats &st)
{
    constexpr int K = D - 2;
    if (r0 >= r1) return;
    int c[K > 0 ? K : 1];
    c[0] = 0;
    td_unrank_colex<K>(r0, nnz, c);
    for (uint64_t r = r0; r < r1; ++r) {
        if (r > r0) td_next_colex<K>(c);
        int64_t s[K > 0 ? K : 1][D];
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int t = 0; t < D; ++t) s[j][t] = xi[(size_t)c[j] * PSI + t];
        TdBasis<D> Bs;
        if (!td_make_basis<D>(s, Bs)) {
            if (lane == 0) st.dependent++;
            continue;
        }
        if (lane == 0) st.sweeps++;
        td_publish_basis<D>(Bs, c, wqa, wqb, wmeta, lane);
        /* exact projections of every point, compacted list of the nonzero ones */
        int base = 0, t = 0;
        bool wide = false; /* some projected coordinate is 2^31 or more in magnitude */
        for (int i0 = 0; i0 < nnz; i0 += 32) {
            int i = i0 + lane;
            int64_t y1 = 0, y2 = 0;
            bool valid = i < nnz;
            if (valid) {
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    int64_t xv = xi[(size_t)i * PSI + k];
                    y1 += Bs.qa[k] * xv;
                    y2 += Bs.qb[k] * xv;
                }
            }
            bool tight = valid && y1 == 0 && y2 == 0;
            bool nonz = valid && !tight;
            int64_t h1 = 0, h2 = 0;
            bool plus = false;
            if (nonz) plus = td_normalise(y1, y2, h1, h2);
            if (valid) {
                H[2 * i] = h1;
                H[2 * i + 1] = h2;
            }
            wide |= (h1 >= ((int64_t)1 << 31)) | (h1 <= -((int64_t)1 << 31)) | (h2 >= ((int64_t)1 << 31));
            unsigned bn = __ballot_sync(TD_FULL, nonz);
            if (nonz) idx[base + __popc(bn & ((1u << lane) - 1u))] = (uint16_t)(i | (plus ? 0x8000 : 0));
            base += __popc(bn);
            t += __popc(__ballot_sync(TD_FULL, tight));
        }
        __syncwarp();
        int G = 0;
        {
            const int npad = td_pow2_at_least(base);
            for (int l = base + lane; l < npad; l += 32) idx[l] = TD_SENT;
            __syncwarp();
            /* the exact comparisons in int64 when every coordinate is below
             * 2^31 (their products then stay below 2^62), else in int128 */
            if (__any_sync(TD_FULL, wide)) {
                td_sort_exact_fast<false>(idx, npad, H, lane, nullptr);
                G = td_walk_sorted<false>(idx, base, H, lane);
            } else {
                td_sort_exact_fast<true>(idx, npad, H, lane, nullptr);
                G = td_walk_sorted<true>(idx, base, H, lane);
            }
        }
        st.exact += (lane == 0) ? nnz : 0;
        int V = G;
        if (t > K && G < best) {
            if (lane == 0) st.tight++;
            V = G + td_tight_correction<D>(wmeta, nullptr, 0, xi, PSI, nnz, nullptr, H, scr, gcount, lane);
        }
        best = min(best, V);
    }
}

template <int D>
__global__ void __launch_bounds__(128, 1) td_k_plain(TdLaunch L, int q)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_tmp[32];
    __shared__ int s_best[TD_WARPS_MAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const TdQuery &Q = L.q[q];
    if (Q.k < 0 || Q.hi <= Q.lo) return;
    const int nnz = Q.nnz, d = Q.d;
    const int nmaxp = td_pow2_at_least(L.nmax);
    const int PSI = L.pmax <= 4 ? 4 : 8;
    /* layout: xi [nmax][PSI] int32 | per warp: H [nmaxp][2] int64, idx [nmaxp] u16, gcount */
    int32_t *xi = reinterpret_cast<int32_t *>(smem);
    size_t off = ((size_t)L.nmax * PSI * 4 + 15) & ~(size_t)15;
    size_t per_warp = ((size_t)nmaxp * 16 + (size_t)nmaxp * 2 + 16 + TD_WARP_META_BYTES + 15) & ~(size_t)15;
    unsigned char *wb = smem + off + per_warp * w;
    int64_t *H = reinterpret_cast<int64_t *>(wb);
    uint16_t *idx = reinterpret_cast<uint16_t *>(wb + (size_t)nmaxp * 16);
    int *gcount = reinterpret_cast<int *>(idx + nmaxp);
    int64_t *wqa = reinterpret_cast<int64_t *>(wb + (size_t)nmaxp * 16 + (size_t)nmaxp * 2 + 16);
    int64_t *wqb = wqa + TD_MAXD;
    int *wmeta = reinterpret_cast<int *>(wqb + TD_MAXD);
    {
        const TdSet S = L.sets[Q.set];
        const int n = S.n, p = S.p;
        const int32_t *X = L.X + S.x_off;
        const int32_t *z = L.Zq + (int64_t)q * TD_MAXD;
        const int T = blockDim.x;
        const int per = (n + T - 1) / T;
        const int beg = min((int)threadIdx.x * per, n), end = min(beg + per, n);
        int cnt = 0;
        for (int i = beg; i < end; ++i) {
            bool nz = false;
            for (int c = 0; c < p; ++c) nz |= X[(int64_t)i * p + c] != z[c];
            cnt += nz;
        }
        int inc = td_wscan_incl(cnt, lane);
        if (lane == 31) s_tmp[w] = inc;
        __syncthreads();
        if (w == 0) {
            int v = lane < nw ? s_tmp[lane] : 0;
            int vi = td_wscan_incl(v, lane);
            if (lane < nw) s_tmp[lane] = vi - v;
        }
        __syncthreads();
        int o = s_tmp[w] + inc - cnt;
        for (int i = beg; i < end; ++i) {
            bool nz = false;
            for (int c = 0; c < p; ++c) nz |= X[(int64_t)i * p + c] != z[c];
            if (!nz) continue;
            for (int c = 0; c < PSI; ++c)
                xi[(size_t)o * PSI + c] = c < d ? (int32_t)((int64_t)X[(int64_t)i * p + Q.piv[c]] - z[Q.piv[c]]) : 0;
            ++o;
        }
        __syncthreads();
    }
    const int gw = blockIdx.x * nw + w;
    const TdScratch scr = td_scratch_at(L.scratch + (size_t)gw * L.scratch_per_warp, nmaxp);
    TdWarpStats st = { 0, 0, 0, 0, 0, 0, 0 };
    const int64_t ts = (int64_t)(L.spw > 0 ? L.spw : 8) * nw;
    const int64_t ntiles = (Q.hi - Q.lo + ts - 1) / ts;
    int best = INT_MAX;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t t0 = Q.lo + tile * ts, t1 = min(t0 + ts, Q.hi);
        const int64_t spw = ts / nw;
        const uint64_t r0 = (uint64_t)min(t0 + spw * w, t1), r1 = (uint64_t)min(t0 + spw * (w + 1), t1);
        if (d == D) td_warp_plain<D>(L, q, xi, PSI, nnz, r0, r1, H, idx, gcount, wqa, wqb, wmeta, scr, lane, best, st);
        else if (lane == 0) st.errors++;
    }
    if (lane == 0) s_best[w] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = INT_MAX;
        for (int k = 0; k < nw; ++k) b = min(b, s_best[k]);
        if (b < INT_MAX) atomicMin(&L.qmin[q], b);
    }
    if (lane == 0) {
        atomicAdd(&L.ctr->sweeps, st.sweeps);
        atomicAdd(&L.ctr->dependent, st.dependent);
        atomicAdd(&L.ctr->exact_points, st.exact);
        atomicAdd(&L.ctr->tight, st.tight);
        atomicAdd(&L.ctr->errors, st.errors);
    }
}

/* ====================================================================== */
/* finalize                                                                */
/* ====================================================================== */

__global__ void td_k_finalize(TdLaunch L)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= L.nq) return;
    const TdQuery &Q = L.q[q];
    int r;
    if (Q.direct >= 0) {
        r = Q.direct;
    } else if (Q.direct == TD_DIRECT_WIDE) {
        r = INT_MIN; /* the wide kernel did not answer it: an error */
        atomicAdd(&L.ctr->errors, 1ull);
    } else if (L.qmin[q] == INT_MAX) {
        /* no independent subset in this shard's (or slice's) range */
        const bool part = L.shard_count > 1 || L.sets[Q.set].slice_count > 1;
        r = part ? INT_MAX : -1;
        if (!part) atomicAdd(&L.ctr->errors, 1ull);
    } else {
        r = Q.Z + L.qmin[q];
    }
    L.out[q] = r;
}

/* ====================================================================== */
/* host-side launch helpers (called from td_api.cu)                        */
/* ====================================================================== */

size_t td_filtered_smem(int nmax, int pmax, int blog2, int warps)
{
    int nmaxp = td_pow2_at_least(nmax);
    nmaxp = nmaxp < 128 ? 128 : nmaxp;
    /* ceil(pmax/2) planes of td_plane_pairs(nmax) pairs, 16 bytes each,
     * shared by the CTA; for the D = 2 kernel (pmax = 2) one plane per warp */
    const size_t hbytes = (size_t)((1 << blog2) + 4) * 4;
    size_t rbytes = hbytes;
    const size_t cbytes = (size_t)TD_COARSE_WORDS * 4 * td_coarse_tables(pmax);
    if (rbytes < cbytes) rbytes = cbytes;
    size_t per_warp = td_warp_region_bytes(rbytes);
    if (pmax == 2) return (td_staging_bytes(nmax, 1) + per_warp) * warps;
    return td_staging_bytes(nmax, (pmax + 1) / 2) + per_warp * warps;
}

size_t td_plain_smem(int nmax, int pmax, int warps)
{
    int nmaxp = td_pow2_at_least(nmax);
    int PSI = pmax <= 4 ? 4 : 8;
    size_t off = ((size_t)nmax * PSI * 4 + 15) & ~(size_t)15;
    size_t per_warp = ((size_t)nmaxp * 16 + (size_t)nmaxp * 2 + 16 + TD_WARP_META_BYTES + 15) & ~(size_t)15;
    return off + per_warp * warps;
}

int64_t td_scratch_per_warp(int nmax) { return (td_scratch_bytes(td_pow2_at_least(nmax)) + 255) & ~(int64_t)255; }

/* the critical-direction kernel lays its scratch out for 2 td_pow2_at_least(nmax) points */
int64_t td_scratch_per_warp_critical(int nmax) { return td_scratch_per_warp(2 * td_pow2_at_least(nmax)); }

/* Set-up, then the data-direction bound (two launches): about 1216 CTAs
 * over the queries (eight per SM on 152 SMs), at least one per query and at
 * most 32 per query, each staging its query's rows (up to 2048 x p int32,
 * 48 KB; longer rows take the global-memory path). */
cudaError_t td_launch_setup(const TdLaunch &L, cudaStream_t s)
{
    td_k_setup<<<L.nq, 256, 0, s>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || L.nq <= 0) return e;
    const int split = std::max(1, std::min(32, (1216 + L.nq - 1) / L.nq));
    const int cap = 2048 * std::max(1, std::min(L.pmax, TD_MAXD)); /* rows of up to 2048 points */
    td_k_bound<<<L.nq * split, 256, (size_t)cap * 4, s>>>(L, split, cap);
    return cudaGetLastError();
}

cudaError_t td_launch_tiles(const TdLaunch &L, cudaStream_t s)
{
    td_k_tiles<<<1, 1024, 0, s>>>(L);
    return cudaGetLastError();
}

/* The dynamic shared memory attribute is set to exactly what a launch uses
 * (td_prepare_*), before any stream capture; the launches do not touch it. */
typedef void (*td_kfn)(TdLaunch);
typedef void (*td_kfn_plain)(TdLaunch, int);

static td_kfn td_filtered_fn(int D)
{
    switch (D) {
    case 2: return td_k_filtered<2>;
    case 3: return td_k_filtered<3>;
    case 4: return td_k_filtered<4>;
    case 5: return td_k_filtered<5>;
    default: return td_k_filtered<6>;
    }
}

static td_kfn_plain td_plain_fn(int D)
{
    switch (D) {
    case 2: return td_k_plain<2>;
    case 3: return td_k_plain<3>;
    case 4: return td_k_plain<4>;
    case 5: return td_k_plain<5>;
    default: return td_k_plain<6>;
    }
}

/* The dynamic shared-memory limit of a kernel is a property of the kernel
 * on the current device, shared by every context, stream and entry point of
 * the process.  It is only ever raised: a call that needs less leaves it
 * where it is, so that a launch another host thread has sized for more is
 * never invalidated between its own attribute call and its launch. */
static std::mutex g_attr_mu;
static std::map<std::pair<int, const void *>, size_t> g_attr_smem;

static cudaError_t td_raise_smem(const void *fn, size_t smem)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    size_t &cur = g_attr_smem[std::make_pair(dev, fn)];
    if (smem <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) cur = smem;
    return e;
}

cudaError_t td_prepare_filtered(int D, size_t smem) { return td_raise_smem((const void *)td_filtered_fn(D), smem); }

cudaError_t td_prepare_plain(int D, size_t smem) { return td_raise_smem((const void *)td_plain_fn(D), smem); }

cudaError_t td_launch_filtered(int D, const TdLaunch &L, int grid, size_t smem, cudaStream_t s)
{
    td_filtered_fn(D)<<<grid, L.warps * 32, smem, s>>>(L);
    return cudaGetLastError();
}

cudaError_t td_launch_plain(int D, const TdLaunch &L, int q, int grid, size_t smem, cudaStream_t s)
{
    td_plain_fn(D)<<<grid, L.warps * 32, smem, s>>>(L, q);
    return cudaGetLastError();
}

/* Algorithm 3 search kernel: the warp form (the D-1 subsets of a node in
 * parallel warps) serves rows of at most 256 points, the block form (each
 * subset by the whole block) longer ones; dynamic shared memory of each. */
bool td_adia_warp_form(int nmax) { return td_pow2_at_least(nmax) <= 256; }

size_t td_adia_smem(int nmax, int D)
{
    const int nmaxp = td_pow2_at_least(nmax);
    const int nwords = nmaxp >> 5;
    const int PSI = D <= 4 ? 4 : 8;
    size_t off = ((size_t)nmax * PSI * 4 + 15) & ~(size_t)15;
    off += ((size_t)nmaxp * 2 + 15) & ~(size_t)15;
    off += ((size_t)nwords * 4 + 15) & ~(size_t)15;
    off += ((size_t)(nwords + 1) * 4 + 15) & ~(size_t)15;
    return off + td_adia_eval_bytes(nmaxp) * (size_t)(td_adia_warp_form(nmax) ? D - 1 : 1);
}

/* global scratch slots (warps) per CTA of the search kernel */
int td_adia_scratch_slots(int nmax) { return td_adia_warp_form(nmax) ? TD_ADIA_THREADS / 32 : 1; }

typedef void (*td_kfn_adia)(TdLaunch);

static td_kfn_adia td_adia_fn(int D, bool warp)
{
    switch (D) {
    case 3: return warp ? td_k_adia<3, true> : td_k_adia<3, false>;
    case 4: return warp ? td_k_adia<4, true> : td_k_adia<4, false>;
    case 5: return warp ? td_k_adia<5, true> : td_k_adia<5, false>;
    default: return warp ? td_k_adia<6, true> : td_k_adia<6, false>;
    }
}

/* the wide kernel: grid, shared memory, launch (every query of the call
 * is looked at; only those flagged TD_DIRECT_WIDE cost work) */
size_t td_wide_smem_for(int nmax) { return td_wide_smem(nmax); }

cudaError_t td_launch_wide(const TdLaunch &L, int sms, cudaStream_t s)
{
    const size_t smem = td_wide_smem(L.nmax);
    cudaError_t e = td_raise_smem((const void *)td_k_wide, smem);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(L.nq, sms));
    td_k_wide<<<grid, TD_WIDE_THREADS, smem, s>>>(L);
    return cudaGetLastError();
}

int td_adia_occupancy(int D, int nmax, size_t smem)
{
    int blocks = 0;
    const td_kfn_adia fn = td_adia_fn(D, td_adia_warp_form(nmax));
    if (td_raise_smem((const void *)fn, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, TD_ADIA_THREADS, smem) != cudaSuccess) return 0;
    return blocks;
}

cudaError_t td_launch_adia(int D, const TdLaunch &L, int grid, size_t smem, cudaStream_t s)
{
    td_adia_fn(D, td_adia_warp_form(L.nmax))<<<grid, TD_ADIA_THREADS, smem, s>>>(L);
    return cudaGetLastError();
}

int64_t td_adia_ws_entries() { return TD_ADIA_CAP; }

/* critical-direction kernel (d = 2..6): shared memory, occupancy, launch */
size_t td_critical_smem(int nmax, int pmax)
{
    const int PSI = pmax <= 4 ? 4 : 8;
    return (((size_t)nmax * PSI * 4 + 15) & ~(size_t)15) + (size_t)td_pow2_at_least(nmax) * 2;
}

static td_kfn_plain td_critical_fn(int D)
{
    switch (D) {
    case 2: return td_k_critical<2>;
    case 3: return td_k_critical<3>;
    case 4: return td_k_critical<4>;
    case 5: return td_k_critical<5>;
    default: return td_k_critical<6>;
    }
}

int td_critical_occupancy(int D, size_t smem)
{
    int blocks = 0;
    if (td_raise_smem((const void *)td_critical_fn(D), smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, td_critical_fn(D), TD_CRIT_THREADS, smem) != cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t td_launch_critical(int D, const TdLaunch &L, int q, int grid, size_t smem, cudaStream_t s)
{
    td_critical_fn(D)<<<grid, TD_CRIT_THREADS, smem, s>>>(L, q);
    return cudaGetLastError();
}

int td_critical_threads() { return TD_CRIT_THREADS; }

cudaError_t td_launch_finalize(const TdLaunch &L, cudaStream_t s)
{
    td_k_finalize<<<(L.nq + 255) / 256, 256, 0, s>>>(L);
    return cudaGetLastError();
}

int td_filtered_occupancy(int D, int warps, size_t smem)
{
    int blocks = 0;
    if (td_prepare_filtered(D, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, td_filtered_fn(D), warps * 32, smem) != cudaSuccess)
        return 0;
    return blocks;
}

int td_plain_occupancy(int D, int warps, size_t smem)
{
    int blocks = 0;
    if (td_prepare_plain(D, smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, td_plain_fn(D), warps * 32, smem) != cudaSuccess)
        return 0;
    return blocks;
}
