/*
 * td_wide.cuh -- the exact path for int32 data beyond td_coord_limit(p)
 * (included by td_kernels.cu).
 *
 * The fast kernels keep every exact intermediate in 64- or 128-bit integers,
 * which bounds the centred coordinates (td_coord_limit).  A query beyond that
 * bound (|X_ij - z_j| up to 2^32 - 1) is flagged by the set-up kernel and
 * answered here with 256-bit integers, by Proposition 1 (Section 2) with
 * r = p - 1 applied recursively -- the form whose predicates are only signs
 * of determinants of original coordinates, so that every intermediate stays
 * below 2^256:
 *
 *   OD_k(P) = min over the (k-1)-subsets F of P spanning a hyperplane H_F of
 *             min(#{x in P : n_F.x < 0}, #{x in P : n_F.x > 0})
 *             + OD_{k-1}(P on H_F)   (only when H_F holds more than F),
 *   OD_1(P) = min(#{x > 0}, #{x < 0}),
 *
 * where n_F.x = det[x_F | x] and the points of P on H_F are taken in the k-1
 * coordinates other than one where n_F is nonzero (injective on H_F).  OD_k
 * is the least number of the nonzero points P (of rank k) strictly on the
 * negative side of a generic direction, the open depth; the depth count is
 * T = Z + OD_d over the nonzero centred points in d pivot coordinates (d
 * their rank, reading R7).  Every set a level sees contains the subset that
 * defines it, so its rank is full and some F is independent.  The largest
 * values: a cofactor n_F,j is a 5x5 determinant of entries below 2^33
 * (< 5! 2^165 < 2^172), n_F.x below 6 2^205 < 2^208.
 *
 * One CTA per query (128 threads): the warps share the top-level subsets F;
 * a warp computes the normal (lane j a cofactor), the signs of every point
 * (lanes over points), and, when H_F holds more than F, the open depth of its
 * points one level down, alone, with the on-hyperplane lists of each level in
 * its own shared memory.  Cost: C(n', d-1) n' determinant-sign evaluations at
 * the top level -- one order of n above Algorithm 1, for the rare inputs that
 * need it.
 */

#define TD_WIDE_THREADS 128
#define TD_WIDE_WARPS (TD_WIDE_THREADS / 32)
#define TD_WIDE_LEVELS 5 /* on-hyperplane lists of dimensions 5, 4, 3, 2, 1 */

/* 256-bit two's complement integer, eight 32-bit limbs (w[0] least
 * significant).  Sums and products are taken modulo 2^256, which is exact
 * while the true values stay below 2^255 in magnitude (here below 2^208). */
struct TdW {
    uint32_t w[8];
};

__device__ __forceinline__ TdW td_w_from(td_i128 v)
{
    TdW r;
    const uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
    r.w[0] = (uint32_t)lo;
    r.w[1] = (uint32_t)(lo >> 32);
    r.w[2] = (uint32_t)hi;
    r.w[3] = (uint32_t)(hi >> 32);
    const uint32_t s = v < 0 ? 0xFFFFFFFFu : 0u;
#pragma unroll
    for (int i = 4; i < 8; ++i) r.w[i] = s;
    return r;
}

__device__ __forceinline__ TdW td_w_add(const TdW &a, const TdW &b)
{
    TdW r;
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c += (uint64_t)a.w[i] + b.w[i];
        r.w[i] = (uint32_t)c;
        c >>= 32;
    }
    return r;
}

__device__ __forceinline__ TdW td_w_neg(const TdW &a)
{
    TdW r;
    uint64_t c = 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c += (uint64_t)(~a.w[i]);
        r.w[i] = (uint32_t)c;
        c >>= 32;
    }
    return r;
}

/* a * b for |b| < 2^63: a times |b| (two limbs) modulo 2^256, negated for
 * b < 0 */
__device__ __forceinline__ TdW td_w_mul(const TdW &a, int64_t b)
{
    const uint64_t m = b < 0 ? (uint64_t)(-b) : (uint64_t)b;
    const uint32_t m0 = (uint32_t)m, m1 = (uint32_t)(m >> 32);
    uint32_t r[8] = { 0, 0, 0, 0, 0, 0, 0, 0 };
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        c += (uint64_t)a.w[i] * m0 + r[i];
        r[i] = (uint32_t)c;
        c >>= 32;
    }
    c = 0;
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        c += (uint64_t)a.w[i] * m1 + r[i + 1];
        r[i + 1] = (uint32_t)c;
        c >>= 32;
    }
    TdW o;
#pragma unroll
    for (int i = 0; i < 8; ++i) o.w[i] = r[i];
    return b < 0 ? td_w_neg(o) : o;
}

__device__ __forceinline__ int td_w_sign(const TdW &a)
{
    if ((int32_t)a.w[7] < 0) return -1;
    uint32_t o = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) o |= a.w[i];
    return o != 0;
}

/* det of the N x N matrix a[r][c] = x[rows[r]] of point cols[c]: points are
 * rows of xs (8 coordinates apart), entries below 2^33.  N <= 3 exactly in
 * 128 bits (below 6 2^99), larger N by expansion along the first row. */
template <int N>
__device__ TdW td_w_det(const int64_t *xs, const int (&rows)[6], const int (&cols)[6])
{
    auto e = [&](int r, int c) -> td_i128 { return (td_i128)xs[8 * cols[c] + rows[r]]; };
    if constexpr (N == 1) {
        return td_w_from(e(0, 0));
    } else if constexpr (N == 2) {
        return td_w_from(e(0, 0) * e(1, 1) - e(0, 1) * e(1, 0));
    } else if constexpr (N == 3) {
        const td_i128 d = e(0, 0) * (e(1, 1) * e(2, 2) - e(1, 2) * e(2, 1)) -
                          e(0, 1) * (e(1, 0) * e(2, 2) - e(1, 2) * e(2, 0)) +
                          e(0, 2) * (e(1, 0) * e(2, 1) - e(1, 1) * e(2, 0));
        return td_w_from(d);
    } else {
        TdW acc = td_w_from(0);
        int sr[6], sc[6];
#pragma unroll
        for (int r = 1; r < N; ++r) sr[r - 1] = rows[r];
#pragma unroll 1
        for (int c = 0; c < N; ++c) {
            int o = 0;
#pragma unroll
            for (int cc = 0; cc < N; ++cc)
                if (cc != c) sc[o++] = cols[cc];
            const TdW t = td_w_mul(td_w_det<N - 1>(xs, sr, sc), xs[8 * cols[c] + rows[0]]);
            acc = (c & 1) ? td_w_add(acc, td_w_neg(t)) : td_w_add(acc, t);
        }
        return acc;
    }
}

__device__ __forceinline__ TdW td_w_det_rt(int n, const int64_t *xs, const int (&rows)[6], const int (&cols)[6])
{
    switch (n) {
    case 1: return td_w_det<1>(xs, rows, cols);
    case 2: return td_w_det<2>(xs, rows, cols);
    case 3: return td_w_det<3>(xs, rows, cols);
    case 4: return td_w_det<4>(xs, rows, cols);
    case 5: return td_w_det<5>(xs, rows, cols);
    default: return td_w_det<6>(xs, rows, cols);
    }
}

/* C(p, k) for 0 <= k <= p <= 6 */
__device__ __forceinline__ int td_small_binom(int p, int k)
{
    if (k < 0 || k > p) return 0;
    int r = 1;
    for (int i = 0; i < k; ++i) r = r * (p - i) / (i + 1);
    return r;
}

/* the t-th k-subset of {0..p-1} in lexicographic order (t < C(p, k)) */
__device__ __forceinline__ bool td_lex_subset(int p, int k, int t, int (&s)[6])
{
    for (int i = 0; i < k; ++i) s[i] = i;
    for (int step = 0; step < t; ++step) {
        int i = k - 1;
        while (i >= 0 && s[i] == p - k + i) --i;
        if (i < 0) return false;
        ++s[i];
        for (int j = i + 1; j < k; ++j) s[j] = s[j - 1] + 1;
    }
    return true;
}

template <int K>
__device__ int td_wide_od(const int64_t *xs, const uint16_t *idx, int t, const int (&coords)[6], uint16_t *lst,
                          int nmax, TdW *wn, int lane);

/* The value of the (K-1)-subset F (indices into the point list idx, or
 * into the points themselves when idx is null) within the K coordinates
 * coords: min of the strict sides of its hyperplane plus, when the
 * hyperplane holds more than F, the open depth of its points one level
 * down.  INT_MAX when F is dependent; any value >= cap when the strict
 * sides alone reach cap.  The points on the hyperplane are listed in lst. */
template <int K>
__device__ int td_wide_eval(const int64_t *xs, const uint16_t *idx, int t, const int (&coords)[6],
                            const int (&F)[6], uint16_t *lst, int nmax, TdW *wn, int lane, int cap)
{
    /* the normal: n_j = (-1)^(j+K-1) det of F's points without coordinate j */
    if (lane < K) {
        int rows[6], cols[6];
        int o = 0;
#pragma unroll
        for (int r = 0; r < K; ++r)
            if (r != lane) rows[o++] = coords[r];
#pragma unroll
        for (int c = 0; c < K - 1; ++c) cols[c] = idx ? idx[F[c]] : F[c];
        TdW n = td_w_det_rt(K - 1, xs, rows, cols);
        wn[lane] = ((lane + K - 1) & 1) ? td_w_neg(n) : n;
    }
    __syncwarp();
    TdW n[K];
    int jstar = -1;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        n[j] = wn[j];
        if (jstar < 0 && td_w_sign(n[j]) != 0) jstar = j;
    }
    __syncwarp();
    if (jstar < 0) return INT_MAX; /* F dependent */
    int neg = 0, pos = 0, on = 0;
    const unsigned below = (1u << lane) - 1u;
    for (int i0 = 0; i0 < t; i0 += 32) {
        const int i = i0 + lane;
        int s = 2;
        if (i < t) {
            const int64_t *x = xs + 8 * (idx ? idx[i] : i);
            TdW acc = td_w_mul(n[0], x[coords[0]]);
#pragma unroll
            for (int j = 1; j < K; ++j) acc = td_w_add(acc, td_w_mul(n[j], x[coords[j]]));
            s = td_w_sign(acc);
        }
        neg += s == -1;
        pos += s == 1;
        const unsigned b = __ballot_sync(TD_FULL, s == 0);
        if (s == 0) lst[on + __popc(b & below)] = (uint16_t)(idx ? idx[i] : i);
        on += __popc(b);
    }
    __syncwarp();
    neg = td_wsum(neg);
    pos = td_wsum(pos);
    int v = min(neg, pos);
    if (v >= cap || on <= K - 1) return v;
    if constexpr (K >= 2) {
        int c2[6];
        int o = 0;
#pragma unroll
        for (int r = 0; r < K; ++r)
            if (r != jstar) c2[o++] = coords[r];
        v += td_wide_od<K - 1>(xs, lst, on, c2, lst + nmax, nmax, wn, lane);
    }
    return v;
}

/* OD_K of the t points idx[0..t) in the coordinates coords (rank K). */
template <int K>
__device__ int td_wide_od(const int64_t *xs, const uint16_t *idx, int t, const int (&coords)[6], uint16_t *lst,
                          int nmax, TdW *wn, int lane)
{
    if constexpr (K == 1) {
        int pos = 0, neg = 0;
        for (int i = lane; i < t; i += 32) {
            const int64_t v = xs[8 * idx[i] + coords[0]];
            pos += v > 0;
            neg += v < 0;
        }
        return min(td_wsum(pos), td_wsum(neg));
    } else {
        int best = INT_MAX;
        int F[6] = { 0, 1, 2, 3, 4, 5 };
        while (F[K - 2] < t) {
            best = min(best, td_wide_eval<K>(xs, idx, t, coords, F, lst, nmax, wn, lane, best));
            /* lexicographic successor of F among the (K-1)-subsets of [0, t) */
            int i = K - 2;
            while (i >= 0 && F[i] == t - (K - 1) + i) --i;
            if (i < 0) break;
            ++F[i];
            for (int j = i + 1; j < K - 1; ++j) F[j] = F[j - 1] + 1;
        }
        return best;
    }
}

/* The top level for effective dimension D: the warps of the CTA share the
 * (D-1)-subsets of the nnz points (colex ranks, strided).  Returns the
 * warp's minimum. */
template <int D>
__device__ int td_wide_top(const int64_t *xs, int nnz, const int (&coords)[6], uint16_t *lst, int nmax, TdW *wn,
                           int lane, int w)
{
    constexpr int K1 = D - 1;
    const uint64_t total = td_binom(nnz, K1);
    int best = INT_MAX;
    for (uint64_t r = (uint64_t)w; r < total; r += TD_WIDE_WARPS) {
        int c[K1 > 0 ? K1 : 1];
        td_unrank_colex<K1>(r, nnz, c);
        int F[6] = { 0, 0, 0, 0, 0, 0 };
#pragma unroll
        for (int i = 0; i < K1; ++i) F[i] = c[i];
        best = min(best, td_wide_eval<D>(xs, nullptr, nnz, coords, F, lst, nmax, wn, lane, best));
    }
    return best;
}

/* Shared memory of td_k_wide: the staged points (8 int64 coordinates
 * each), the per-warp lists of every level and the per-warp normals. */
size_t td_wide_smem(int nmax)
{
    return (size_t)nmax * 64 + (size_t)TD_WIDE_WARPS * TD_WIDE_LEVELS * nmax * 2 + TD_WIDE_WARPS * 6 * sizeof(TdW) + 256;
}

/* Every query flagged TD_DIRECT_WIDE by the set-up kernel: the depth count
 * into Q.direct (the finalize kernel writes it out).  Grid: any number of
 * CTAs, each takes queries q = blockIdx.x, blockIdx.x + gridDim.x, ... */
__global__ void __launch_bounds__(TD_WIDE_THREADS) td_k_wide(TdLaunch L)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_tmp[TD_WIDE_WARPS], s_d, s_piv[6], s_best, s_cnt, s_pn[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nmax = L.nmax;
    int64_t *xs = reinterpret_cast<int64_t *>(smem);
    uint16_t *lists = reinterpret_cast<uint16_t *>(smem + (size_t)nmax * 64);
    TdW *wn = reinterpret_cast<TdW *>(smem + (size_t)nmax * 64 + (size_t)TD_WIDE_WARPS * TD_WIDE_LEVELS * nmax * 2);
    uint16_t *lst = lists + (size_t)w * TD_WIDE_LEVELS * nmax;
    TdW *wnw = wn + 6 * w;
    /* the set-up kernel counted the flagged queries: none, nothing to walk */
    if (*reinterpret_cast<volatile unsigned long long *>(&L.ctr->wide) == 0ull) return;
    for (int q = blockIdx.x; q < L.nq; q += gridDim.x) {
        TdQuery *Q = &L.q[q];
        if (Q->direct != TD_DIRECT_WIDE) continue; /* uniform over the CTA */
        const TdSet S = L.sets[Q->set];
        const int n = S.n, p = S.p;
        if (n > nmax) {
            if (threadIdx.x == 0) atomicAdd(&L.ctr->errors, 1ull);
            continue;
        }
        const int32_t *X = L.X + S.x_off;
        const int32_t *z = L.Zq + (int64_t)q * TD_MAXD;
        /* stage the nonzero centred points in data order (block compaction) */
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        for (int i0 = 0; i0 < n; i0 += TD_WIDE_THREADS) {
            const int i = i0 + (int)threadIdx.x;
            bool nz = false;
            int64_t v[6] = { 0, 0, 0, 0, 0, 0 };
            if (i < n)
                for (int c = 0; c < p; ++c) {
                    v[c] = (int64_t)X[(int64_t)i * p + c] - z[c];
                    nz |= v[c] != 0;
                }
            const unsigned b = __ballot_sync(TD_FULL, nz);
            if (lane == 0) s_tmp[w] = __popc(b);
            __syncthreads();
            int base = s_cnt;
            for (int k = 0; k < w; ++k) base += s_tmp[k];
            if (nz) {
                int64_t *dst = xs + 8 * (base + __popc(b & ((1u << lane) - 1u)));
                for (int c = 0; c < 8; ++c) dst[c] = c < p ? v[c] : 0;
            }
            __syncthreads();
            if (threadIdx.x == 0)
                for (int k = 0; k < TD_WIDE_WARPS; ++k) s_cnt += s_tmp[k];
            __syncthreads();
        }
        const int nnz = s_cnt;
        /* rank and pivot coordinates (reading R7), warp 0: a point joins the
         * independent set when some minor of the enlarged set is nonzero; the
         * pivots are the lexicographically first coordinates whose minor of
         * the independent set is nonzero */
        if (w == 0) {
            int sel[6] = { 0, 0, 0, 0, 0, 0 };
            int r = 0;
            for (int i = 0; i < nnz && r < p; ++i) {
                sel[r] = i;
                const int nsub = td_small_binom(p, r + 1);
                bool nzm = false;
                int rows[6];
                if (lane < nsub && td_lex_subset(p, r + 1, lane, rows))
                    nzm = td_w_sign(td_w_det_rt(r + 1, xs, rows, sel)) != 0;
                if (__any_sync(TD_FULL, nzm)) ++r;
            }
            const int nsub = td_small_binom(p, r);
            bool nzm = false;
            int rows[6] = { 0, 1, 2, 3, 4, 5 };
            if (r > 0 && lane < nsub && td_lex_subset(p, r, lane, rows))
                nzm = td_w_sign(td_w_det_rt(r, xs, rows, sel)) != 0;
            const unsigned bm = __ballot_sync(TD_FULL, nzm);
            const int first = bm ? __ffs(bm) - 1 : 0;
            int prow[6] = { 0, 1, 2, 3, 4, 5 };
            if (r > 0) td_lex_subset(p, r, first, prow);
            if (lane == 0) {
                s_d = r;
                for (int c = 0; c < 6; ++c) s_piv[c] = prow[c];
                s_best = INT_MAX;
            }
        }
        __syncthreads();
        const int d = s_d;
        int coords[6];
        for (int c = 0; c < 6; ++c) coords[c] = s_piv[c];
        const int Z = n - nnz;
        int T;
        if (nnz == 0) {
            T = n;
        } else if (d == 1) {
            /* the p = 1 case of Section 3 along the one pivot coordinate */
            int pos = 0, neg = 0;
            for (int i = threadIdx.x; i < nnz; i += TD_WIDE_THREADS) {
                pos += xs[8 * i + coords[0]] > 0;
                neg += xs[8 * i + coords[0]] < 0;
            }
            pos = td_wsum(pos);
            neg = td_wsum(neg);
            if (threadIdx.x == 0) s_pn[0] = s_pn[1] = 0;
            __syncthreads();
            if (lane == 0) {
                atomicAdd(&s_pn[0], pos);
                atomicAdd(&s_pn[1], neg);
            }
            __syncthreads();
            T = Z + min(s_pn[0], s_pn[1]);
        } else {
            int wb = INT_MAX;
            switch (d) {
            case 2: wb = td_wide_top<2>(xs, nnz, coords, lst, nmax, wnw, lane, w); break;
            case 3: wb = td_wide_top<3>(xs, nnz, coords, lst, nmax, wnw, lane, w); break;
            case 4: wb = td_wide_top<4>(xs, nnz, coords, lst, nmax, wnw, lane, w); break;
            case 5: wb = td_wide_top<5>(xs, nnz, coords, lst, nmax, wnw, lane, w); break;
            default: wb = td_wide_top<6>(xs, nnz, coords, lst, nmax, wnw, lane, w); break;
            }
            if (lane == 0) atomicMin(&s_best, wb);
            __syncthreads();
            T = s_best == INT_MAX ? -1 : Z + s_best;
        }
        if (threadIdx.x == 0) {
            if (T < 0) atomicAdd(&L.ctr->errors, 1ull);
            else Q->direct = T;
        }
        __syncthreads();
    }
}
