/*
 * td_adia.cuh -- Algorithm 3 (ADIA, Section 4) on the device; included by
 * td_kernels.cu after the exact sweep helpers it uses.
 *
 * td_k_adia<D, WARP> runs Steps 2-4 and Step 5(a) for the queries of
 * effective dimension D (persistent CTAs of 256 threads, one query at a time
 * per CTA, in work order), and hands Step 5(b) to the filtered sweep: it
 * writes the staging order of
 * the query's nonzero points with the union of Step 5(a) first, the subset
 * range [0, C(|union|, D-2)) and the running minimum d0, so that the sweep
 * visits exactly the subsets of the union and returns min(d0, their V(S)).
 *
 * Readings (the paper states Algorithm 3 for data in general position and
 * fixes no order for its choices):
 *   - depths are counts V(S) (the paper's D_n(S) - (p-2)/n), exact;
 *   - the critical points of S (Step 2(c), Step 4(a)(ii)) are the points
 *     whose projected line bounds a cell of the quotient's line arrangement
 *     whose count is G(S);
 *   - the subsets of a node are taken in lexicographic order, critical points
 *     in increasing index, N is a stack, nodes are identified by their index
 *     set and "not in Q" ignores deleted nodes;
 *   - Step 2 ranks the data directions +-x_j by #{i : u'x_i <= 0} in the
 *     input coordinates, ties to the smaller j and then to +x_j; its order
 *     is by u'x_i, ties by index; when no nonzero point has u'x_i <= 0 the
 *     result is Z; the start subset is taken greedily after the negative
 *     points (wrapping round), skipping dependent points; Step 2(c) takes the
 *     critical point of least index;
 *   - Step 5(a): X_F is the closed side of the hyperplane through 0 and F
 *     with fewer points, or on a tie the side holding the point of least
 *     index off the hyperplane;
 *   - with no more than 2D nonzero points (the paper's n <= 2p) the query
 *     keeps the full subset range (Algorithm 1).
 * A query whose search needs more than TD_ADIA_CAP nodes or TD_ADIA_MAX_POPS
 * iterations keeps the full subset range too (the exact count) and is
 * counted in the fallback statistic.
 *
 * A subset is evaluated exactly (projections, comparison sort with the
 * FP32-filtered exact comparator, the count of every cell of the line
 * arrangement) either by one warp (WARP: rows of at most 256 points, the D-1
 * subsets of a node in parallel) or by the whole block (longer rows, the
 * subsets one after another).  A subset with V(S) > d0 changes nothing (its
 * nodes would be deleted by Step 4(b) before any later step reads them, and
 * two subsets of one node cannot produce the same node), so the critical set
 * and the exact tight correction are computed only when G(S) <= d0, and
 * thread 0 applies (iii) and (iv) in lexicographic order, stopping at the
 * first subset that lowers d0 (the block form then evaluates no further
 * subset of the node).
 */

#define TD_ADIA_CAP_LOG2 11
#define TD_ADIA_CAP (1 << TD_ADIA_CAP_LOG2)
#define TD_ADIA_MAX_POPS 20000
#define TD_ADIA_THREADS 256

/* Node key: the sorted point indices (< 4096), 12 bits each, shifted left
 * by one with the low bit set (0 marks an empty slot). */
__device__ __forceinline__ uint64_t td_adia_pack(const int *idx, int k1)
{
    uint64_t v = 0;
    for (int j = 0; j < k1; ++j) v |= (uint64_t)idx[j] << (12 * j);
    return (v << 1) | 1ull;
}

__device__ __forceinline__ void td_adia_unpack(uint64_t key, int *idx, int k1)
{
    key >>= 1;
    for (int j = 0; j < k1; ++j) idx[j] = (int)((key >> (12 * j)) & 0xFFF);
}

/* Insert (or revive) a node in the open-addressing table.  Returns its slot
 * when it was absent or deleted, -1 when a live node holds the key, -2 when
 * the table is full. */
__device__ int td_adia_insert(uint64_t *keys, int32_t *dep, uint64_t key, int depth)
{
    const unsigned h = (unsigned)((key * 0x9E3779B97F4A7C15ull) >> (64 - TD_ADIA_CAP_LOG2));
    for (int probe = 0; probe < TD_ADIA_CAP; ++probe) {
        const unsigned s = (h + (unsigned)probe) & (TD_ADIA_CAP - 1);
        const uint64_t k = keys[s];
        if (k == 0) {
            keys[s] = key;
            dep[s] = depth;
            return (int)s;
        }
        if (k == key) {
            if (dep[s] >= 0) return -1;
            dep[s] = depth;
            return (int)s;
        }
    }
    return -2;
}

/* Rank of cnt rows (length d) by fraction-free elimination in __int128. */
__device__ int td_adia_rank(const int64_t (*rows)[TD_MAXD], int cnt, int d)
{
    td_i128 m[TD_MAXD][TD_MAXD];
    for (int r = 0; r < cnt; ++r)
        for (int c = 0; c < d; ++c) m[r][c] = rows[r][c];
    int rank = 0;
    for (int c = 0; c < d && rank < cnt; ++c) {
        int piv = -1;
        for (int r = rank; r < cnt; ++r)
            if (m[r][c] != 0) { piv = r; break; }
        if (piv < 0) continue;
        for (int cc = 0; cc < d; ++cc) {
            td_i128 t = m[rank][cc];
            m[rank][cc] = m[piv][cc];
            m[piv][cc] = t;
        }
        for (int r = rank + 1; r < cnt; ++r) {
            td_i128 f = m[r][c], e = m[rank][c];
            td_i128 g = 0;
            for (int cc = 0; cc < d; ++cc) {
                m[r][cc] = e * m[r][cc] - f * m[rank][cc];
                g = td_i128_gcd(g, m[r][cc]);
            }
            if (g > 1)
                for (int cc = 0; cc < d; ++cc) m[r][cc] = td_i128_div_exact(m[r][cc], g);
        }
        ++rank;
    }
    return rank;
}

/* Shared buffers of one subset evaluation (nmaxp points): H (exact
 * projections, int64 pairs) | Hf (their binary32 copies) | idx (sort list) |
 * gcount | basis and meta rows | crit (critical-point bits) | cell flags. */
__host__ __device__ inline size_t td_adia_crit_off(int nmaxp)
{
    return (size_t)nmaxp * 26 + 16 + TD_WARP_META_BYTES;
}

__host__ __device__ inline size_t td_adia_eval_bytes(int nmaxp)
{
    return (td_adia_crit_off(nmaxp) + (size_t)(nmaxp >> 3) + (size_t)nmaxp + 16 + 15) & ~(size_t)15;
}

/* Block-wide exclusive prefix sum of v and the total (s_w: 32 ints). */
__device__ __forceinline__ int td_block_excl(int v, int *s_w, int &tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int inc = td_wscan_incl(v, lane);
    __syncthreads();
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    int base = 0, t = 0;
    for (int k = 0; k < nw; ++k) {
        const int x = s_w[k];
        base += k < w ? x : 0;
        t += x;
    }
    tot = t;
    return base + inc - v;
}

/* Block-wide minimum (op 0) or maximum (op 1) of v (s_w: 32 ints). */
__device__ __forceinline__ int td_block_minmax(int v, int *s_w, int op)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int r = op ? td_wmax(v) : td_wmin(v);
    __syncthreads();
    if (lane == 0) s_w[w] = r;
    __syncthreads();
    int t = s_w[0];
    for (int k = 1; k < nw; ++k) t = op ? max(t, s_w[k]) : min(t, s_w[k]);
    return t;
}

/* Bitonic sort of idx[0..npad) by increasing line direction with the whole
 * block, FP32-filtered exact comparisons (td_cross_sign_f).  For strides up
 * to 32 the pairs of a warp stay inside the warp's own 64-entry windows in
 * every step, so those steps are separated by warp barriers only. */
__device__ void td_sort_block(uint16_t *idx, int npad, const int64_t *H, const float2 *Hf)
{
    const int half = npad >> 1, T = blockDim.x;
    for (int size = 2; size <= npad; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t0 = threadIdx.x; t0 < half; t0 += 2 * T) {
                int ii[2], cr[2];
                uint16_t u[2], v[2];
                float2 fa[2], fb[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int tt = min(t0 + k * T, half - 1);
                    ii[k] = ((tt & ~(stride - 1)) << 1) | (tt & (stride - 1));
                    u[k] = idx[ii[k]];
                    v[k] = idx[ii[k] + stride];
                    fa[k] = Hf[u[k] == TD_SENT ? 0 : (u[k] & 0x7FFF)];
                    fb[k] = Hf[v[k] == TD_SENT ? 0 : (v[k] & 0x7FFF)];
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float p2 = fa[k].y * fb[k].x;
                    const float p1 = fa[k].x * fb[k].y;
                    const float c = fmaf(fa[k].x, fb[k].y, -p2);
                    const float bnd = (8.0f * TD_U) * (fabsf(p1) + fabsf(p2));
                    cr[k] = c > bnd ? 1 : (c < -bnd ? -1 : 2);
                    if (cr[k] == 2 && u[k] != TD_SENT && v[k] != TD_SENT) {
                        const int ia = u[k] & 0x7FFF, ib = v[k] & 0x7FFF;
                        cr[k] = td_cross_sign(H[2 * ia], H[2 * ia + 1], H[2 * ib], H[2 * ib + 1]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (t0 + k * T >= half) continue;
                    /* u before v iff u is valid and (v is padding or u x v > 0) */
                    const bool uv = u[k] != TD_SENT && (v[k] == TD_SENT || cr[k] == 1);
                    const bool vu = v[k] != TD_SENT && (u[k] == TD_SENT || cr[k] == -1);
                    const bool up = (ii[k] & size) == 0;
                    if (up ? vu : uv) {
                        idx[ii[k]] = v[k];
                        idx[ii[k] + stride] = u[k];
                    }
                }
            }
            if (stride > 32 || stride == 1) __syncthreads();
            else __syncwarp();
        }
}

/* Exact V(S) of one subset c (compact point indices) by one warp, and, when
 * G(S) <= d0, the critical points of S as bits crit[i >> 5] of the warp's
 * buffer (cleared first).  The projections are exact int64, the lines are
 * ordered by a comparison sort with the exact cross-product comparator, and
 * the walk reads the count of every cell of the line arrangement.  Returns
 * INT_MAX for a dependent subset; V(S) when G(S) <= d0, else G(S) (> d0). */
template <int D>
__device__ int td_adia_eval(const int32_t *xi, int PSI, int nnz, const int (&c)[D - 2], unsigned char *wb,
                            int nmaxp, const TdScratch &scr, int d0, int lane)
{
    constexpr int K = D - 2;
    int64_t *H = reinterpret_cast<int64_t *>(wb);
    float2 *Hf = reinterpret_cast<float2 *>(wb + (size_t)nmaxp * 16);
    uint16_t *idx = reinterpret_cast<uint16_t *>(wb + (size_t)nmaxp * 24);
    int *gcount = reinterpret_cast<int *>(wb + (size_t)nmaxp * 26);
    int64_t *wqa = reinterpret_cast<int64_t *>(wb + (size_t)nmaxp * 26 + 16);
    int64_t *wqb = wqa + TD_MAXD;
    int *wmeta = reinterpret_cast<int *>(wqb + TD_MAXD);
    uint32_t *crit = reinterpret_cast<uint32_t *>(wb + td_adia_crit_off(nmaxp));
    unsigned char *cell = reinterpret_cast<unsigned char *>(crit + (nmaxp >> 5));
    for (int i = lane; i < (nmaxp >> 5); i += 32) crit[i] = 0u;
    int64_t s[K][D];
#pragma unroll
    for (int j = 0; j < K; ++j)
#pragma unroll
        for (int t = 0; t < D; ++t) s[j][t] = xi[(size_t)c[j] * PSI + t];
    TdBasis<D> Bs;
    if (!td_make_basis<D>(s, Bs)) return INT_MAX;
    td_publish_basis<D>(Bs, c, wqa, wqb, wmeta, lane);
    /* exact projections; compacted list of the nonzero ones (orientation in bit 15) */
    int m = 0, t = 0;
    for (int i0 = 0; i0 < nnz; i0 += 32) {
        const int i = i0 + lane;
        int64_t y1 = 0, y2 = 0;
        const bool valid = i < nnz;
        if (valid) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const int64_t xv = xi[(size_t)i * PSI + k];
                y1 += Bs.qa[k] * xv;
                y2 += Bs.qb[k] * xv;
            }
        }
        const bool tight = valid && y1 == 0 && y2 == 0;
        const bool nonz = valid && !tight;
        int64_t h1 = 0, h2 = 0;
        bool plus = false;
        if (nonz) plus = td_normalise(y1, y2, h1, h2);
        if (valid) {
            H[2 * i] = h1;
            H[2 * i + 1] = h2;
            Hf[i] = make_float2(__ll2float_rn(h1), __ll2float_rn(h2));
        }
        const unsigned bn = __ballot_sync(TD_FULL, nonz);
        if (nonz) idx[m + __popc(bn & ((1u << lane) - 1u))] = (uint16_t)(i | (plus ? 0x8000 : 0));
        m += __popc(bn);
        t += __popc(__ballot_sync(TD_FULL, tight));
    }
    __syncwarp();
    int G = 0;
    if (m > 0) {
        const int npad = td_pow2_at_least(m);
        for (int l = m + lane; l < npad; l += 32) idx[l] = TD_SENT;
        __syncwarp();
        td_sort_exact_fast(idx, npad, H, lane, Hf);
        auto same_line = [&](int l0, int l1) -> bool {
            const int a = idx[l0] & 0x7FFF, b = idx[l1] & 0x7FFF;
            return td_cross_sign_f(Hf[a], Hf[b], H[2 * a], H[2 * a + 1], H[2 * b], H[2 * b + 1]) == 0;
        };
        int A = 0;
        for (int l = lane; l < m; l += 32) A += (idx[l] >> 15) & 1;
        A = td_wsum(A);
        const int C = (m + 31) >> 5;
        const int beg = min(lane * C, m), end = min(beg + C, m);
        int sev = 0, nst = 0;
        for (int l = beg; l < end; ++l) {
            sev += (idx[l] & 0x8000) ? -1 : 1;
            nst += (l == 0 || !same_line(l - 1, l)) ? 1 : 0;
        }
        const int vexcl = A + td_wscan_incl(sev, lane) - sev;
        const int gexcl = td_wscan_incl(nst, lane) - nst;
        /* walk value after each group = count of the cell that follows it;
         * A is the count of the cell before the first line (the same cell as
         * the one after the last line, turned by pi) */
        int v = vexcl, mn = A, mx = A;
        for (int l = beg; l < end; ++l) {
            v += (idx[l] & 0x8000) ? -1 : 1;
            if (l + 1 == m || !same_line(l, l + 1)) {
                mn = min(mn, v);
                mx = max(mx, v);
            }
        }
        G = min(td_wmin(mn), m - td_wmax(mx));
        if (G <= d0) {
            /* cell[g] = 1 when the cell before line group g has count G;
             * cell[L] (after the last group) equals cell[0] */
            if (lane == 0) cell[0] = (unsigned char)(min(A, m - A) == G);
            v = vexcl;
            int g = gexcl - 1;
            for (int l = beg; l < end; ++l) {
                v += (idx[l] & 0x8000) ? -1 : 1;
                if (l == 0 || !same_line(l - 1, l)) ++g;
                if (l + 1 == m || !same_line(l, l + 1)) cell[g + 1] = (unsigned char)(min(v, m - v) == G);
            }
            __syncwarp();
            g = gexcl - 1;
            for (int l = beg; l < end; ++l) {
                if (l == 0 || !same_line(l - 1, l)) ++g;
                if (cell[g] | cell[g + 1]) {
                    const int i = idx[l] & 0x7FFF;
                    atomicOr(&crit[i >> 5], 1u << (i & 31));
                }
            }
            __syncwarp();
        }
    }
    int V = G;
    if (t > K && G <= d0)
        V = G + td_tight_correction<D>(wmeta, nullptr, 0, xi, PSI, nnz, nullptr, H, scr, gcount, lane);
    return V;
}

/* Exact V(S) of one subset c (compact point indices, the same in every
 * thread) by the whole block, and, when G(S) <= d0, the critical points of S
 * as bits of crit (cleared first).  The projections are exact int64, the
 * lines are ordered by a comparison sort with the exact (FP32-filtered)
 * comparator, and the walk reads the count of every cell of the line
 * arrangement.  Returns, in every thread, INT_MAX for a dependent subset;
 * V(S) when G(S) <= d0, else G(S) (> d0). */
template <int D>
__device__ int td_adia_eval_block(const int32_t *xi, int PSI, int nnz, const int (&c)[D - 2], unsigned char *eb,
                                  int nmaxp, const TdScratch &scr, int d0, int *s_w, int *s_res)
{
    constexpr int K = D - 2;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, w = tid >> 5;
    int64_t *H = reinterpret_cast<int64_t *>(eb);
    float2 *Hf = reinterpret_cast<float2 *>(eb + (size_t)nmaxp * 16);
    uint16_t *idx = reinterpret_cast<uint16_t *>(eb + (size_t)nmaxp * 24);
    int *gcount = reinterpret_cast<int *>(eb + (size_t)nmaxp * 26);
    int64_t *wqa = reinterpret_cast<int64_t *>(eb + (size_t)nmaxp * 26 + 16);
    int64_t *wqb = wqa + TD_MAXD;
    int *wmeta = reinterpret_cast<int *>(wqb + TD_MAXD);
    uint32_t *crit = reinterpret_cast<uint32_t *>(eb + td_adia_crit_off(nmaxp));
    unsigned char *cell = reinterpret_cast<unsigned char *>(crit + (nmaxp >> 5));
    for (int i = tid; i < (nmaxp >> 5); i += T) crit[i] = 0u;
    /* the subset's basis, by warp 0, read by every thread from wqa / wqb */
    if (w == 0) {
        int64_t s[K][D];
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int t = 0; t < D; ++t) s[j][t] = xi[(size_t)c[j] * PSI + t];
        TdBasis<D> Bs;
        const bool ok = td_make_basis<D>(s, Bs);
        if (ok) td_publish_basis<D>(Bs, c, wqa, wqb, wmeta, lane);
        if (lane == 0) s_res[1] = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_res[1]) return INT_MAX; /* the same in every thread */
    int64_t qa[D], qb[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        qa[k] = wqa[k];
        qb[k] = wqb[k];
    }
    /* exact projections; compacted list of the nonzero ones (orientation in bit 15) */
    int m = 0, tcount = 0;
    for (int i0 = 0; i0 < nnz; i0 += T) {
        const int i = i0 + tid;
        int64_t y1 = 0, y2 = 0;
        const bool valid = i < nnz;
        if (valid) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const int64_t xv = xi[(size_t)i * PSI + k];
                y1 += qa[k] * xv;
                y2 += qb[k] * xv;
            }
        }
        const bool tight = valid && y1 == 0 && y2 == 0;
        const bool nonz = valid && !tight;
        int64_t h1 = 0, h2 = 0;
        bool plus = false;
        if (nonz) plus = td_normalise(y1, y2, h1, h2);
        if (valid) {
            H[2 * i] = h1;
            H[2 * i + 1] = h2;
            Hf[i] = make_float2(__ll2float_rn(h1), __ll2float_rn(h2));
        }
        int tot = 0, ttot = 0;
        const int pos = td_block_excl(nonz ? 1 : 0, s_w, tot);
        if (nonz) idx[m + pos] = (uint16_t)(i | (plus ? 0x8000 : 0));
        td_block_excl(tight ? 1 : 0, s_w, ttot);
        m += tot;
        tcount += ttot;
    }
    int G = 0;
    if (m > 0) {
        const int npad = td_pow2_at_least(m);
        for (int l = m + tid; l < npad; l += T) idx[l] = TD_SENT;
        __syncthreads();
        td_sort_block(idx, npad, H, Hf);
        auto same_line = [&](int l0, int l1) -> bool {
            const int a = idx[l0] & 0x7FFF, b = idx[l1] & 0x7FFF;
            return td_cross_sign_f(Hf[a], Hf[b], H[2 * a], H[2 * a + 1], H[2 * b], H[2 * b + 1]) == 0;
        };
        const int C = (m + T - 1) / T;
        const int beg = min(tid * C, m), end = min(beg + C, m);
        int pl = 0, sev = 0, nst = 0;
        for (int l = beg; l < end; ++l) {
            pl += (idx[l] >> 15) & 1;
            sev += (idx[l] & 0x8000) ? -1 : 1;
            nst += (l == 0 || !same_line(l - 1, l)) ? 1 : 0;
        }
        int A = 0, tmp = 0;
        td_block_excl(pl, s_w, A);
        const int vexcl = A + td_block_excl(sev, s_w, tmp);
        const int gexcl = td_block_excl(nst, s_w, tmp);
        /* walk value after each group = count of the cell that follows it;
         * A is the count of the cell before the first line (the same cell as
         * the one after the last line, turned by pi) */
        int v = vexcl, mn = A, mx = A;
        for (int l = beg; l < end; ++l) {
            v += (idx[l] & 0x8000) ? -1 : 1;
            if (l + 1 == m || !same_line(l, l + 1)) {
                mn = min(mn, v);
                mx = max(mx, v);
            }
        }
        mn = td_block_minmax(mn, s_w, 0);
        mx = td_block_minmax(mx, s_w, 1);
        G = min(mn, m - mx);
        if (G <= d0) {
            /* cell[g] = 1 when the cell before line group g has count G;
             * cell[L] (after the last group) equals cell[0] */
            if (tid == 0) cell[0] = (unsigned char)(min(A, m - A) == G);
            v = vexcl;
            int g = gexcl - 1;
            for (int l = beg; l < end; ++l) {
                v += (idx[l] & 0x8000) ? -1 : 1;
                if (l == 0 || !same_line(l - 1, l)) ++g;
                if (l + 1 == m || !same_line(l, l + 1)) cell[g + 1] = (unsigned char)(min(v, m - v) == G);
            }
            __syncthreads();
            g = gexcl - 1;
            for (int l = beg; l < end; ++l) {
                if (l == 0 || !same_line(l - 1, l)) ++g;
                if (cell[g] | cell[g + 1]) {
                    const int i = idx[l] & 0x7FFF;
                    atomicOr(&crit[i >> 5], 1u << (i & 31));
                }
            }
        }
    }
    __syncthreads();
    int V = G;
    if (tcount > K && G <= d0) {
        if (w == 0) {
            const int mS = td_tight_correction<D>(wmeta, nullptr, 0, xi, PSI, nnz, nullptr, H, scr, gcount, lane);
            if (lane == 0) s_res[0] = mS;
        }
        __syncthreads();
        V = G + s_res[0];
        __syncthreads();
    }
    return V;
}

/* Exact staging of query q's nonzero centred points (pivot coordinates,
 * int32, row stride PSI) in data order, and their data indices. */
__device__ int td_adia_stage(const TdLaunch &L, int q, int32_t *xi, int PSI, uint16_t *orig, int *s_tmp)
{
    const TdQuery &Q = L.q[q];
    const TdSet S = L.sets[Q.set];
    const int n = S.n, p = S.p, d = Q.d;
    const int32_t *X = L.X + S.x_off;
    const int32_t *z = L.Zq + (int64_t)q * TD_MAXD;
    const int T = blockDim.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = T >> 5;
    const int per = (n + T - 1) / T;
    const int beg = min((int)threadIdx.x * per, n), end = min(beg + per, n);
    int cnt = 0;
    for (int i = beg; i < end; ++i) {
        bool nz = false;
        for (int c = 0; c < p; ++c) nz |= X[(int64_t)i * p + c] != z[c];
        cnt += nz;
    }
    const int inc = td_wscan_incl(cnt, lane);
    if (lane == 31) s_tmp[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int v = lane < nw ? s_tmp[lane] : 0;
        const int vi = td_wscan_incl(v, lane);
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
        orig[o] = (uint16_t)i;
        ++o;
    }
    __syncthreads();
    return Q.nnz;
}

template <int D, bool WARP>
__global__ void __launch_bounds__(TD_ADIA_THREADS, 1) td_k_adia(TdLaunch L)
{
    constexpr int K = D - 2, K1 = D - 1;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_tmp[32], s_w[32], s_res[4];
    __shared__ int s_node[TD_MAXD], s_S[TD_MAXD], s_V[TD_MAXD];
    __shared__ int s_d0, s_ns, s_done, s_fail, s_improved, s_pick, s_nk;
    __shared__ unsigned s_dkey;
    __shared__ unsigned long long s_okey, s_prev;
    __shared__ int s_le, s_ge, s_low, s_side;
    __shared__ int64_t s_qa[TD_MAXD], s_qb[TD_MAXD], s_yt[2];
    const int T = blockDim.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nmaxp = td_pow2_at_least(L.nmax);
    const int nwords = nmaxp >> 5;
    const int PSI = D <= 4 ? 4 : 8;
    int32_t *xi = reinterpret_cast<int32_t *>(smem);
    size_t off = ((size_t)L.nmax * PSI * 4 + 15) & ~(size_t)15;
    uint16_t *orig = reinterpret_cast<uint16_t *>(smem + off);
    off += ((size_t)nmaxp * 2 + 15) & ~(size_t)15;
    uint32_t *inK = reinterpret_cast<uint32_t *>(smem + off);
    off += ((size_t)nwords * 4 + 15) & ~(size_t)15;
    int *wpre = reinterpret_cast<int *>(smem + off);
    off += ((size_t)(nwords + 1) * 4 + 15) & ~(size_t)15;
    /* evaluation buffers: one for the block, or (WARP) one per warp w < D-1 */
    const size_t ebytes = td_adia_eval_bytes(nmaxp);
    const int wslot = (WARP && w < K1) ? w : 0;
    unsigned char *eb = smem + off + ebytes * (size_t)wslot;
    auto crit_of = [&](int slot) -> const uint32_t * {
        return reinterpret_cast<const uint32_t *>(smem + off + ebytes * (size_t)slot + td_adia_crit_off(nmaxp));
    };
    const uint32_t *crit = crit_of(0);
    const TdScratch scr = td_scratch_at(
        L.scratch + ((size_t)blockIdx.x * (WARP ? TD_ADIA_THREADS / 32 : 1) + wslot) * L.scratch_per_warp, nmaxp);
    uint64_t *keys = L.adia_keys + (size_t)blockIdx.x * TD_ADIA_CAP;
    int32_t *dep = L.adia_dep + (size_t)blockIdx.x * TD_ADIA_CAP;
    int32_t *stk = L.adia_stack + (size_t)blockIdx.x * TD_ADIA_CAP;
    unsigned long long st_pops = 0, st_sub = 0, st_union = 0, st_fb = 0, st_err = 0;

    for (int jq = blockIdx.x; jq < L.nq; jq += gridDim.x) {
        const int q = L.order[jq];
        TdQuery *Q = &L.q[q];
        if (Q->d != D || Q->k != K || Q->direct >= 0) continue;
        const int nnz = Q->nnz, Z = Q->Z;
        uint16_t *perm = L.perm + (size_t)q * L.perm_stride;
        if (nnz <= 2 * D) { /* Algorithm 1 directly (the paper's n <= 2p) */
            for (int i = threadIdx.x; i < nnz; i += T) perm[i] = (uint16_t)i;
            continue;
        }
        const TdSet S = L.sets[Q->set];
        const int p = S.p;
        const int32_t *X = L.X + S.x_off;
        const int32_t *z = L.Zq + (int64_t)q * TD_MAXD;
        td_adia_stage(L, q, xi, PSI, orig, s_tmp);
        const bool same_coords = Q->d == p; /* pivot coordinates are the input coordinates */
        auto xorig = [&](int i, int c) -> int64_t {
            if (same_coords) return xi[(size_t)i * PSI + c];
            return (int64_t)X[(int64_t)orig[i] * p + c] - z[c];
        };
        for (int s2 = threadIdx.x; s2 < TD_ADIA_CAP; s2 += T) keys[s2] = 0ull;
        if (threadIdx.x == 0) {
            s_dkey = 0xFFFFFFFFu;
            s_okey = ~0ull;
            s_prev = ~0ull;
            s_ns = 0;
            s_fail = 0;
            s_done = 0;
            s_d0 = INT_MAX;
        }
        for (int wd = threadIdx.x; wd < nwords; wd += T) inK[wd] = 0u;
        __syncthreads();
        /* Step 2(a): data direction u = +-x_j with the least closed count;
         * key = count * 2^13 + 2 j + (1 for -x_j) orders count, j, sign */
        unsigned best = 0xFFFFFFFFu;
        for (int a = threadIdx.x; a < nnz; a += T) {
            int le = Z, ge = Z;
            if (same_coords) { /* p == D: registers, unrolled */
                int64_t u[D];
#pragma unroll
                for (int c = 0; c < D; ++c) u[c] = xi[(size_t)a * PSI + c];
                for (int i = 0; i < nnz; ++i) {
                    int64_t dot = 0;
#pragma unroll
                    for (int c = 0; c < D; ++c) dot += u[c] * xi[(size_t)i * PSI + c];
                    le += dot <= 0;
                    ge += dot >= 0;
                }
            } else {
                int64_t u[TD_MAXD];
                for (int c = 0; c < p; ++c) u[c] = xorig(a, c);
                for (int i = 0; i < nnz; ++i) {
                    int64_t dot = 0;
                    for (int c = 0; c < p; ++c) dot += u[c] * xorig(i, c);
                    le += dot <= 0;
                    ge += dot >= 0;
                }
            }
            const unsigned j = orig[a];
            best = min(best, min(((unsigned)le << 13) | (j << 1), ((unsigned)ge << 13) | (j << 1) | 1u));
        }
        atomicMin(&s_dkey, best);
        __syncthreads();
        const int U = (int)(s_dkey >> 13);
        if (U - Z == 0) { /* no nonzero point in the closed halfspace: T = Z */
            if (threadIdx.x == 0) {
                Q->direct = Z;
                Q->lo = Q->hi = 0;
            }
            for (int i = threadIdx.x; i < nnz; i += T) perm[i] = (uint16_t)i;
            __syncthreads();
            continue;
        }
        int64_t umin[TD_MAXD];
        {
            const int jd = (int)((s_dkey >> 1) & 0xFFFu);
            const int sg = (s_dkey & 1u) ? -1 : 1;
            for (int c = 0; c < p; ++c) umin[c] = sg * ((int64_t)X[(int64_t)jd * p + c] - z[c]);
        }
        /* Step 2(b)-(c): start subset, greedily in the order of u_min'x_i
         * (ties by index) from the first point with u_min'x_i >= 0, wrapping
         * round; a point dependent on those taken is skipped.  Order keys:
         * (projection + 2^48) * 2^12 + index. */
        auto okey = [&](int i) -> unsigned long long {
            int64_t dot = 0;
            if (same_coords) {
#pragma unroll
                for (int c = 0; c < D; ++c) dot += umin[c] * xi[(size_t)i * PSI + c];
            } else {
                for (int c = 0; c < p; ++c) dot += umin[c] * xorig(i, c);
            }
            return ((unsigned long long)(dot + ((int64_t)1 << 48)) << 12) | (unsigned long long)i;
        };
        const unsigned long long zero_key = (unsigned long long)((int64_t)1 << 48) << 12;
        int taken = 0;
        for (int it = 0; it < nnz && taken < K; ++it) {
            /* successor of s_prev in key order (the first key >= zero_key at the start) */
            unsigned long long mine = ~0ull, wrapmin = ~0ull;
            const unsigned long long lo = (it == 0) ? zero_key : s_prev + 1;
            for (int i = threadIdx.x; i < nnz; i += T) {
                const unsigned long long kk = okey(i);
                if (kk >= lo) mine = min(mine, kk);
                wrapmin = min(wrapmin, kk);
            }
            if (threadIdx.x == 0) s_okey = ~0ull;
            __syncthreads();
            atomicMin(&s_okey, mine);
            __syncthreads();
            if (s_okey == ~0ull) { /* wrap round to the smallest key */
                __syncthreads();
                if (threadIdx.x == 0) s_okey = ~0ull;
                __syncthreads();
                atomicMin(&s_okey, wrapmin);
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                const int cand = (int)(s_okey & 0xFFFull);
                s_prev = s_okey;
                int64_t rows[TD_MAXD][TD_MAXD];
                for (int b = 0; b <= taken; ++b)
                    for (int cc = 0; cc < D; ++cc)
                        rows[b][cc] = xi[(size_t)(b < taken ? s_S[b] : cand) * PSI + cc];
                s_pick = td_adia_rank(rows, taken + 1, D) == taken + 1 ? cand : -1;
                if (s_pick >= 0) s_S[taken] = cand;
            }
            __syncthreads();
            if (s_pick >= 0) ++taken;
        }
        if (taken < K) { /* cannot happen for data of rank D; keep Algorithm 1 */
            if (threadIdx.x == 0) ++st_err;
            for (int i = threadIdx.x; i < nnz; i += T) perm[i] = (uint16_t)i;
            __syncthreads();
            continue;
        }
        if (threadIdx.x == 0) /* sort the start subset */
            for (int a = 1; a < K; ++a)
                for (int b = a; b > 0 && s_S[b - 1] > s_S[b]; --b) {
                    const int tt = s_S[b];
                    s_S[b] = s_S[b - 1];
                    s_S[b - 1] = tt;
                }
        __syncthreads();
        /* Step 2(c): V of the start subset and its critical point of least index */
        {
            int c[K];
#pragma unroll
            for (int b = 0; b < K; ++b) c[b] = s_S[b];
            int V0 = 0;
            if constexpr (WARP) {
                if (w == 0) {
                    const int v = td_adia_eval<D>(xi, PSI, nnz, c, eb, nmaxp, scr, INT_MAX, lane);
                    if (lane == 0) s_res[2] = v;
                }
                __syncthreads();
                V0 = s_res[2];
            } else {
                V0 = td_adia_eval_block<D>(xi, PSI, nnz, c, eb, nmaxp, scr, INT_MAX, s_w, s_res);
            }
            if (threadIdx.x == 0) {
                ++st_sub;
                int h0 = -1;
                for (int wd = 0; wd < nwords && h0 < 0; ++wd)
                    if (crit[wd]) h0 = wd * 32 + __ffs(crit[wd]) - 1;
                if (V0 == INT_MAX || h0 < 0) {
                    s_fail = 1;
                } else {
                    int Cn[TD_MAXD];
                    for (int b = 0; b < K; ++b) Cn[b] = s_S[b];
                    Cn[K] = h0;
                    for (int a = 1; a < K1; ++a)
                        for (int b = a; b > 0 && Cn[b - 1] > Cn[b]; --b) {
                            const int tt = Cn[b];
                            Cn[b] = Cn[b - 1];
                            Cn[b - 1] = tt;
                        }
                    /* Step 3 */
                    const int sl = td_adia_insert(keys, dep, td_adia_pack(Cn, K1), V0);
                    stk[0] = sl;
                    s_ns = 1;
                    s_d0 = V0;
                }
            }
        }
        __syncthreads();
        /* Step 4: pop a node; its subsets in lexicographic order (subset j
         * omits member K1-1-j), each evaluated by the whole block; thread 0
         * pushes the new nodes of a subset with V <= d0 and stops at the
         * first subset that lowers d0 */
        for (int pops = 0; !s_fail; ++pops) {
            if (threadIdx.x == 0) {
                if (s_ns == 0) {
                    s_done = 1;
                } else if (pops >= TD_ADIA_MAX_POPS) {
                    s_fail = 1;
                } else {
                    const int sl = stk[--s_ns];
                    td_adia_unpack(keys[sl], s_node, K1);
                    ++st_pops;
                }
                s_improved = 0;
            }
            __syncthreads();
            if (s_done || s_fail) break;
            const int d0 = s_d0;
            /* thread 0: apply (iii) and (iv) for subset sidx with value V and
             * critical bits cb */
            auto apply = [&](int sidx, int V, const uint32_t *cb) {
                ++st_sub;
                if (V > s_d0) return;
                int c[K];
#pragma unroll
                for (int b = 0; b < K; ++b) c[b] = s_node[b < K1 - 1 - sidx ? b : b + 1];
                for (int wd = 0; wd < nwords && !s_fail; ++wd) {
                    uint32_t bits = cb[wd];
                    for (int b = 0; b < K1; ++b)
                        if ((s_node[b] >> 5) == wd) bits &= ~(1u << (s_node[b] & 31));
                    while (bits) {
                        const int tpt = wd * 32 + __ffs(bits) - 1;
                        bits &= bits - 1;
                        int Nn[TD_MAXD];
                        for (int b = 0; b < K; ++b) Nn[b] = c[b];
                        Nn[K] = tpt;
                        for (int a = 1; a < K1; ++a)
                            for (int b = a; b > 0 && Nn[b - 1] > Nn[b]; --b) {
                                const int tt = Nn[b];
                                Nn[b] = Nn[b - 1];
                                Nn[b - 1] = tt;
                            }
                        const int sl = td_adia_insert(keys, dep, td_adia_pack(Nn, K1), V);
                        if (sl == -2 || s_ns >= TD_ADIA_CAP) {
                            s_fail = 1;
                            break;
                        }
                        if (sl >= 0) stk[s_ns++] = sl;
                    }
                }
                if (V < s_d0) { /* (iv) */
                    s_d0 = V;
                    s_improved = 1;
                }
            };
            if constexpr (WARP) {
                /* the D-1 subsets in parallel, one warp each */
                if (w < K1) {
                    int c[K];
#pragma unroll
                    for (int b = 0; b < K; ++b) c[b] = s_node[b < K1 - 1 - w ? b : b + 1];
                    const int V = td_adia_eval<D>(xi, PSI, nnz, c, eb, nmaxp, scr, d0, lane);
                    if (lane == 0) s_V[w] = V;
                }
                __syncthreads();
                if (threadIdx.x == 0)
                    for (int sidx = 0; sidx < K1 && !s_improved && !s_fail; ++sidx) apply(sidx, s_V[sidx], crit_of(sidx));
                __syncthreads();
            } else {
                for (int sidx = 0; sidx < K1; ++sidx) {
                    int c[K];
#pragma unroll
                    for (int b = 0; b < K; ++b) c[b] = s_node[b < K1 - 1 - sidx ? b : b + 1];
                    const int V = td_adia_eval_block<D>(xi, PSI, nnz, c, eb, nmaxp, scr, d0, s_w, s_res);
                    if (threadIdx.x == 0) apply(sidx, V, crit);
                    __syncthreads();
                    if (s_improved || s_fail) break;
                }
            }
            if (s_improved && !s_fail) {
                /* Step 4(b): delete the nodes deeper than d0 */
                const int nd0 = s_d0;
                for (int s2 = threadIdx.x; s2 < TD_ADIA_CAP; s2 += T)
                    if (keys[s2] != 0ull && dep[s2] > nd0) dep[s2] = -1;
                __syncthreads();
                if (threadIdx.x == 0) {
                    int wr = 0;
                    for (int r = 0; r < s_ns; ++r)
                        if (dep[stk[r]] >= 0) stk[wr++] = stk[r];
                    s_ns = wr;
                }
            }
            __syncthreads();
        }
        __syncthreads();
        if (s_fail) { /* too large a search: the full subset range (exact) */
            for (int i = threadIdx.x; i < nnz; i += T) perm[i] = (uint16_t)i;
            if (threadIdx.x == 0) {
                ++st_fb;
                if (s_d0 < L.qmin[q]) L.qmin[q] = s_d0; /* still an upper bound */
            }
            __syncthreads();
            continue;
        }
        /* Step 5(a): the closed side with fewer points of every node left.
         * For F = S + {t} (t its largest index) the functional
         * x -> y_t x y_x of the projections by the basis of S vanishes on
         * span(S) and on x_t, so it is det[x_F | x] up to a sign that is the
         * same for every x; the choice of side below does not depend on that
         * sign (fewer points, or on a tie the side of the least index off
         * the hyperplane).  The nodes left are listed in stk first (the
         * stack is empty now). */
        if (threadIdx.x == 0) s_ns = 0;
        __syncthreads();
        for (int s2 = threadIdx.x; s2 < TD_ADIA_CAP; s2 += T)
            if (keys[s2] != 0ull && dep[s2] >= 0) stk[atomicAdd(&s_ns, 1)] = s2;
        __syncthreads();
        const int nlive = s_ns;
        for (int f = 0; f < nlive; ++f) {
            if (threadIdx.x == 0) {
                int F[TD_MAXD];
                td_adia_unpack(keys[stk[f]], F, K1);
                int64_t sm[K][D];
#pragma unroll
                for (int j = 0; j < K; ++j)
#pragma unroll
                    for (int cc = 0; cc < D; ++cc) sm[j][cc] = xi[(size_t)F[j] * PSI + cc];
                TdBasis<D> Bs;
                if (!td_make_basis<D>(sm, Bs)) ++st_err; /* F is independent: cannot happen */
                int64_t y1 = 0, y2 = 0;
#pragma unroll
                for (int cc = 0; cc < D; ++cc) {
                    s_qa[cc] = Bs.qa[cc];
                    s_qb[cc] = Bs.qb[cc];
                    y1 += Bs.qa[cc] * (int64_t)xi[(size_t)F[K] * PSI + cc];
                    y2 += Bs.qb[cc] * (int64_t)xi[(size_t)F[K] * PSI + cc];
                }
                s_yt[0] = y1;
                s_yt[1] = y2;
                s_le = Z;
                s_ge = Z;
                s_low = INT_MAX;
            }
            __syncthreads();
            int64_t qa[D], qb[D];
#pragma unroll
            for (int cc = 0; cc < D; ++cc) {
                qa[cc] = s_qa[cc];
                qb[cc] = s_qb[cc];
            }
            const int64_t t1 = s_yt[0], t2 = s_yt[1];
            auto side_of = [&](int i) -> int {
                int64_t y1 = 0, y2 = 0;
#pragma unroll
                for (int cc = 0; cc < D; ++cc) {
                    const int64_t xv = xi[(size_t)i * PSI + cc];
                    y1 += qa[cc] * xv;
                    y2 += qb[cc] * xv;
                }
                return td_cross_sign(t1, t2, y1, y2);
            };
            int le = 0, ge = 0, low = INT_MAX;
            for (int i = threadIdx.x; i < nnz; i += T) {
                const int sg = side_of(i);
                le += sg <= 0;
                ge += sg >= 0;
                if (sg != 0) low = min(low, i);
            }
            atomicAdd(&s_le, le);
            atomicAdd(&s_ge, ge);
            atomicMin(&s_low, low);
            __syncthreads();
            if (threadIdx.x == 0) {
                int side = 0; /* -1: <= 0, +1: >= 0, 0: every point */
                if (s_le < s_ge) side = -1;
                else if (s_ge < s_le) side = 1;
                else if (s_low != INT_MAX) side = side_of(s_low);
                s_side = side;
            }
            __syncthreads();
            const int side = s_side;
            for (int i = threadIdx.x; i < nnz; i += T) {
                const int sg = side_of(i);
                if (side == 0 || sg == 0 || sg == side) atomicOr(&inK[i >> 5], 1u << (i & 31));
            }
            __syncthreads();
        }
        /* Step 5(b) hand-off: union first in the staging order */
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int wd = 0; wd < nwords; ++wd) {
                wpre[wd] = acc;
                acc += __popc(inK[wd]);
            }
            wpre[nwords] = acc;
            s_nk = acc;
        }
        __syncthreads();
        const int nk = s_nk;
        for (int i = threadIdx.x; i < nnz; i += T) {
            const uint32_t wd = inK[i >> 5];
            const int before = wpre[i >> 5] + __popc(wd & ((1u << (i & 31)) - 1u));
            perm[i] = (uint16_t)(((wd >> (i & 31)) & 1u) ? before : nk + (i - before));
        }
        if (threadIdx.x == 0) {
            st_union += (unsigned long long)nk;
            const int d0 = s_d0;
            Q->lo = 0;
            Q->hi = (d0 <= 0 || nk < K) ? 0 : (int64_t)td_binom(nk, K);
            L.qmin[q] = d0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&L.ctr->adia_pops, st_pops);
        atomicAdd(&L.ctr->adia_fallback, st_fb);
        atomicAdd(&L.ctr->adia_union, st_union);
        atomicAdd(&L.ctr->errors, st_err);
    }
    if (threadIdx.x == 0) atomicAdd(&L.ctr->adia_subsets, st_sub);
}
