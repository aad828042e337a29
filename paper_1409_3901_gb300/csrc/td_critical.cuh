/*
 * td_critical.cuh -- Proposition 1 with r = p - 1 (the critical-direction
 * form) on the device; included by td_kernels.cu after the tight-set path.
 *
 * For every (d-1)-subset F of the nonzero centred points (d the effective
 * dimension) the hyperplane H = span(F) has the integer normal n_F, the
 * cofactor vector of the d x (d-1) matrix of F (n_F . x = det[x_F | x]).
 * Every point lies strictly on one side of H or on it.  For a direction
 * u = +-n_F + eps v (v in H, generic) the points off H keep their side and
 * the points on H are split by v alone, so the fewest points strictly on the
 * negative side is
 *
 *     V'(F) = min(#{n_F . x < 0}, #{n_F . x > 0}) + m_F,
 *
 * m_F the open depth of the nonzero points on H inside H (0 when H holds no
 * data point besides F, as in general position, where this is the paper's
 * P_n(u'X <= 0) - (p-1)/n of Proposition 1).  Every generic direction lies in
 * an open cell of the arrangement of the hyperplanes x_i^perp whose closure
 * has a ray spanned by some n_F, so T = Z + min_F V'(F), exactly.
 *
 * Exact int64 arithmetic: the caller guarantees d! max|x|^d < 2^62, so the
 * cofactors ((d-1)! max|x|^(d-1)) and every n_F . x fit.  m_F is computed by
 * the tight-set recursion (td_open_depth<d-1>, or td_open_depth_s<5> at
 * d = 6) on the points of H in the d - 1 coordinates other than one where
 * n_F is nonzero (injective on H).
 */

#define TD_CRIT_THREADS 256

template <int D>
__device__ void td_warp_critical(const int32_t *xi, int PSI, int nnz, uint64_t r0, uint64_t r1,
                                 const TdScratch &scr, int lane, int &best, TdWarpStats &st)
{
    constexpr int K1 = D - 1;
    if (r0 >= r1) return;
    int c[K1];
    c[0] = 0;
    td_unrank_colex<K1>(r0, nnz, c);
    for (uint64_t r = r0; r < r1; ++r) {
        if (r > r0) td_next_colex<K1>(c);
        /* the normal: n_j = (-1)^(j + D - 1) det(F's coordinates without row
         * j), cofactor j by lane j, shared by shuffles */
        int64_t mine = 0;
        if (lane < D) {
            constexpr int MS = K1 > 4 ? K1 : 4;
            int64_t M[MS][MS];
#pragma unroll
            for (int o = 0; o < MS; ++o)
#pragma unroll
                for (int a = 0; a < MS; ++a)
                    M[o][a] = (o < K1 && a < K1) ? xi[(size_t)c[a] * PSI + (o < lane ? o : o + 1)] : 0;
            const int64_t m = td_detn<K1>(M);
            mine = ((lane + D - 1) & 1) ? -m : m;
        }
        int64_t n[D];
        bool nz = false;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            n[j] = td_shfl64(mine, j);
            nz |= n[j] != 0;
        }
        if (!nz) { /* dependent subset */
            if (lane == 0) st.dependent++;
            continue;
        }
        if (lane == 0) st.sweeps++;
        int neg = 0, pos = 0, on = 0;
        for (int i = lane; i < nnz; i += 32) {
            int64_t s = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) s += n[k] * (int64_t)xi[(size_t)i * PSI + k];
            neg += s < 0;
            pos += s > 0;
            on += s == 0;
        }
        neg = td_wsum(neg);
        pos = td_wsum(pos);
        on = td_wsum(on);
        int V = min(neg, pos);
        if (on > K1 && V < best) {
            /* m_F: the points on H in the coordinates other than jd */
            int jd = 0;
#pragma unroll
            for (int j = D - 1; j >= 0; --j)
                if (n[j] != 0) jd = j;
            int t = 0;
            const unsigned below = (1u << lane) - 1u;
            for (int i0 = 0; i0 < nnz; i0 += 32) {
                const int i = i0 + lane;
                bool g = false;
                if (i < nnz) {
                    int64_t s = 0;
#pragma unroll
                    for (int k = 0; k < D; ++k) s += n[k] * (int64_t)xi[(size_t)i * PSI + k];
                    g = s == 0;
                }
                const unsigned bg = __ballot_sync(TD_FULL, g);
                if (g) {
                    const int slot = t + __popc(bg & below);
                    constexpr int CS = K1 > 4 ? 8 : 4; /* see td_k_critical's scratch */
                    int o = 0;
#pragma unroll
                    for (int k = 0; k < D; ++k)
                        if (k != jd) scr.c0[CS * slot + o++] = xi[(size_t)i * PSI + k];
                }
                t += __popc(bg);
            }
            __syncwarp();
            if (lane == 0) st.tight++;
            if constexpr (K1 == 5) V += td_open_depth_s<5, 8>(scr.c0, t, scr, lane);
            else V += td_open_depth<K1>(scr.c0, t, scr, lane, 0);
        }
        best = min(best, V);
    }
}

/* One query per launch; CTAs take tiles of its (d-1)-subset positions. */
template <int D>
__global__ void __launch_bounds__(TD_CRIT_THREADS, 1) td_k_critical(TdLaunch L, int q)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int s_tmp[32];
    __shared__ int s_best[TD_CRIT_THREADS / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const TdQuery &Q = L.q[q];
    if (Q.k != D - 1 || Q.hi <= Q.lo || Q.d != D) return;
    const int nnz = Q.nnz;
    const int nmaxp = td_pow2_at_least(L.nmax);
    const int PSI = D <= 4 ? 4 : 8;
    int32_t *xi = reinterpret_cast<int32_t *>(smem);
    uint16_t *orig = reinterpret_cast<uint16_t *>(smem + (((size_t)L.nmax * PSI * 4 + 15) & ~(size_t)15));
    td_adia_stage(L, q, xi, PSI, orig, s_tmp);
    const int gw = blockIdx.x * nw + w;
    /* scratch laid out for 2 nmaxp points: c0 then holds 8 coordinates for
     * each of nmaxp points (the 5-D hyperplane sets at d = 6) */
    const TdScratch scr = td_scratch_at(L.scratch + (size_t)gw * L.scratch_per_warp, 2 * nmaxp);
    TdWarpStats st = { 0, 0, 0, 0, 0, 0, 0 };
    const int64_t ts = (int64_t)(L.spw > 0 ? L.spw : 16) * nw;
    const int64_t ntiles = (Q.hi - Q.lo + ts - 1) / ts;
    int best = INT_MAX;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t t0 = Q.lo + tile * ts, t1 = min(t0 + ts, Q.hi);
        const int64_t spw = ts / nw;
        const uint64_t r0 = (uint64_t)min(t0 + spw * w, t1), r1 = (uint64_t)min(t0 + spw * (w + 1), t1);
        td_warp_critical<D>(xi, PSI, nnz, r0, r1, scr, lane, best, st);
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
        atomicAdd(&L.ctr->tight, st.tight);
    }
}
