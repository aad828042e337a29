/*
 * td_api.cu -- host side of the C ABI declared in include/tukey_depth.h.
 *
 * A call packs its datasets into device arenas, then runs on one CUDA stream
 *   set-up kernel -> tile-prefix kernel -> persistent sweep kernel -> finalize
 * (TD_MODE_FILTERED; the launch sequence is captured once as a CUDA graph and
 * replayed while the shapes repeat), or
 *   set-up kernel -> one plain exact launch per query -> finalize
 * (TD_MODE_PLAIN_EXACT), and copies the outputs out after checking the
 * device-side error counter, so that no partial result is ever written.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/tukey_depth.h"
#include "td_internal.h"

/* kernels and launch helpers (td_kernels.cu) */
size_t td_filtered_smem(int nmax, int pmax, int blog2, int warps);
size_t td_plain_smem(int nmax, int pmax, int warps);
int64_t td_scratch_per_warp(int nmax);
int64_t td_scratch_per_warp_critical(int nmax);
cudaError_t td_launch_setup(const TdLaunch &L, cudaStream_t s);
cudaError_t td_launch_tiles(const TdLaunch &L, cudaStream_t s);
cudaError_t td_launch_filtered(int D, const TdLaunch &L, int grid, size_t smem, cudaStream_t s);
cudaError_t td_launch_plain(int D, const TdLaunch &L, int q, int grid, size_t smem, cudaStream_t s);
cudaError_t td_launch_finalize(const TdLaunch &L, cudaStream_t s);
cudaError_t td_launch_wide(const TdLaunch &L, int sms, cudaStream_t s);
int td_filtered_occupancy(int D, int warps, size_t smem);
int td_plain_occupancy(int D, int warps, size_t smem);
size_t td_adia_smem(int nmax, int D);
int td_adia_occupancy(int D, int nmax, size_t smem);
int td_adia_scratch_slots(int nmax);
cudaError_t td_launch_adia(int D, const TdLaunch &L, int grid, size_t smem, cudaStream_t s);
int64_t td_adia_ws_entries();
size_t td_critical_smem(int nmax, int pmax);
int td_critical_occupancy(int D, size_t smem);
cudaError_t td_launch_critical(int D, const TdLaunch &L, int q, int grid, size_t smem, cudaStream_t s);
int td_critical_threads();

namespace {

/* Warps per CTA of the sweep kernels.  The warps of a CTA meet at a
 * barrier at the end of each tile, and in CTAs of 4 they wait less for the
 * slowest than in CTAs of 8: W2 31.5 to 31.1 ms, W4 147 to 145 ms, W3 5.50
 * to 5.45 s -- W3 even where its rows of up to 2000 points (each CTA
 * stages its own copy) leave 12 warps resident per SM instead of 16. */
const int kWarpsFiltered = 4;
const int kWarpsPlain = 4;

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

/* Grow-only device buffer. */
cudaError_t grow(DevBuf &b, size_t bytes)
{
    if (bytes <= b.cap) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t want = std::max(bytes, (size_t)256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e == cudaSuccess) b.cap = want;
    return e;
}

struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
};

cudaError_t grow_host(HostBuf &b, size_t bytes)
{
    if (bytes <= b.cap) return cudaSuccess;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t want = std::max(bytes, (size_t)256);
    cudaError_t e = cudaMallocHost(&b.p, want);
    if (e == cudaSuccess) b.cap = want;
    return e;
}

/* Device state of one batched call (or one stream request). */
struct Work {
    DevBuf X, Zq, sets, q, order, prefix, tsize, ticket, qmin, out, ctr, scratch;
    DevBuf perm, akeys, adep, astk; /* Algorithm 3: staging order per query, node tables per CTA */
    int grid[TD_NDIM] = { 0, 0, 0, 0, 0 }; /* persistent grid of the sweep kernel of dimension D = 2 + i */
    int agrid[TD_NDIM] = { 0, 0, 0, 0, 0 }; /* Algorithm 3 search kernel of dimension D = 2 + i: */
    size_t asmem[TD_NDIM] = { 0, 0, 0, 0, 0 }; /* grid and shared memory */
};

struct GraphKey {
    int nq, nsets, nmax, pmax, grid[TD_NDIM], nmaxD[TD_NDIM], blog2, spw, early_exit, algorithm, unseeded, warps;
    uint16_t spw_tab[TD_NDIM][TD_NOCT];
    size_t smem;
    const void *ptrs[17];
    int64_t shard_index, shard_count;
    bool operator==(const GraphKey &o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

}  // namespace

struct td_ctx {
    int device = 0;
    int sms = 0;
    int smem_optin = 0; /* largest dynamic shared memory per block */
    td_options opt;
    cudaStream_t own = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evs0 = nullptr, evs1 = nullptr;
    Work w;
    HostBuf hstage, hout;
    std::string cuda_err;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    bool gvalid = false;
    uint16_t tune[TD_NDIM][TD_NOCT] = {}; /* td_autotune: subsets per warp by dimension and octave */
};

/* one request of a stream: a copy of its inputs until its last slice has
 * run.  Its subset loop is cut into nslices contiguous ranges of subset
 * positions (time slices of bounded work); each slice's counts are merged
 * into acc by a minimum. */
struct td_stream_req {
    uint64_t ticket;
    int32_t n, p, m;
    std::vector<int32_t> X, Z;
    std::vector<int32_t> acc; /* minimum over the finished slices */
    int32_t *user_out;
    size_t bytes;
    int nslices, next_slice, done_slices;
    double slice_work;        /* point evaluations of one slice */
    bool finished;
    int status;
};

/* one slice of one request inside a batch */
struct td_slice_entry {
    td_stream_req *r;
    int slice;
    int64_t out_off; /* offset of its outputs in the batch's output */
};

/* a batch of coalesced slices in flight */
struct td_stream_slot {
    Work w;
    HostBuf hstage, hout;
    cudaEvent_t done = nullptr;
    bool busy = false;
    int nq = 0;
    std::vector<td_slice_entry> ents;
};

struct td_stream {
    td_ctx *ctx;
    cudaStream_t s;
    size_t budget, inflight;
    uint64_t next;
    DevBuf scratch;
    std::vector<td_stream_req *> pending;   /* admitted, with slices not yet launched */
    std::vector<td_stream_req *> reqs;      /* every request not yet reaped */
    td_stream_slot slot[2];
};

namespace {

int fail_cuda(td_ctx *c, cudaError_t e, const char *what)
{
    if (c) {
        c->cuda_err = std::string(what) + ": " + cudaGetErrorString(e);
    }
    return e == cudaErrorMemoryAllocation ? TD_ERR_OOM : TD_ERR_CUDA;
}

#define TDCK(call)                                              \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return fail_cuda(ctx, _e, #call); \
    } while (0)

td_options default_options()
{
    td_options o;
    memset(&o, 0, sizeof(o));
    o.mode = TD_MODE_FILTERED;
    o.use_graph = 1;
    o.shard_count = 1;
    return o;
}

cudaStream_t stream_of(td_ctx *c) { return c->opt.stream ? (cudaStream_t)c->opt.stream : c->own; }

int validate_options(const td_options &o)
{
    if (o.mode != TD_MODE_FILTERED && o.mode != TD_MODE_PLAIN_EXACT) return TD_ERR_INVALID;
    if (o.shard_count > 1 && (o.shard_index < 0 || o.shard_index >= o.shard_count)) return TD_ERR_INVALID;
    if (o.algorithm != TD_ALG_RCOM && o.algorithm != TD_ALG_ADIA && o.algorithm != TD_ALG_CRITICAL)
        return TD_ERR_INVALID;
    if (o.algorithm == TD_ALG_ADIA && (o.mode != TD_MODE_FILTERED || o.shard_count > 1)) return TD_ERR_INVALID;
    return TD_OK;
}

int validate_set(const td_dataset &d)
{
    if (d.n < 1 || d.n > TD_MAX_N || d.p < 1 || d.p > TD_MAX_P || d.m < 0) return TD_ERR_INVALID;
    if (!d.X || (d.m > 0 && (!d.Z || !d.out))) return TD_ERR_INVALID;
    return TD_OK;
}

struct Plan {
    int nq = 0, nsets = 0, nmax = 1, pmax = 1;
    int nmaxD[TD_NDIM] = { 1, 1, 1, 1, 1 }; /* largest n over the datasets with p >= D (D = 2 + i) */
    size_t x_elems = 0;
    std::vector<TdSet> sets;
    std::vector<TdQuery> q;
    std::vector<int32_t> order;
};

Plan make_plan(const td_dataset *sets, int k)
{
    Plan P;
    P.nsets = k;
    std::vector<std::pair<double, int>> cost;
    for (int s = 0; s < k; ++s) {
        TdSet t;
        t.x_off = (int64_t)P.x_elems;
        t.n = sets[s].n;
        t.p = sets[s].p;
        t.slice_index = 0;
        t.slice_count = 1;
        P.sets.push_back(t);
        /* every dataset starts on a 16-byte boundary of the arena (the
         * sweep kernels copy a dataset into shared memory with one bulk
         * copy, which needs that alignment) */
        P.x_elems += ((size_t)t.n * t.p + 3) & ~(size_t)3;
        P.nmax = std::max(P.nmax, t.n);
        P.pmax = std::max(P.pmax, t.p);
        for (int D = 2; D <= std::min(t.p, 6); ++D) P.nmaxD[D - 2] = std::max(P.nmaxD[D - 2], t.n);
        double c = 1.0;
        for (int i = 0; i < t.p - 2; ++i) c *= (double)(t.n - i) / (i + 1);
        c *= t.n;
        for (int j = 0; j < sets[s].m; ++j) {
            TdQuery Q;
            memset(&Q, 0, sizeof(Q));
            Q.set = s;
            cost.push_back({-c, P.nq});
            P.q.push_back(Q);
            ++P.nq;
        }
    }
    /* longest work first */
    std::stable_sort(cost.begin(), cost.end());
    for (auto &c : cost) P.order.push_back(c.second);
    return P;
}

cudaError_t alloc_work(Work &w, const Plan &P, int grid_warps, bool need_x_arena)
{
    cudaError_t e;
    if (need_x_arena && (e = grow(w.X, std::max<size_t>(P.x_elems, 1) * 4)) != cudaSuccess) return e;
    if ((e = grow(w.Zq, (size_t)std::max(P.nq, 1) * TD_MAXD * 4)) != cudaSuccess) return e;
    if ((e = grow(w.sets, (size_t)std::max(P.nsets, 1) * sizeof(TdSet))) != cudaSuccess) return e;
    if ((e = grow(w.q, (size_t)std::max(P.nq, 1) * sizeof(TdQuery))) != cudaSuccess) return e;
    if ((e = grow(w.order, (size_t)std::max(P.nq, 1) * 4)) != cudaSuccess) return e;
    if ((e = grow(w.prefix, (size_t)TD_NDIM * (P.nq + 1) * 8)) != cudaSuccess) return e;
    if ((e = grow(w.tsize, (size_t)std::max(P.nq, 1) * 4)) != cudaSuccess) return e;
    if ((e = grow(w.ticket, (size_t)TD_NDIM * TD_TICKET_STRIDE * 8)) != cudaSuccess) return e;
    if ((e = grow(w.qmin, (size_t)std::max(P.nq, 1) * 4)) != cudaSuccess) return e;
    if ((e = grow(w.out, (size_t)std::max(P.nq, 1) * 4)) != cudaSuccess) return e;
    if ((e = grow(w.ctr, sizeof(TdCounters))) != cudaSuccess) return e;
    size_t sc = (size_t)grid_warps * (size_t)td_scratch_per_warp(P.nmax);
    if ((e = grow(w.scratch, sc)) != cudaSuccess) return e;
    return cudaSuccess;
}

/* Histogram size of the sweep kernels (shared memory sizing): 2^blog2 angular
 * buckets, about one per two points and at least 128 (four per lane, the
 * 128-bit scan granularity). */
int blog2_for(int nmax, const td_options &o)
{
    if (o.buckets_log2 > 0) return std::max(7, std::min(o.buckets_log2, 12));
    int b = 7;
    while ((2 << b) < nmax && b < 11) ++b;
    return b;
}

/* Pack the host-side inputs into pinned staging and enqueue the copies. */
int stage_inputs(td_ctx *ctx, Work &w, HostBuf &stage, const Plan &P, const td_dataset *sets, int k,
                 bool devptr, cudaStream_t s, const int32_t **x_arena)
{
    size_t zq_bytes = (size_t)P.nq * TD_MAXD * 4;
    size_t small = P.nsets * sizeof(TdSet) + P.nq * sizeof(TdQuery) + P.nq * 4;
    size_t host_bytes = zq_bytes + small + (devptr ? 0 : P.x_elems * 4) + 64;
    TDCK(grow_host(stage, host_bytes));
    char *h = (char *)stage.p;
    /* queries, row stride TD_MAXD */
    int32_t *hz = (int32_t *)h;
    memset(hz, 0, zq_bytes);
    if (!devptr) {
        int qi = 0;
        for (int s2 = 0; s2 < k; ++s2)
            for (int j = 0; j < sets[s2].m; ++j, ++qi)
                memcpy(hz + (size_t)qi * TD_MAXD, sets[s2].Z + (size_t)j * sets[s2].p, sets[s2].p * 4);
        TDCK(cudaMemcpyAsync(w.Zq.p, hz, zq_bytes, cudaMemcpyHostToDevice, s));
    } else {
        int qi = 0;
        for (int s2 = 0; s2 < k; ++s2) {
            if (sets[s2].m > 0)
                TDCK(cudaMemcpy2DAsync((int32_t *)w.Zq.p + (size_t)qi * TD_MAXD, TD_MAXD * 4, sets[s2].Z,
                                       sets[s2].p * 4, sets[s2].p * 4, sets[s2].m, cudaMemcpyDeviceToDevice, s));
            qi += sets[s2].m;
        }
    }
    char *hs = h + zq_bytes;
    memcpy(hs, P.sets.data(), P.nsets * sizeof(TdSet));
    memcpy(hs + P.nsets * sizeof(TdSet), P.q.data(), P.nq * sizeof(TdQuery));
    memcpy(hs + P.nsets * sizeof(TdSet) + P.nq * sizeof(TdQuery), P.order.data(), P.nq * 4);
    TDCK(cudaMemcpyAsync(w.sets.p, hs, P.nsets * sizeof(TdSet), cudaMemcpyHostToDevice, s));
    if (P.nq > 0) {
        TDCK(cudaMemcpyAsync(w.q.p, hs + P.nsets * sizeof(TdSet), P.nq * sizeof(TdQuery), cudaMemcpyHostToDevice, s));
        TDCK(cudaMemcpyAsync(w.order.p, hs + P.nsets * sizeof(TdSet) + P.nq * sizeof(TdQuery), P.nq * 4,
                             cudaMemcpyHostToDevice, s));
    }
    if (devptr && k == 1) {
        *x_arena = sets[0].X; /* used in place */
    } else if (devptr) {
        for (int s2 = 0; s2 < k; ++s2)
            TDCK(cudaMemcpyAsync((int32_t *)w.X.p + P.sets[s2].x_off, sets[s2].X,
                                 (size_t)sets[s2].n * sets[s2].p * 4, cudaMemcpyDeviceToDevice, s));
        *x_arena = (const int32_t *)w.X.p;
    } else {
        int32_t *hx = (int32_t *)(((uintptr_t)(hs + small) + 63) & ~(uintptr_t)63);
        for (int s2 = 0; s2 < k; ++s2)
            memcpy(hx + P.sets[s2].x_off, sets[s2].X, (size_t)sets[s2].n * sets[s2].p * 4);
        TDCK(cudaMemcpyAsync(w.X.p, hx, P.x_elems * 4, cudaMemcpyHostToDevice, s));
        *x_arena = (const int32_t *)w.X.p;
    }
    return TD_OK;
}

TdLaunch make_launch(const Work &w, const Plan &P, const int32_t *x_arena, const td_options &o, int warps,
                     int blog2, const uint16_t (*tune)[TD_NOCT])
{
    TdLaunch L;
    memset(&L, 0, sizeof(L));
    if (tune) memcpy(L.spw_tab, tune, sizeof(L.spw_tab));
    L.X = x_arena;
    L.Zq = (const int32_t *)w.Zq.p;
    L.sets = (const TdSet *)w.sets.p;
    L.q = (TdQuery *)w.q.p;
    L.nq = P.nq;
    L.warps = warps;
    L.order = (const int32_t *)w.order.p;
    L.tile_prefix = (int64_t *)w.prefix.p;
    L.tile_size = (int32_t *)w.tsize.p;
    L.ticket = (unsigned long long *)w.ticket.p;
    L.qmin = (int32_t *)w.qmin.p;
    L.out = (int32_t *)w.out.p;
    L.ctr = (TdCounters *)w.ctr.p;
    L.shard_index = o.shard_count > 1 ? o.shard_index : 0;
    L.shard_count = o.shard_count > 1 ? o.shard_count : 1;
    L.spw = o.subsets_per_warp;
    L.blog2 = blog2;
    L.nmax = P.nmax;
    L.pmax = P.pmax;
    L.scratch = (char *)w.scratch.p;
    L.scratch_per_warp = td_scratch_per_warp(P.nmax);
    L.early_exit = o.early_exit != 0;
    L.unseeded = o.unseeded != 0;
    L.adia = o.algorithm == TD_ALG_ADIA;
    L.critical = o.algorithm == TD_ALG_CRITICAL;
    if (L.adia) {
        L.perm = (uint16_t *)w.perm.p;
        L.perm_stride = P.nmax;
        L.adia_keys = (uint64_t *)w.akeys.p;
        L.adia_dep = (int32_t *)w.adep.p;
        L.adia_stack = (int32_t *)w.astk.p;
    }
    return L;
}

/* Enqueue the kernels of one call on stream s.  Returns launches issued.
 * ev_a / ev_b (may be null) are recorded around the sweep kernel(s).  The
 * plain form needs each query's effective dimension, read back after the
 * set-up kernel (so it is never captured in a graph). */
int enqueue_kernels(td_ctx *ctx, Work &w, const Plan &P, const TdLaunch &Lf, const td_options &o, int blog2,
                    cudaStream_t s, int *launches, cudaEvent_t ev_a = nullptr, cudaEvent_t ev_b = nullptr)
{
    int nl = 0;
    if (o.algorithm == TD_ALG_CRITICAL) {
        /* Proposition 1 with r = p-1: one launch per query, after reading
         * back each query's effective dimension */
        TdLaunch L = Lf;
        L.warps = td_critical_threads() / 32;
        L.scratch_per_warp = td_scratch_per_warp_critical(P.nmax);
        const size_t smem = td_critical_smem(P.nmax, P.pmax);
        TDCK(td_launch_setup(L, s));
        nl += 2; /* set-up and the data-direction bound */
        std::vector<TdQuery> hq(P.nq);
        TDCK(cudaMemcpyAsync(hq.data(), w.q.p, P.nq * sizeof(TdQuery), cudaMemcpyDeviceToHost, s));
        TDCK(cudaStreamSynchronize(s));
        if (ev_a) TDCK(cudaEventRecord(ev_a, s));
        for (int q = 0; q < P.nq; ++q) {
            const int D = hq[q].d;
            if (hq[q].k < 0 || hq[q].hi <= hq[q].lo || D < 2 || D > 6) continue;
            const int occ = td_critical_occupancy(D, smem);
            if (occ < 1) return TD_ERR_INVALID;
            TDCK(td_launch_critical(D, L, q, ctx->sms * occ, smem, s));
            ++nl;
        }
        if (ev_b) TDCK(cudaEventRecord(ev_b, s));
        TDCK(td_launch_wide(L, ctx->sms, s));
        TDCK(td_launch_finalize(L, s));
        nl += 2;
    } else if (o.mode == TD_MODE_PLAIN_EXACT) {
        TdLaunch L = Lf;
        L.warps = kWarpsPlain;
        size_t smem = td_plain_smem(P.nmax, P.pmax, kWarpsPlain);
        TDCK(td_launch_setup(L, s));
        nl += 2; /* set-up and the data-direction bound */
        std::vector<TdQuery> hq(P.nq);
        TDCK(cudaMemcpyAsync(hq.data(), w.q.p, P.nq * sizeof(TdQuery), cudaMemcpyDeviceToHost, s));
        TDCK(cudaStreamSynchronize(s));
        if (ev_a) TDCK(cudaEventRecord(ev_a, s));
        for (int q = 0; q < P.nq; ++q) {
            const int D = hq[q].d;
            if (hq[q].k < 0 || hq[q].hi <= hq[q].lo || D < 2 || D > 6) continue;
            int occ = td_plain_occupancy(D, kWarpsPlain, smem);
            if (occ < 1) return TD_ERR_INVALID;
            TDCK(td_launch_plain(D, L, q, ctx->sms * occ, smem, s));
            ++nl;
        }
        if (ev_b) TDCK(cudaEventRecord(ev_b, s));
        TDCK(td_launch_wide(L, ctx->sms, s));
        TDCK(td_launch_finalize(L, s));
        nl += 2;
    } else {
        TDCK(td_launch_setup(Lf, s));
        nl = 2; /* set-up and the data-direction bound */
        if (Lf.adia) {
            /* Algorithm 3, Steps 2-5(a): the search sets each query's subset
             * range, staging order and running minimum for the sweep */
            for (int D = 3; D <= std::min(P.pmax, 6); ++D) {
                TdLaunch LD = Lf;
                LD.nmax = P.nmaxD[D - 2];
                LD.pmax = D;
                LD.scratch_per_warp = td_scratch_per_warp(LD.nmax);
                TDCK(td_launch_adia(D, LD, w.agrid[D - 2], w.asmem[D - 2], s));
                ++nl;
            }
        }
        TDCK(td_launch_tiles(Lf, s));
        ++nl;
        /* inside a stream capture only an "external" record becomes an event
         * node of the graph; outside a capture the flag changes nothing */
        if (ev_a) TDCK(cudaEventRecordWithFlags(ev_a, s, cudaEventRecordExternal));
        for (int D = 2; D <= std::min(P.pmax, 6); ++D) {
            /* each dimension's kernel is sized for the datasets that can
             * hold queries of that dimension (p >= D) */
            TdLaunch LD = Lf;
            LD.nmax = P.nmaxD[D - 2];
            LD.pmax = D;
            LD.blog2 = blog2_for(LD.nmax, o);
            LD.scratch_per_warp = td_scratch_per_warp(LD.nmax);
            const size_t smemD = td_filtered_smem(LD.nmax, D, LD.blog2, LD.warps);
            TDCK(td_launch_filtered(D, LD, w.grid[D - 2], smemD, s));
            ++nl;
        }
        if (ev_b) TDCK(cudaEventRecordWithFlags(ev_b, s, cudaEventRecordExternal));
        TDCK(td_launch_wide(Lf, ctx->sms, s));
        TDCK(td_launch_finalize(Lf, s));
        nl += 2;
    }
    *launches = nl;
    return TD_OK;
}

/* Persistent grids of the sweep kernels (D = 2 .. min(pmax, 6)), each sized
 * for its own dimension (rows of at most nmaxD points, stride 4 or 8 floats),
 * in CTAs of kWarpsFiltered warps; sets the dynamic shared memory attribute
 * of each.  Returns the scratch bytes the largest grid needs, or 0 if a
 * kernel cannot be resident. */
size_t filtered_grids(td_ctx *ctx, const Plan &P, const td_options &o, int *grid)
{
    const int wsel = kWarpsFiltered;
    size_t scratch = 256;
    for (int i = 0; i < TD_NDIM; ++i) grid[i] = 0;
    for (int D = 2; D <= std::min(P.pmax, 6); ++D) {
        const int nmaxD = P.nmaxD[D - 2];
        const size_t smem = td_filtered_smem(nmaxD, D, blog2_for(nmaxD, o), wsel);
        int occ = td_filtered_occupancy(D, wsel, smem);
        if (occ < 1) return 0;
        grid[D - 2] = ctx->sms * occ;
        scratch = std::max(scratch, (size_t)grid[D - 2] * wsel * (size_t)td_scratch_per_warp(nmaxD));
    }
    return scratch;
}

/* Algorithm 3: grid and shared memory of the search kernel of every
 * dimension D = 3 .. min(pmax, 6), and its buffers (staging order per query,
 * node tables per CTA).  Returns the scratch bytes it needs, or 0 if a kernel
 * cannot be resident. */
size_t adia_prepare(td_ctx *ctx, Work &w, const Plan &P, cudaError_t *err)
{
    *err = cudaSuccess;
    size_t scratch = 256;
    int gmax = 0;
    for (int D = 3; D <= std::min(P.pmax, 6); ++D) {
        const int nmaxD = P.nmaxD[D - 2];
        const size_t smem = td_adia_smem(nmaxD, D);
        if (smem > (size_t)ctx->smem_optin) return 0;
        const int occ = td_adia_occupancy(D, nmaxD, smem);
        if (occ < 1) return 0;
        const int grid = std::max(1, std::min(P.nq, ctx->sms * occ));
        w.agrid[D - 2] = grid;
        w.asmem[D - 2] = smem;
        gmax = std::max(gmax, grid);
        scratch = std::max(scratch, (size_t)grid * td_adia_scratch_slots(nmaxD) * (size_t)td_scratch_per_warp(nmaxD));
    }
    const size_t ent = (size_t)std::max(gmax, 1) * (size_t)td_adia_ws_entries();
    cudaError_t e = grow(w.perm, (size_t)std::max(P.nq, 1) * P.nmax * 2);
    if (e == cudaSuccess) e = grow(w.akeys, ent * 8);
    if (e == cudaSuccess) e = grow(w.adep, ent * 4);
    if (e == cudaSuccess) e = grow(w.astk, ent * 4);
    *err = e;
    return scratch;
}

/* One synchronous batched call. */
int run_batch(td_ctx *ctx, const td_dataset *sets, int k, td_stats *st)
{
    if (!ctx || (!sets && k > 0) || k < 0) return TD_ERR_INVALID;
    const bool devptr = ctx->opt.device_pointers != 0;
    for (int s2 = 0; s2 < k; ++s2) {
        int v = validate_set(sets[s2]);
        if (v != TD_OK) return v;
    }
    if (st) memset(st, 0, sizeof(*st));
    Plan P = make_plan(sets, k);
    if (P.nq == 0) return TD_OK;
    const td_options &o = ctx->opt;
    cudaStream_t s = stream_of(ctx);
    const int blog2 = blog2_for(P.nmax, o);
    int grid = 0, warps_total = 0;
    (void)cudaGetLastError(); /* clear any stale error of an earlier call */
    int grids[TD_NDIM] = { 0, 0, 0, 0, 0 };
    if (o.algorithm == TD_ALG_CRITICAL) {
        const size_t smem = td_critical_smem(P.nmax, P.pmax);
        int occ = 0;
        for (int D = 2; D <= 6; ++D) occ = std::max(occ, td_critical_occupancy(D, smem));
        if (occ < 1) return TD_ERR_INVALID;
        grid = ctx->sms * occ;
        warps_total = grid * (td_critical_threads() / 32);
        TDCK(alloc_work(ctx->w, P, warps_total, true));
        /* the critical kernel lays its per-warp scratch out for 2 nmax points */
        TDCK(grow(ctx->w.scratch, (size_t)warps_total * (size_t)td_scratch_per_warp_critical(P.nmax)));
    } else if (o.mode == TD_MODE_PLAIN_EXACT) {
        size_t smem = td_plain_smem(P.nmax, P.pmax, kWarpsPlain);
        int occ = 0;
        for (int D = 2; D <= 6; ++D) occ = std::max(occ, td_plain_occupancy(D, kWarpsPlain, smem));
        if (occ < 1) return TD_ERR_INVALID;
        grid = ctx->sms * occ;
        warps_total = grid * kWarpsPlain;
        TDCK(alloc_work(ctx->w, P, warps_total, true));
    } else {
        size_t scratch = filtered_grids(ctx, P, o, grids);
        if (scratch < 1) return TD_ERR_INVALID;
        TDCK(alloc_work(ctx->w, P, 0, true));
        if (o.algorithm == TD_ALG_ADIA) {
            cudaError_t ae;
            const size_t as = adia_prepare(ctx, ctx->w, P, &ae);
            TDCK(ae);
            if (as < 1) return TD_ERR_INVALID;
            scratch = std::max(scratch, as);
        }
        TDCK(grow(ctx->w.scratch, scratch));
    }
    memcpy(ctx->w.grid, grids, sizeof(grids));
    const int32_t *x_arena = nullptr;
    int rc = stage_inputs(ctx, ctx->w, ctx->hstage, P, sets, k, devptr, s, &x_arena);
    if (rc != TD_OK) return rc;
    TDCK(cudaMemsetAsync(ctx->w.ctr.p, 0, sizeof(TdCounters), s));
    TdLaunch L = make_launch(ctx->w, P, x_arena, o, kWarpsFiltered, blog2, ctx->tune);
    TDCK(cudaEventRecord(ctx->ev0, s));
    int launches = 0;
    if (o.mode == TD_MODE_FILTERED && o.use_graph && o.algorithm != TD_ALG_CRITICAL) {
        GraphKey key;
        memset(&key, 0, sizeof(key));
        key.nq = P.nq;
        key.nsets = P.nsets;
        key.nmax = P.nmax;
        key.pmax = P.pmax;
        memcpy(key.grid, grids, sizeof(grids));
        memcpy(key.nmaxD, P.nmaxD, sizeof(P.nmaxD));
        key.blog2 = blog2;
        key.spw = o.subsets_per_warp;
        key.early_exit = L.early_exit;
        key.unseeded = L.unseeded;
        memcpy(key.spw_tab, L.spw_tab, sizeof(key.spw_tab));
        key.algorithm = o.algorithm;
        key.warps = L.warps;
        key.smem = td_filtered_smem(P.nmax, P.pmax, blog2, L.warps);
        const Work &cw = ctx->w;
        const void *pp[17] = { x_arena,     cw.Zq.p,   cw.sets.p,  cw.q.p,     cw.order.p, cw.prefix.p,
                               cw.tsize.p,  cw.ticket.p, cw.qmin.p, cw.out.p,   cw.ctr.p,   cw.scratch.p,
                               cw.X.p,      cw.perm.p, cw.akeys.p, cw.adep.p,  cw.astk.p };
        memcpy(key.ptrs, pp, sizeof(pp));
        key.shard_index = L.shard_index;
        key.shard_count = L.shard_count;
        if (!ctx->gvalid || !(key == ctx->gkey)) {
            if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
            ctx->gexec = nullptr;
            ctx->gvalid = false;
            cudaStream_t cs = nullptr;
            TDCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                cudaStreamDestroy(cs);
                return fail_cuda(ctx, e, "cudaStreamBeginCapture");
            }
            int nl = 0;
            int rc2 = enqueue_kernels(ctx, ctx->w, P, L, o, blog2, cs, &nl, ctx->evs0, ctx->evs1);
            e = cudaStreamEndCapture(cs, &g);
            cudaStreamDestroy(cs);
            if (rc2 != TD_OK) {
                if (g) cudaGraphDestroy(g);
                return rc2;
            }
            if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ctx->gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail_cuda(ctx, e, "cudaGraphInstantiate");
            ctx->gkey = key;
            ctx->gvalid = true;
        }
        TDCK(cudaGraphLaunch(ctx->gexec, s));
        launches = 5 + std::min(P.pmax, 6) - 1; /* set-up, bound, tiles, sweeps for D = 2..min(p,6), wide, finalize */
        if (L.adia) launches += std::max(0, std::min(P.pmax, 6) - 2); /* search kernels, D = 3..min(p,6) */
    } else {
        rc = enqueue_kernels(ctx, ctx->w, P, L, o, blog2, s, &launches, ctx->evs0, ctx->evs1);
        if (rc != TD_OK) return rc;
    }
    TDCK(cudaEventRecord(ctx->ev1, s));
    /* check the device-side error counter before any output is written */
    TdCounters C;
    TDCK(cudaMemcpyAsync(&C, ctx->w.ctr.p, sizeof(C), cudaMemcpyDeviceToHost, s));
    TDCK(cudaStreamSynchronize(s));
    if (C.errors != 0) return TD_ERR_INTERNAL;
    if (devptr) {
        int qi = 0;
        for (int s2 = 0; s2 < k; ++s2) {
            if (sets[s2].m > 0)
                TDCK(cudaMemcpyAsync(sets[s2].out, (int32_t *)ctx->w.out.p + qi, sets[s2].m * 4,
                                     cudaMemcpyDeviceToDevice, s));
            qi += sets[s2].m;
        }
        TDCK(cudaStreamSynchronize(s));
    } else {
        TDCK(grow_host(ctx->hout, (size_t)P.nq * 4));
        TDCK(cudaMemcpyAsync(ctx->hout.p, ctx->w.out.p, (size_t)P.nq * 4, cudaMemcpyDeviceToHost, s));
        TDCK(cudaStreamSynchronize(s));
        int qi = 0;
        for (int s2 = 0; s2 < k; ++s2) {
            memcpy(sets[s2].out, (int32_t *)ctx->hout.p + qi, (size_t)sets[s2].m * 4);
            qi += sets[s2].m;
        }
    }
    if (st) {
        st->sweeps = C.sweeps;
        st->skipped_dependent = C.dependent;
        st->filtered_points = C.filtered_points;
        st->exact_points = C.exact_points;
        st->tight_exceptions = C.tight;
        st->resolved_buckets = C.resolved;
        st->early_skipped = C.early;
        st->rescanned_sweeps = C.rescanned;
        st->adia_pops = C.adia_pops;
        st->adia_subsets = C.adia_subsets;
        st->adia_union_points = C.adia_union;
        st->adia_fallbacks = C.adia_fallback;
        st->kernel_launches = (uint64_t)launches;
        float ms = 0.f, mss = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1) != cudaSuccess) ms = -1.f;
        if (cudaEventElapsedTime(&mss, ctx->evs0, ctx->evs1) != cudaSuccess) mss = -1.f;
        st->ms = ms;
        st->ms_sweep = mss;
    }
    return TD_OK;
}

}  // namespace

/* ======================================================================= */
/* exported entry points                                                    */
/* ======================================================================= */

extern "C" int64_t td_coord_limit(int32_t p) { return td_coord_limit_of(p); }

extern "C" const char *td_strerror(int code)
{
    switch (code) {
    case TD_OK: return "ok";
    case TD_ERR_INVALID: return "invalid argument";
    case TD_ERR_RANGE: return "coordinates exceed the exact-arithmetic limit";
    case TD_ERR_OOM: return "out of memory";
    case TD_ERR_BUSY: return "stream admission refused (memory budget)";
    case TD_ERR_TIMEOUT: return "timed out";
    case TD_ERR_CUDA: return "CUDA error";
    case TD_ERR_NOTFOUND: return "unknown ticket";
    case TD_ERR_INTERNAL: return "device-side consistency check failed";
    default: return "unknown error";
    }
}

extern "C" const char *td_last_cuda_error(td_ctx *ctx) { return ctx ? ctx->cuda_err.c_str() : ""; }

extern "C" int td_create(td_ctx **out, int device, const td_options *opt)
{
    if (!out) return TD_ERR_INVALID;
    *out = nullptr;
    td_ctx *ctx = new (std::nothrow) td_ctx();
    if (!ctx) return TD_ERR_OOM;
    ctx->device = device;
    ctx->opt = opt ? *opt : default_options();
    if (ctx->opt.shard_count < 1) ctx->opt.shard_count = 1;
    if (validate_options(ctx->opt) != TD_OK) {
        delete ctx;
        return TD_ERR_INVALID;
    }
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->evs0);
    if (e == cudaSuccess) e = cudaEventCreate(&ctx->evs1);
    if (e != cudaSuccess) {
        int rc = fail_cuda(ctx, e, "td_create");
        td_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return TD_OK;
}

extern "C" int td_set_options(td_ctx *ctx, const td_options *opt)
{
    if (!ctx || !opt) return TD_ERR_INVALID;
    td_options o = *opt;
    if (o.shard_count < 1) o.shard_count = 1;
    if (validate_options(o) != TD_OK) return TD_ERR_INVALID;
    ctx->opt = *opt;
    if (ctx->opt.shard_count < 1) ctx->opt.shard_count = 1;
    ctx->gvalid = false;
    return TD_OK;
}

extern "C" int td_destroy(td_ctx *ctx)
{
    if (!ctx) return TD_ERR_INVALID;
    cudaSetDevice(ctx->device);
    if (ctx->own) cudaStreamSynchronize(ctx->own);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    Work &w = ctx->w;
    DevBuf *bufs[] = { &w.X,      &w.Zq,  &w.sets, &w.q,     &w.order, &w.prefix, &w.tsize, &w.ticket,
                       &w.qmin,   &w.out, &w.ctr,  &w.scratch, &w.perm, &w.akeys, &w.adep,  &w.astk };
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (ctx->hstage.p) cudaFreeHost(ctx->hstage.p);
    if (ctx->hout.p) cudaFreeHost(ctx->hout.p);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    if (ctx->evs0) cudaEventDestroy(ctx->evs0);
    if (ctx->evs1) cudaEventDestroy(ctx->evs1);
    if (ctx->own) cudaStreamDestroy(ctx->own);
    delete ctx;
    return TD_OK;
}

extern "C" int td_depth(td_ctx *ctx, const int32_t *X, int32_t n, int32_t p, const int32_t *Z, int32_t m,
                        int32_t *out, td_stats *st)
{
    if (!ctx) return TD_ERR_INVALID;
    td_dataset d;
    d.n = n;
    d.p = p;
    d.X = X;
    d.m = m;
    d.Z = Z;
    d.out = out;
    cudaSetDevice(ctx->device);
    return run_batch(ctx, &d, 1, st);
}

extern "C" int td_depth_batched(td_ctx *ctx, const td_dataset *sets, int32_t k, td_stats *st)
{
    if (!ctx) return TD_ERR_INVALID;
    cudaSetDevice(ctx->device);
    return run_batch(ctx, sets, k, st);
}

/* ----------------------------------------------------------------------- */
/* autotuner                                                                */
/* ----------------------------------------------------------------------- */

namespace {

/* candidates of the work-tile size (subsets per warp) */
const int kTuneSpw[TD_TUNE_MAX] = { 16, 32, 64, 128, 192, 256, 512, 1024 };
const int kTuneCount = 8;
/* a candidate replaces the size rule only when it is faster by more than
 * this fraction: the synthetic problem is a proxy, and closer times say
 * more about it and about timing noise than about the caller's data */
constexpr float kTuneMargin = 0.01f;

/* A seeded synthetic dataset of n points in dimension p, uniform integers in
 * [-127, 127] (a 64-bit xorshift generator), and m queries: data rows and
 * uniform points alternately. */
void tune_data(int n, int p, int m, std::vector<int32_t> &X, std::vector<int32_t> &Z)
{
    uint64_t x = 0x9E3779B97F4A7C15ull ^ ((uint64_t)n << 8) ^ (uint64_t)p;
    auto next = [&]() {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        return (int32_t)((x >> 11) % 255) - 127;
    };
    X.resize((size_t)n * p);
    for (auto &v : X) v = next();
    Z.resize((size_t)m * p);
    for (int q = 0; q < m; ++q)
        for (int c = 0; c < p; ++c) Z[(size_t)q * p + c] = (q & 1) ? next() : X[(size_t)((q * 7919) % n) * p + c];
}

/* Median device time of the sweep kernels over three calls (one untimed
 * call first, which also captures the graph). */
int tune_time(td_ctx *ctx, const td_dataset &d, float *ms)
{
    float t[3];
    td_stats st;
    int rc = run_batch(ctx, &d, 1, &st);
    for (int r = 0; r < 3 && rc == TD_OK; ++r) {
        rc = run_batch(ctx, &d, 1, &st);
        t[r] = st.ms_sweep;
    }
    if (rc != TD_OK) return rc;
    std::sort(t, t + 3);
    *ms = t[1];
    return TD_OK;
}

}  // namespace

extern "C" int td_autotune(td_ctx *ctx, int32_t p, int32_t n, td_tune_result *res)
{
    if (!ctx || p < 3 || p > TD_MAX_P || n < p + 1 || n > TD_MAX_N) return TD_ERR_INVALID;
    cudaSetDevice(ctx->device);
    /* queries enough for about 10 ms of sweeping: about 1e10 point
     * evaluations (C(n, p-2) n each), so that the launch's last partial
     * wave of tiles weighs little */
    double cost = (double)n;
    for (int i = 0; i < p - 2; ++i) cost *= (double)(n - i) / (i + 1);
    const int m = (int)std::max(1.0, std::min(256.0, 1e10 / cost));
    std::vector<int32_t> X, Z, out((size_t)m);
    tune_data(n, p, m, X, Z);
    td_dataset d;
    d.n = n;
    d.p = p;
    d.X = X.data();
    d.m = m;
    d.Z = Z.data();
    d.out = out.data();
    const td_options saved = ctx->opt;
    uint16_t saved_tab[TD_NDIM][TD_NOCT];
    memcpy(saved_tab, ctx->tune, sizeof(saved_tab));
    td_options o = saved;
    o.mode = TD_MODE_FILTERED;
    o.device_pointers = 0;
    o.early_exit = 0;
    o.algorithm = TD_ALG_RCOM;
    o.unseeded = 0;
    o.shard_index = 0;
    o.shard_count = 1;
    o.buckets_log2 = 0;
    ctx->opt = o;
    const int D = p, oct = td_octave(n), oct1 = td_octave(n - 1);
    td_tune_result r;
    memset(&r, 0, sizeof(r));
    r.p = p;
    r.n = n;
    r.queries = m;
    int rc = TD_OK;
    /* the size rule (no table entry, subsets_per_warp = 0) first */
    ctx->tune[D - 2][oct] = ctx->tune[D - 2][oct1] = 0;
    ctx->opt.subsets_per_warp = 0;
    rc = tune_time(ctx, d, &r.ms_default);
    r.best_ms = r.ms_default;
    r.best_spw = 0;
    for (int k = 0; k < kTuneCount && rc == TD_OK; ++k) {
        ctx->opt.subsets_per_warp = kTuneSpw[k];
        float ms = 0.f;
        rc = tune_time(ctx, d, &ms);
        r.spw[k] = kTuneSpw[k];
        r.ms[k] = ms;
        if (rc == TD_OK && ms < r.best_ms && ms < r.ms_default * (1.0f - kTuneMargin)) {
            r.best_ms = ms;
            r.best_spw = kTuneSpw[k];
        }
    }
    r.candidates = kTuneCount;
    ctx->opt = saved;
    memcpy(ctx->tune, saved_tab, sizeof(saved_tab));
    if (rc != TD_OK) return rc;
    /* the fastest, kept for rows of this dimension and octave (0: the size
     * rule was fastest) */
    ctx->tune[D - 2][oct] = (uint16_t)r.best_spw;
    ctx->tune[D - 2][oct1] = (uint16_t)r.best_spw;
    ctx->gvalid = false;
    if (res) *res = r;
    return TD_OK;
}

extern "C" int td_set_tuned(td_ctx *ctx, int32_t d, int32_t octave, int32_t subsets_per_warp)
{
    if (!ctx || d < 2 || d > 6 || octave < 0 || octave >= TD_NOCT || subsets_per_warp < 0 ||
        subsets_per_warp > 4096)
        return TD_ERR_INVALID;
    ctx->tune[d - 2][octave] = (uint16_t)subsets_per_warp;
    ctx->gvalid = false;
    return TD_OK;
}

/* ----------------------------------------------------------------------- */
/* stream API                                                               */
/* ----------------------------------------------------------------------- */

namespace {

size_t request_bytes(int n, int p, int m)
{
    return (size_t)n * p * 4 + (size_t)m * (TD_MAXD * 4 + sizeof(TdQuery) + 4 + 8 * TD_NDIM + 4 + 4 + 4) + 4096;
}

/* Point evaluations (C(n, p-2) n a query) of a stream slice: about 25 ms
 * of sweeping on one GB300.  A batch takes every waiting request of one
 * slice and the next slice of the sliced ones in arrival order while their
 * work stays within kBatchWork (at least one), so that a small request waits
 * behind at most a batch of bounded work however large the requests before
 * it are. */
constexpr double kSliceWork = 1.5e10;
constexpr double kBatchWork = 3.0e10;

/* Finish a slot whose event completed: merge every slice's counts into its
 * request, and hand a request its outputs once its last slice is in. */
void complete_slot(td_stream *s, int k)
{
    td_stream_slot &sl = s->slot[k];
    const int32_t *h = (const int32_t *)sl.hout.p;
    const TdCounters *c = (const TdCounters *)(h + ((sl.nq + 3) & ~3));
    const bool ok = c->errors == 0;
    for (const td_slice_entry &e : sl.ents) {
        td_stream_req *r = e.r;
        if (ok) {
            for (int j = 0; j < r->m; ++j) r->acc[j] = std::min(r->acc[j], h[e.out_off + j]);
        } else {
            r->status = TD_ERR_INTERNAL;
        }
        if (++r->done_slices == r->nslices) {
            if (r->status == TD_OK) memcpy(r->user_out, r->acc.data(), (size_t)r->m * 4);
            r->finished = true;
            s->inflight -= r->bytes;
            std::vector<int32_t>().swap(r->X);
            std::vector<int32_t>().swap(r->Z);
            std::vector<int32_t>().swap(r->acc);
        }
    }
    sl.ents.clear();
    sl.busy = false;
}

/* Reap finished slots, then launch the next slices of the waiting requests
 * as one batch into a free slot.  Returns TD_OK or a CUDA error code. */
int pump(td_stream *s)
{
    td_ctx *ctx = s->ctx;
    for (int k = 0; k < 2; ++k)
        if (s->slot[k].busy) {
            cudaError_t e = cudaEventQuery(s->slot[k].done);
            if (e == cudaSuccess) complete_slot(s, k);
            else if (e != cudaErrorNotReady) return fail_cuda(ctx, e, "cudaEventQuery");
        }
    if (s->pending.empty()) return TD_OK;
    int k = !s->slot[0].busy ? 0 : (!s->slot[1].busy ? 1 : -1);
    if (k < 0) return TD_OK;
    td_stream_slot &sl = s->slot[k];
    std::vector<td_dataset> sets;
    std::vector<td_slice_entry> ents;
    int64_t off = 0;
    double work = 0.0;
    for (td_stream_req *r : s->pending) {
        /* the next slice of a sliced request joins while the batch's work
         * stays within kBatchWork; a request of one slice always joins */
        if (r->nslices > 1 && !ents.empty() && work + r->slice_work > kBatchWork) continue;
        td_dataset d;
        d.n = r->n;
        d.p = r->p;
        d.X = r->X.data();
        d.m = r->m;
        d.Z = r->Z.data();
        d.out = nullptr;
        sets.push_back(d);
        ents.push_back({ r, r->next_slice++, off });
        off += r->m;
        work += r->slice_work;
    }
    s->pending.erase(std::remove_if(s->pending.begin(), s->pending.end(),
                                    [](td_stream_req *r) { return r->next_slice >= r->nslices; }),
                     s->pending.end());
    Plan P = make_plan(sets.data(), (int)sets.size());
    for (size_t i = 0; i < ents.size(); ++i) {
        P.sets[i].slice_index = ents[i].slice;
        P.sets[i].slice_count = ents[i].r->nslices;
    }
    td_options o = ctx->opt;
    o.mode = TD_MODE_FILTERED;
    o.device_pointers = 0;
    o.shard_count = 1;
    o.shard_index = 0;
    const int blog2 = blog2_for(P.nmax, o);
    (void)cudaGetLastError();
    int grids[TD_NDIM] = { 0, 0, 0, 0, 0 };
    size_t scratch = filtered_grids(ctx, P, o, grids);
    if (scratch < 1) return TD_ERR_INVALID;
    cudaError_t e = alloc_work(sl.w, P, 0, true);
    if (e == cudaSuccess && o.algorithm == TD_ALG_ADIA) {
        const size_t as = adia_prepare(ctx, sl.w, P, &e);
        if (e == cudaSuccess && as < 1) return TD_ERR_INVALID;
        scratch = std::max(scratch, as);
    }
    if (e == cudaSuccess) e = grow(s->scratch, scratch);
    if (e == cudaSuccess && !sl.done) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    const size_t outb = (size_t)((P.nq + 3) & ~3) * 4 + sizeof(TdCounters);
    if (e == cudaSuccess) e = grow_host(sl.hout, outb);
    if (e != cudaSuccess) return fail_cuda(ctx, e, "stream batch buffers");
    memcpy(sl.w.grid, grids, sizeof(grids));
    const int32_t *x_arena = nullptr;
    int rc = stage_inputs(ctx, sl.w, sl.hstage, P, sets.data(), (int)sets.size(), false, s->s, &x_arena);
    if (rc != TD_OK) return rc;
    TdLaunch L = make_launch(sl.w, P, x_arena, o, kWarpsFiltered, blog2, ctx->tune);
    L.scratch = (char *)s->scratch.p;
    TDCK(cudaMemsetAsync(sl.w.ctr.p, 0, sizeof(TdCounters), s->s));
    int nl = 0;
    rc = enqueue_kernels(ctx, sl.w, P, L, o, blog2, s->s, &nl);
    if (rc != TD_OK) return rc;
    TDCK(cudaMemcpyAsync(sl.hout.p, sl.w.out.p, (size_t)P.nq * 4, cudaMemcpyDeviceToHost, s->s));
    TDCK(cudaMemcpyAsync((int32_t *)sl.hout.p + ((P.nq + 3) & ~3), sl.w.ctr.p, sizeof(TdCounters),
                         cudaMemcpyDeviceToHost, s->s));
    TDCK(cudaEventRecord(sl.done, s->s));
    sl.ents.swap(ents);
    sl.nq = P.nq;
    sl.busy = true;
    return TD_OK;
}

td_stream_req *find_req(td_stream *s, uint64_t ticket)
{
    for (td_stream_req *r : s->reqs)
        if (r->ticket == ticket) return r;
    return nullptr;
}

}  // namespace

extern "C" int td_stream_create(td_ctx *ctx, size_t mem_budget_bytes, td_stream **out)
{
    if (!ctx || !out) return TD_ERR_INVALID;
    *out = nullptr;
    if (ctx->opt.algorithm == TD_ALG_CRITICAL) return TD_ERR_INVALID; /* a synchronous cross-check form */
    td_stream *s = new (std::nothrow) td_stream();
    if (!s) return TD_ERR_OOM;
    s->ctx = ctx;
    s->budget = mem_budget_bytes;
    s->inflight = 0;
    s->next = 1;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return fail_cuda(ctx, e, "td_stream_create");
    }
    *out = s;
    return TD_OK;
}

extern "C" int td_stream_submit(td_stream *s, const td_dataset *d, uint64_t *ticket)
{
    if (!s || !d || !ticket) return TD_ERR_INVALID;
    td_ctx *ctx = s->ctx;
    if (ctx->opt.device_pointers) return TD_ERR_INVALID; /* the stream takes host inputs */
    int v = validate_set(*d);
    if (v != TD_OK) return v;
    cudaSetDevice(ctx->device);
    int rc = pump(s); /* reaps finished batches first (frees budget) */
    if (rc != TD_OK) return rc;
    size_t bytes = request_bytes(d->n, d->p, d->m);
    if (ctx->opt.algorithm == TD_ALG_ADIA) bytes += (size_t)d->m * d->n * 2; /* staging order per query */
    if (s->inflight + bytes > s->budget) return TD_ERR_BUSY;
    td_stream_req *r = new (std::nothrow) td_stream_req();
    if (!r) return TD_ERR_OOM;
    r->ticket = s->next++;
    r->n = d->n;
    r->p = d->p;
    r->m = d->m;
    r->X.assign(d->X, d->X + (size_t)d->n * d->p); /* the caller may reuse its inputs on return */
    if (d->m > 0) r->Z.assign(d->Z, d->Z + (size_t)d->m * d->p);
    r->user_out = d->out;
    r->bytes = bytes;
    /* time slices: about kSliceWork point evaluations each (Algorithm 3's
     * search is not sliced) */
    double work = (double)d->n * d->m;
    for (int i = 0; i < d->p - 2; ++i) work *= (double)(d->n - i) / (i + 1);
    int ns = (int)std::min(std::ceil(work / kSliceWork), 1048576.0);
    if (ctx->opt.algorithm == TD_ALG_ADIA || ns < 1) ns = 1;
    r->nslices = ns;
    r->next_slice = 0;
    r->done_slices = 0;
    r->slice_work = work / ns;
    r->acc.assign((size_t)d->m, INT32_MAX);
    r->finished = d->m == 0;
    r->status = TD_OK;
    s->reqs.push_back(r);
    if (!r->finished) {
        s->inflight += bytes;
        s->pending.push_back(r);
        rc = pump(s);
        if (rc != TD_OK) return rc;
    }
    *ticket = r->ticket;
    return TD_OK;
}

extern "C" int td_stream_poll(td_stream *s, uint64_t ticket, int *done)
{
    if (!s || !done) return TD_ERR_INVALID;
    td_stream_req *r = find_req(s, ticket);
    if (!r) return TD_ERR_NOTFOUND;
    if (!r->finished) {
        cudaSetDevice(s->ctx->device);
        int rc = pump(s);
        if (rc != TD_OK) return rc;
    }
    *done = r->finished ? 1 : 0;
    if (!r->finished) return TD_OK;
    /* reported: the ticket is forgotten */
    const int status = r->status;
    s->reqs.erase(std::find(s->reqs.begin(), s->reqs.end(), r));
    delete r;
    return status;
}

extern "C" int td_stream_wait(td_stream *s, uint64_t ticket, int64_t timeout_us)
{
    if (!s) return TD_ERR_INVALID;
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        int done = 0;
        int rc = td_stream_poll(s, ticket, &done);
        if (rc != TD_OK || done) return rc;
        if (timeout_us >= 0) {
            auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
            if (el >= timeout_us) return TD_ERR_TIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

extern "C" int td_stream_destroy(td_stream *s)
{
    if (!s) return TD_ERR_INVALID;
    cudaSetDevice(s->ctx->device);
    cudaStreamSynchronize(s->s);
    for (td_stream_req *r : s->reqs) delete r;
    for (int k = 0; k < 2; ++k) {
        td_stream_slot &sl = s->slot[k];
        Work &w = sl.w;
        DevBuf *bufs[] = { &w.X,    &w.Zq,  &w.sets, &w.q,       &w.order, &w.prefix, &w.tsize, &w.ticket,
                           &w.qmin, &w.out, &w.ctr,  &w.scratch, &w.perm,  &w.akeys,  &w.adep,  &w.astk };
        for (DevBuf *b : bufs)
            if (b->p) cudaFree(b->p);
        if (sl.hstage.p) cudaFreeHost(sl.hstage.p);
        if (sl.hout.p) cudaFreeHost(sl.hout.p);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    if (s->scratch.p) cudaFree(s->scratch.p);
    cudaStreamDestroy(s->s);
    delete s;
    return TD_OK;
}
