/*
 * td_noalloc.cu -- td_depth_noalloc: the depth computation for callers that
 * must not allocate device memory.
 *
 * Who needs it: code that runs where device memory is owned by someone else
 * -- inside a framework whose caching allocator holds the whole GPU and
 * forbids direct cudaMalloc, inside a process with a device-memory budget
 * fixed at load time, or on a latency-critical path where a cudaMalloc /
 * cudaFree pair would synchronise the device.  Such a caller passes its
 * device inputs and output buffer; every other buffer the kernels need lives
 * in one file-scope __device__ array of TD_NOALLOC_BYTES bytes, which the
 * module loader reserves on every GPU that loads this library and which stays
 * reserved until the process exits.
 *
 * The kernels are the ones of td_kernels.cu (set-up, tile prefix, persistent
 * sweep per dimension, finalize), launched with their work buffers carved out
 * of that array; two small kernels of this file initialise the tables and
 * fold the device-side checks into one status word.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "../../include/tukey_depth.h"
#include "td_internal.h"

size_t td_filtered_smem(int nmax, int pmax, int blog2, int warps);
int64_t td_scratch_per_warp(int nmax);
cudaError_t td_launch_setup(const TdLaunch &L, cudaStream_t s);
cudaError_t td_launch_tiles(const TdLaunch &L, cudaStream_t s);
cudaError_t td_launch_filtered(int D, const TdLaunch &L, int grid, size_t smem, cudaStream_t s);
cudaError_t td_launch_finalize(const TdLaunch &L, cudaStream_t s);
int td_filtered_occupancy(int D, int warps, size_t smem);

namespace {

constexpr int kWarps = 8;
constexpr size_t al256(size_t v) { return (v + 255) & ~(size_t)255; }

/* layout of the array (byte offsets, each region 256-byte aligned) */
constexpr size_t kZq = 0;
constexpr size_t kQ = kZq + al256((size_t)TD_NOALLOC_MAX_M * TD_MAXD * 4);
constexpr size_t kOrder = kQ + al256((size_t)TD_NOALLOC_MAX_M * sizeof(TdQuery));
constexpr size_t kPrefix = kOrder + al256((size_t)TD_NOALLOC_MAX_M * 4);
constexpr size_t kTsize = kPrefix + al256((size_t)TD_NDIM * (TD_NOALLOC_MAX_M + 1) * 8);
constexpr size_t kTicket = kTsize + al256((size_t)TD_NOALLOC_MAX_M * 4);
constexpr size_t kQmin = kTicket + al256((size_t)TD_NDIM * TD_TICKET_STRIDE * 8);
constexpr size_t kOut = kQmin + al256((size_t)TD_NOALLOC_MAX_M * 4);
constexpr size_t kCtr = kOut + al256((size_t)TD_NOALLOC_MAX_M * 4);
constexpr size_t kSets = kCtr + al256(sizeof(TdCounters));
constexpr size_t kStatus = kSets + al256(sizeof(TdSet));
constexpr size_t kScratch = kStatus + al256(4 * sizeof(unsigned long long));
/* per-warp scratch of the exact tight-set path, sized for TD_NOALLOC_MAX_N */
constexpr size_t kPerWarp = al256((size_t)256 * 72 * ((TD_NOALLOC_MAX_N + 255) / 256) + 256);
constexpr size_t kBytes = kScratch + (size_t)TD_NOALLOC_CTAS * kWarps * kPerWarp;
static_assert(kBytes <= (size_t)TD_NOALLOC_BYTES, "TD_NOALLOC_BYTES too small for the layout");

}  // namespace

/* The scratch.  Device code may name it; host code only ever uses the address
 * that cudaGetSymbolAddress returns for the current device (the host-side
 * symbol is a stand-in, not a device address). */
static __device__ __align__(256) unsigned char td_noalloc_scratch[TD_NOALLOC_BYTES];

/* initialise the tables one call needs (the array keeps the previous call's
 * contents): queries of dataset 0, identity work order, zero counters */
__global__ void td_k_noalloc_init(TdLaunch L, TdSet set, unsigned long long *status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < L.nq) {
        TdQuery Q;
        memset(&Q, 0, sizeof(Q));
        Q.set = 0;
        L.q[i] = Q;
        const_cast<int32_t *>(L.order)[i] = i;
    }
    if (i == 0) {
        const_cast<TdSet *>(L.sets)[0] = set;
        memset(L.ctr, 0, sizeof(TdCounters));
        status[0] = status[1] = 0ull;
    }
}

/* status[0] = device-side consistency failures, status[1] = queries with a
 * centred coordinate (any of the p) beyond the fast kernels' limit.  The
 * set-up kernel makes that test before anything else and gives such a query
 * no subset loop; this entry point does not run the wide kernel, so it
 * refuses them. */
__global__ void td_k_noalloc_status(TdLaunch L, unsigned long long *status)
{
    unsigned long long bad = 0;
    for (int i = threadIdx.x; i < L.nq; i += blockDim.x) bad += L.q[i].direct == TD_DIRECT_WIDE ? 1ull : 0ull;
    if (bad) atomicAdd(&status[1], bad);
    if (threadIdx.x == 0) status[0] = L.ctr->errors;
}

namespace {

std::mutex g_mu;
void *g_base[256];

/* Device address of the array on the current device, looked up once per
 * device.  The first call on a device does the lookup (and so makes the
 * module load there); make that first call before any stream capture. */
int scratch_base(void **base)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return TD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, td_noalloc_scratch) != cudaSuccess || !p) return TD_ERR_CUDA;
        g_base[dev] = p;
    }
    *base = g_base[dev];
    return TD_OK;
}

}  // namespace

extern "C" int td_depth_noalloc(const int32_t *X, int32_t n, int32_t p, const int32_t *Z, int32_t m,
                                int32_t *out, void *stream)
{
    if (!X || p < 1 || p > TD_MAX_P || n < 1 || m < 0) return TD_ERR_INVALID;
    if (n > TD_NOALLOC_MAX_N || m > TD_NOALLOC_MAX_M) return TD_ERR_INVALID; /* beyond the array's capacity */
    if (m == 0) return TD_OK;
    if (!Z || !out) return TD_ERR_INVALID;
    void *vbase = nullptr;
    int rc = scratch_base(&vbase);
    if (rc != TD_OK) return rc;
    char *base = (char *)vbase;
    cudaStream_t s = (cudaStream_t)stream;
    (void)cudaGetLastError();

    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TD_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TD_ERR_CUDA;
    int blog2 = 7;
    while ((2 << blog2) < n && blog2 < 11) ++blog2;

    TdLaunch L;
    memset(&L, 0, sizeof(L));
    L.X = X;
    L.Zq = (const int32_t *)(base + kZq);
    L.sets = (const TdSet *)(base + kSets);
    L.q = (TdQuery *)(base + kQ);
    L.nq = m;
    L.warps = kWarps;
    L.order = (const int32_t *)(base + kOrder);
    L.tile_prefix = (int64_t *)(base + kPrefix);
    L.tile_size = (int32_t *)(base + kTsize);
    L.ticket = (unsigned long long *)(base + kTicket);
    L.qmin = (int32_t *)(base + kQmin);
    L.out = (int32_t *)(base + kOut);
    L.ctr = (TdCounters *)(base + kCtr);
    L.shard_index = 0;
    L.shard_count = 1;
    L.spw = 0;
    L.blog2 = blog2;
    L.nmax = n;
    L.pmax = p;
    L.scratch = base + kScratch;
    L.scratch_per_warp = td_scratch_per_warp(n);
    if ((size_t)L.scratch_per_warp > kPerWarp) return TD_ERR_INVALID;
    unsigned long long *status = (unsigned long long *)(base + kStatus);

    TdSet set;
    set.x_off = 0;
    set.n = n;
    set.p = p;
    set.slice_index = 0;
    set.slice_count = 1;
    if (cudaMemcpy2DAsync(base + kZq, TD_MAXD * 4, Z, (size_t)p * 4, (size_t)p * 4, m, cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return TD_ERR_CUDA;
    td_k_noalloc_init<<<(m + 255) / 256, 256, 0, s>>>(L, set, status);
    if (cudaGetLastError() != cudaSuccess) return TD_ERR_CUDA;
    if (td_launch_setup(L, s) != cudaSuccess) return TD_ERR_CUDA;
    if (td_launch_tiles(L, s) != cudaSuccess) return TD_ERR_CUDA;
    for (int D = 2; D <= std::min((int)p, 6); ++D) {
        /* each dimension's kernel sized for its own layout (pmax = D) */
        TdLaunch LD = L;
        LD.pmax = D;
        const size_t smemD = td_filtered_smem(n, D, blog2, kWarps);
        const int occ = td_filtered_occupancy(D, kWarps, smemD);
        if (occ < 1) return TD_ERR_INVALID;
        const int grid = std::min(sms * occ, TD_NOALLOC_CTAS);
        if (td_launch_filtered(D, LD, grid, smemD, s) != cudaSuccess) return TD_ERR_CUDA;
    }
    if (td_launch_finalize(L, s) != cudaSuccess) return TD_ERR_CUDA;
    td_k_noalloc_status<<<1, 256, 0, s>>>(L, status);
    if (cudaGetLastError() != cudaSuccess) return TD_ERR_CUDA;
    unsigned long long hs[2] = { 0, 0 };
    if (cudaMemcpyAsync(hs, status, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TD_ERR_CUDA;
    if (hs[1] != 0) return TD_ERR_RANGE;
    if (hs[0] != 0) return TD_ERR_INTERNAL;
    if (cudaMemcpyAsync(out, base + kOut, (size_t)m * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return TD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TD_ERR_CUDA;
    return TD_OK;
}
