/* Issue-rate probe: sustained lane operations per second of the instruction
 * kinds the depth sweep is made of (FP32 multiply-add, packed f32x2
 * multiply-add, 32-bit integer add/xor).  The sweep's roofline is this
 * issue rate (its data stay in shared memory), so its peak is checked here
 * by measurement. */
#include <cuda_runtime.h>

#include "td_issue_rate.h"

namespace {

constexpr int kChains = 8;   /* independent chains per thread and kind */
constexpr int kUnroll = 8;   /* chain steps per loop iteration */
constexpr int kThreads = 256;
constexpr int kIters = 4096;

__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b,
                                                        unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

/* Lane operations per thread and loop iteration, as written below. */
__host__ __device__ constexpr int ops_per_iter(int kind)
{
    return kind == TD_ISSUE_FFMA    ? kChains * kUnroll
           : kind == TD_ISSUE_FFMA2 ? 2 * kChains * kUnroll
           : kind == TD_ISSUE_INT   ? 2 * kChains * kUnroll
                                    : 4 * kChains * kUnroll;
}

/* The multipliers and addends are kernel arguments, so nothing folds at
 * compile time; FP32 arithmetic is not reassociated, and the integer chains
 * a += b; b ^= a have no algebraic shortcut. */
template <int KIND>
__global__ void __launch_bounds__(kThreads) td_k_issue(unsigned *out, int iters, float s, float t, unsigned w)
{
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    float f[kChains], g[kChains];
    unsigned a[kChains], b[kChains];
    unsigned long long q[kChains];
    const unsigned long long s2 = __float_as_uint(s) | ((unsigned long long)__float_as_uint(s) << 32);
    const unsigned long long t2 = __float_as_uint(t) | ((unsigned long long)__float_as_uint(t) << 32);
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
        f[j] = (float)(tid & 255) * 1e-3f + (float)j;
        g[j] = f[j] + 0.5f;
        a[j] = tid * 2654435761u + (unsigned)j;
        b[j] = a[j] ^ w;
        q[j] = __float_as_uint(f[j]) | ((unsigned long long)__float_as_uint(g[j]) << 32);
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
            for (int j = 0; j < kChains; ++j) {
                if (KIND == TD_ISSUE_FFMA) {
                    f[j] = fmaf(f[j], s, t);
                } else if (KIND == TD_ISSUE_FFMA2) {
                    q[j] = fma_f32x2(q[j], s2, t2);
                } else if (KIND == TD_ISSUE_INT) {
                    a[j] += b[j];
                    b[j] ^= a[j];
                } else {
                    f[j] = fmaf(f[j], s, t);
                    a[j] += b[j];
                    g[j] = fmaf(g[j], s, t);
                    b[j] ^= a[j];
                }
            }
        }
    }
    unsigned acc = 0;
#pragma unroll
    for (int j = 0; j < kChains; ++j)
        acc ^= __float_as_uint(f[j]) ^ __float_as_uint(g[j]) ^ a[j] ^ b[j] ^ (unsigned)q[j] ^ (unsigned)(q[j] >> 32);
    out[tid] = acc;
}

template <int KIND>
int run_kind(int device, double *rate, float *ms_out)
{
    int sms = 0, per_sm = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, td_k_issue<KIND>, kThreads, 0) != cudaSuccess ||
        sms <= 0 || per_sm <= 0)
        return TD_ERR_CUDA;
    const int blocks = sms * per_sm; /* one full wave */
    unsigned *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TD_OK;
    float best = 0.f;
    if (cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(unsigned)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = TD_ERR_CUDA;
    } else {
        for (int rep = 0; rep < 4 && rc == TD_OK; ++rep) {
            cudaEventRecord(e0, st);
            td_k_issue<KIND><<<blocks, kThreads, 0, st>>>(out, kIters, 0.9999f, 1e-4f, 0x9E3779B9u);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
                cudaGetLastError() != cudaSuccess) {
                rc = TD_ERR_CUDA;
            } else if (rep > 0 && (best == 0.f || ms < best)) {
                best = ms; /* launch 0 is the warm-up */
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (rc == TD_OK && best > 0.f) {
        const double ops = (double)blocks * kThreads * kIters * ops_per_iter(KIND);
        *rate = ops / (best * 1e-3);
        if (ms_out) *ms_out = best;
    } else if (rc == TD_OK) {
        rc = TD_ERR_CUDA;
    }
    return rc;
}

} // namespace

extern "C" int td_issue_rate(int device, int kind, double *lane_ops_per_s, float *ms)
{
    if (!lane_ops_per_s) return TD_ERR_INVALID;
    switch (kind) {
    case TD_ISSUE_FFMA: return run_kind<TD_ISSUE_FFMA>(device, lane_ops_per_s, ms);
    case TD_ISSUE_FFMA2: return run_kind<TD_ISSUE_FFMA2>(device, lane_ops_per_s, ms);
    case TD_ISSUE_INT: return run_kind<TD_ISSUE_INT>(device, lane_ops_per_s, ms);
    case TD_ISSUE_MIXED: return run_kind<TD_ISSUE_MIXED>(device, lane_ops_per_s, ms);
    default: return TD_ERR_INVALID;
    }
}
