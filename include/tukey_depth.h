/*
 * tukey_depth.h -- C ABI of libtukeydepth.so: the exact sample Tukey
 * (halfspace) depth on an NVIDIA GB300 (sm_103a).
 *
 * The operation (Eq. 1, Section 1): for n data points X_1..X_n in Z^p and a
 * query point z, the depth count
 *
 *     T(z) = n * D_n(z) = min over unit u of #{ i : u'(X_i - z) <= 0 },
 *
 * the fewest data points in a closed halfspace whose boundary passes through
 * z.  It is computed by the paper's first exact algorithm (Algorithm 1,
 * Section 3): the minimum over all (p-2)-subsets S of the centred data of a
 * bivariate count (Algorithm 2, Section 3) of the data projected onto the 2-D
 * quotient of R^p by span(S), made exact for data that are not in general
 * position (Section 2 assumes general position):
 *
 *   - comparisons of projected directions are decided in FP32 when a forward
 *     error bound certifies them and otherwise by exact integer determinants;
 *   - equal directions are flipped together (Algorithm 2, step 1(e));
 *   - the "- (p-2)" of Algorithm 1, step 2 is replaced per subset by the
 *     number of data points in span(S) that a tilt out of the quotient can
 *     move off the closed halfspace (exact for every input);
 *   - data whose centred points span fewer than p dimensions are solved in
 *     that many coordinates; p = 1 is the trivial case of Section 3 and p = 2
 *     is Algorithm 2 alone.
 * The result is the integer count T in [0, n] (the paper returns T / n).
 *
 * Conventions for every entry point:
 *   - X is n x p int32, row-major (point i at X[i*p .. i*p+p-1]); query points
 *     Z are m x p int32, row-major; out is m int32.
 *   - Pointers are host pointers unless the context was created (or set) with
 *     td_options.device_pointers != 0, in which case they are device pointers
 *     of the context's device, used in stream order on the context's stream.
 *   - The caller owns every buffer.  Host inputs are copied before the call
 *     returns (td_depth, td_depth_batched) or before td_stream_submit returns.
 *     Results are written before td_depth / td_depth_batched return, or before
 *     td_stream_wait returns (td_stream_poll reports done).
 *   - Limits: 1 <= p <= TD_MAX_P, 1 <= n <= TD_MAX_N, m >= 0.  Any int32
 *     values: a query with some |X_ij - z_j| above td_coord_limit(p) (the
 *     fast kernels keep every exact intermediate in 64- or 128-bit integers
 *     below it) is answered by an exact 256-bit path instead (Proposition 1
 *     of Section 2 with r = p - 1, one order of n slower), with the same
 *     result.
 *   - Return value 0 (TD_OK) or a negative TD_ERR_* code; on error no output
 *     element is written (no partial results).  td_strerror() names a code.
 *   - Results are bit-exact and independent of scheduling; the statistics
 *     counters may vary with scheduling.
 */
#ifndef TUKEY_DEPTH_H
#define TUKEY_DEPTH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TD_OK 0
#define TD_ERR_INVALID (-1) /* null pointer, n < 1, m < 0, p outside [1, TD_MAX_P], n > TD_MAX_N */
#define TD_ERR_RANGE (-2)   /* td_depth_noalloc only: some |X_ij - z_j| exceeds td_coord_limit(p) */
#define TD_ERR_OOM (-3)     /* device or pinned host allocation failed */
#define TD_ERR_BUSY (-4)    /* stream admission refused: request exceeds the memory budget now */
#define TD_ERR_TIMEOUT (-5) /* td_stream_wait expired before the request finished */
#define TD_ERR_CUDA (-6)    /* a CUDA runtime call failed (see td_last_cuda_error) */
#define TD_ERR_NOTFOUND (-7) /* unknown stream ticket */
#define TD_ERR_INTERNAL (-8) /* a device-side consistency check failed */

#define TD_MAX_P 6
#define TD_MAX_N 2048

typedef struct td_ctx td_ctx;
typedef struct td_stream td_stream;

/* Algorithms (td_options.algorithm). */
#define TD_ALG_RCOM 0 /* Algorithm 1 (Section 3) over every (p-2)-subset: the exact count T */
#define TD_ALG_ADIA 1 /* Algorithm 3 (Section 4): an adaptive search from the best data direction
                         (Steps 2-4), then Algorithm 1 over the subsets of the points in the
                         halfspaces of the nodes it ends with (Step 5).  Every value it takes is
                         some V(S), so out[q] >= T.  The paper reports out[q] == T in all its
                         experiments, without proof; it is not so for every input (a query with
                         T = 32 and out[q] = 33 is among the tests).  Filtered mode, unsharded
                         only.  A query beyond td_coord_limit(p) gets the exact count T from
                         the 256-bit path. */
#define TD_ALG_CRITICAL 2 /* Proposition 1 (Section 2) with r = p-1: the minimum over the
                             hyperplanes spanned by p-1 centred points of the points strictly on
                             the smaller side, plus the open depth of the points on the hyperplane
                             inside it: the exact count T by a second route, O(n^(p-1)) normals
                             of O(n) work each, one launch per query (a cross-check of
                             Algorithm 1) in int64 while p! M^p < 2^62 for the largest
                             centred coordinate M, in the 256-bit form beyond;
                             td_options.mode is ignored; not served by the stream API
                             (td_stream_create returns TD_ERR_INVALID). */

/* Execution forms of the same computation (identical results). */
#define TD_MODE_FILTERED 0    /* persistent launch over (dataset, query, subset-tile) work,
                                 FP32 filter with exact fallback, angular buckets */
#define TD_MODE_PLAIN_EXACT 1 /* one launch per query, every projection and comparison in
                                 exact integer arithmetic, comparison sort */

typedef struct {
    int32_t mode;             /* TD_MODE_FILTERED (default) or TD_MODE_PLAIN_EXACT */
    int32_t device_pointers;  /* nonzero: X, Z, out are device pointers */
    int32_t use_graph;        /* nonzero (default): replay the launch sequence of a batched call
                                 from a captured CUDA graph when the shapes repeat */
    int32_t subsets_per_warp; /* work-tile size (subsets per warp per tile); 0 = the value td_autotune
                                 (or td_set_tuned) stored in the context for the query's effective
                                 dimension and octave of its nonzero point count, else a size rule
                                 (about 3 * 2^16 point evaluations per warp and tile, 4 to 1024) */
    int32_t buckets_log2;     /* angular buckets of the rare exact path = 2^buckets_log2; 0 = about
                                 one per two points (7 to 11); measured to make no difference */
    int32_t early_exit;       /* nonzero: filtered mode stops sweeping a query once its running
                                 minimum of V(S) reaches 0, the least value (then T = Z).  The
                                 running minimum always starts at the upper bound of data
                                 directions u = +-x_j (Algorithm 3, Step 2).  The depths are
                                 unchanged; stats.early_skipped counts the subsets not swept.
                                 0 (default): every subset is swept. */
    int32_t algorithm;        /* TD_ALG_RCOM (default), TD_ALG_ADIA or TD_ALG_CRITICAL */
    int32_t unseeded;         /* nonzero: each query's running minimum starts at +infinity instead
                                 of the data-direction upper bound, so that under sharding out[q]
                                 is exactly Z + the minimum of V(S) over the shard's own range
                                 (INT32_MAX if it holds no independent subset) -- the form in
                                 which a range can be checked against a reference.  Same depths
                                 unsharded; slower.  0 (default): seeded. */
    int64_t shard_index;      /* multi-GPU sharding of Algorithm 1's subset loop: process only the */
    int64_t shard_count;      /* shard_index-th of shard_count contiguous ranges of subset positions
                                 of every query (0 or 1: all).  The positions are the colex ranks
                                 r = sum_i C(c_i, i+1) of the (d-2)-subsets c_0 < .. < c_(d-3) of
                                 the query's nnz nonzero centred points in data order (d its
                                 effective dimension); shard s of S takes the ranks
                                 [floor(N s / S), floor(N (s+1) / S)), N = C(nnz, d-2), and a
                                 query without a subset loop is answered by shard 0 alone (the
                                 others report INT32_MAX).  out[q] is then Z + the minimum of
                                 V(S) over that range, or the data-direction bound if that is
                                 smaller (see unseeded), or INT32_MAX if the range holds no subset
                                 and the bound was not taken; the minimum of out[q] over all shards
                                 is the depth. */
    void *stream;             /* cudaStream_t to run on; NULL = the context's own stream */
} td_options;

/* One dataset with its queries, for td_depth_batched and td_stream_submit. */
typedef struct {
    int32_t n, p;
    const int32_t *X; /* n x p */
    int32_t m;
    const int32_t *Z; /* m x p */
    int32_t *out;     /* m */
} td_dataset;

/* Per-call statistics (counts summed over queries). */
typedef struct {
    uint64_t sweeps;            /* (query, subset of rank p-2) pairs swept (Algorithm 1 step 1) */
    uint64_t skipped_dependent; /* subsets of rank < p-2, skipped */
    uint64_t filtered_points;   /* projected points (over all sweeps) whose angular range the FP32
                                   filter certified (plain mode: 0) */
    uint64_t exact_points;      /* projected points it could not certify (the subset's own points
                                   among them); in the sweeps that need their order they are placed
                                   with exact integer arithmetic (plain mode: every point) */
    uint64_t tight_exceptions;  /* subsets whose span holds more data points than the subset */
    uint64_t resolved_buckets;  /* sweeps whose extremum needed an exact in-bucket order */
    uint64_t kernel_launches;   /* CUDA kernels launched by the call */
    float ms;                   /* device time from first to last kernel of the call */
    float ms_sweep;             /* device time of the sweep kernel(s) alone (CUDA events on the
                                   launch stream around them) */
    uint64_t early_skipped;     /* subsets not swept because their query had reached 0
                                   (td_options.early_exit) */
    uint64_t adia_pops;         /* Algorithm 3: nodes popped in Step 4 */
    uint64_t adia_subsets;      /* Algorithm 3: subsets evaluated in Steps 2(c) and 4 (exact sort) */
    uint64_t adia_union_points; /* Algorithm 3: points in the unions of Step 5(a), summed over queries
                                   (Step 5(b) sweeps are counted in sweeps) */
    uint64_t adia_fallbacks;    /* Algorithm 3: queries whose search outgrew its node table or
                                   iteration bound and were swept in full (exact count) */
    uint64_t rescanned_sweeps;  /* sweeps whose bound over the FP32-certified points did not reach
                                   the query's running minimum: their points were projected again at
                                   the fine bucket level and the uncertain ones placed exactly (the
                                   exact path's hit rate per sweep; plain mode: 0) */
} td_stats;

/* The fast kernels' coordinate bound for dimension p: queries with every
 * |X_ij - z_j| <= td_coord_limit(p) run on them, the others on the exact
 * 256-bit path (td_depth_noalloc refuses them with TD_ERR_RANGE). */
int64_t td_coord_limit(int32_t p);

/* Create a context on CUDA device `device`; opt may be NULL (defaults).
 * The context owns a CUDA stream, device work buffers (grown on demand) and
 * pinned staging memory.  Not thread-safe: one host thread per context. */
int td_create(td_ctx **ctx, int device, const td_options *opt);

/* Replace the context's options (same meaning as in td_create). */
int td_set_options(td_ctx *ctx, const td_options *opt);

/* Wait for outstanding work and free everything the context owns. */
int td_destroy(td_ctx *ctx);

/* out[q] = T(Z_q) for the m queries Z (m x p) against data X (n x p).
 * Algorithm 1 (Section 3) with Algorithm 2 as the inner count; Eq. (1). */
int td_depth(td_ctx *ctx, const int32_t *X, int32_t n, int32_t p,
             const int32_t *Z, int32_t m, int32_t *out, td_stats *st);

/* The same for k independent datasets (each with its own n, p and queries),
 * served by one persistent launch over (dataset, query, subset-tile) work. */
int td_depth_batched(td_ctx *ctx, const td_dataset *sets, int32_t k, td_stats *st);

/* Asynchronous request stream.  A request is admitted only while the device
 * memory it needs fits under mem_budget_bytes together with the requests in
 * flight; otherwise td_stream_submit returns TD_ERR_BUSY and changes nothing.
 * td_stream_submit copies the request's inputs before it returns.  A large
 * request's subset loop is cut into time slices: contiguous ranges of each
 * query's subset positions of about 1.5e10 point evaluations (C(n, p-2) n a
 * query), whose counts are merged by a minimum.  Admitted requests are
 * coalesced: whenever one of the stream's two batch slots is free, one
 * batched launch (as td_depth_batched) on the stream's own CUDA stream takes
 * every waiting request of a single slice and the next slice of the sliced
 * requests in arrival order while their work stays within about 3e10 point
 * evaluations, so that a small request never waits behind the whole of a
 * large one.  Progress (reaping finished batches, launching the waiting
 * slices) is made inside td_stream_submit, td_stream_poll and td_stream_wait.
 * A ticket is forgotten once poll or wait has reported it done
 * (TD_ERR_NOTFOUND afterwards).  Algorithm 3 requests are not sliced. */
int td_stream_create(td_ctx *ctx, size_t mem_budget_bytes, td_stream **s);
int td_stream_submit(td_stream *s, const td_dataset *d, uint64_t *ticket);
/* *done = 1 once the request's outputs have been written to its out buffer. */
int td_stream_poll(td_stream *s, uint64_t ticket, int *done);
/* Block until done or until timeout_us microseconds pass (TD_ERR_TIMEOUT;
 * the request stays in flight).  timeout_us < 0 waits without limit. */
int td_stream_wait(td_stream *s, uint64_t ticket, int64_t timeout_us);
int td_stream_destroy(td_stream *s);

/* Autotuner (no counterpart in the paper: the choice of work-tile size of
 * the persistent sweep).  Times the filtered sweep kernel of dimension p on a
 * seeded synthetic dataset of n points (uniform integers in [-127, 127]) with
 * enough queries for about 10 ms of sweeping (at most 256), first with the
 * size rule and then with each candidate work-tile size (16 to 1024 subsets
 * per warp), the median of three calls each (td_stats.ms_sweep), and keeps
 * the fastest -- a candidate only when it beats the size rule by more than
 * 1% -- in the context for queries of effective dimension p whose nonzero point count lies
 * in the octave of n (ceil(log2 n), and that of n - 1); later calls with
 * subsets_per_warp = 0 use it.  The results never depend on the choice.
 * res (may be NULL) receives the candidates, their times and the choice
 * (best_spw = 0: the size rule was fastest).  Runs synchronously on the
 * context's stream; the context's options are unchanged on return.  Limits:
 * 3 <= p <= TD_MAX_P, p < n <= TD_MAX_N (TD_ERR_INVALID). */
#define TD_TUNE_MAX 8
typedef struct {
    int32_t p, n, queries, candidates;
    int32_t spw[TD_TUNE_MAX]; /* candidate subsets per warp */
    float ms[TD_TUNE_MAX];    /* their sweep-kernel times (ms, median of three calls) */
    float ms_default;         /* the size rule's time */
    int32_t best_spw;         /* the choice stored in the context (0 = the size rule) */
    float best_ms;
} td_tune_result;
int td_autotune(td_ctx *ctx, int32_t p, int32_t n, td_tune_result *res);

/* Store a work-tile size for effective dimension d (2..6) and octave
 * (0..11: queries with 2^(octave-1) < nonzero points <= 2^octave), e.g. one
 * that td_autotune chose in an earlier process; 0 restores the size rule. */
int td_set_tuned(td_ctx *ctx, int32_t d, int32_t octave, int32_t subsets_per_warp);

/* Allocation-free depth (no counterpart in the paper; a deployment need).
 * For callers that must not allocate device memory: code running under a
 * framework whose memory pool owns the GPU, processes with a device-memory
 * budget fixed when they load, or latency-critical paths where cudaMalloc
 * and cudaFree would synchronise the device.  Same operation and results as
 * td_depth, but needs no context and calls no allocating routine: X (n x p),
 * Z (m x p) and out (m) are DEVICE pointers of the current device, used on
 * `stream` (a cudaStream_t; NULL = the default stream); every other buffer is
 * carved out of one file-scope __device__ array of TD_NOALLOC_BYTES bytes
 * that each GPU loading this library holds until the process exits.
 *   - Limits: n <= TD_NOALLOC_MAX_N, m <= TD_NOALLOC_MAX_M (TD_ERR_INVALID
 *     beyond them: the array has no room), p <= TD_MAX_P, and the coordinate
 *     limit of td_coord_limit on every coordinate (TD_ERR_RANGE: the first
 *     kernel tests it and gives an out-of-range query no further work).
 *   - The first call on a device looks the array up (cudaGetSymbolAddress)
 *     and so loads the module there; make that first call before any stream
 *     capture.
 *   - Returns after the results are in out (it synchronises `stream`); on an
 *     error out is left untouched.
 *   - All calls share the one array: calls that overlap on the GPU (other
 *     host threads, or other streams still running an earlier call) race and
 *     must be serialised by the caller.  The sweep uses at most
 *     TD_NOALLOC_CTAS thread blocks.  Its shared-memory limits are raised,
 *     never lowered, so it can run beside td_depth calls of other threads. */
#define TD_NOALLOC_MAX_N 512
#define TD_NOALLOC_MAX_M 4096
#define TD_NOALLOC_CTAS 80
#define TD_NOALLOC_BYTES (24u << 20)
int td_depth_noalloc(const int32_t *X, int32_t n, int32_t p, const int32_t *Z, int32_t m,
                     int32_t *out, void *stream);

const char *td_strerror(int code);
/* Text of the last CUDA error seen by this context (empty if none). */
const char *td_last_cuda_error(td_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* TUKEY_DEPTH_H */
