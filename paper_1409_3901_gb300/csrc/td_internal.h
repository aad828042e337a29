/*
 * td_internal.h -- structures shared by the host side and the kernels of
 * libtukeydepth.so (not part of the public ABI).
 */
#pragma once
#include <stdint.h>

#define TD_MAXD 6
#define TD_NDIM 5            /* effective dimensions 2..6 with a subset loop */
#define TD_TICKET_STRIDE 16  /* work counters 128 bytes apart */
#define TD_DIRECT_WIDE (-2)  /* TdQuery.direct of a query whose centred coordinates exceed the fast
                                kernels' limit: answered by the wide kernel (td_wide.cuh) */
#define TD_NOCT 12           /* octaves of the nonzero point count: ceil(log2 nnz) in [0, 11] */

/* octave of a row of nnz nonzero points (1 <= nnz <= 2048): ceil(log2 nnz) */
static inline __host__ __device__ int td_octave(int nnz)
{
    int b = 0;
    while (b < TD_NOCT - 1 && (1 << b) < nnz) ++b;
    return b;
}

/* Largest |X_ij - z_j| (every coordinate) the fast kernels take for
 * dimension p: it keeps every exact intermediate in 64-bit (coordinates,
 * minors, projections) or 128-bit (cross products) integers, every
 * coordinate exact in binary32, and inside the window of the magic-constant
 * float-to-int conversion (|v| <= 2^22).  Queries beyond it go to the wide
 * kernel. */
static inline __host__ __device__ int64_t td_coord_limit_of(int p)
{
    switch (p) {
    case 1:
    case 2:
    case 3: return 4194303; /* 2^22 - 1 */
    case 4: return 524287;  /* 4 * 2 M^2 * M < 2^62 */
    case 5: return 16383;   /* 5 * 3^(3/2) M^3 * M < 2^62 */
    case 6: return 2047;    /* 6 * (2M)^4 * M < 2^62 */
    default: return 0;
    }
}

/* Per-query state written by the set-up kernel (one per query). */
struct TdQuery {
    int32_t set;           /* dataset index */
    int32_t n;             /* data points of the dataset */
    int32_t nnz;           /* centred points x_i = X_i - z that are nonzero */
    int32_t Z;             /* centred points equal to zero (counted by every closed halfspace) */
    int32_t d;             /* rank of the nonzero centred points (effective dimension) */
    int32_t k;             /* subset size d - 2 of Algorithm 1, or -1 when there is no subset loop */
    int32_t direct;        /* final count when there is no subset loop (nnz == 0 or d <= 1, or the
                              wide kernel's result), -1 when there is one, TD_DIRECT_WIDE while a
                              query beyond the fast kernels' limit waits for the wide kernel */
    int32_t amax;          /* max |x_ij| over every coordinate (saturated at INT32_MAX) */
    int32_t piv[TD_MAXD];  /* coordinates on which the span of the points projects injectively */
    int32_t mx[TD_MAXD];   /* max |x_i| per projected coordinate (FP32 error bounds) */
    int64_t nsub;          /* subset positions C(nnz, k) of the whole loop */
    int64_t lo, hi;        /* subset positions [lo, hi) handled by this call (shard) */
};

/* One dataset inside the device arenas. */
struct TdSet {
    int64_t x_off;  /* offset of X (n x p int32) in the data arena, in int32 elements */
    int32_t n, p;
    int32_t slice_index, slice_count; /* this call handles slice slice_index of slice_count contiguous
                                         ranges of each query's subset positions (the stream's time
                                         slices; slice_count <= 1: the call's shard) */
};

/* Statistics counters accumulated on the device. */
struct TdCounters {
    unsigned long long sweeps, dependent, filtered_points, exact_points, tight, resolved;
    unsigned long long errors;  /* device-side consistency failures (must stay 0) */
    unsigned long long early;   /* subsets not swept because their query had reached 0 (early exit) */
    unsigned long long adia_pops, adia_subsets, adia_union, adia_fallback; /* Algorithm 3 search */
    unsigned long long rescanned; /* sweeps that went past the coarse bound */
    unsigned long long wide;      /* queries the set-up flagged TD_DIRECT_WIDE */
};

/* Parameters of the work-queue launches. */
struct TdLaunch {
    const int32_t *X;        /* data arena */
    const int32_t *Zq;       /* query points, m_total x p_q (row stride TD_MAXD) */
    const TdSet *sets;
    TdQuery *q;              /* per query */
    int32_t nq;              /* number of queries */
    int32_t warps;           /* warps per CTA */
    const int32_t *order;    /* work order of the queries (a permutation of [0, nq)) */
    int64_t *tile_prefix;    /* TD_NDIM x (nq + 1) prefix sums of tiles, per dimension, in work order */
    int32_t *tile_size;      /* subsets per tile, per query */
    unsigned long long *ticket;  /* work-queue counters, one per dimension (stride TD_TICKET_STRIDE) */
    int32_t *qmin;           /* per-query minimum of V(S) over the processed subsets */
    int32_t *out;            /* per-query output */
    TdCounters *ctr;
    int64_t shard_index, shard_count;
    int32_t spw;             /* subsets per warp per tile (0 = the tuned table, else by size) */
    uint16_t spw_tab[TD_NDIM][TD_NOCT]; /* tuned subsets per warp by dimension and octave (0 = by size) */
    int32_t blog2;           /* angular buckets log2 (0 = by size) */
    int32_t nmax;            /* largest nnz over the queries (smem sizing) */
    int32_t pmax;            /* largest p over the datasets */
    char *scratch;           /* per-warp global scratch for the exact tight-set path */
    int64_t scratch_per_warp;
    int32_t early_exit;      /* nonzero: seed qmin with the data-direction bound, stop a query at 0 */
    int32_t adia;            /* nonzero: Algorithm 3 (search kernel before the sweep) */
    int32_t critical;        /* nonzero: Proposition 1 with r = p-1 (subsets of d-1 points) */
    int32_t unseeded;        /* nonzero: qmin starts at +inf, not at the data-direction bound */
    uint16_t *perm;          /* Algorithm 3: staging position of every nonzero point, per query, or null */
    int64_t perm_stride;     /* entries per query in perm */
    uint64_t *adia_keys;     /* Algorithm 3 node tables, per CTA of the search kernel */
    int32_t *adia_dep;
    int32_t *adia_stack;
};
