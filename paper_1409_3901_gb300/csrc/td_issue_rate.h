/*
 * td_issue_rate.h -- issue-rate probe exported by libtdprobe.so, the small
 * measurement library that the benchmark loads beside libtukeydepth.so (the
 * depth library itself does not contain it).
 *
 * The depth sweep (Algorithm 1 with Algorithm 2 inside, Section 3) is bound
 * by plain FP32/INT32 instruction issue, not by memory or tensor cores, so
 * its roofline is lane operations per second.  The derived peak is
 * SMs x 128 lanes x SM clock.  td_issue_rate measures what the GPU actually
 * sustains for the instruction kinds the sweep uses, so that the derived peak
 * can be checked against a measurement instead of a vendor figure.
 *
 * Each kind runs a kernel of independent dependency chains (enough per
 * thread to hide the pipe latency) over one full wave of resident thread
 * blocks (SMs x the occupancy limit), for a few milliseconds, and counts the
 * lane operations in its source:
 *
 *   TD_ISSUE_FFMA   scalar FP32 fused multiply-add, 1 operation each;
 *   TD_ISSUE_FFMA2  packed fma.rn.f32x2, 2 operations (one per half) each;
 *   TD_ISSUE_INT    32-bit integer add and xor alternating, 1 operation each;
 *   TD_ISSUE_MIXED  FP32 multiply-add and the integer add/xor pair, 1:1.
 *
 * The loop counter's own instructions (about 2% of the issued ones) are not
 * counted, so the figure is a slight underestimate of the issue rate.
 */
#ifndef TD_ISSUE_RATE_H
#define TD_ISSUE_RATE_H

#include "tukey_depth.h"

#ifdef __cplusplus
extern "C" {
#endif

#define TD_ISSUE_FFMA 0
#define TD_ISSUE_FFMA2 1
#define TD_ISSUE_INT 2
#define TD_ISSUE_MIXED 3

/* Measure the sustained rate of instruction kind `kind` on device `device`.
 *   - *lane_ops_per_s receives lane operations per second (best of three
 *     timed launches after one warm-up launch, CUDA events on a stream of
 *     its own); *ms receives that launch's duration.  Either pointer may be
 *     NULL except lane_ops_per_s.
 *   - The call allocates and frees its own small device buffer (one word per
 *     thread) and synchronises its stream; it does not touch any td_ctx.
 *   - Returns TD_OK, TD_ERR_INVALID (unknown kind, null lane_ops_per_s) or
 *     TD_ERR_CUDA (no device, launch or timing failure). */
int td_issue_rate(int device, int kind, double *lane_ops_per_s, float *ms);

#ifdef __cplusplus
}
#endif
#endif /* TD_ISSUE_RATE_H */
