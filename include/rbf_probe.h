/*
 * rbf_probe.h - measurement helper of librbf.so (not part of the paper's method).
 *
 * Measures the per-SM issue rates that bound the Gaussian product kernels:
 * ex2.approx.f32 (the special-function unit), scalar FP32 FMA and packed
 * f32x2 FMA, each as operations per SM per clock, with the SM clock derived
 * from the cycle counter and the global nanosecond timer of the probe run.
 * These are the denominators of the product kernels' roofline.  The float64
 * FMA rate bounds the float64 Gram-Schmidt vector work of FGMRES (one FMA per
 * 8-byte element it streams).  It also times,
 * on one thread per SM, the issue-to-completion latency of the tensor-core step
 * of the product (two dependent tcgen05.mma of kind::tf32, M = 128, N = 32,
 * K = 8, then tcgen05.commit to an mbarrier), alone and four in a row.
 */
#ifndef RBF_PROBE_H
#define RBF_PROBE_H

#include "rbf.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int num_sms;
    double sm_mhz;                  /* SM clock during the probe (cycles / ns * 1000) */
    double ex2_per_clk_sm;          /* MUFU.EX2 results per SM per clock */
    double ffma_per_clk_sm;         /* scalar FP32 FMA per SM per clock */
    double ffma2_lanes_per_clk_sm;  /* packed f32x2 FMA, FP32 lanes per SM per clock */
    double mma_commit_cycles;       /* SM cycles from issuing one MMA pair + commit to the mbarrier phase */
    double mma_commit4_cycles;      /* the same for four pairs (each with its commit) issued back to back */
    double dfma_per_clk_sm;         /* float64 FMA per SM per clock */
} rbf_probe_result;

/* Runs four short kernels (about 10 ms each) and the latency kernel (under 1 ms)
 * on `device` (default stream) and fills *r.  Errors: RBF_ERR_INVALID (null r),
 * RBF_ERR_CUDA, RBF_ERR_TIMEOUT (an mbarrier wait of the latency kernel expired;
 * its waits are bounded at 100 ms). */
rbf_status rbf_probe_peaks(int device, rbf_probe_result *r);

/* Failure-detection check of the bounded waits (no fault involved): one thread
 * waits, with the wait the tensor-core kernels use, for an mbarrier phase that
 * nothing completes; after limit_ns (clamped to [1 us, 1 s]) the wait gives up,
 * raises the context's device error word and the kernel returns.  The call then
 * synchronises `stream` and reports what a product launch that gave up would:
 * RBF_ERR_TIMEOUT, with rbf_last_error set and the word cleared; the context
 * stays usable.  Returns RBF_OK only if the phase completed (it cannot). */
rbf_status rbf_probe_wait_expiry(rbf_ctx *ctx, uint64_t limit_ns, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RBF_PROBE_H */
