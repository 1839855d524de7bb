/*
 * Test and profiling hooks of the transport library (not part of the transport
 * interface in et.h; same conventions: status codes, host pointers unless a name
 * says "_device").
 */
#ifndef ET_DEBUG_H
#define ET_DEBUG_H

#include "et.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Record the start time (%globaltimer, ns) of every iteration the persistent driver
 * runs (enable = 1; allocates max_iters entries once) or stop recording (0).
 */
et_status et_debug_iteration_times(et_ctx* ctx, int enable);

/* Copy the recorded start times (n = iterations so far, at most max_iters) into out[cap]. */
et_status et_debug_read_iteration_times(et_ctx* ctx, uint64_t* out, uint64_t cap, uint64_t* n);

/*
 * Host-side fault injection for the persistent driver's grid barrier: block skip_block
 * (-1: none) returns at the start of the launch and never arrives, so the other blocks'
 * bounded waits run out after timeout_ns (0: keep the current limit) and the run ends
 * with ET_ERR_TIMEOUT.  No GPU fault is caused.
 */
et_status et_debug_set_barrier_fault(et_ctx* ctx, int skip_block, uint64_t timeout_ns);

/*
 * Evaluate one of the transport's device primitives on n inputs (device buffers, one
 * thread per input, on cuda_stream; returns after the stream finished):
 *   ET_EVAL_PHILOX        in uint32[n][6] = counter c0..c3, key k0, k1 (Philox4x32-10,
 *                         Salmon et al. SC'11)             -> out uint32[n][4]
 *   ET_EVAL_U01           in uint32[n]  -> out float[n]: ((x >> 8) + 1) 2^-24
 *   ET_EVAL_LOG, _EXP     in float[n]   -> out float[n]: the strict model's log / exp
 *   ET_EVAL_SINCOS2PI     in float[n]   -> out float[n][2]: sin, cos of 2 pi u (strict)
 * ET_ERR_INVALID for an unknown `what` or null buffers with n > 0.
 */
enum { ET_EVAL_PHILOX = 0, ET_EVAL_U01 = 1, ET_EVAL_LOG = 2, ET_EVAL_EXP = 3, ET_EVAL_SINCOS2PI = 4 };
et_status et_debug_eval(int what, const void* in_device, void* out_device, size_t n,
                        void* cuda_stream);

/*
 * The column of each slab in an event's row of the device deposit array (out[s] for
 * s < n_slabs; 1 <= n_slabs <= 128): within each complete group of 32 slabs, adjacent
 * slabs sit in the group's two 128-byte halves alternately; an incomplete last group
 * keeps its order.  The read calls return deposits in slab order; this only exposes
 * the device layout to tests.  Host only; ET_ERR_INVALID for a bad count or null out.
 */
et_status et_debug_score_columns(uint32_t n_slabs, uint32_t* out);

#ifdef __cplusplus
}
#endif
#endif
