/* Test hooks of libmls: device self-checks that the test suite calls
 * through the same C ABI as the renderer.  None of them is needed to
 * render; each allocates its own device memory, runs on the current device
 * and synchronises before it returns. */
#ifndef MLS_DEBUG_H
#define MLS_DEBUG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Bounded waits (the failure detection of the tensor-core kernel).  Launches
 * one warp that waits on an mbarrier phase nothing completes; the wait gives
 * up after limit_ns nanoseconds of the device clock, records its error code
 * (1 = a wait for a filled operand stage gave up) and the kernel returns.
 * *code_out receives that code (0 = no wait gave up).  Returns MLS_OK when
 * the kernel ran and the context is still usable, MLS_E_CUDA otherwise. */
int mls_debug_wait_selftest(int64_t limit_ns, int *code_out);

/* The double-float weight functions of the hand-over path, evaluated on n
 * arguments a = arg_hi[i] + arg_lo[i] (host arrays of float; out a host
 * array of n doubles receiving hi + lo of the result):
 *   kind 0: exp(a), for -70 <= a <= 1 (the Gaussian weight of Section 3.3,
 *           Eq. eq-weights, relative to the stabiliser: exp(-(r^2 - m)/h^2));
 *   kind 1: the Wendland C2 weight (1 - q)^4 (4 q + 1), q = sqrt(a), 0 <= a < 1
 *           (the compactly supported weight of the Section 3.3 weight family);
 *   kind 2: sqrt(a), a >= 0.
 * Returns MLS_E_INVAL for a bad kind, n < 0 or a null array with n > 0,
 * MLS_E_NOMEM / MLS_E_CUDA on device failures, MLS_OK otherwise. */
int mls_debug_df_weight(int kind, const float *arg_hi, const float *arg_lo, int64_t n, double *out);

/* Reduced-precision Gaussian renders visit, per 16 x 16 tile, only the points
 * whose weight at some pixel of the tile is at least e^-28 of that pixel's
 * largest (below it an FP16 weight rounds to exactly zero and a BF16 / FP32
 * product lies below the FP32 resolution of the sums).  on = 0 makes the
 * handle's later renders visit every point, so that a test can check that
 * the cut changes nothing beyond FP32 rounding.  Returns MLS_E_INVAL for a
 * null handle, MLS_OK otherwise. */
struct mls_handle;
int mls_debug_operand_cut(struct mls_handle *h, int32_t on);

/* Pixels that the reduced-precision passes hand over are recomputed by four
 * kernels (setup, moments, degree policy, values) for the first entries of
 * the list, up to a state capacity of an eighth of the W H pixels (at least
 * min(W H, 1024) entries, at most 2^19), when the list holds at least
 * 19,456 entries; by one fused kernel for shorter lists and for the entries
 * past that capacity.  For the handle's later renders, cap >= 0 lowers the
 * capacity (0: every entry through the fused kernel) and least >= 0 sets the
 * shortest list the four kernels take, so that a test can check both
 * paths; -1 restores either.  Returns MLS_E_INVAL for a null handle or an
 * argument below -1, MLS_OK otherwise. */
int mls_debug_handover_split(struct mls_handle *h, int64_t cap, int64_t least);

/* Page-locked host outputs of mls_render (on_device = 0): with a field of at
 * most 256 MiB the kernels write them directly; above it the render goes to
 * device staging and one copy kernel writes them.  mode 1 takes the staged
 * copy and mode 2 the direct writes for the handle's later renders whatever
 * the size, so that a test can check both; 0 restores the choice by size.
 * Returns MLS_E_INVAL for a null handle or another mode, MLS_OK otherwise. */
int mls_debug_host_output(struct mls_handle *h, int32_t mode);

#ifdef __cplusplus
}
#endif

#endif /* MLS_DEBUG_H */
