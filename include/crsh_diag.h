/* crsh_diag.h - diagnostics of the CRSH library (not steps of the method).
 *
 * These calls measure the GPU or exercise the library's failure paths; the
 * path of the paper (include/crsh.h) never calls them.  Same conventions as
 * crsh.h: device pointers, asynchronous on `stream`, argument errors returned
 * synchronously, device-side errors in crsh_counters.status.
 */
#ifndef CRSH_DIAG_H
#define CRSH_DIAG_H

#include "crsh.h"

#ifdef __cplusplus
extern "C" {
#endif

/* FP32 peak probe for roofline measurements (measurement only): launches
 * `blocks` x 256 threads, each running 8 independent FMA chains for 4 x iters
 * steps, and writes one float per block to `out` (device, `blocks` entries).
 * *flops (host) receives the FP32 operations launched (2 per FMA); time the
 * call with events on `stream`.  blocks in [1, 2^20], iters >= 1. */
crsh_status crsh_fma_probe(float *out, uint32_t iters, uint32_t blocks, unsigned long long *flops, void *stream);

/* Bounded-wait self-test of the decoupled look-back that the single-pass scans
 * and the radix sort use (their waits for a predecessor tile are bounded; a
 * wait that runs out records CRSH_ERR_TIMEOUT and the kernel finishes).  One
 * warp resolves tile `tile` (>= 1) against caller-prepared status words with
 * at most `spin_limit` polls:
 *   wide = 1: 64-bit words (bits 63:62 flag: 0 not published, 1 tile total,
 *             2 inclusive prefix; bits 61:0 value), status64 has tile + 1
 *             entries;
 *   wide = 0: 32-bit words (bits 31:30 flag, 29:0 value), status32 likewise.
 * The tile publishes its own aggregate `aggregate` first and its inclusive
 * prefix last (entry `tile` is overwritten).  *prefix_out (device, 8 bytes)
 * receives the exclusive prefix found; counters->status receives
 * CRSH_ERR_TIMEOUT if a predecessor never published within the limit.
 * spin_limit in [1, 2^22]. */
crsh_status crsh_lookback_selftest(unsigned long long *status64, uint32_t *status32, uint32_t wide, uint32_t tile,
                                   uint32_t aggregate, uint32_t spin_limit, unsigned long long *prefix_out,
                                   crsh_counters *counters, void *stream);

/* crsh_closest_hit with its final-test kernel timed (measurement only): the
 * same arguments, validation and results as crsh_closest_hit (include/crsh.h,
 * Section 3.3.8), plus *kernel_ms (host) = the duration of the final-test
 * kernel (k_closest, or k_closest_words for level 1 in word form), measured
 * with two CUDA events recorded on `stream` immediately before and after that
 * kernel's launch.  Synchronous: returns after the call has completed on
 * `stream`.  Errors: those of crsh_closest_hit; CRSH_ERR_INVALID_ARG if
 * kernel_ms is NULL; CRSH_ERR_CUDA if an event call or the synchronisation
 * fails (*kernel_ms is then not written). */
crsh_status crsh_closest_hit_timed(const crsh_hierarchy *h, const crsh_rays *rays, const uint32_t *n_rays,
                                   const crsh_scene *scene, const crsh_pairs *pairs, crsh_hits *out,
                                   crsh_counters *counters, void *workspace, size_t workspace_bytes,
                                   float *kernel_ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CRSH_DIAG_H */
