/*
 * vr_inject.h -- fault-injection hooks of the Vietoris-Rips library, for
 * tests of its failure handling.  The paper has no counterpart: these hooks
 * exist so that every failure path (out of memory, a device wait that gives
 * up, a refused admission) can be exercised without faulting, trapping or
 * hanging a GPU.  Every fault is made on the host or by a kernel that
 * withholds a signal under a short, bounded wait; the CUDA context stays
 * usable and the next call works normally.
 *
 * The hooks are process-wide and one-shot (each arms the next matching
 * event only); vr_inject_clear disarms them all.  Not for production use.
 */
#ifndef VR_INJECT_H
#define VR_INJECT_H

#include "vr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The nth device allocation of the library from now on (1 = the next) fails
 * as if the device were out of memory; the failing call returns VR_ERR_OOM
 * and releases what it had allocated.  0 disarms.  nth < 0: VR_ERR_ARG. */
VR_API vr_status vr_inject_alloc_failure(int64_t nth);

/* In the next radix digit pass with more than `tile` tiles (the sorts of the
 * edge keys and of the triangle keys), tile `tile` publishes no count, so the
 * later tiles' look-back waits give up after `wait_limit` polls: the build
 * (or vr_sort_keys) reports VR_ERR_TIMEOUT.  tile < 0 or wait_limit < 1:
 * VR_ERR_ARG. */
VR_API vr_status vr_inject_lookback_stall(int64_t tile, int64_t wait_limit);

/* In the next tensor-core distance launch with more than `tile` tiles, CTA
 * `tile` issues no MMA and no completion signal, so its wait gives up after
 * `wait_limit` polls (its operand loads are waited for in full, so nothing
 * is in flight when it releases its tensor memory): the build reports
 * VR_ERR_TIMEOUT.  tile < 0 or wait_limit < 1: VR_ERR_ARG. */
VR_API vr_status vr_inject_gram_stall(int32_t tile, int64_t wait_limit);

/* The request server's next k memory-admission decisions refuse every cloud
 * of their micro-batch; refused clouds go back to the queue and are admitted
 * later (vr_server_stats.deferred counts them).  0 disarms. */
VR_API vr_status vr_inject_admission_refusals(int64_t k);

/* Disarm every hook above. */
VR_API vr_status vr_inject_clear(void);

/* Bytes currently allocated from the current device's stream-ordered pool
 * (where the library's device memory comes from): a leak check for tests. */
VR_API vr_status vr_pool_used_bytes(int64_t *bytes);

#ifdef __cplusplus
}
#endif

#endif /* VR_INJECT_H */
