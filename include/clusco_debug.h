/* clusco_debug.h -- test hooks of the debug build of libclusco (libclusco_debug.so).
 *
 * The debug library is the production source compiled with -DCLUSCO_DEBUG_HOOKS and a short
 * device wait limit (-DCLUSCO_WAIT_NS=200000000, 0.2 s); the production library (libclusco.so)
 * exports none of this. The hooks let tests reach two failure paths without faulting or hanging
 * a GPU: a bounded wait that gives up, a near-duplicate queue that overflows, and lists of
 * flagged pairs that overflow into the flag mask.
 */
#ifndef CLUSCO_DEBUG_H
#define CLUSCO_DEBUG_H

#include <stdint.h>

#include "clusco.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Set the hooks for the calls that follow (process-wide; not thread-safe against running calls).
 *  skip_arrive != 0 -- in every tensor-core all-pairs forward, CTA 0's TMA producer skips its
 *     first pipeline stage: no arrive and no copy on that stage's barrier. The MMA issuer's and
 *     the producer's bounded waits then give up, the CTA drains its copies in flight and leaves,
 *     the other CTAs finish normally, and clusco_sync_status() returns CLUSCO_ETIMEOUT. Values
 *     of the pairs of CTA 0's first tile are then undefined.
 *  nd_cap > 0 -- capacity of the adjoints' near-duplicate queues (pairs with cRMSD below the
 *     near-duplicate threshold that take the direct FP64 path); pairs past it are counted, not
 *     stored, and clusco_sync_status() reports the overflow (CLUSCO_ECUDA, bounds). 0 restores
 *     the default capacity, min(P, 2^22).
 * Returns CLUSCO_OK, CLUSCO_EINVAL (nd_cap < 0) or CLUSCO_ECUDA. */
int clusco_debug_hooks(int skip_arrive, int64_t nd_cap);

/* Capacity of each epilogue warp's list of flagged pairs in the exact-digit forward, for the
 * calls that follow (process-wide): cap > 0 caps the lists at cap entries, so that the pairs
 * past them take the refinement's mask path (results are unchanged); 0 restores the default
 * (1/32 of the pairs, at least 2^16 entries, over all lists).
 * Returns CLUSCO_OK or CLUSCO_EINVAL (cap < 0). */
int clusco_debug_flag_list_cap(int cap);

#ifdef __cplusplus
}
#endif

#endif /* CLUSCO_DEBUG_H */
