// chunk_rule.h -- the chunk rules of the scheduled image loop (Sec. 2.2,
// Algorithm 3's getChunk), as one function that host code (the chunk tables
// of every entry point) and device code (the allocation-free entry point's
// table build) both call.
//
// Readings: the scheduling step advances by one per assignment and every
// chunk is clamped to the iterations that remain; SS hands out min_chunk
// iterations; GSS ceil(R / P), never below min_chunk; FAC hands out batches of
// P equal chunks of ceil(R / (2P)) (FAC2), R being what remains when the batch
// starts, never below min_chunk.  STATIC has no per-step rule (worker k takes
// the block [floor(kN/P), floor((k+1)N/P))), nor has the probabilistic FAC
// batch size, which is IEEE double arithmetic done on the host only.
#pragma once

#include <cstdint>

#include "../../include/spin.h"

#ifdef __CUDACC__
#define SI_HOST_DEVICE __host__ __device__
#else
#define SI_HOST_DEVICE
#endif

namespace si {

// Chunk of scheduling step `step` under `kind` (SI_SCHED_SS, SI_SCHED_GSS or
// SI_SCHED_FAC) with `rem` > 0 iterations left, P workers and lower bound mc.
// `fac_c` carries FAC's batch chunk from the batch's first step to the others.
SI_HOST_DEVICE inline int64_t chunk_rule_next(int kind, int64_t step, int64_t rem, int64_t P, int64_t mc,
                                              int64_t *fac_c) {
    int64_t c;
    if (kind == SI_SCHED_SS) {
        c = mc;
    } else if (kind == SI_SCHED_GSS) {
        c = (rem + P - 1) / P;
        if (c < mc) c = mc;
    } else {  // SI_SCHED_FAC
        if (step % P == 0) {
            *fac_c = (rem + 2 * P - 1) / (2 * P);
            if (*fac_c < mc) *fac_c = mc;
        }
        c = *fac_c;
    }
    return c < rem ? c : rem;
}

}  // namespace si
