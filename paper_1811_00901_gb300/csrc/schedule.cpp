// schedule.cpp -- chunk rules of the scheduled image loop (Sec. 2.2 and
// Algorithm 3's getChunk).  The master loop of Algorithm 3 is run once on the
// host to completion; the resulting boundary table is what the persistent
// kernel's workers claim, one atomic increment of the step index per request.
//
// Readings: the scheduling step advances by one per assignment and every chunk
// is clamped to the iterations that remain; GSS never goes below min_chunk;
// FAC hands out batches of P equal chunks of ceil(R / (2P)) (FAC2), R being
// what remains when the batch starts; STATIC gives worker k the block
// [floor(kN/P), floor((k+1)N/P)).
#include <algorithm>
#include <vector>

#include "internal.h"

namespace si {

int64_t chunk_table(int kind, int64_t units, int workers, int min_chunk, std::vector<int64_t> *starts) {
    starts->clear();
    starts->push_back(0);
    const int64_t P = std::max(1, workers);
    const int64_t mc = std::max(1, min_chunk);
    if (units <= 0 && kind != SI_SCHED_STATIC) return 0;
    if (kind == SI_SCHED_STATIC) {
        for (int64_t k = 0; k < P; ++k) starts->push_back((k + 1) * units / P);
        return P;
    }
    int64_t done = 0, step = 0, fac_c = 0;
    while (done < units) {
        const int64_t rem = units - done;
        int64_t c;
        switch (kind) {
            case SI_SCHED_SS:
                c = mc;
                break;
            case SI_SCHED_GSS:
                c = std::max(mc, (rem + P - 1) / P);
                break;
            default:  // SI_SCHED_FAC
                if (step % P == 0) fac_c = std::max(mc, (rem + 2 * P - 1) / (2 * P));
                c = fac_c;
                break;
        }
        c = std::min(c, rem);
        done += c;
        starts->push_back(done);
        ++step;
    }
    return step;
}

}  // namespace si

extern "C" si_status si_chunk_table(int32_t kind, int64_t units, int32_t workers, int32_t min_chunk,
                                    int64_t *starts, int64_t capacity, int64_t *nsteps) {
    if (kind < SI_SCHED_STATIC || kind > SI_SCHED_FAC || units < 0 || workers < 1 || min_chunk < 0 || !nsteps) {
        si::set_error("si_chunk_table: bad arguments");
        return SI_ERR_INVALID;
    }
    std::vector<int64_t> s;
    *nsteps = si::chunk_table(kind, units, workers, min_chunk, &s);
    if (!starts || capacity < (int64_t)s.size()) {
        si::set_error("si_chunk_table: need capacity for %lld entries", (long long)s.size());
        return SI_ERR_INVALID;
    }
    std::copy(s.begin(), s.end(), starts);
    return SI_OK;
}
