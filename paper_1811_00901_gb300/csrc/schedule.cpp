// schedule.cpp -- chunk rules of the scheduled image loop (Sec. 2.2 and
// Algorithm 3's getChunk).  The master loop of Algorithm 3 is run once on the
// host to completion; the resulting boundary table is what the persistent
// kernel's workers claim, one atomic increment of the step index per request.
//
// Readings: the scheduling step advances by one per assignment and every chunk
// is clamped to the iterations that remain; SS, GSS and FAC (FAC2) take their
// chunks from chunk_rule_next (chunk_rule.h, shared with the device code of the
// allocation-free entry point); FAC_PROB takes the batch chunk from the
// original factoring rule (Hummel, Schonberg and Flynn 1992) for iterations
// whose times have coefficient of variation cov; STATIC gives worker k the
// block [floor(kN/P), floor((k+1)N/P)).
#include <algorithm>
#include <cmath>
#include <vector>

#include "chunk_rule.h"
#include "internal.h"

namespace si {

// Batch chunk of probabilistic factoring for batch j with R iterations left:
// b = P / (2 sqrt(R)) * cov, x_0 = 1 + b^2 + b sqrt(b^2 + 2), x_j = 2 + b^2 +
// b sqrt(b^2 + 4), chunk = ceil(R / (x P)); IEEE double, in this order.
int64_t fac_prob_chunk(int64_t batch, int64_t R, int64_t P, double cov) {
    const double b = (double)P / (2.0 * std::sqrt((double)R)) * cov;
    const double x = batch == 0 ? 1.0 + b * b + b * std::sqrt(b * b + 2.0) : 2.0 + b * b + b * std::sqrt(b * b + 4.0);
    return (int64_t)std::ceil((double)R / (x * (double)P));
}

int64_t chunk_table(int kind, int64_t units, int workers, int min_chunk, double cov, std::vector<int64_t> *starts) {
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
        if (kind == SI_SCHED_FAC_PROB) {
            if (step % P == 0) fac_c = std::max(mc, fac_prob_chunk(step / P, rem, P, cov));
            c = std::min(fac_c, rem);
        } else {
            // SS, GSS, FAC (and any other kind as FAC): the rule every caller shares
            c = chunk_rule_next(kind == SI_SCHED_SS || kind == SI_SCHED_GSS ? kind : SI_SCHED_FAC, step, rem, P, mc,
                                &fac_c);
        }
        done += c;
        starts->push_back(done);
        ++step;
    }
    return step;
}

}  // namespace si

extern "C" si_status si_schedule_chunks(const si_schedule *sc, int64_t units, int32_t workers, int64_t *starts,
                                        int64_t capacity, int64_t *nsteps) {
    if (!sc || sc->kind < SI_SCHED_STATIC || sc->kind > SI_SCHED_FAC_PROB || units < 0 || workers < 1 ||
        sc->min_chunk < 0 || !(sc->fac_cov >= 0.0f && sc->fac_cov <= 1e6f) || !nsteps) {
        si::set_error("si_schedule_chunks: bad arguments");
        return SI_ERR_INVALID;
    }
    std::vector<int64_t> s;
    *nsteps = si::chunk_table(sc->kind, units, workers, sc->min_chunk, sc->fac_cov, &s);
    if (!starts || capacity < (int64_t)s.size()) {
        si::set_error("si_schedule_chunks: need capacity for %lld entries", (long long)s.size());
        return SI_ERR_INVALID;
    }
    std::copy(s.begin(), s.end(), starts);
    return SI_OK;
}

extern "C" si_status si_chunk_table(int32_t kind, int64_t units, int32_t workers, int32_t min_chunk,
                                    int64_t *starts, int64_t capacity, int64_t *nsteps) {
    si_schedule sc{};
    sc.kind = kind;
    sc.min_chunk = min_chunk;
    return si_schedule_chunks(&sc, units, workers, starts, capacity, nsteps);
}
