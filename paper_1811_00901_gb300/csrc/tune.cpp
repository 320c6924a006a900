// tune.cpp -- the autotuner: the GPU analogue of the paper's scheduling study
// (Sec. 5 compares STATIC, SS, GSS and FAC on each machine).  For one mesh and
// request shape it times candidate launch settings -- loop rule, minimum chunk,
// image group size, grid resolution and worker count -- with CUDA events on
// the caller's stream, and records the fastest per size class
// (W, floor(log2 n), floor(log2 m)).  The table can be saved to and loaded
// from a small JSON file; si_generate_batched consults it for every item.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace si {
namespace {

struct Entry {
    si_schedule s;
    double ms;
};
using Key = std::tuple<int, int, int>;
std::map<Key, Entry> g_table;
std::mutex g_table_mu;

int ilog2(int64_t v) {
    int l = 0;
    while (v > 1) {
        v >>= 1;
        ++l;
    }
    return l;
}

Key key_of(int W, int64_t n, int64_t m) { return Key{W, ilog2(std::max<int64_t>(1, n)), ilog2(std::max<int64_t>(1, m))}; }

si_status time_one(si_mesh_t mesh, const int32_t *q, int64_t m, int W, float B, float c, si_schedule s, int32_t *out,
                   int reps, cudaStream_t st, double *ms) {
    cudaEvent_t e0, e1;
    SI_CUDA(cudaEventCreate(&e0));
    SI_CUDA(cudaEventCreate(&e1));
    // warm-up (also builds the grid of this resolution)
    si_status r = si_generate(mesh, q, m, W, B, c, s, out, (si_stream)st);
    std::vector<double> t;
    for (int k = 0; r == SI_OK && k < reps; ++k) {
        // each repetition on a freshly built grid (untimed): a grid's order of
        // points within a cell comes from atomics, so rebuilding changes which
        // points share a group, and with it how a rule's chunks balance (most
        // for the cost order, whose first chunks hold the costliest groups);
        // the median then stands for a new mesh, not for one lucky build
        mesh_drop_grids(reinterpret_cast<Mesh *>(mesh));
        r = si_mesh_prepare(mesh, W, B, &s, (si_stream)st);
        if (r != SI_OK) break;
        cudaEventRecord(e0, st);
        r = si_generate(mesh, q, m, W, B, c, s, out, (si_stream)st);
        cudaEventRecord(e1, st);
        if (r != SI_OK) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) {
            r = cuda_fail(e, "tuning run");
            break;
        }
        float f = 0.f;
        cudaEventElapsedTime(&f, e0, e1);
        t.push_back(f);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != SI_OK) return r;
    std::sort(t.begin(), t.end());
    *ms = t.empty() ? 1e30 : t[t.size() / 2];
    return SI_OK;
}

}  // namespace
}  // namespace si

using namespace si;

extern "C" {

si_status si_tune_mesh(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W, float bin_size,
                       float cos_support_angle, int32_t *scratch_out, int32_t reps, si_schedule *best,
                       double *best_ms, si_stream stream) {
    if (!mesh || !scratch_out || m <= 0 || reps < 1 || !best) {
        set_error("si_tune_mesh: bad arguments");
        return SI_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const Mesh *me = reinterpret_cast<const Mesh *>(mesh);
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    const int auto_l2 = choose_log2_group(W, 0);
    // stage 1: group size x grid resolution under FAC (GSS's large first
    // chunks make it the rule most sensitive to which groups come first, a
    // poor guide for the grid the other rules will run on)
    std::vector<int> groups;
    for (int l = auto_l2; l >= 0 && l >= auto_l2 - 2; --l) groups.push_back(1 << l);
    const int divs[] = {4, 6, 8, 12};
    si_schedule cur{SI_SCHED_FAC, 1, 0, 1 << auto_l2, 4};
    double cur_ms = 1e30;
    for (int g : groups)
        for (int d : divs) {
            si_schedule s{SI_SCHED_FAC, 1, 0, g, d};
            double ms;
            si_status r = time_one(mesh, query_idx, m, W, bin_size, cos_support_angle, s, scratch_out, reps, st, &ms);
            if (r != SI_OK) return r;
            if (ms < cur_ms) {
                cur_ms = ms;
                cur = s;
            }
        }
    // stage 2: loop rule x minimum chunk x worker count x group order (the
    // dynamic rules in grid order and in decreasing estimated cost)
    const int l2 = choose_log2_group(W, cur.group);
    const size_t smem = spin_smem_bytes(W, l2);
    const int per_sm = std::max(1, blocks_per_sm_for(smem, ring_mode(l2)));
    const int sms = num_sms(dev);
    const int worker_opts[] = {0, sms * per_sm / 2, sms * per_sm * 2};
    for (int kind = SI_SCHED_STATIC; kind <= SI_SCHED_FAC; ++kind)
        for (int mc : {1, 2, 4}) {
            if (kind == SI_SCHED_STATIC && mc != 1) continue;
            for (int w : worker_opts)
                // (GSS's chunks shrink with the remaining work: its runs of equal chunks
                // to deal the costliest groups over are short, and its first chunks are
                // its largest, so it stays in grid order)
                for (int order = 0; order <= (kind == SI_SCHED_STATIC || kind == SI_SCHED_GSS ? 0 : 1); ++order) {
                    si_schedule s{kind, mc, w, cur.group, cur.grid_div};
                    s.order = order;
                    double ms;
                    si_status r =
                        time_one(mesh, query_idx, m, W, bin_size, cos_support_angle, s, scratch_out, reps, st, &ms);
                    if (r != SI_OK) return r;
                    if (ms < cur_ms) {
                        cur_ms = ms;
                        cur = s;
                    }
                }
        }
    *best = cur;
    if (best_ms) *best_ms = cur_ms;
    std::lock_guard<std::mutex> lk(g_table_mu);
    g_table[key_of(W, me->n, m)] = Entry{cur, cur_ms};
    return SI_OK;
}

si_status si_tune_lookup(int32_t W, int64_t n, int64_t m, si_schedule *out) {
    if (!out) {
        set_error("si_tune_lookup: NULL output");
        return SI_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_table_mu);
    const Key k = key_of(W, n, m);
    auto it = g_table.find(k);
    if (it == g_table.end()) {
        // nearest size class with the same W
        int bestd = 1 << 30;
        for (auto &e : g_table) {
            if (std::get<0>(e.first) != W) continue;
            int d = std::abs(std::get<1>(e.first) - std::get<1>(k)) + std::abs(std::get<2>(e.first) - std::get<2>(k));
            if (d < bestd) {
                bestd = d;
                it = g_table.find(e.first);
            }
        }
        if (it == g_table.end() || bestd > 4) {
            set_error("no tuning entry for W=%d near n=%lld, m=%lld", W, (long long)n, (long long)m);
            return SI_ERR_INVALID;
        }
    }
    *out = it->second.s;
    return SI_OK;
}

si_status si_tune_save(const char *path) {
    if (!path) {
        set_error("si_tune_save: NULL path");
        return SI_ERR_INVALID;
    }
    FILE *f = std::fopen(path, "w");
    if (!f) {
        set_error("si_tune_save: cannot open %s", path);
        return SI_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_table_mu);
    std::fprintf(f, "{\"entries\": [\n");
    size_t k = 0;
    for (auto &e : g_table) {
        const si_schedule &s = e.second.s;
        std::fprintf(f,
                     "  {\"W\": %d, \"log2n\": %d, \"log2m\": %d, \"kind\": %d, \"min_chunk\": %d, "
                     "\"num_workers\": %d, \"group\": %d, \"grid_div\": %d, \"order\": %d, \"ms\": %.6f}%s\n",
                     std::get<0>(e.first), std::get<1>(e.first), std::get<2>(e.first), s.kind, s.min_chunk,
                     s.num_workers, s.group, s.grid_div, s.order, e.second.ms, ++k < g_table.size() ? "," : "");
    }
    std::fprintf(f, "]}\n");
    std::fclose(f);
    return SI_OK;
}

// Reads the format written by si_tune_save: one object per entry with the
// nine numeric fields in any order, and "order" (0 when absent).
si_status si_tune_load(const char *path) {
    if (!path) {
        set_error("si_tune_load: NULL path");
        return SI_ERR_INVALID;
    }
    FILE *f = std::fopen(path, "r");
    if (!f) {
        set_error("si_tune_load: cannot open %s", path);
        return SI_ERR_INVALID;
    }
    std::string txt;
    char buf[4096];
    size_t r;
    while ((r = std::fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, r);
    std::fclose(f);
    std::map<Key, Entry> loaded;
    size_t pos = txt.find('[');
    if (pos == std::string::npos) pos = 0;
    while (true) {
        size_t a = txt.find('{', pos);
        if (a == std::string::npos) break;
        size_t b = txt.find('}', a);
        if (b == std::string::npos) break;
        std::string obj = txt.substr(a, b - a);
        auto field = [&](const char *name, double *v) {
            std::string pat = std::string("\"") + name + "\"";
            size_t p = obj.find(pat);
            if (p == std::string::npos) return false;
            p = obj.find(':', p);
            if (p == std::string::npos) return false;
            *v = std::strtod(obj.c_str() + p + 1, nullptr);
            return true;
        };
        double W, ln, lm, kind, mc, nw, g, d, ms;
        if (field("W", &W) && field("log2n", &ln) && field("log2m", &lm) && field("kind", &kind) &&
            field("min_chunk", &mc) && field("num_workers", &nw) && field("group", &g) && field("grid_div", &d)) {
            if (!field("ms", &ms)) ms = 0;
            double ord = 0;
            if (!field("order", &ord)) ord = 0;  // tables written before the field existed
            si_schedule s{(int)kind, (int)mc, (int)nw, (int)g, (int)d};
            s.order = (int)ord;
            if (s.kind < 0 || s.kind > 3 || s.grid_div < 0 || s.grid_div > 16 || s.order < 0 || s.order > 1) {
                set_error("si_tune_load: bad entry in %s", path);
                return SI_ERR_INVALID;
            }
            loaded[Key{(int)W, (int)ln, (int)lm}] = Entry{s, ms};
        }
        pos = b + 1;
    }
    std::lock_guard<std::mutex> lk(g_table_mu);
    for (auto &e : loaded) g_table[e.first] = e.second;
    return SI_OK;
}

si_status si_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_table_mu);
    g_table.clear();
    return SI_OK;
}

}  // extern "C"
