// batch.cu -- turning a batch of items (meshes with their own parameters) into
// device work: the plan (grids, the step table of the scheduled loop, query
// sorting, scratch layout), the descriptor blob, and the recorded commands
// (counter reset, grid-order query sort, persistent spin kernel).  Single-mesh
// calls are batches of one.  Batched calls additionally keep CUDA graphs: the
// first call with a given batch captures its commands once, later identical
// calls replay the graph (one graph launch for the whole batch).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <list>
#include <numeric>

#include "device_common.cuh"
#include "internal.h"
#include "scan.h"

namespace si {

namespace {

// What the query-sort kernels need per item that sorts its queries.
struct SortItem {
    const float4 *pn;
    const int *sorted_pos;
    const int *query_idx;
    int64_t qbase;  // first query of the item in the concatenated query space
    int64_t hbase;  // first histogram bin of the item
    int n_points;
    const GridGeom *geom;
};

__device__ __forceinline__ int find_item(const int64_t *qbase, int nitems, int64_t g) {
    int lo = 0, hi = nitems - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (qbase[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int query_cell(const SortItem &s, int64_t q) {
    int src = s.query_idx ? s.query_idx[q] : (int)q;
    if ((unsigned)src >= (unsigned)s.n_points) src = 0;  // reported by the spin kernel
    const int sp = s.sorted_pos[src];
    const float4 p = s.pn[2 * (int64_t)sp];
    const GridGeom &g = *s.geom;
    const int cx = cell_coord(p.x, g.origin[0], g.inv_cell, g.dims[0]);
    const int cy = cell_coord(p.y, g.origin[1], g.inv_cell, g.dims[1]);
    const int cz = cell_coord(p.z, g.origin[2], g.inv_cell, g.dims[2]);
    return (cz * g.dims[1] + cy) * g.dims[0] + cx;
}

__global__ void qsort_count_kernel(const SortItem *__restrict__ items, const int64_t *__restrict__ qbase,
                                   int nitems, int64_t total, int *__restrict__ hist) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const SortItem &s = items[find_item(qbase, nitems, g)];
        atomicAdd(&hist[s.hbase + query_cell(s, g - s.qbase)], 1);
    }
}

// Exact overflow check of sliced items after the spin kernel: an image's
// pixels (int32 read as signed) sum to 65536 x its contributing pairs unless
// a pixel wrapped.  One warp per image.
__global__ void split_check_kernel(const ItemDesc *__restrict__ items, const int64_t *__restrict__ base,
                                   const int *__restrict__ which, int nsplit, int64_t total) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < total; g += warps) {
        int lo = 0, hi = nsplit - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (base[mid] <= g)
                lo = mid;
            else
                hi = mid - 1;
        }
        const ItemDesc &it = items[which[lo]];
        const int64_t q = g - base[lo];
        const int npix = it.W * it.W;
        const int32_t *img = it.out + q * npix;
        long long s = 0;
        for (int p = lane; p < npix; p += 32) s += img[p];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        const long long w = it.binning == SI_BIN_NEAREST ? 1ll : 65536ll;  // weight of one pair
        if (lane == 0 && s != w * it.counts[q]) atomicOr(it.flags, kFlagOverflow);
    }
}

// hist holds exclusive offsets on entry and is consumed as a cursor.
__global__ void qsort_scatter_kernel(const SortItem *__restrict__ items, const int64_t *__restrict__ qbase,
                                     int nitems, int64_t total, int *__restrict__ hist, int *__restrict__ perm) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const SortItem &s = items[find_item(qbase, nitems, g)];
        const int64_t q = g - s.qbase;
        const int pos = atomicAdd(&hist[s.hbase + query_cell(s, q)], 1);
        perm[pos] = (int)q;
    }
}

int clamp_blocks(int64_t work) {
    int64_t b = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Host-side plan of one batch.
struct Plan {
    int nitems = 0;
    std::vector<Grid *> grids;
    std::vector<int> log2S, units;
    size_t max_img_words = 4, smem = 0;
    int workers = 0;
    int modes = 0;  // tile-ring disciplines of the items' group shapes
    int slow_workers = 0;
    float slowdown = 1.0f;
    std::vector<int> binning;  // per item: si_binning
    // adaptive rules (AWF, AF): unit bases of the items; af: the rule is AF
    bool awf = false;
    bool af = false;
    // cost order (si_schedule.order = 1): the ordered items, their first group
    // in the concatenated group space and their deal batches
    std::vector<int> ord;  // ord_items[n_ord], gbase[n_ord + 1], dbase[n_ord + 1], deal[3 x batches]
    int n_ord = 0, ord_groups = 0;
    int awf_min_chunk = 1;
    std::vector<int> awf_ubase;
    bool all_static = true;
    int nsteps = 0;
    std::vector<Piece> pieces;
    std::vector<int> step_piece;
    std::vector<SortItem> sitems;
    std::vector<int64_t> sqbase;
    std::vector<int> sort_of;
    int64_t qtot = 0, htot = 0;
    // sliced items: their index, first image in the concatenated check space,
    // and the offset of their pair counts
    std::vector<int> slices;
    std::vector<int> split_items;
    std::vector<int64_t> split_base, counts_off;
    int64_t split_images = 0;
    size_t o_ctr = 0, o_items = 0, o_pieces = 0, o_steps = 0, o_sitems = 0, o_sqbase = 0, o_split = 0,
           o_split_items = 0, o_awf_ubase = 0, o_af = 0, o_ord = 0, o_hist = 0, o_perm = 0, o_counts = 0,
           o_gorder = 0, o_gkey = 0, o_ghist = 0,
           total_bytes = 0;
    bool empty = false;
};

si_status plan_batch(const std::vector<si_batch_item> &items, const std::vector<si_schedule> &scheds,
                     int forced_workers, bool probe, cudaStream_t stream, Plan *p) {
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    const int nitems = (int)items.size();
    p->nitems = nitems;
    for (int k = 0; k < nitems; ++k) {
        si_status st = check_item(items[k], scheds[k], dev);
        if (st != SI_OK) return st;
    }
    // ---- grids and per-item shapes
    p->grids.assign(nitems, nullptr);
    p->log2S.resize(nitems);
    p->units.resize(nitems);
    int64_t total_units = 0;
    for (int k = 0; k < nitems; ++k) {
        const si_batch_item &it = items[k];
        Mesh *m = reinterpret_cast<Mesh *>(it.mesh);
        p->log2S[k] = choose_log2_group(it.W, scheds[k].group);
        p->units[k] = (int)((it.m + (1 << p->log2S[k]) - 1) >> p->log2S[k]);
        total_units += p->units[k];
        if (it.m == 0) continue;
        si_status st;
        p->grids[k] = mesh_grid(m, grid_cell_for(m, it.W, it.bin_size, scheds[k].grid_div), stream, &st);
        if (!p->grids[k]) return st;
        p->max_img_words = std::max(p->max_img_words, image_words(it.W, p->log2S[k]));
    }
    if (total_units == 0) {
        p->empty = true;
        return SI_OK;
    }
    if (total_units > INT32_MAX) {
        set_error("too many image groups in one call");
        return SI_ERR_INVALID;
    }
    // heterogeneity emulation: from the override, or the first item's rule
    p->slow_workers = scheds[0].slow_workers;
    p->slowdown = scheds[0].slowdown >= 1.0f ? scheds[0].slowdown : 1.0f;
    p->binning.resize(nitems);
    p->modes = 0;
    for (int k = 0; k < nitems; ++k) {
        p->binning[k] = scheds[k].binning;
        p->modes |= ring_mode(p->log2S[k]) | (scheds[k].binning == SI_BIN_NEAREST ? kModeNearest : 0);
    }
    p->smem = 0;
    for (int k = 0; k < nitems; ++k)
        if (items[k].m > 0) p->smem = std::max(p->smem, spin_smem_bytes(items[k].W, p->log2S[k]));
    p->modes = launch_modes_for(p->modes, p->smem, probe);
    SI_CUDA(setup_spin_kernel_attributes(p->smem));
    const int per_sm = blocks_per_sm_for(p->smem, p->modes);
    if (per_sm < 1) {
        set_error("spin kernel does not fit on an SM with %zu bytes of shared memory", p->smem);
        return SI_ERR_INVALID;
    }
    int workers = forced_workers > 0 ? forced_workers : 0;
    if (!workers)
        for (int k = 0; k < nitems; ++k) workers = std::max(workers, scheds[k].num_workers);
    if (!workers) workers = num_sms(dev) * per_sm;
    p->workers = workers;

    // ---- candidate slices: a call with few groups would leave most workers
    // idle (a group is one block's work), so each group's candidate stream is
    // split over several blocks; probes need whole groups
    p->slices.assign(nitems, 1);
    const int auto_k = total_units >= 2 * (int64_t)workers
                           ? 1
                           : (int)std::min<int64_t>(64, (2 * (int64_t)workers + total_units - 1) / total_units);
    total_units = 0;
    for (int k = 0; k < nitems; ++k) {
        int K = scheds[k].slices > 0 ? std::min(scheds[k].slices, 64) : auto_k;
        if (probe) K = 1;
        p->slices[k] = K;
        p->units[k] *= K;
        total_units += p->units[k];
        if (K > 1 && items[k].m > 0) {
            p->split_items.push_back(k);
            p->split_base.push_back(p->split_images);
            p->counts_off.push_back(p->split_images);
            p->split_images += items[k].m;
        }
    }
    if (total_units > INT32_MAX) {
        set_error("too many image groups in one call");
        return SI_ERR_INVALID;
    }
    p->split_base.push_back(p->split_images);

    // ---- the scheduled loop: steps made of pieces
    int n_awf = 0, n_af = 0, n_used = 0;
    for (int k = 0; k < nitems; ++k) {
        if (items[k].m > 0 && scheds[k].kind != SI_SCHED_STATIC) p->all_static = false;
        if (items[k].m > 0) {
            ++n_used;
            if (scheds[k].kind == SI_SCHED_AWF) ++n_awf;
            if (scheds[k].kind == SI_SCHED_AF) ++n_af;
        }
    }
    if ((n_awf > 0 && n_awf != n_used) || (n_af > 0 && n_af != n_used)) {
        set_error("an adaptive rule (AWF, AF) must be the rule of every item of a call");
        return SI_ERR_INVALID;
    }
    p->af = n_af > 0;
    n_awf += n_af;
    p->step_piece.assign(1, 0);
    std::vector<std::vector<int64_t>> tables(nitems);  // each item's chunk table (dynamic rules)
    if (n_awf > 0) {
        // one loop over the concatenated units, chunk sizes decided on the device
        p->awf = true;
        p->awf_ubase.assign(nitems + 1, 0);
        for (int k = 0; k < nitems; ++k) p->awf_ubase[k + 1] = p->awf_ubase[k] + p->units[k];
        int mc = 1;
        for (int k = 0; k < nitems; ++k)
            if (items[k].m > 0) {
                mc = std::max(1, scheds[k].min_chunk);
                break;
            }
        p->awf_min_chunk = mc;
        p->nsteps = 0;
    } else if (p->all_static) {
        // PSIA: block b gets the contiguous block [floor(bU/P), floor((b+1)U/P)) of
        // the concatenated group space; a block may span item boundaries.
        std::vector<int64_t> ubase(nitems + 1, 0);
        for (int k = 0; k < nitems; ++k) ubase[k + 1] = ubase[k] + p->units[k];
        int k = 0;
        for (int b = 0; b < workers; ++b) {
            int64_t lo = (int64_t)b * total_units / workers, hi = (int64_t)(b + 1) * total_units / workers;
            while (lo < hi) {
                while (ubase[k + 1] <= lo) ++k;
                const int64_t e = std::min(hi, ubase[k + 1]);
                p->pieces.push_back(Piece{k, (int)(lo - ubase[k]), (int)(e - ubase[k]), 0});
                lo = e;
            }
            p->step_piece.push_back((int)p->pieces.size());
        }
    } else {
        // each item's own rule; items with more work first
        std::vector<int> order(nitems);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const Mesh *ma = reinterpret_cast<const Mesh *>(items[a].mesh);
            const Mesh *mb = reinterpret_cast<const Mesh *>(items[b].mesh);
            return (double)items[a].m * ma->n > (double)items[b].m * mb->n;
        });
        std::vector<int64_t> st;
        for (int k : order) {
            if (p->units[k] == 0) continue;
            chunk_table(scheds[k].kind, p->units[k], workers, scheds[k].min_chunk, scheds[k].fac_cov, &st);
            tables[k] = st;
            for (size_t s = 0; s + 1 < st.size(); ++s) {
                if (st[s + 1] == st[s]) continue;
                p->pieces.push_back(Piece{k, (int)st[s], (int)st[s + 1], 0});
                p->step_piece.push_back((int)p->pieces.size());
            }
        }
    }
    if (!p->awf) p->nsteps = (int)p->step_piece.size() - 1;

    // ---- cost order of the groups of the dynamic rules' items that ask for it.
    // Deal batches: within a run of equal chunks of the item's table (a FAC
    // batch), the cost-sorted groups are dealt round-robin over the run's
    // chunks, so that no chunk bundles the costliest groups (a chunk of c
    // groups from the top of the order could outlast a worker's whole share)
    {
        std::vector<int> oi, gb(1, 0), db(1, 0), deal;
        for (int k = 0; k < nitems; ++k) {
            if (items[k].m == 0 || scheds[k].order != 1 || scheds[k].kind == SI_SCHED_STATIC || p->all_static)
                continue;
            const int groups = p->units[k] / p->slices[k];
            if (groups < 2) continue;
            oi.push_back(k);
            gb.push_back(gb.back() + groups);
            const std::vector<int64_t> &t = tables[k];
            if (p->slices[k] == 1 && t.size() > 2) {
                size_t s = 0;
                while (s + 1 < t.size()) {
                    const int64_t c = t[s + 1] - t[s];
                    size_t e = s + 1;
                    while (e + 1 < t.size() && t[e + 1] - t[e] == c && (int64_t)(e - s) < workers) ++e;
                    const int64_t nc = (int64_t)(e - s);
                    if (c >= 2 && nc >= 2) {
                        deal.push_back((int)t[s]);
                        deal.push_back((int)nc);
                        deal.push_back((int)c);
                    }
                    s = e;
                }
            }
            db.push_back((int)deal.size() / 3);
        }
        p->n_ord = (int)oi.size();
        p->ord_groups = gb.back();
        p->ord = oi;
        if (p->n_ord > 0) {
            p->ord.insert(p->ord.end(), gb.begin(), gb.end());
            p->ord.insert(p->ord.end(), db.begin(), db.end());
            p->ord.insert(p->ord.end(), deal.begin(), deal.end());
        }
    }

    // ---- query sorting (items that are not "all points of the mesh")
    p->sort_of.assign(nitems, -1);
    for (int k = 0; k < nitems; ++k) {
        const si_batch_item &it = items[k];
        const Mesh *m = reinterpret_cast<const Mesh *>(it.mesh);
        if (it.m == 0) continue;
        if (!it.query_idx && it.m == m->n) continue;  // grid order is the query order
        const Grid *g = p->grids[k];
        SortItem s;
        s.pn = g->pn;
        s.sorted_pos = g->sorted_pos;
        s.query_idx = it.query_idx;
        s.n_points = (int)m->n;
        s.qbase = p->qtot;
        s.hbase = p->htot;
        s.geom = g->geom;
        p->sort_of[k] = (int)p->sitems.size();
        p->sitems.push_back(s);
        p->sqbase.push_back(p->qtot);
        p->qtot += it.m;
        p->htot += g->ncell_cap;  // the device geometry's cells fit within the cap
    }
    if (p->htot + 1 > INT32_MAX || p->qtot > INT32_MAX) {
        set_error("query sort too large for one call");
        return SI_ERR_INVALID;
    }

    // ---- scratch layout (one allocation per call)
    p->o_ctr = 0;
    p->o_items = align_up(p->o_ctr + sizeof(LaunchCounters), 256);
    p->o_pieces = align_up(p->o_items + sizeof(ItemDesc) * nitems, 256);
    p->o_steps = align_up(p->o_pieces + sizeof(Piece) * p->pieces.size(), 256);
    p->o_sitems = align_up(p->o_steps + sizeof(int) * p->step_piece.size(), 256);
    p->o_sqbase = align_up(p->o_sitems + sizeof(SortItem) * p->sitems.size(), 256);
    p->o_split = align_up(p->o_sqbase + sizeof(int64_t) * p->sqbase.size(), 256);
    p->o_split_items = align_up(p->o_split + sizeof(int64_t) * p->split_base.size(), 256);
    p->o_awf_ubase = align_up(p->o_split_items + sizeof(int) * p->split_items.size(), 256);
    p->o_af = align_up(p->o_awf_ubase + sizeof(int) * p->awf_ubase.size(), 256);
    p->o_ord = align_up(p->o_af + (p->af ? sizeof(AfWorker) * (size_t)p->workers : 0), 256);
    p->o_hist = align_up(p->o_ord + sizeof(int) * p->ord.size(), 256);
    p->o_perm = align_up(p->o_hist + sizeof(int) * (p->htot + 1), 256);
    p->o_counts = align_up(p->o_perm + sizeof(int) * p->qtot, 256);
    p->o_gorder = align_up(p->o_counts + sizeof(int) * p->split_images, 256);
    p->o_gkey = align_up(p->o_gorder + sizeof(int) * (size_t)p->ord_groups, 256);
    p->o_ghist = align_up(p->o_gkey + sizeof(uint16_t) * (size_t)p->ord_groups, 256);
    p->total_bytes = align_up(p->o_ghist + sizeof(int) * (size_t)p->n_ord * kCostBuckets, 256);
    return SI_OK;
}

// Descriptors, pieces, steps and sort items for a scratch at `scratch`.
void fill_blob(const Plan &p, const std::vector<si_batch_item> &items, const std::vector<const si_probe *> &probes,
               char *scratch, std::vector<char> *blob) {
    blob->assign(p.o_hist - p.o_items, 0);
    int *d_perm = reinterpret_cast<int *>(scratch + p.o_perm);
    std::vector<ItemDesc> descs(p.nitems);
    for (int k = 0; k < p.nitems; ++k) {
        const si_batch_item &it = items[k];
        const Mesh *m = reinterpret_cast<const Mesh *>(it.mesh);
        ItemDesc &d = descs[k];
        std::memset(&d, 0, sizeof(d));
        d.m = it.m;
        d.n_points = (int)m->n;
        d.W = it.W;
        d.log2S = p.log2S[k];
        d.units = p.units[k];
        d.out = it.out;
        d.flags = m->flags;
        d.query_idx = it.query_idx;
        if (it.m == 0) continue;
        const Grid *g = p.grids[k];
        d.pn = g->pn;
        d.cell_start = g->cell_start;
        d.sorted_pos = g->sorted_pos;
        d.geom = g->geom;
        if (p.sort_of[k] < 0) {
            d.perm = g->orig_idx;
            d.perm_is_grid = 1;
        } else {
            d.perm = d_perm + p.sitems[p.sort_of[k]].qbase;
            d.perm_is_grid = 0;
        }
        const float rc2 = candidate_rc2(it.W, it.bin_size, p.binning[k]);
        d.binning = p.binning[k];
        d.B = it.bin_size;
        d.Rc2 = rc2;
        d.Rc = std::sqrt(rc2);
        d.cosS = it.cos_support_angle;
        d.invB = 1.0f / it.bin_size;
        d.halfW = 0.5f * (float)it.W;
        d.umax = (float)(it.W - 1);
        const si_probe *pr = probes.empty() ? nullptr : probes[k];
        if (pr) {
            d.p_culled = pr->culled;
            d.p_hash = pr->cand_hash;
            d.p_support = pr->support;
            d.p_worker = pr->worker;
            d.p_step = pr->step;
            d.p_examined = pr->examined;
            d.p_angle = pr->angle;
        }
    }
    int *d_counts = reinterpret_cast<int *>(scratch + p.o_counts);
    for (int k = 0; k < p.nitems; ++k) descs[k].slices = p.slices[k];
    for (size_t s = 0; s < p.split_items.size(); ++s) descs[p.split_items[s]].counts = d_counts + p.counts_off[s];
    int *d_gorder = reinterpret_cast<int *>(scratch + p.o_gorder);
    for (int j = 0; j < p.n_ord; ++j) descs[p.ord[j]].gorder = d_gorder + p.ord[p.n_ord + j];
    char *h = blob->data();
    std::memcpy(h, descs.data(), sizeof(ItemDesc) * p.nitems);
    std::memcpy(h + (p.o_pieces - p.o_items), p.pieces.data(), sizeof(Piece) * p.pieces.size());
    std::memcpy(h + (p.o_steps - p.o_items), p.step_piece.data(), sizeof(int) * p.step_piece.size());
    if (!p.sitems.empty()) {
        std::memcpy(h + (p.o_sitems - p.o_items), p.sitems.data(), sizeof(SortItem) * p.sitems.size());
        std::memcpy(h + (p.o_sqbase - p.o_items), p.sqbase.data(), sizeof(int64_t) * p.sqbase.size());
    }
    if (!p.split_items.empty()) {
        std::memcpy(h + (p.o_split - p.o_items), p.split_base.data(), sizeof(int64_t) * p.split_base.size());
        std::memcpy(h + (p.o_split_items - p.o_items), p.split_items.data(), sizeof(int) * p.split_items.size());
    }
    if (p.awf) {
        std::memcpy(h + (p.o_awf_ubase - p.o_items), p.awf_ubase.data(), sizeof(int) * p.awf_ubase.size());
    }
    if (p.n_ord > 0) std::memcpy(h + (p.o_ord - p.o_items), p.ord.data(), sizeof(int) * p.ord.size());
}

// Device commands of a planned batch on `stream` (also what a graph captures).
// Returns the number of kernels recorded in *kernels.
si_status record_batch(const Plan &p, const std::vector<si_batch_item> &items, char *scratch, bool probe,
                       cudaStream_t stream, int *kernels, const si_trace *trace = nullptr) {
    int nk = 0;
    cudaError_t e = cudaMemsetAsync(scratch + p.o_ctr, 0, sizeof(LaunchCounters), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counters)");
    // sliced items accumulate into zeroed outputs and pair counts
    for (int k : p.split_items) {
        const si_batch_item &it = items[k];
        e = cudaMemsetAsync(it.out, 0, sizeof(int32_t) * (size_t)it.m * it.W * it.W, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(sliced output)");
    }
    if (p.split_images > 0) {
        e = cudaMemsetAsync(scratch + p.o_counts, 0, sizeof(int) * p.split_images, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(pair counts)");
    }
    if (p.qtot > 0) {
        int *hist = reinterpret_cast<int *>(scratch + p.o_hist);
        int *perm = reinterpret_cast<int *>(scratch + p.o_perm);
        const SortItem *d_sitems = reinterpret_cast<const SortItem *>(scratch + p.o_sitems);
        const int64_t *d_sqbase = reinterpret_cast<const int64_t *>(scratch + p.o_sqbase);
        e = cudaMemsetAsync(hist, 0, sizeof(int) * (p.htot + 1), stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(hist)");
        qsort_count_kernel<<<clamp_blocks(p.qtot), 256, 0, stream>>>(d_sitems, d_sqbase, (int)p.sitems.size(),
                                                                     p.qtot, hist);
        ++nk;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "query sort");
        const int64_t before = si_kernel_launches();
        si_status st = scan_exclusive(hist, hist, p.htot + 1, stream);
        if (st != SI_OK) return st;
        const int scan_k = (int)(si_kernel_launches() - before);
        note_launches(-scan_k);  // the caller counts every recorded kernel once per run
        nk += scan_k;
        qsort_scatter_kernel<<<clamp_blocks(p.qtot), 256, 0, stream>>>(d_sitems, d_sqbase, (int)p.sitems.size(),
                                                                       p.qtot, hist, perm);
        ++nk;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "query sort");
    }
    if (p.n_ord > 0) {
        // the query order (above) first: the cost estimate reads each group's queries
        const int *d_ord = reinterpret_cast<const int *>(scratch + p.o_ord);
        int kk = 0;
        si_status st = enqueue_group_order(reinterpret_cast<const ItemDesc *>(scratch + p.o_items), d_ord,
                                           d_ord + p.n_ord, d_ord + 2 * p.n_ord + 1, d_ord + 3 * p.n_ord + 2,
                                           p.n_ord, p.ord_groups,
                                           reinterpret_cast<uint16_t *>(scratch + p.o_gkey),
                                           reinterpret_cast<int *>(scratch + p.o_ghist),
                                           reinterpret_cast<int *>(scratch + p.o_gorder), stream, &kk);
        if (st != SI_OK) return st;
        nk += kk;
    }
    LaunchArgs a;
    a.items = reinterpret_cast<const ItemDesc *>(scratch + p.o_items);
    a.pieces = reinterpret_cast<const Piece *>(scratch + p.o_pieces);
    a.step_piece = reinterpret_cast<const int *>(scratch + p.o_steps);
    a.nsteps = p.nsteps;
    a.is_static = p.all_static ? 1 : 0;
    a.ctr = reinterpret_cast<LaunchCounters *>(scratch + p.o_ctr);
    a.nitems = p.nitems;
    a.img_words = (int)p.max_img_words;
    a.probe = probe ? 1 : 0;
    a.modes = p.modes;
    if (p.awf) {
        a.awf = 1;
        a.total_units = p.awf_ubase.back();
        a.unit_base = reinterpret_cast<const int *>(scratch + p.o_awf_ubase);
        a.min_chunk = p.awf_min_chunk;
        if (p.af) {
            a.af = 1;
            a.af_workers = reinterpret_cast<AfWorker *>(scratch + p.o_af);
        }
    }
    // heterogeneity emulation: at most every launched block is slow
    const int blocks = p.all_static ? p.nsteps : p.workers;
    a.slow_workers = std::min(p.slow_workers, blocks);
    a.slowdown = p.slowdown;
    if (trace) {
        a.trace = trace->claims;
        a.trace_cap = trace->capacity;
        a.trace_count = trace->count;
    }
    launch_spin_kernel(a, p.all_static ? p.nsteps : p.workers, p.smem, stream);
    ++nk;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "spin kernel launch");
    if (p.split_images > 0) {
        const int blocks = (int)std::min<int64_t>((p.split_images + 7) / 8, 152 * 8);
        split_check_kernel<<<blocks, 256, 0, stream>>>(
            a.items, reinterpret_cast<const int64_t *>(scratch + p.o_split),
            reinterpret_cast<const int *>(scratch + p.o_split_items), (int)p.split_items.size(), p.split_images);
        ++nk;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "overflow check launch");
    }
    *kernels = nk;
    return SI_OK;
}

void note_calls(const std::vector<si_batch_item> &items) {
    for (const auto &it : items) {
        Mesh *m = reinterpret_cast<Mesh *>(it.mesh);
        std::lock_guard<std::mutex> lk(m->mu);
        m->calls += 1;
        m->images += it.m;
    }
}

// Brackets the spin work of a call with timing events when timing is on.
struct TimedRegion {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Mesh *mesh = nullptr;
    TimedRegion(Mesh *m, cudaStream_t s) {
        if (!timing_enabled()) return;
        mesh = m;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, s);
    }
    void end(cudaStream_t s) {
        if (!mesh) return;
        cudaEventRecord(e1, s);
        std::lock_guard<std::mutex> lk(mesh->mu);
        mesh->pending_events.emplace_back(e0, e1);
        mesh = nullptr;
    }
};

// ------------------------------------------------------------ graph cache --
struct GraphEntry {
    std::vector<char> key;
    std::vector<const Mesh *> meshes;
    cudaGraphExec_t exec = nullptr;
    char *scratch = nullptr;  // pool memory, persistent for the entry's lifetime
    cudaEvent_t last = nullptr;
    int kernels = 0;
    int device = 0;
};
std::list<GraphEntry> g_graphs;  // most recently used first
std::mutex g_graphs_mu;
constexpr size_t kMaxGraphs = 8;

void destroy_entry(GraphEntry &e) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(e.device);
    if (e.last) {
        cudaEventSynchronize(e.last);
        cudaEventDestroy(e.last);
    }
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.scratch) {
        dev_free(e.scratch, nullptr);
        cudaStreamSynchronize(nullptr);
    }
    cudaSetDevice(prev);
}

std::vector<char> batch_key(const std::vector<si_batch_item> &items, const std::vector<si_schedule> &scheds,
                            int forced_workers, int dev) {
    std::vector<char> k(sizeof(int) * 2 + items.size() * (sizeof(si_batch_item) + sizeof(si_schedule)));
    char *p = k.data();
    std::memcpy(p, &dev, sizeof(int));
    std::memcpy(p + sizeof(int), &forced_workers, sizeof(int));
    p += 2 * sizeof(int);
    for (size_t i = 0; i < items.size(); ++i) {
        std::memcpy(p, &items[i], sizeof(si_batch_item));
        p += sizeof(si_batch_item);
        std::memcpy(p, &scheds[i], sizeof(si_schedule));
        p += sizeof(si_schedule);
    }
    return k;
}

}  // namespace

si_status enqueue_batch(const std::vector<si_batch_item> &items, const std::vector<si_schedule> &scheds,
                        const std::vector<const si_probe *> &probes, cudaStream_t stream, int forced_workers,
                        const si_trace *trace) {
    bool probe = false;
    for (auto *pr : probes)
        if (pr) probe = true;
    Plan p;
    si_status st = plan_batch(items, scheds, forced_workers, probe, stream, &p);
    if (st != SI_OK || p.empty) return st;
    char *scratch = nullptr;
    st = dev_alloc((void **)&scratch, p.total_bytes, stream);
    if (st != SI_OK) return st;
    std::vector<char> blob;
    fill_blob(p, items, probes, scratch, &blob);
    st = stage_upload(scratch + p.o_items, blob.data(), blob.size(), stream);
    if (st == SI_OK) {
        TimedRegion tr(reinterpret_cast<Mesh *>(items[0].mesh), stream);
        int nk = 0;
        st = record_batch(p, items, scratch, probe, stream, &nk, trace);
        tr.end(stream);
        note_launches(nk);
        if (st == SI_OK) note_calls(items);
    }
    dev_free(scratch, stream);
    return st;
}

// Batched calls: replay a cached graph when the same batch comes again,
// capture one otherwise.  The legacy default stream cannot be captured; such
// calls take the direct path.
si_status enqueue_batch_graph(const std::vector<si_batch_item> &items, const std::vector<si_schedule> &scheds,
                              cudaStream_t stream, int forced_workers) {
    if (stream == nullptr) return enqueue_batch(items, scheds, {}, stream, forced_workers);
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    std::vector<char> key = batch_key(items, scheds, forced_workers, dev);
    {
        std::lock_guard<std::mutex> lk(g_graphs_mu);
        for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
            if (it->key != key) continue;
            g_graphs.splice(g_graphs.begin(), g_graphs, it);  // most recently used
            GraphEntry &e = g_graphs.front();
            TimedRegion tr(reinterpret_cast<Mesh *>(items[0].mesh), stream);
            cudaError_t err = cudaGraphLaunch(e.exec, stream);
            tr.end(stream);
            if (err == cudaSuccess) err = cudaEventRecord(e.last, stream);
            if (err != cudaSuccess) return cuda_fail(err, "cudaGraphLaunch");
            note_launches(e.kernels);
            note_calls(items);
            return SI_OK;
        }
    }
    Plan p;
    si_status st = plan_batch(items, scheds, forced_workers, false, stream, &p);
    if (st != SI_OK || p.empty) return st;
    GraphEntry e;
    e.key = key;
    e.device = dev;
    for (const auto &it : items) e.meshes.push_back(reinterpret_cast<const Mesh *>(it.mesh));
    // the entry's scratch lives as long as the entry: taken from the pool in
    // stream order before capture, returned when the entry is destroyed
    st = dev_alloc((void **)&e.scratch, p.total_bytes, stream);
    if (st != SI_OK) return st;
    cudaError_t err = cudaSuccess;
    std::vector<char> blob;
    fill_blob(p, items, {}, e.scratch, &blob);
    // the descriptor blob is uploaded once, outside the graph, in stream order
    st = stage_upload(e.scratch + p.o_items, blob.data(), blob.size(), stream);
    cudaGraph_t graph = nullptr;
    if (st == SI_OK) {
        err = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) st = cuda_fail(err, "cudaStreamBeginCapture");
    }
    if (st == SI_OK) {
        st = record_batch(p, items, e.scratch, false, stream, &e.kernels);
        err = cudaStreamEndCapture(stream, &graph);
        if (err != cudaSuccess && st == SI_OK) st = cuda_fail(err, "cudaStreamEndCapture");
    }
    if (st == SI_OK) {
        err = cudaGraphInstantiate(&e.exec, graph, 0);
        if (err != cudaSuccess) st = cuda_fail(err, "cudaGraphInstantiate");
    }
    if (graph) cudaGraphDestroy(graph);
    if (st == SI_OK) {
        err = cudaEventCreateWithFlags(&e.last, cudaEventDisableTiming);
        if (err != cudaSuccess) st = cuda_fail(err, "cudaEventCreate");
    }
    if (st == SI_OK) {
        TimedRegion tr(reinterpret_cast<Mesh *>(items[0].mesh), stream);
        err = cudaGraphLaunch(e.exec, stream);
        tr.end(stream);
        if (err == cudaSuccess) err = cudaEventRecord(e.last, stream);
        if (err != cudaSuccess) st = cuda_fail(err, "cudaGraphLaunch");
    }
    if (st != SI_OK) {
        cudaStreamSynchronize(stream);
        destroy_entry(e);
        return st;
    }
    note_launches(e.kernels);
    note_calls(items);
    std::lock_guard<std::mutex> lk(g_graphs_mu);
    g_graphs.push_front(std::move(e));
    while (g_graphs.size() > kMaxGraphs) {
        destroy_entry(g_graphs.back());
        g_graphs.pop_back();
    }
    return SI_OK;
}

// Drops cached graphs that reference a mesh (called when the mesh goes away).
void forget_mesh_graphs(const void *mesh) {
    std::lock_guard<std::mutex> lk(g_graphs_mu);
    for (auto it = g_graphs.begin(); it != g_graphs.end();) {
        if (std::find(it->meshes.begin(), it->meshes.end(), mesh) != it->meshes.end()) {
            destroy_entry(*it);
            it = g_graphs.erase(it);
        } else {
            ++it;
        }
    }
}

size_t cached_batch_graphs() {
    std::lock_guard<std::mutex> lk(g_graphs_mu);
    return g_graphs.size();
}

}  // namespace si
