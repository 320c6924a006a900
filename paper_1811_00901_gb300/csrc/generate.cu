// generate.cu -- enqueueing spin-image generation: argument checks, grids,
// grid-order query sorting, the step table of the scheduled loop, item
// descriptors, and the persistent launch.  Single-mesh, batched and
// host-buffer entry points all go through enqueue_batch.
#include <algorithm>
#include <cmath>
#include <cstring>
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
    float origin[3];
    float inv;
    int dims[3];
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

__device__ __forceinline__ int query_cell(const SortItem &s, int64_t q, int *out_q) {
    int src = s.query_idx ? s.query_idx[q] : (int)q;
    if ((unsigned)src >= (unsigned)s.n_points) src = 0;  // reported by the spin kernel
    const int sp = s.sorted_pos[src];
    const float4 p = s.pn[2 * (int64_t)sp];
    const int cx = cell_coord(p.x, s.origin[0], s.inv, s.dims[0]);
    const int cy = cell_coord(p.y, s.origin[1], s.inv, s.dims[1]);
    const int cz = cell_coord(p.z, s.origin[2], s.inv, s.dims[2]);
    *out_q = (int)q;
    return (cz * s.dims[1] + cy) * s.dims[0] + cx;
}

__global__ void qsort_count_kernel(const SortItem *__restrict__ items, const int64_t *__restrict__ qbase,
                                   int nitems, int64_t total, int *__restrict__ hist) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_item(qbase, nitems, g);
        const SortItem &s = items[k];
        int q;
        const int c = query_cell(s, g - s.qbase, &q);
        atomicAdd(&hist[s.hbase + c], 1);
    }
}

// hist holds exclusive offsets on entry and is consumed as a cursor.
__global__ void qsort_scatter_kernel(const SortItem *__restrict__ items, const int64_t *__restrict__ qbase,
                                     int nitems, int64_t total, int *__restrict__ hist, int *__restrict__ perm) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
        const int k = find_item(qbase, nitems, g);
        const SortItem &s = items[k];
        int q;
        const int c = query_cell(s, g - s.qbase, &q);
        const int pos = atomicAdd(&hist[s.hbase + c], 1);
        perm[pos] = q;
    }
}

int clamp_blocks(int64_t work) {
    int64_t b = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 8));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool valid_group(int g) { return g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32; }

}  // namespace

si_status check_item(const si_batch_item &it, const si_schedule &sc, int dev) {
    if (!it.mesh) {
        set_error("NULL mesh");
        return SI_ERR_INVALID;
    }
    const Mesh *m = reinterpret_cast<const Mesh *>(it.mesh);
    if (m->device != dev) {
        set_error("mesh lives on device %d, current device is %d", m->device, dev);
        return SI_ERR_INVALID;
    }
    if (it.W < 2 || it.W > kMaxW) {
        set_error("W = %d outside [2, %d]", it.W, kMaxW);
        return SI_ERR_INVALID;
    }
    if (!(it.bin_size > 0.0f) || !std::isfinite(it.bin_size)) {
        set_error("bin size must be positive and finite");
        return SI_ERR_INVALID;
    }
    if (!(it.cos_support_angle >= -1.0f && it.cos_support_angle <= 1.0f)) {
        set_error("cos of the support angle must lie in [-1, 1]");
        return SI_ERR_INVALID;
    }
    if (it.m < 0 || it.m > INT32_MAX) {
        set_error("m = %lld out of range", (long long)it.m);
        return SI_ERR_INVALID;
    }
    if (!it.query_idx && it.m > m->n) {
        set_error("m = %lld exceeds the mesh size %lld with NULL query_idx", (long long)it.m, (long long)m->n);
        return SI_ERR_INVALID;
    }
    if (it.m > 0 && !it.out) {
        set_error("NULL output");
        return SI_ERR_INVALID;
    }
    if (sc.kind < SI_SCHED_STATIC || sc.kind > SI_SCHED_FAC || sc.min_chunk < 0 || sc.num_workers < 0 ||
        !valid_group(sc.group) || sc.grid_div < 0 || sc.grid_div > 16) {
        set_error("bad schedule (kind %d, min_chunk %d, workers %d, group %d, grid_div %d)", sc.kind, sc.min_chunk,
                  sc.num_workers, sc.group, sc.grid_div);
        return SI_ERR_INVALID;
    }
    const int l2 = choose_log2_group(it.W, sc.group);
    if (spin_smem_bytes(image_words(it.W, l2)) > (size_t)227 * 1024) {
        set_error("W = %d with group %d needs more shared memory than a block has", it.W, 1 << l2);
        return SI_ERR_INVALID;
    }
    return SI_OK;
}

si_status enqueue_batch(const std::vector<si_batch_item> &items, const std::vector<si_schedule> &scheds,
                        const std::vector<const si_probe *> &probes, cudaStream_t stream, int forced_workers) {
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    const int nitems = (int)items.size();
    for (int k = 0; k < nitems; ++k) {
        si_status st = check_item(items[k], scheds[k], dev);
        if (st != SI_OK) return st;
    }
    // ---- grids and per-item shapes (host)
    std::vector<Grid *> grids(nitems, nullptr);
    std::vector<int> log2S(nitems), units(nitems);
    size_t max_img_words = 4;
    int64_t total_units = 0;
    for (int k = 0; k < nitems; ++k) {
        const si_batch_item &it = items[k];
        Mesh *m = reinterpret_cast<Mesh *>(it.mesh);
        log2S[k] = choose_log2_group(it.W, scheds[k].group);
        units[k] = (int)((it.m + (1 << log2S[k]) - 1) >> log2S[k]);
        total_units += units[k];
        if (it.m == 0) continue;
        si_status st;
        grids[k] = mesh_grid(m, grid_cell_for(m, it.W, it.bin_size, scheds[k].grid_div), stream, &st);
        if (!grids[k]) return st;
        max_img_words = std::max(max_img_words, image_words(it.W, log2S[k]));
    }
    if (total_units == 0) return SI_OK;
    if (total_units > INT32_MAX) {
        set_error("too many image groups in one call");
        return SI_ERR_INVALID;
    }
    const size_t smem = spin_smem_bytes(max_img_words);
    SI_CUDA(setup_spin_kernel_attributes(smem));
    int per_sm = blocks_per_sm_for(smem);
    if (per_sm < 1) {
        set_error("spin kernel does not fit on an SM with %zu bytes of shared memory", smem);
        return SI_ERR_INVALID;
    }
    int workers = forced_workers > 0 ? forced_workers : 0;
    if (!workers)
        for (int k = 0; k < nitems; ++k) workers = std::max(workers, scheds[k].num_workers);
    if (!workers) workers = num_sms(dev) * per_sm;

    // ---- the scheduled loop: steps made of pieces
    bool all_static = true;
    for (int k = 0; k < nitems; ++k)
        if (items[k].m > 0 && scheds[k].kind != SI_SCHED_STATIC) all_static = false;
    std::vector<Piece> pieces;
    std::vector<int> step_piece(1, 0);
    if (all_static) {
        // PSIA: block b gets the contiguous block [floor(bU/P), floor((b+1)U/P)) of
        // the concatenated group space; a block may span item boundaries.
        std::vector<int64_t> ubase(nitems + 1, 0);
        for (int k = 0; k < nitems; ++k) ubase[k + 1] = ubase[k] + units[k];
        int k = 0;
        for (int b = 0; b < workers; ++b) {
            int64_t lo = (int64_t)b * total_units / workers, hi = (int64_t)(b + 1) * total_units / workers;
            while (lo < hi) {
                while (ubase[k + 1] <= lo) ++k;
                const int64_t e = std::min(hi, ubase[k + 1]);
                pieces.push_back(Piece{k, (int)(lo - ubase[k]), (int)(e - ubase[k]), 0});
                lo = e;
            }
            step_piece.push_back((int)pieces.size());
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
            if (units[k] == 0) continue;
            chunk_table(scheds[k].kind, units[k], workers, scheds[k].min_chunk, &st);
            for (size_t s = 0; s + 1 < st.size(); ++s) {
                if (st[s + 1] == st[s]) continue;
                pieces.push_back(Piece{k, (int)st[s], (int)st[s + 1], 0});
                step_piece.push_back((int)pieces.size());
            }
        }
    }
    const int nsteps = (int)step_piece.size() - 1;

    // ---- query sorting needs (items that are not "all points of the mesh")
    std::vector<SortItem> sitems;
    std::vector<int64_t> sqbase;
    std::vector<int> sort_of(nitems, -1);
    int64_t qtot = 0, htot = 0;
    for (int k = 0; k < nitems; ++k) {
        const si_batch_item &it = items[k];
        const Mesh *m = reinterpret_cast<const Mesh *>(it.mesh);
        if (it.m == 0) continue;
        if (!it.query_idx && it.m == m->n) continue;  // grid order is the query order
        const Grid *g = grids[k];
        SortItem s;
        s.pn = g->pn;
        s.sorted_pos = g->sorted_pos;
        s.query_idx = it.query_idx;
        s.n_points = (int)m->n;
        s.qbase = qtot;
        s.hbase = htot;
        for (int d = 0; d < 3; ++d) {
            s.origin[d] = g->origin[d];
            s.dims[d] = g->dims[d];
        }
        s.inv = g->inv_cell;
        sort_of[k] = (int)sitems.size();
        sitems.push_back(s);
        sqbase.push_back(qtot);
        qtot += it.m;
        htot += g->ncell;
    }
    if (htot + 1 > INT32_MAX || qtot > INT32_MAX) {
        set_error("query sort too large for one call");
        return SI_ERR_INVALID;
    }

    // ---- one scratch allocation for the call
    const size_t o_ctr = 0;
    const size_t o_items = align_up(o_ctr + sizeof(LaunchCounters), 256);
    const size_t o_pieces = align_up(o_items + sizeof(ItemDesc) * nitems, 256);
    const size_t o_steps = align_up(o_pieces + sizeof(Piece) * pieces.size(), 256);
    const size_t o_sitems = align_up(o_steps + sizeof(int) * step_piece.size(), 256);
    const size_t o_sqbase = align_up(o_sitems + sizeof(SortItem) * sitems.size(), 256);
    const size_t o_hist = align_up(o_sqbase + sizeof(int64_t) * sqbase.size(), 256);
    const size_t o_perm = align_up(o_hist + sizeof(int) * (htot + 1), 256);
    const size_t total_bytes = align_up(o_perm + sizeof(int) * qtot, 256);
    char *scratch = nullptr;
    si_status st = dev_alloc((void **)&scratch, total_bytes, stream);
    if (st != SI_OK) return st;
    LaunchCounters *ctr = reinterpret_cast<LaunchCounters *>(scratch + o_ctr);
    ItemDesc *d_items = reinterpret_cast<ItemDesc *>(scratch + o_items);
    int *d_perm = reinterpret_cast<int *>(scratch + o_perm);

    std::vector<ItemDesc> descs(nitems);
    for (int k = 0; k < nitems; ++k) {
        const si_batch_item &it = items[k];
        Mesh *m = reinterpret_cast<Mesh *>(it.mesh);
        ItemDesc &d = descs[k];
        std::memset(&d, 0, sizeof(d));
        d.m = it.m;
        d.n_points = (int)m->n;
        d.W = it.W;
        d.log2S = log2S[k];
        d.units = units[k];
        d.out = it.out;
        d.flags = m->flags;
        d.query_idx = it.query_idx;
        if (it.m == 0) continue;
        const Grid *g = grids[k];
        d.pn = g->pn;
        d.cell_start = g->cell_start;
        d.sorted_pos = g->sorted_pos;
        for (int a = 0; a < 3; ++a) {
            d.origin[a] = g->origin[a];
            d.dims[a] = g->dims[a];
        }
        d.cell = g->cell_len;
        d.inv_cell = g->inv_cell;
        if (sort_of[k] < 0) {
            d.perm = g->orig_idx;
            d.perm_is_grid = 1;
        } else {
            d.perm = d_perm + sitems[sort_of[k]].qbase;
            d.perm_is_grid = 0;
        }
        const float rc2 = si_candidate_rc2(it.W, it.bin_size);
        d.Rc2 = rc2;
        d.Rc = std::sqrt(rc2);
        d.cosS = it.cos_support_angle;
        d.invB = 1.0f / it.bin_size;
        d.halfW = 0.5f * (float)it.W;
        d.umax = (float)(it.W - 1);
        d.amax2 = support_alpha2(it.W, it.bin_size);
        double mag = 0.0;
        for (int a = 0; a < 3; ++a)
            mag = std::max(mag, std::max(std::fabs((double)m->bmin[a]), std::fabs((double)m->bmax[a])));
        d.margin = (float)(1e-5 * (mag + d.Rc + g->cell_len) + 1e-30);
        const si_probe *pr = probes.empty() ? nullptr : probes[k];
        if (pr) {
            d.p_culled = pr->culled;
            d.p_hash = pr->cand_hash;
            d.p_support = pr->support;
            d.p_worker = pr->worker;
            d.p_step = pr->step;
        }
        std::lock_guard<std::mutex> lk(m->mu);
        m->calls += 1;
        m->images += it.m;
    }

    cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(LaunchCounters), stream);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync(counters)");
    // one upload for descriptors, pieces, steps and sort items (contiguous region)
    std::vector<char> host(o_hist - o_items, 0);
    std::memcpy(host.data(), descs.data(), sizeof(ItemDesc) * nitems);
    std::memcpy(host.data() + (o_pieces - o_items), pieces.data(), sizeof(Piece) * pieces.size());
    std::memcpy(host.data() + (o_steps - o_items), step_piece.data(), sizeof(int) * step_piece.size());
    if (!sitems.empty()) {
        std::memcpy(host.data() + (o_sitems - o_items), sitems.data(), sizeof(SortItem) * sitems.size());
        std::memcpy(host.data() + (o_sqbase - o_items), sqbase.data(), sizeof(int64_t) * sqbase.size());
    }
    if (st == SI_OK) st = stage_upload(scratch + o_items, host.data(), host.size(), stream);
    if (st == SI_OK && qtot > 0) {
        int *hist = reinterpret_cast<int *>(scratch + o_hist);
        const SortItem *d_sitems = reinterpret_cast<const SortItem *>(scratch + o_sitems);
        const int64_t *d_sqbase = reinterpret_cast<const int64_t *>(scratch + o_sqbase);
        e = cudaMemsetAsync(hist, 0, sizeof(int) * (htot + 1), stream);
        if (e == cudaSuccess) {
            qsort_count_kernel<<<clamp_blocks(qtot), 256, 0, stream>>>(d_sitems, d_sqbase, (int)sitems.size(), qtot,
                                                                       hist);
            note_launches(1);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) st = scan_exclusive(hist, hist, htot + 1, stream);
        if (e == cudaSuccess && st == SI_OK) {
            qsort_scatter_kernel<<<clamp_blocks(qtot), 256, 0, stream>>>(d_sitems, d_sqbase, (int)sitems.size(),
                                                                         qtot, hist, d_perm);
            note_launches(1);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess && st == SI_OK) st = cuda_fail(e, "query sort");
    }
    if (st == SI_OK) {
        LaunchArgs a;
        a.items = d_items;
        a.pieces = reinterpret_cast<const Piece *>(scratch + o_pieces);
        a.step_piece = reinterpret_cast<const int *>(scratch + o_steps);
        a.nsteps = nsteps;
        a.is_static = all_static ? 1 : 0;
        a.ctr = ctr;
        a.nitems = nitems;
        a.img_words = (int)max_img_words;
        a.probe = 0;
        for (auto *p : probes)
            if (p) a.probe = 1;
        const int blocks = all_static ? nsteps : workers;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        const bool timed = timing_enabled();
        if (timed) {
            cudaEventCreate(&ev0);
            cudaEventCreate(&ev1);
            cudaEventRecord(ev0, stream);
        }
        launch_spin_kernel(a, blocks, smem, stream);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "spin kernel launch");
        if (timed) {
            cudaEventRecord(ev1, stream);
            Mesh *m0 = reinterpret_cast<Mesh *>(items[0].mesh);
            std::lock_guard<std::mutex> lk(m0->mu);
            m0->pending_events.emplace_back(ev0, ev1);
        }
    }
    dev_free(scratch, stream);
    return st;
}

}  // namespace si

using namespace si;

static si_schedule norm_sched(si_schedule s) { return s; }

extern "C" {

si_status si_generate_probe(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W, float bin_size,
                            float cos_support_angle, si_schedule schedule, int32_t *out, const si_probe *probe,
                            si_stream stream) {
    si_batch_item it{mesh, query_idx, m, W, bin_size, cos_support_angle, out};
    std::vector<si_batch_item> items{it};
    std::vector<si_schedule> sc{norm_sched(schedule)};
    std::vector<const si_probe *> pr;
    if (probe) pr.push_back(probe);
    return enqueue_batch(items, sc, pr, (cudaStream_t)stream, 0);
}

si_status si_generate(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W, float bin_size,
                      float cos_support_angle, si_schedule schedule, int32_t *out, si_stream stream) {
    return si_generate_probe(mesh, query_idx, m, W, bin_size, cos_support_angle, schedule, out, nullptr, stream);
}

si_status si_mesh_prepare(si_mesh_t mesh, int32_t W, float bin_size, const si_schedule *schedule,
                          si_stream stream) {
    if (!mesh || W < 2 || W > kMaxW || !(bin_size > 0.0f) || !std::isfinite(bin_size)) {
        set_error("si_mesh_prepare: bad arguments");
        return SI_ERR_INVALID;
    }
    Mesh *m = reinterpret_cast<Mesh *>(mesh);
    si_status st;
    Grid *g = mesh_grid(m, grid_cell_for(m, W, bin_size, schedule ? schedule->grid_div : 0), (cudaStream_t)stream,
                        &st);
    if (!g) return st;
    const int l2 = choose_log2_group(W, schedule ? schedule->group : 0);
    SI_CUDA(setup_spin_kernel_attributes(spin_smem_bytes(image_words(W, l2))));
    return SI_OK;
}

si_status si_generate_host(const float *points, const float *normals, int64_t n, const int32_t *query_idx,
                           int64_t m, int32_t W, float bin_size, float cos_support_angle, si_schedule schedule,
                           int32_t *out, si_stream stream) {
    if (!out && m > 0) {
        set_error("si_generate_host: NULL output");
        return SI_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    si_mesh_t mesh = nullptr;
    si_status st = si_mesh_create(points, normals, n, stream, &mesh);
    if (st != SI_OK) return st;
    int32_t *d_q = nullptr, *d_out = nullptr;
    const size_t out_bytes = sizeof(int32_t) * (size_t)m * W * W;
    do {
        if (query_idx && m > 0) {
            if ((st = dev_alloc((void **)&d_q, sizeof(int32_t) * m, s)) != SI_OK) break;
            cudaError_t e = cudaMemcpyAsync(d_q, query_idx, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "query upload");
                break;
            }
        }
        if ((st = dev_alloc((void **)&d_out, out_bytes, s)) != SI_OK) break;
        st = si_generate(mesh, d_q, m, W, bin_size, cos_support_angle, schedule, d_out, stream);
        if (st != SI_OK) break;
        if (m > 0) {
            cudaError_t e = cudaMemcpyAsync(out, d_out, out_bytes, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "image download");
                break;
            }
        }
    } while (0);
    if (d_q) dev_free(d_q, s);
    if (d_out) dev_free(d_out, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == SI_OK) st = cuda_fail(e, "cudaStreamSynchronize");
    si_stats stats;
    si_status st2 = si_get_stats(mesh, &stats);
    si_mesh_destroy(mesh);
    if (st == SI_OK && st2 != SI_OK) st = st2;
    return st;
}

si_status si_generate_batched(const si_batch_item *items, int32_t count, const si_schedule *override_or_null,
                              si_stream stream) {
    if (count < 0 || (count > 0 && !items)) {
        set_error("si_generate_batched: bad item array");
        return SI_ERR_INVALID;
    }
    if (count == 0) return SI_OK;
    std::vector<si_batch_item> v(items, items + count);
    std::vector<si_schedule> sc(count);
    for (int k = 0; k < count; ++k) {
        if (override_or_null) {
            sc[k] = *override_or_null;
        } else {
            const Mesh *m = items[k].mesh ? reinterpret_cast<const Mesh *>(items[k].mesh) : nullptr;
            si_schedule t{SI_SCHED_GSS, 1, 0, 0, 0};
            if (!m || si_tune_lookup(items[k].W, m->n, items[k].m, &t) != SI_OK) t = si_schedule{SI_SCHED_GSS, 1, 0, 0, 0};
            t.num_workers = 0;  // one launch: the worker count is the launch's
            sc[k] = t;
        }
    }
    std::vector<const si_probe *> pr;
    return enqueue_batch(v, sc, pr, (cudaStream_t)stream, override_or_null ? override_or_null->num_workers : 0);
}

si_status si_get_stats(si_mesh_t mesh, si_stats *out) {
    if (!mesh || !out) {
        set_error("si_get_stats: NULL argument");
        return SI_ERR_INVALID;
    }
    Mesh *m = reinterpret_cast<Mesh *>(mesh);
    SI_CUDA(cudaDeviceSynchronize());
    unsigned flags = 0;
    SI_CUDA(cudaMemcpy(&flags, m->flags, sizeof(unsigned), cudaMemcpyDeviceToHost));
    {
        std::lock_guard<std::mutex> lk(m->mu);
        for (auto &pe : m->pending_events) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pe.first, pe.second) == cudaSuccess) {
                m->timed_ms += ms;
                m->timed_launches += 1;
            }
            cudaEventDestroy(pe.first);
            cudaEventDestroy(pe.second);
        }
        m->pending_events.clear();
        out->calls = m->calls;
        out->images = m->images;
        out->grid_cells = m->last_cells;
        out->kernel_launches = m->timed_launches;
        out->kernel_ms = m->timed_ms;
    }
    out->overflow = (flags & kFlagOverflow) ? 1 : 0;
    out->timeout = (flags & kFlagTimeout) ? 1 : 0;
    out->bad_query = (flags & kFlagBadQuery) ? 1 : 0;
    if (out->overflow) {
        set_error("a pixel exceeded INT32_MAX");
        return SI_ERR_OVERFLOW;
    }
    if (out->timeout) {
        set_error("a bounded device wait gave up");
        return SI_ERR_TIMEOUT;
    }
    if (out->bad_query) {
        set_error("a query index was outside [0, n); its image was not written");
        return SI_ERR_INVALID;
    }
    return SI_OK;
}

si_status si_reset_stats(si_mesh_t mesh) {
    if (!mesh) {
        set_error("si_reset_stats: NULL mesh");
        return SI_ERR_INVALID;
    }
    Mesh *m = reinterpret_cast<Mesh *>(mesh);
    SI_CUDA(cudaDeviceSynchronize());
    SI_CUDA(cudaMemset(m->flags, 0, sizeof(unsigned)));
    std::lock_guard<std::mutex> lk(m->mu);
    for (auto &pe : m->pending_events) {
        cudaEventDestroy(pe.first);
        cudaEventDestroy(pe.second);
    }
    m->pending_events.clear();
    m->timed_launches = 0;
    m->timed_ms = 0.0;
    m->calls = 0;
    m->images = 0;
    return SI_OK;
}

}  // extern "C"
