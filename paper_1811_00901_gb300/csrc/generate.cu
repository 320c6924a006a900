// generate.cu -- the generation entry points: argument checks, single-mesh,
// host-buffer and batched calls, grid preparation and statistics.  The device
// work of every call is planned and recorded in batch.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace si {

namespace {
bool valid_group(int g) { return g == 0 || g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32; }

__global__ void iota_kernel(int32_t *q, int64_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        q[i] = (int32_t)i;
}

// One non-blocking stream per device for si_generate_host's image downloads.
cudaStream_t download_stream(int dev, cudaError_t *err) {
    static std::mutex mu;
    static cudaStream_t streams[128] = {};
    std::lock_guard<std::mutex> lk(mu);
    *err = cudaSuccess;
    if (dev < 0 || dev >= 128) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    if (!streams[dev]) *err = cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
    return streams[dev];
}

// si_generate_host splits calls of at least kPipeMinImages images into
// kPipeChunks query ranges: the download of one range's images overlaps the
// generation of the next.
#ifndef SI_PIPE_CHUNKS
#define SI_PIPE_CHUNKS 2
#endif
constexpr int64_t kPipeMinImages = 32768;
constexpr int kPipeChunks = SI_PIPE_CHUNKS;
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
    if (sc.kind < SI_SCHED_STATIC || sc.kind > SI_SCHED_AF || sc.min_chunk < 0 || sc.num_workers < 0 ||
        !valid_group(sc.group) || sc.grid_div < 0 || sc.grid_div > 16 || sc.slices < 0 || sc.slices > 64) {
        set_error("bad schedule (kind %d, min_chunk %d, workers %d, group %d, grid_div %d)", sc.kind, sc.min_chunk,
                  sc.num_workers, sc.group, sc.grid_div);
        return SI_ERR_INVALID;
    }
    if ((sc.binning != SI_BIN_BILINEAR && sc.binning != SI_BIN_NEAREST) || sc.slow_workers < 0 ||
        !(sc.slowdown == 0.0f || (sc.slowdown >= 1.0f && sc.slowdown <= 1000.0f)) ||
        !(sc.fac_cov >= 0.0f && sc.fac_cov <= 1e6f) || sc.order < 0 || sc.order > 1) {
        set_error("bad schedule (binning %d, slow_workers %d, slowdown %g, fac_cov %g, order %d)", sc.binning,
                  sc.slow_workers, (double)sc.slowdown, (double)sc.fac_cov, sc.order);
        return SI_ERR_INVALID;
    }
    const int l2 = choose_log2_group(it.W, sc.group);
    if (spin_smem_bytes(it.W, l2) > kMaxBlockSmem) {
        set_error("W = %d with group %d needs more shared memory than a block has", it.W, 1 << l2);
        return SI_ERR_INVALID;
    }
    return SI_OK;
}

}  // namespace si

using namespace si;

static si_schedule norm_sched(si_schedule s) { return s; }

extern "C" {

si_status si_generate_traced(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W, float bin_size,
                             float cos_support_angle, si_schedule schedule, int32_t *out, const si_trace *trace,
                             si_stream stream) {
    if (!trace || !trace->claims || !trace->count || trace->capacity < 0) {
        set_error("si_generate_traced: need claims, count and capacity >= 0");
        return SI_ERR_INVALID;
    }
    si_batch_item it{mesh, query_idx, m, W, bin_size, cos_support_angle, out};
    std::vector<si_batch_item> items{it};
    std::vector<si_schedule> sc{norm_sched(schedule)};
    return enqueue_batch(items, sc, {}, (cudaStream_t)stream, 0, trace);
}

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
    SI_CUDA(setup_spin_kernel_attributes(spin_smem_bytes(W, l2)));
    return SI_OK;
}

si_status si_default_workers(int32_t W, const si_schedule *schedule, int32_t *workers) {
    const int group = schedule ? schedule->group : 0;
    const int binning = schedule ? schedule->binning : SI_BIN_BILINEAR;
    if (!workers || W < 2 || W > kMaxW || !valid_group(group) ||
        (binning != SI_BIN_BILINEAR && binning != SI_BIN_NEAREST)) {
        set_error("si_default_workers: bad arguments");
        return SI_ERR_INVALID;
    }
    const int l2 = choose_log2_group(W, group);
    const size_t smem = spin_smem_bytes(W, l2);
    if (smem > kMaxBlockSmem) {
        set_error("W = %d with group %d needs more shared memory than a block has", W, 1 << l2);
        return SI_ERR_INVALID;
    }
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    const int modes = launch_modes_for(ring_mode(l2) | (binning == SI_BIN_NEAREST ? kModeNearest : 0), smem, false);
    SI_CUDA(setup_spin_kernel_attributes(smem));
    const int per_sm = blocks_per_sm_for(smem, modes);
    if (per_sm < 1) {
        set_error("spin kernel does not fit on an SM with %zu bytes of shared memory", smem);
        return SI_ERR_INVALID;
    }
    *workers = num_sms(dev) * per_sm;
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
    // the inputs are checked on the device; si_get_stats below reports a bad point
    si_status st = mesh_create(points, normals, n, stream, &mesh, false);
    if (st != SI_OK) return st;
    int32_t *d_q = nullptr, *d_out = nullptr;
    const size_t img_words = (size_t)W * W;
    const size_t out_bytes = sizeof(int32_t) * (size_t)m * img_words;
    // A large call whose output is page-locked host memory mapped into the
    // device's address space is written there by the kernel itself, over the
    // host link, while it runs (no download afterwards); whole groups only, so
    // no atomics go to host memory.
    int32_t *direct = nullptr;
    if (m >= kPipeMinImages) {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
            direct = static_cast<int32_t *>(pa.devicePointer);
        cudaGetLastError();  // clear a failed attribute query
    }
    const int chunks = direct ? 1 : (m >= kPipeMinImages ? kPipeChunks : 1);
    cudaEvent_t ev[kPipeChunks + 1] = {};
    do {
        if (direct) {
            if (query_idx) {
                if ((st = dev_alloc((void **)&d_q, sizeof(int32_t) * m, s)) != SI_OK) break;
                cudaError_t e = cudaMemcpyAsync(d_q, query_idx, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s);
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "query upload");
                    break;
                }
            }
            si_schedule whole = schedule;
            whole.slices = 1;
            st = si_generate(mesh, d_q, m, W, bin_size, cos_support_angle, whole, direct, stream);
            break;
        }
        if (query_idx && m > 0) {
            if ((st = dev_alloc((void **)&d_q, sizeof(int32_t) * m, s)) != SI_OK) break;
            cudaError_t e = cudaMemcpyAsync(d_q, query_idx, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "query upload");
                break;
            }
        } else if (chunks > 1) {
            // query ranges of the all-points call as explicit index lists
            if ((st = dev_alloc((void **)&d_q, sizeof(int32_t) * m, s)) != SI_OK) break;
            iota_kernel<<<256, 256, 0, s>>>(d_q, m);
            note_launches(1);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) {
                st = cuda_fail(e, "iota_kernel");
                break;
            }
        }
        if ((st = dev_alloc((void **)&d_out, out_bytes, s)) != SI_OK) break;
        if (chunks == 1) {
            st = si_generate(mesh, d_q, m, W, bin_size, cos_support_angle, schedule, d_out, stream);
            if (st != SI_OK) break;
            if (m > 0) {
                cudaError_t e = cudaMemcpyAsync(out, d_out, out_bytes, cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "image download");
                    break;
                }
            }
            break;
        }
        // generate range k on `s` while the download stream copies range k-1 out
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        cudaStream_t cs = e == cudaSuccess ? download_stream(dev, &e) : nullptr;
        for (int k = 0; k <= chunks && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "download stream / events");
            break;
        }
        for (int k = 0; k < chunks && st == SI_OK; ++k) {
            const int64_t a = m * k / chunks, b = m * (k + 1) / chunks;
            st = si_generate(mesh, d_q + a, b - a, W, bin_size, cos_support_angle, schedule, d_out + a * img_words,
                             stream);
            if (st != SI_OK) break;
            e = cudaEventRecord(ev[k], s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[k], 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(out + a * img_words, d_out + a * img_words,
                                    sizeof(int32_t) * (size_t)(b - a) * img_words, cudaMemcpyDeviceToHost, cs);
            if (e != cudaSuccess) st = cuda_fail(e, "image download");
        }
        // the output buffer is released on `s`, after the last download
        e = cudaEventRecord(ev[chunks], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[chunks], 0);
        if (e != cudaSuccess && st == SI_OK) st = cuda_fail(e, "download completion");
    } while (0);
    if (d_q) dev_free(d_q, s);
    if (d_out) dev_free(d_out, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == SI_OK) st = cuda_fail(e, "cudaStreamSynchronize");
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
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
    return enqueue_batch_graph(v, sc, (cudaStream_t)stream, override_or_null ? override_or_null->num_workers : 0);
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
    int cells = 0;  // the most recently built grid's cells (its geometry lives on the device)
    {
        std::lock_guard<std::mutex> lk(m->mu);
        if (!m->grids.empty())
            SI_CUDA(cudaMemcpy(&cells, &m->grids.back()->geom->ncell, sizeof(int), cudaMemcpyDeviceToHost));
    }
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
        out->grid_cells = cells;
        out->kernel_launches = m->timed_launches;
        out->kernel_ms = m->timed_ms;
    }
    out->overflow = (flags & kFlagOverflow) ? 1 : 0;
    out->timeout = (flags & kFlagTimeout) ? 1 : 0;
    out->bad_query = (flags & kFlagBadQuery) ? 1 : 0;
    out->bad_input = (flags & kFlagBadInput) ? 1 : 0;
    if (out->overflow) {
        set_error("a pixel exceeded INT32_MAX");
        return SI_ERR_OVERFLOW;
    }
    if (out->timeout) {
        set_error("a bounded device wait gave up");
        return SI_ERR_TIMEOUT;
    }
    if (flags & kFlagBounds) {
        set_error("an index check of the bounds-checking build failed (the access was skipped)");
        return SI_ERR_CUDA;
    }
    if (flags & kFlagLaunch) {
        set_error("internal error: a spin-kernel launch had less shared memory than its layout");
        return SI_ERR_CUDA;
    }
    if (out->bad_input) {
        set_error("a point of the mesh had a non-finite coordinate or a zero normal (its images are unspecified)");
        return SI_ERR_INVALID;
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
