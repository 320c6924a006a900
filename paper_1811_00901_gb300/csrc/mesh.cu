// mesh.cu -- oriented-point sets resident in HBM and their uniform grids.
//
// si_mesh_create replicates the input once on the device (the "input data is
// replicated" design of Sec. 3): positions and FP32-normalised normals as
// float4.  Grids are built lazily per cell size and cached on the mesh: a
// counting sort of the points by cell (cell ids -> histogram -> exclusive
// scan -> scatter), giving cell_start[] and the points in cell order.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_common.cuh"
#include "internal.h"
#include "scan.h"

namespace si {

namespace {

__global__ void mesh_ingest_kernel(const float *__restrict__ pts, const float *__restrict__ nrm, int64_t n,
                                   float4 *__restrict__ pos, float4 *__restrict__ nrm_out,
                                   unsigned *__restrict__ keys /* [6]: min xyz, max xyz */,
                                   unsigned *__restrict__ flags) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    unsigned my_bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        float a = nrm[3 * i], b = nrm[3 * i + 1], c = nrm[3 * i + 2];
        // unit normal in IEEE FP32, each rounding spelled out (the nearest-bin
        // count's pixel indices depend on these exact values)
        float l2 = __fmaf_rn(c, c, __fmaf_rn(b, b, __fmul_rn(a, a)));
        bool ok = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(l2) && l2 > 0.0f;
        if (!ok) {
            my_bad = 1;
            l2 = 1.0f;
            x = isfinite(x) ? x : 0.0f;  // keep the bounding box finite
            y = isfinite(y) ? y : 0.0f;
            z = isfinite(z) ? z : 0.0f;
        }
        float inv = __fdiv_rn(1.0f, __fsqrt_rn(l2));
        pos[i] = make_float4(x, y, z, 0.0f);
        nrm_out[i] = make_float4(__fmul_rn(a, inv), __fmul_rn(b, inv), __fmul_rn(c, inv), 0.0f);
        lo[0] = fminf(lo[0], x);
        lo[1] = fminf(lo[1], y);
        lo[2] = fminf(lo[2], z);
        hi[0] = fmaxf(hi[0], x);
        hi[1] = fmaxf(hi[1], y);
        hi[2] = fmaxf(hi[2], z);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], d));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], d));
        }
    }
    my_bad = __any_sync(0xffffffffu, my_bad);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (lo[k] <= hi[k]) {
                atomicMin(&keys[k], float_key(lo[k]));
                atomicMax(&keys[3 + k], float_key(hi[k]));
            }
        }
        if (my_bad) atomicOr(flags, kFlagBadInput);
    }
}

// Decodes an order-preserving key (float_key) back to the float.
__device__ __forceinline__ float key_float(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// The grid's geometry from the mesh's bounding box: cells of edge `cell`
// (coarsened by 1.25x until at most `cap` cells cover the box), origin at the
// box's minimum corner.  One thread.
__global__ void grid_geom_kernel(const unsigned *__restrict__ keys, float cell, int64_t cap, GridGeom *g) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double lo[3], hi[3];
    const bool empty = keys[0] == 0xffffffffu;  // no point reached the box (cannot happen for n >= 1)
    for (int k = 0; k < 3; ++k) {
        lo[k] = empty ? 0.0 : (double)key_float(keys[k]);
        hi[k] = empty ? 0.0 : (double)key_float(keys[3 + k]);
    }
    double cellv = cell;
    int dims[3] = {1, 1, 1};
    int64_t ncell = 1;
    for (int guard = 0; guard < 64; ++guard) {
        ncell = 1;
        for (int k = 0; k < 3; ++k) {
            double d = ceil((hi[k] - lo[k]) / cellv);
            if (d < 1) d = 1;
            if (d > (1 << 20)) d = 1 << 20;
            dims[k] = (int)d;
            ncell *= dims[k];
        }
        if (ncell <= cap) break;
        cellv *= 1.25;
    }
    if (ncell > cap) {  // unreachable for finite boxes; one cell keeps every index in range
        dims[0] = dims[1] = dims[2] = 1;
        ncell = 1;
    }
    double mag = 0.0;
    for (int k = 0; k < 3; ++k) {
        g->origin[k] = (float)lo[k];
        g->dims[k] = dims[k];
        mag = fmax(mag, fmax(fabs(lo[k]), fabs(hi[k])));
    }
    g->cell_len = (float)cellv;
    g->inv_cell = (float)(1.0 / cellv);
    g->mag = (float)mag;
    g->ncell = (int)ncell;
}

__device__ __forceinline__ int cell_of(const GridGeom &g, float4 p) {
    int cx = cell_coord(p.x, g.origin[0], g.inv_cell, g.dims[0]);
    int cy = cell_coord(p.y, g.origin[1], g.inv_cell, g.dims[1]);
    int cz = cell_coord(p.z, g.origin[2], g.inv_cell, g.dims[2]);
    return (cz * g.dims[1] + cy) * g.dims[0] + cx;
}

__global__ void grid_count_kernel(const float4 *__restrict__ pos, int64_t n, const GridGeom *__restrict__ gp,
                                  int *__restrict__ hist) {
    const GridGeom g = *gp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        atomicAdd(&hist[cell_of(g, pos[i])], 1);
    }
}

// Scatter into cell order.  Lanes of a warp that share a cell take
// consecutive slots (warp-aggregated atomics); the order of warps within a
// cell is whatever the atomics give.  Every result of the library is
// independent of that order (integer accumulation).
__global__ void grid_scatter_kernel(const float4 *__restrict__ pos, const float4 *__restrict__ nrm, int64_t n,
                                    const GridGeom *__restrict__ gp, int *__restrict__ cursor, float4 *__restrict__ pn,
                                    int *__restrict__ sorted_pos, int *__restrict__ orig_idx) {
    const GridGeom g = *gp;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; base < n;
         base += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = base + lane;
        bool live = i < n;
        float4 p = live ? pos[i] : make_float4(0, 0, 0, 0);
        int c = live ? cell_of(g, p) : -1;
        unsigned peers = __match_any_sync(0xffffffffu, c);
        int leader = __ffs(peers) - 1;
        int rank = __popc(peers & ((1u << lane) - 1u));
        int slot0 = 0;
        if (live && lane == leader) slot0 = atomicAdd(&cursor[c], __popc(peers));
        slot0 = __shfl_sync(0xffffffffu, slot0, leader);
        if (live) {
            int s = slot0 + rank;
            pn[2 * (int64_t)s] = make_float4(p.x, p.y, p.z, __int_as_float((int)i));
            pn[2 * (int64_t)s + 1] = nrm[i];
            sorted_pos[i] = s;
            orig_idx[s] = (int)i;
        }
    }
}

int grid_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

// Grids and meshes live in the device's stream-ordered pool (its release
// threshold keeps freed blocks for reuse, so a new mesh of the same size
// allocates in microseconds); callers free them with no work pending.
void free_grid(Grid *g, cudaStream_t stream) {
    if (!g) return;
    dev_free(g->geom, stream);
    dev_free(g->cell_start, stream);
    dev_free(g->pn, stream);
    dev_free(g->sorted_pos, stream);
    dev_free(g->orig_idx, stream);
    if (g->ready) cudaEventDestroy(g->ready);
    delete g;
}

bool is_device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// Cell edge for a call: the candidate radius divided by grid_div, rounded down
// to a quarter octave so that calls with nearby (W, B) share one grid.
// A contributing pair has |beta| <= h and alpha < (W-1) B (bilinear: all four
// corners inside), or |beta| < (W/2 + 1) B and alpha <= (W-1) B (nearest bin:
// -1 < u <= W-1); the 1e-5 inflation keeps FP32 rounding of |X-P|^2 from
// dropping such a pair.
float candidate_rc2(int W, float bin_size, int binning) {
    const double B = (double)bin_size;
    const double h = binning == SI_BIN_NEAREST ? ((double)W / 2.0 + 1.0) * B : (double)W * B / 2.0;
    const double r = (double)(W - 1) * B;
    return (float)((h * h + r * r) * (1.0 + 1e-5));
}

// At most 8 cells per point (and 2^24): a grid whose requested cells would
// outnumber that is coarsened; the bound sizes the cell array before the
// geometry is known on the host.
int64_t grid_cell_cap(int64_t n) { return std::min<int64_t>(int64_t(1) << 24, 8 * n + 4096); }

float grid_cell_for(const Mesh *m, int W, float bin, int grid_div) {
    (void)m;
    double R = std::sqrt((double)si_candidate_rc2(W, bin));
    int div = grid_div > 0 ? grid_div : (W >= 64 ? 6 : 8);  // measured defaults: wide images prefer coarser cells
    double c = R / div;
    double e = std::floor(std::log2(c) * 4.0) / 4.0;
    return (float)std::exp2(e);
}

// Drops the mesh's grids; the next call that needs one builds it again.  The
// cached batch graphs that hold the grids' pointers go first, then the device
// finishes its work, as in si_mesh_destroy.
void mesh_drop_grids(Mesh *m) {
    forget_mesh_graphs(m);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaDeviceSynchronize();
    for (Grid *g : m->grids) free_grid(g, nullptr);
    m->grids.clear();
}

Grid *mesh_grid(Mesh *m, float cell, cudaStream_t stream, si_status *st) {
    *st = SI_OK;
    std::lock_guard<std::mutex> lk(m->mu);
    for (Grid *g : m->grids)
        if (g->cell == cell) {
            cudaError_t e = cudaStreamWaitEvent(stream, g->ready, 0);
            if (e != cudaSuccess) {
                *st = cuda_fail(e, "cudaStreamWaitEvent(grid)");
                return nullptr;
            }
            return g;
        }
    // build a new grid: its geometry comes from the bounding box on the device
    const int64_t cap = grid_cell_cap(m->n);
    Grid *g = new Grid();
    g->cell = cell;
    g->ncell_cap = cap;
    cudaError_t e = cudaSuccess;
    *st = dev_alloc((void **)&g->geom, sizeof(GridGeom), stream);
    if (*st == SI_OK) *st = dev_alloc((void **)&g->cell_start, sizeof(int) * (cap + 1), stream);
    if (*st == SI_OK) *st = dev_alloc((void **)&g->pn, sizeof(float4) * 2 * m->n, stream);
    if (*st == SI_OK) *st = dev_alloc((void **)&g->sorted_pos, sizeof(int) * m->n, stream);
    if (*st == SI_OK) *st = dev_alloc((void **)&g->orig_idx, sizeof(int) * m->n, stream);
    if (*st == SI_OK) {
        e = cudaEventCreateWithFlags(&g->ready, cudaEventDisableTiming);
        if (e != cudaSuccess) *st = cuda_fail(e, "grid event");
    }
    if (*st != SI_OK) {
        free_grid(g, stream);
        return nullptr;
    }
    int *cursor = nullptr;
    do {
        e = cudaStreamWaitEvent(stream, m->ready, 0);
        if (e != cudaSuccess) break;
        grid_geom_kernel<<<1, 32, 0, stream>>>(m->bbox_keys, cell, cap, g->geom);
        note_launches(1);
        e = cudaMemsetAsync(g->cell_start, 0, sizeof(int) * (cap + 1), stream);
        if (e != cudaSuccess) break;
        grid_count_kernel<<<grid_blocks(m->n), 256, 0, stream>>>(m->pos, m->n, g->geom, g->cell_start);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        *st = scan_exclusive(g->cell_start, g->cell_start, cap + 1, stream);
        if (*st != SI_OK) break;
        *st = dev_alloc((void **)&cursor, sizeof(int) * cap, stream);
        if (*st != SI_OK) break;
        e = cudaMemcpyAsync(cursor, g->cell_start, sizeof(int) * cap, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) break;
        grid_scatter_kernel<<<grid_blocks(m->n), 256, 0, stream>>>(m->pos, m->nrm, m->n, g->geom, cursor, g->pn,
                                                                  g->sorted_pos, g->orig_idx);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        e = cudaEventRecord(g->ready, stream);
    } while (0);
    if (cursor) dev_free(cursor, stream);
    if (e != cudaSuccess && *st == SI_OK) *st = cuda_fail(e, "grid build");
    if (*st != SI_OK) {
        cudaStreamSynchronize(stream);
        free_grid(g, stream);
        return nullptr;
    }
    m->grids.push_back(g);
    return g;
}

}  // namespace si

using namespace si;

namespace si {
// si_mesh_create; with check_host false, host inputs are checked on the device
// like device inputs (for callers that read si_get_stats before returning).
si_status mesh_create(const float *points, const float *normals, int64_t n, si_stream stream,
                      si_mesh_t *out_mesh, bool check_host) {
    if (!out_mesh) {
        set_error("si_mesh_create: out_mesh is NULL");
        return SI_ERR_INVALID;
    }
    *out_mesh = nullptr;
    if (!points || !normals || n < 1 || n > (int64_t(1) << 30)) {
        set_error("si_mesh_create: need non-NULL points/normals and 1 <= n <= 2^30 (n = %lld)", (long long)n);
        return SI_ERR_INVALID;
    }
    const bool dev_p = is_device_pointer(points), dev_n = is_device_pointer(normals);
    // host inputs are checked here, synchronously; device inputs by the ingest
    // kernel, which flags the mesh (si_get_stats reports it)
    for (int64_t i = 0; check_host && !dev_p && i < 3 * n; ++i)
        if (!std::isfinite(points[i])) {
            set_error("si_mesh_create: coordinate %lld is not finite", (long long)i);
            return SI_ERR_INVALID;
        }
    for (int64_t i = 0; check_host && !dev_n && i < n; ++i) {
        const float a = normals[3 * i], b = normals[3 * i + 1], c = normals[3 * i + 2];
        const float l2 = std::fma(c, c, std::fma(b, b, a * a));
        if (!std::isfinite(l2) || !(l2 > 0.0f)) {
            set_error("si_mesh_create: normal %lld is zero or not finite", (long long)i);
            return SI_ERR_INVALID;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    Mesh *m = new Mesh();
    SI_CUDA(cudaGetDevice(&m->device));
    m->n = n;
    const float *dp = points, *dn = normals;
    float *tmp_p = nullptr, *tmp_n = nullptr;
    si_status st = SI_OK;
    cudaError_t e = cudaSuccess;
    do {
        if ((st = dev_alloc((void **)&m->pos, sizeof(float4) * n, s)) != SI_OK) break;
        if ((st = dev_alloc((void **)&m->nrm, sizeof(float4) * n, s)) != SI_OK) break;
        if ((st = dev_alloc((void **)&m->flags, sizeof(unsigned), s)) != SI_OK) break;
        if ((st = dev_alloc((void **)&m->bbox_keys, sizeof(unsigned) * 8, s)) != SI_OK) break;
        e = cudaEventCreateWithFlags(&m->ready, cudaEventDisableTiming);
        if (e != cudaSuccess) break;
        e = cudaMemsetAsync(m->flags, 0, sizeof(unsigned), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->bbox_keys, 0xff, sizeof(unsigned) * 3, s);  // min keys
        if (e == cudaSuccess) e = cudaMemsetAsync(m->bbox_keys + 3, 0, sizeof(unsigned) * 5, s);  // max keys
        if (e != cudaSuccess) break;
        if (!dev_p) {
            if ((st = dev_alloc((void **)&tmp_p, sizeof(float) * 3 * n, s)) != SI_OK) break;
            e = cudaMemcpyAsync(tmp_p, points, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) break;
            dp = tmp_p;
        }
        if (!dev_n) {
            if ((st = dev_alloc((void **)&tmp_n, sizeof(float) * 3 * n, s)) != SI_OK) break;
            e = cudaMemcpyAsync(tmp_n, normals, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) break;
            dn = tmp_n;
        }
        mesh_ingest_kernel<<<grid_blocks(n), 256, 0, s>>>(dp, dn, n, m->pos, m->nrm, m->bbox_keys, m->flags);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        e = cudaEventRecord(m->ready, s);
    } while (0);
    if (tmp_p) dev_free(tmp_p, s);
    if (tmp_n) dev_free(tmp_n, s);
    if (e != cudaSuccess && st == SI_OK) st = cuda_fail(e, "si_mesh_create");
    if (st != SI_OK) {
        cudaStreamSynchronize(s);
        dev_free(m->pos, s);
        dev_free(m->nrm, s);
        dev_free(m->flags, s);
        dev_free(m->bbox_keys, s);
        if (m->ready) cudaEventDestroy(m->ready);
        cudaStreamSynchronize(s);
        delete m;
        return st;
    }
    *out_mesh = reinterpret_cast<si_mesh_t>(m);
    return SI_OK;
}
}  // namespace si

extern "C" {

si_status si_mesh_create(const float *points, const float *normals, int64_t n, si_stream stream,
                         si_mesh_t *out_mesh) {
    return si::mesh_create(points, normals, n, stream, out_mesh, true);
}

si_status si_mesh_destroy(si_mesh_t mesh) {
    if (!mesh) {
        set_error("si_mesh_destroy: NULL mesh");
        return SI_ERR_INVALID;
    }
    Mesh *m = reinterpret_cast<Mesh *>(mesh);
    forget_mesh_graphs(m);  // cached batch graphs hold this mesh's grid pointers
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    for (Grid *g : m->grids) free_grid(g, nullptr);
    for (auto &pe : m->pending_events) {
        cudaEventDestroy(pe.first);
        cudaEventDestroy(pe.second);
    }
    dev_free(m->pos, nullptr);
    dev_free(m->nrm, nullptr);
    dev_free(m->flags, nullptr);
    dev_free(m->bbox_keys, nullptr);
    cudaStreamSynchronize(nullptr);
    if (m->ready) cudaEventDestroy(m->ready);
    delete m;
    cudaSetDevice(prev);
    return SI_OK;
}

float si_candidate_rc2(int32_t W, float bin_size) { return si::candidate_rc2(W, bin_size, SI_BIN_BILINEAR); }

float si_candidate_rc2_binned(int32_t W, float bin_size, int32_t binning) {
    return si::candidate_rc2(W, bin_size, binning);
}

}  // extern "C"
