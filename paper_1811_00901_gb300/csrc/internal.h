// internal.h -- shared declarations of the spin-image library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/spin.h"

namespace si {

// ----------------------------------------------------------------- errors --
void set_error(const char *fmt, ...);
si_status cuda_fail(cudaError_t e, const char *what);

#define SI_CUDA(call)                                              \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::si::cuda_fail(_e, #call);  \
    } while (0)

// ------------------------------------------------------------- constants --
// Build-time shape of the spin kernel (defaults measured best on GB300):
// 12-warp blocks, two per SM, up to 113 KB of shared memory each.
#ifndef SI_THREADS
#define SI_THREADS 384
#endif
#ifndef SI_MIN_BLOCKS
#define SI_MIN_BLOCKS 2
#endif
#ifndef SI_SMEM_BUDGET_KB
#define SI_SMEM_BUDGET_KB 113
#endif
constexpr int kThreads = SI_THREADS;  // threads per spin-kernel block
#ifndef SI_TILE_MAX
#define SI_TILE_MAX 576
#endif
#ifndef SI_TILE_MIN
#define SI_TILE_MIN 448
#endif
#ifndef SI_STAGES
#define SI_STAGES 2
#endif
// Candidate points per staged tile (32 B each): the larger the tile, the fewer
// block barriers or stage hand-offs per candidate.  Each group shape takes the
// largest tile in [kTileMin, kTileMax] that keeps its blocks-per-SM target
// (tile_for_shape in spin_kernel.cu).
constexpr int kTileMax = SI_TILE_MAX;
constexpr int kTileMin = SI_TILE_MIN;
constexpr int kStages = SI_STAGES;  // tile ring depth
constexpr int kMaxRows = 512;       // stencil rows held in shared memory at once
constexpr int kMaxW = 128;
constexpr size_t kMaxBlockSmem = (size_t)227 * 1024;  // dynamic shared memory one block may opt into
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // bounded device waits: 2 s
constexpr uint64_t kSlowIdleCapNs = 1000000000ull;  // heterogeneity emulation: idle at most 1 s per step

// Device flags (per mesh).
constexpr unsigned kFlagOverflow = 1u;
constexpr unsigned kFlagTimeout = 2u;
constexpr unsigned kFlagBadQuery = 4u;  // a query index outside [0, n): its image is left unwritten
constexpr unsigned kFlagLaunch = 8u;    // the kernel's shared-memory layout did not fit its launch: no work done
constexpr unsigned kFlagBadInput = 16u; // a device input point had a non-finite coordinate or a zero normal
constexpr unsigned kFlagBounds = 32u;   // SI_DEBUG_BOUNDS builds: an index check failed (the access was skipped)

// ------------------------------------------------------------------- grid --
// Geometry of a uniform grid over the mesh's bounding box, computed on the
// device (grid_geom_kernel) from the bounding box the mesh's ingest kernel
// left there, so that building and using a grid needs no host round trip.
struct GridGeom {
    float origin[3];  // the bounding box's minimum corner
    float cell_len;   // cell edge (>= the requested edge when the grid was coarsened)
    float inv_cell;   // 1 / cell_len
    float mag;        // largest |coordinate| of the bounding box (stencil margin)
    int dims[3];
    int ncell;        // dims[0] dims[1] dims[2] <= the grid's ncell_cap
};

// A uniform grid over the mesh's bounding box; points counting-sorted by cell.
struct Grid {
    float cell = 0.f;           // cache key: the requested edge
    int64_t ncell_cap = 0;      // cells the arrays are sized for (the device geometry stays within it)
    GridGeom *geom = nullptr;   // device
    int *cell_start = nullptr;  // [ncell_cap + 1]
    float4 *pn = nullptr;       // [2n]: (x, y, z, orig index bits), (nx, ny, nz, 0)
    int *sorted_pos = nullptr;  // [n]: original index -> sorted position
    int *orig_idx = nullptr;    // [n]: sorted position -> original index
    cudaEvent_t ready = nullptr;
};

struct Mesh {
    int device = 0;
    int64_t n = 0;
    float4 *pos = nullptr;  // original order, w = 0
    float4 *nrm = nullptr;  // original order, normalised
    unsigned *bbox_keys = nullptr;  // device [8]: order-preserving keys of min xyz, max xyz
    std::vector<Grid *> grids;
    unsigned *flags = nullptr;  // device word: kFlag*
    cudaEvent_t ready = nullptr;
    std::mutex mu;
    int64_t calls = 0, images = 0;
    // timing
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending_events;
    int64_t timed_launches = 0;
    double timed_ms = 0.0;
};

// ---------------------------------------------------------- device items --
// Everything the persistent kernel needs to know about one item (one mesh
// with its own parameters).  Lives in device memory.
struct ItemDesc {
    const float4 *pn;
    const int *cell_start;
    const int *sorted_pos;
    const int *query_idx;  // [m] or null (0..m-1)
    const int *perm;       // [m] grid-ordered query t -> query slot q; null: identity order
    int32_t *out;          // [m][W][W]
    unsigned *flags;
    const GridGeom *geom;  // the grid's geometry (device)
    int64_t m;
    int n_points;          // mesh size (query indices are checked against it)
    int W;
    int log2S;             // group = 1 << log2S images
    float invB, halfW, umax, Rc2, Rc, cosS;
    int units;             // ceil(m / group)
    int perm_is_grid;      // perm holds grid orig_idx (all-points query of the mesh)
    // probes (device, may be null)
    int64_t *p_culled;
    uint32_t *p_hash;
    int64_t *p_support;
    int32_t *p_worker;
    int32_t *p_step;
    int64_t *p_examined;
    int64_t *p_angle;
    // candidate slices per group (>= 1); with more than one, slices add
    // partial images into a zeroed `out` and per-image pair counts into `counts`
    int slices;
    int *counts;  // [m], zeroed, when slices > 1
    int binning;  // si_binning: SI_BIN_NEAREST counts 1 per pair at (ceil(u), ceil(v))
    float B;      // bin size (the nearest-bin count divides by it)
    const int *gorder;  // [groups] loop position -> group (decreasing estimated cost), or null: grid order
};

// Cost order of the groups (si_schedule.order = 1): for the `n_ord` items
// ord_items[0..n_ord) of a launch, whose groups occupy [gbase[j], gbase[j+1])
// of a concatenated group space, estimate each group's cost (the candidates
// of its stencil), bucket it by log cost and write each item's groups in
// decreasing bucket order to gorder[gbase[j] ..].  Item j's deal batches,
// deal[3b .. 3b+2] = (first position, chunks nc, chunk size c) for b in
// [dbase[j], dbase[j+1]), spread the positions of such a run of equal chunks
// round-robin: sorted rank start + i goes to chunk i mod nc, slot i div nc.
// Scratch: key[gbase[n_ord]] and hist[n_ord * kCostBuckets].  Four
// stream-ordered operations (a memset and three kernels); returns the
// kernels launched in *kernels.
constexpr int kCostBuckets = 1024;
si_status enqueue_group_order(const ItemDesc *items, const int *ord_items, const int *gbase, const int *dbase,
                              const int *deal, int n_ord, int total_groups, uint16_t *key, int *hist, int *gorder,
                              cudaStream_t st, int *kernels);

// A piece of the scheduled loop: units [u0, u1) of item `item`.
struct Piece {
    int item, u0, u1, pad;
};

// Launch-wide scratch counters, reset by the last block of each launch.
struct LaunchCounters {
    unsigned long long step;         // next dynamic step to hand out
    unsigned long long done_blocks;  // blocks finished
    unsigned long long awf_next;     // AWF: next unit of the call's concatenated unit space
    unsigned long long awf_claims;   // AWF: chunks handed out
    double awf_rate_sum;             // AWF: sum of the measured worker rates (units per ns)
    unsigned awf_rated;              // AWF and AF: workers with a measurement
    unsigned pad;
    double af_d_sum;                 // AF: sum over measured workers of sigma^2 / mu (ns)
    double af_e_sum;                 // AF: sum over measured workers of 1 / mu (units per ns)
};

// Adaptive factoring: one worker's statistics of its per-unit times (ns), kept
// in global memory by the worker's thread 0.  A unit's time is scaled by its
// chunk's wall time over the chunk's summed unit times, so the claim overhead
// and a slow worker's idle are spread over the units.
struct AfWorker {
    double sum, sumsq;  // scaled unit times of the finished chunks
    double cs, cs2;     // unit times of the current chunk
    double d, e;        // the worker's published sigma^2 / mu and 1 / mu (e = 0: none yet)
    int n, cn;          // units in sum; units timed in the current chunk
};

struct LaunchArgs {
    const ItemDesc *items;
    const Piece *pieces;
    const int *step_piece;  // [nsteps + 1]: pieces of step s are step_piece[s] .. step_piece[s+1]
    int nsteps;
    int is_static;          // 1: block b runs step b (no claims)
    LaunchCounters *ctr;
    int nitems;
    int img_words;          // shared words reserved for images (max over items)
    int probe;
    int slow_workers = 0;   // heterogeneity emulation: blocks 0..slow_workers-1 are slow and request first
    float slowdown = 1.0f;  // a slow block idles (slowdown - 1) x each step's time
    int modes = 0;          // tile-ring disciplines present (kModeBarrier | kModeProducer); 0 = both
    // adaptive rules (chunk sizes decided on the device): awf = 1 for AWF and
    // AF, af = 1 for AF, whose per-worker statistics live in af_workers[gridDim.x]
    int awf = 0;
    int af = 0;
    AfWorker *af_workers = nullptr;
    int total_units = 0;             // units of all items
    const int *unit_base = nullptr;  // [nitems + 1]: first unit of each item in the concatenation
    int min_chunk = 1;
    // claim trace (si_generate_traced): [trace_cap][4] worker, step, start, end
    int64_t *trace = nullptr;
    int64_t trace_cap = 0;
    unsigned long long *trace_count = nullptr;
};

// Tile-ring discipline of a group shape: groups of <= 4 images run a producer
// warp, larger groups a block barrier per tile.
constexpr int kModeBarrier = 1, kModeProducer = 2;
constexpr int kModeNearest = 4;  // some group uses the nearest-bin count (runtime-shape path)
constexpr int kModeWide = 8;     // the launch's shared memory allows fewer blocks per SM than SI_MIN_BLOCKS
inline int ring_mode(int log2S) { return log2S <= 2 ? kModeProducer : kModeBarrier; }
// Disciplines compiled into the kernel instance that runs a launch whose
// groups use `modes`: one discipline alone gets its own instance; mixed
// launches and probe launches run the instance with both.
// A mixed launch whose shared memory leaves room for two blocks per SM only
// (kModeWide) runs a mixed instance built for two blocks, with their registers.
inline int launch_modes(int modes, bool probe) {
    if (probe || (modes & kModeNearest)) return kModeBarrier | kModeProducer | kModeNearest;
    const int rings = modes & (kModeBarrier | kModeProducer);
    if (rings == kModeBarrier || rings == kModeProducer) return rings;
    return (kModeBarrier | kModeProducer) | (modes & kModeWide);
}
// The same from the groups' own modes (ring_mode, kModeNearest) and the
// launch's dynamic shared memory.
inline int launch_modes_for(int modes, size_t smem_bytes, bool probe) {
    if (smem_bytes > (size_t)SI_SMEM_BUDGET_KB * 1024) modes |= kModeWide;
    return launch_modes(modes, probe);
}

// ---------------------------------------------------------- host helpers --
si_status mesh_create(const float *points, const float *normals, int64_t n, si_stream stream, si_mesh_t *out_mesh,
                      bool check_host);
Grid *mesh_grid(Mesh *m, float cell, cudaStream_t stream, si_status *st);
void mesh_drop_grids(Mesh *m);
// Cells a grid of a mesh of n points may have (the coarsening bound).
int64_t grid_cell_cap(int64_t n);
// Candidate threshold of a binning: fl32(R^2 (1 + 1e-5)) with R^2 = h^2 +
// ((W-1)B)^2 (bilinear, h = W B / 2) or ((W/2 + 1) B)^2 + ((W-1)B)^2 (nearest).
float candidate_rc2(int W, float bin_size, int binning);
float grid_cell_for(const Mesh *m, int W, float bin, int grid_div);
int choose_log2_group(int W, int requested_group);
size_t image_words(int W, int log2S);
// Dynamic shared memory a group of shape (W, 2^log2S images) needs in the
// spin kernel; a launch takes the maximum over its items.
size_t spin_smem_bytes(int W, int log2S);
// Resident spin-kernel blocks per SM for the instance that runs `modes`.
int blocks_per_sm_for(size_t smem_bytes, int modes);
int num_sms(int device);

// Chunk rules (host side, one implementation for every caller).
int64_t chunk_table(int kind, int64_t units, int workers, int min_chunk, double cov,
                    std::vector<int64_t> *starts);

// Synchronous argument checks of one item.
si_status check_item(const si_batch_item &it, const si_schedule &sc, int dev);

// Enqueue the generation of a batch of items (host-validated) on `stream`.
si_status enqueue_batch(const std::vector<si_batch_item> &items, const std::vector<si_schedule> &scheds,
                        const std::vector<const si_probe *> &probes, cudaStream_t stream,
                        int forced_workers, const si_trace *trace = nullptr);
// The same for batched calls through the CUDA-graph cache (capture once,
// replay for identical batches); the legacy default stream goes direct.
si_status enqueue_batch_graph(const std::vector<si_batch_item> &items, const std::vector<si_schedule> &scheds,
                              cudaStream_t stream, int forced_workers);
void forget_mesh_graphs(const void *mesh);
size_t cached_batch_graphs();

// Pinned staging ring for host->device uploads.
si_status stage_upload(void *dev_dst, const void *src, size_t bytes, cudaStream_t stream);

// Stream-ordered device allocation (pool-backed).
si_status dev_alloc(void **p, size_t bytes, cudaStream_t stream);
void dev_free(void *p, cudaStream_t stream);

// Library kernels launched from host code in other translation units.
void launch_spin_kernel(const LaunchArgs &a, int blocks, size_t smem, cudaStream_t stream);
cudaError_t setup_spin_kernel_attributes(size_t smem_bytes);

bool timing_enabled();

// Count of kernels launched by the library (diagnostics).
void note_launches(int k);

}  // namespace si
