// noalloc.cu -- si_generate_noalloc: spin-image generation that allocates
// nothing, for callers that must not allocate device memory at the point of
// the call.
//
// si_generate takes its per-call scratch (the dynamic-schedule step counter,
// the item descriptor, the chunk table and the query permutation) from the
// stream-ordered pool, and builds a missing grid on the fly.  Some callers
// cannot let that happen: a process whose device memory is fully reserved by
// another allocator (every cudaMalloc there fails or evicts someone else's
// cache), or a frame loop with a fixed memory footprint that must not enter
// the allocator between frames.  This variant keeps its scratch in one
// file-scope __device__ array of kNoAllocScratchBytes (2 MiB), which every GPU
// that loads the library holds until the process exits, and it never builds
// a grid: the mesh's grid for (W, bin size, grid_div) must already exist
// (si_mesh_prepare).
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address once (cudaGetSymbolAddress); make that first call
// before any stream capture.  Every call reuses the same array and leaves the
// last call's contents behind; the set-up kernel of each call clears the
// counters that must start at zero.  Two calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on the array.
//
// Differences from si_generate: explicit query lists are generated in the
// order given (no grid-order sort, so there is no permutation to store); the
// images are the same, bit for bit.
#include <cmath>
#include <cstring>
#include <mutex>

#include "chunk_rule.h"
#include "device_common.cuh"
#include "internal.h"

namespace si {

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(2) << 20;  // 2 MiB
constexpr size_t kOffDesc = 256;
constexpr size_t kOffPieces = 1024;
// each scheduling step needs one Piece (16 B) and one step_piece entry (4 B)
constexpr int kNoAllocMaxSteps = 100000;
static_assert(kOffPieces + (size_t)kNoAllocMaxSteps * sizeof(Piece) + (kNoAllocMaxSteps + 1) * sizeof(int) <=
                  kNoAllocScratchBytes,
              "scratch layout exceeds the array");
static_assert(sizeof(LaunchCounters) <= kOffDesc && sizeof(ItemDesc) <= kOffPieces - kOffDesc,
              "scratch header exceeds its slots");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_addr_mu;
void *g_addr[64] = {nullptr};

// Scheduling steps of a call under `kind`, counted with the library's one
// chunk rule (chunk_rule_next); the count stops at `limit` + 1, so a call
// with far more steps than the scratch holds is refused without walking them.
int64_t count_steps(int kind, int64_t units, int64_t P, int64_t mc, int64_t limit) {
    if (kind == SI_SCHED_STATIC) return P;
    int64_t done = 0, step = 0, fac_c = 0;
    while (done < units && step <= limit) {
        done += chunk_rule_next(kind, step, units - done, P, mc, &fac_c);
        ++step;
    }
    return step;
}

// Writes the descriptor, zeroes the launch counters and builds the chunk
// table of the call inside the static scratch.  One block.
__global__ void noalloc_setup_kernel(ItemDesc desc, int kind, int units, int P, int mc, int nsteps,
                                     unsigned char *scratch) {
    LaunchCounters *ctr = reinterpret_cast<LaunchCounters *>(scratch);
    ItemDesc *d = reinterpret_cast<ItemDesc *>(scratch + kOffDesc);
    Piece *pieces = reinterpret_cast<Piece *>(scratch + kOffPieces);
    int *step_piece = reinterpret_cast<int *>(pieces + kNoAllocMaxSteps);
    const int tid = threadIdx.x;
    if (tid == 0) {
        ctr->step = 0;
        ctr->done_blocks = 0;
        *d = desc;
    }
    for (int s = tid; s <= nsteps; s += blockDim.x) step_piece[s] = s;
    if (kind == SI_SCHED_STATIC) {
        for (int s = tid; s < nsteps; s += blockDim.x)
            pieces[s] = Piece{0, (int)((int64_t)s * units / P), (int)((int64_t)(s + 1) * units / P), 0};
    } else if (kind == SI_SCHED_SS) {
        for (int s = tid; s < nsteps; s += blockDim.x) {
            const int64_t lo = (int64_t)s * mc;
            const int64_t hi = lo + mc < units ? lo + mc : units;
            pieces[s] = Piece{0, (int)lo, (int)hi, 0};
        }
    } else if (tid == 0) {
        // GSS and FAC: each chunk depends on what the earlier ones left, so one
        // thread walks the steps with the library's chunk rule
        int64_t done = 0, fac_c = 0;
        for (int s = 0; s < nsteps; ++s) {
            const int64_t c = chunk_rule_next(kind, s, units - done, P, mc, &fac_c);
            pieces[s] = Piece{0, (int)done, (int)(done + c), 0};
            done += c;
        }
    }
}

si_status scratch_address(int dev, unsigned char **out) {
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (dev < 0 || dev >= 64) {
        set_error("si_generate_noalloc: device index %d out of range", dev);
        return SI_ERR_INVALID;
    }
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_addr[dev] = p;
    }
    *out = reinterpret_cast<unsigned char *>(g_addr[dev]);
    return SI_OK;
}

}  // namespace

}  // namespace si

using namespace si;

extern "C" si_status si_generate_noalloc(si_mesh_t mesh, const int32_t *query_idx, int64_t m, int32_t W,
                                         float bin_size, float cos_support_angle, si_schedule schedule,
                                         int32_t *out, si_stream stream) {
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    const si_batch_item it{mesh, query_idx, m, W, bin_size, cos_support_angle, out};
    si_status s = check_item(it, schedule, dev);
    if (s != SI_OK) return s;
    if (schedule.kind >= SI_SCHED_FAC_PROB || schedule.binning != SI_BIN_BILINEAR || schedule.slow_workers != 0 ||
        schedule.slices > 1 || schedule.order != 0) {
        set_error("si_generate_noalloc: takes STATIC, SS, GSS or FAC, bilinear binning, no slow workers, one "
                  "slice per group and grid order");
        return SI_ERR_INVALID;
    }
    if (m == 0) return SI_OK;
    Mesh *me = reinterpret_cast<Mesh *>(mesh);
    // the grid must exist already: look it up, never build it
    const float cell = grid_cell_for(me, W, bin_size, schedule.grid_div);
    const Grid *g = nullptr;
    {
        std::lock_guard<std::mutex> lk(me->mu);
        for (const Grid *c : me->grids)
            if (c->cell == cell) g = c;
    }
    if (!g) {
        set_error("si_generate_noalloc: no grid for W=%d, bin size %g, grid_div %d; call si_mesh_prepare first", W,
                  (double)bin_size, schedule.grid_div);
        return SI_ERR_INVALID;
    }
    const int log2S = choose_log2_group(W, schedule.group);
    const int64_t units = (m + (1 << log2S) - 1) >> log2S;
    const int modes = launch_modes(ring_mode(log2S), false);
    const size_t smem = spin_smem_bytes(W, log2S);
    SI_CUDA(setup_spin_kernel_attributes(smem));
    const int per_sm = blocks_per_sm_for(smem, modes);
    if (per_sm < 1) {
        set_error("si_generate_noalloc: the spin kernel does not fit on an SM");
        return SI_ERR_INVALID;
    }
    const int P = schedule.num_workers > 0 ? schedule.num_workers : num_sms(dev) * per_sm;
    const int mc = schedule.min_chunk > 0 ? schedule.min_chunk : 1;
    const int64_t nsteps = count_steps(schedule.kind, units, P, mc, kNoAllocMaxSteps);
    if (nsteps > kNoAllocMaxSteps) {
        set_error("si_generate_noalloc: more than the %d scheduling steps that fit in its %zu-byte scratch; "
                  "use a larger min_chunk, group or fewer workers",
                  kNoAllocMaxSteps, kNoAllocScratchBytes);
        return SI_ERR_INVALID;
    }
    unsigned char *scratch = nullptr;
    s = scratch_address(dev, &scratch);
    if (s != SI_OK) return s;

    ItemDesc d;
    std::memset(&d, 0, sizeof(d));
    d.pn = g->pn;
    d.cell_start = g->cell_start;
    d.sorted_pos = g->sorted_pos;
    d.query_idx = query_idx;
    d.out = out;
    d.flags = me->flags;
    d.geom = g->geom;
    d.m = m;
    d.n_points = (int)me->n;
    d.W = W;
    d.log2S = log2S;
    d.units = (int)units;
    if (!query_idx && m == me->n) {
        d.perm = g->orig_idx;  // all points: grid order is the query order
        d.perm_is_grid = 1;
    } else {
        d.perm = nullptr;  // queries in the order given
        d.perm_is_grid = 0;
    }
    const float rc2 = si_candidate_rc2(W, bin_size);
    d.Rc2 = rc2;
    d.Rc = sqrtf(rc2);
    d.cosS = cos_support_angle;
    d.invB = 1.0f / bin_size;
    d.halfW = 0.5f * (float)W;
    d.umax = (float)(W - 1);

    SI_CUDA(cudaStreamWaitEvent(st, g->ready, 0));
    noalloc_setup_kernel<<<1, 256, 0, st>>>(d, schedule.kind, (int)units, P, mc, (int)nsteps, scratch);
    note_launches(1);
    SI_CUDA(cudaGetLastError());
    LaunchArgs a;
    a.items = reinterpret_cast<const ItemDesc *>(scratch + kOffDesc);
    a.pieces = reinterpret_cast<const Piece *>(scratch + kOffPieces);
    a.step_piece = reinterpret_cast<const int *>(a.pieces + kNoAllocMaxSteps);
    a.nsteps = (int)nsteps;
    a.is_static = schedule.kind == SI_SCHED_STATIC ? 1 : 0;
    a.ctr = reinterpret_cast<LaunchCounters *>(scratch);
    a.nitems = 1;
    a.img_words = (int)image_words(W, log2S);
    a.probe = 0;
    a.modes = modes;
    launch_spin_kernel(a, a.is_static ? (int)nsteps : P, smem, st);
    note_launches(1);
    SI_CUDA(cudaGetLastError());
    {
        std::lock_guard<std::mutex> lk(me->mu);
        me->calls += 1;
        me->images += m;
    }
    return SI_OK;
}
