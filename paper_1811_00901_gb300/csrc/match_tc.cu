// match_tc.cu -- spin-image matching on the fifth-generation tensor cores:
// the all-pairs correlation of BF16 centred images as a tcgen05 GEMM whose
// epilogue keeps each scene image's k best model images, so the correlation
// tile never leaves the chip.
//
// Work decomposition (one CTA per (scene block, model part)):
//   * a CTA owns 128 scene rows (the MMA's M) and a contiguous range of model
//     tiles of 256 images (the MMA's N); the model tiles are cut into `parts`
//     ranges so that the grid fills whole waves of the GPU's SMs;
//   * warp 0 (one lane) streams 64-element K slices of the scene block and of
//     the current model tile into a 4-stage shared-memory ring with 2-D TMA
//     loads (128-byte swizzle), completion on per-stage mbarriers;
//   * warp 1 allocates 512 TMEM columns (two 128 x 256 FP32 accumulators) and
//     one of its lanes issues tcgen05.mma (kind::f16, BF16 operands from shared
//     memory descriptors, FP32 accumulation in TMEM); tcgen05.commit releases a
//     ring stage when the MMAs reading it are done, and hands a finished
//     accumulator to the epilogue;
//   * warps 2-9 read the accumulator out of TMEM (tcgen05.ld, lane i = scene
//     row i of the block): two threads per row, one for each half of the
//     tile's columns, each loading its whole share into registers before it
//     hands the buffer back, so the next tile's MMAs overlap the scan; each
//     thread keeps a running list of its row's k best in registers (higher
//     value first; model indices arrive in increasing order, so equal values
//     keep the smaller index).
// Each CTA writes two lists per row (one per column half);
// merge_parts_kernel combines the lists of all parts.
//
// Every mbarrier wait is bounded (kWaitLimitNs of %globaltimer): on expiry the
// CTA sets the error word, stops issuing, waits (bounded) for the copies and
// MMAs it has in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <climits>
#include <mutex>

#include "device_common.cuh"
#include "internal.h"
#include "match_tc.h"

namespace si {
namespace {

constexpr int kBM = 128;             // scene rows per CTA (MMA M)
constexpr int kBN = 256;             // model images per tile (MMA N)
constexpr int kBK = 64;              // K elements per ring stage (128 bytes of BF16: one swizzle row)
constexpr int kStagesTc = 4;         // shared-memory ring depth
constexpr int kAStageBytes = kBM * kBK * 2;   // 16 KB
constexpr int kBStageBytes = kBN * kBK * 2;   // 32 KB
constexpr int kStageBytes = kAStageBytes + kBStageBytes;
constexpr int kTmemCols = 2 * kBN;   // two FP32 accumulators of 128 lanes x 256 columns
constexpr int kEpiWarps = 8;         // two per TMEM lane quarter, each scanning half of a tile's columns
constexpr int kTcThreads = 32 * (2 + kEpiWarps);  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kTcSmem = 1024 + kStagesTc * kStageBytes + 256;

struct TcBarriers {
    uint64_t full[kStagesTc];
    uint64_t empty[kStagesTc];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};
static_assert(sizeof(TcBarriers) <= 256, "barrier block");

// ---- PTX wrappers (tcgen05, TMA) ----
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Issues a load of 32 consecutive FP32 columns of this thread's TMEM lane;
// the registers hold them after tc_wait_ld().
__device__ __forceinline__ void tc_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Ties the registers of an issued TMEM load to this point of the program, so
// that no use of them is scheduled above the preceding tc_wait_ld().
__device__ __forceinline__ void tc_pin(uint32_t (&r)[32]) {
#pragma unroll
    for (int i = 0; i < 32; ++i) asm volatile("" : "+r"(r[i]));
}

// Shared-memory matrix descriptor of a K-major BF16 tile written by TMA with
// the 128-byte swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart (the
// stride byte offset); the leading byte offset is unused for this layout.
// Fields: start address >> 4 (bits 0-13), leading offset >> 4 (16-29),
// stride offset >> 4 (32-45), descriptor version 1 (46-47), swizzle mode
// 2 = 128-byte (61-63).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

// Bounded wait on an mbarrier phase; false (and the abort flag set) on expiry.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!*abort_flag) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) {
            *abort_flag = 1;
            return false;
        }
    }
    return false;
}

// The largest of 32 values by a balanced tree.
__device__ __forceinline__ float chunk_max(const float (&x)[32]) {
    float m[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) m[u] = fmaxf(x[u], x[u + 16]);
#pragma unroll
    for (int w = 8; w > 0; w >>= 1)
#pragma unroll
        for (int u = 0; u < w; ++u) m[u] = fmaxf(m[u], m[u + w]);
    return m[0];
}

// Inserts (x, j) into a descending list held in the first k of L register
// slots (x strictly better than the k-th, which the caller checked): one pass
// in which every index is compile-time, so the list stays in registers.  From
// the first slot x beats on, the entries shift down one place; an equal value
// stays ahead of x (x comes from a later column).  Returns the new k-th value.
template <int L>
__device__ __forceinline__ float topk_push(float (&v)[L], int (&ix)[L], int k, float x, int j) {
    float cv = x;
    int ci = j;
    bool moving = false;
    float kth = v[0];
#pragma unroll
    for (int q = 0; q < L; ++q) {
        moving = moving || cv > v[q];
        const bool sw = moving && q < k;
        const float tv = v[q];
        const int ti = ix[q];
        v[q] = sw ? cv : tv;
        ix[q] = sw ? ci : ti;
        cv = sw ? tv : cv;
        ci = sw ? ti : ci;
        if (q == k - 1) kth = v[q];
    }
    return kth;
}

// L = register slots of each thread's list (k <= L).  A block of ten warps
// gets at most 168 registers a thread (three of its warps share one
// sub-partition's 16K registers), which a tile share of 128 values and a
// 16-slot list overflow; k <= 8 runs with 8 slots.
template <int L>
__global__ void __launch_bounds__(kTcThreads, 1)
    match_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                    const int n_scene, const int n_model, const int k_slices, const int tiles, const int parts,
                    const int band_m, const int k, float *__restrict__ part_v, int *__restrict__ part_i,
                    unsigned *err) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 128-byte swizzle atoms need 1024-byte alignment
    unsigned char *const sbase = smem_raw + (base - raw);
    TcBarriers &B = *reinterpret_cast<TcBarriers *>(sbase + kStagesTc * kStageBytes);
    volatile int *abort_flag = &B.abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // banded part-major order: the scene blocks are taken in bands of band_m,
    // and within a band the CTAs run part by part, so the CTAs resident at one
    // time share a model range (its tiles come from DRAM once, then from L2)
    // and hold at most a band's scene operands, which stay in L2 while the
    // band's parts stream past them
    const int mblocks = (n_scene + kBM - 1) / kBM;
    const int full_bands = mblocks / band_m, per_band = band_m * parts;
    int band = blockIdx.x / per_band, bm_eff = band_m;
    if (band >= full_bands) {
        band = full_bands;
        bm_eff = mblocks - full_bands * band_m;
    }
    const int idx = blockIdx.x - band * per_band;
    const int part = idx / bm_eff, mb = band * band_m + (idx - (idx / bm_eff) * bm_eff);
    const int t0 = (int)((int64_t)tiles * part / parts), t1 = (int)((int64_t)tiles * (part + 1) / parts);
    const int ntile = t1 - t0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStagesTc; ++s) {
            mbar_init(&B.full[s], 1);
            mbar_init(&B.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&B.tfull[b], 1);
            mbar_init(&B.tempty[b], kEpiWarps);
        }
        mbar_init(&B.drain, 1);
        B.abort = 0;
        fence_mbar_init();
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_a)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_b)) : "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&B.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = B.tmem_base;

    if (warp == 0) {
        // ---- producer: K slices of the scene block and of each model tile
        if (lane == 0) {
            int it = 0, issued = 0;
            for (int t = 0; t < ntile && !*abort_flag; ++t) {
                const int ncol0 = (t0 + t) * kBN;
                for (int ks = 0; ks < k_slices; ++ks, ++it) {
                    const int s = it % kStagesTc;
                    const uint32_t ph = (uint32_t)(it / kStagesTc) & 1u;
                    if (!tc_wait(&B.empty[s], ph ^ 1u, abort_flag)) break;
                    const uint32_t a_dst = base + s * kStageBytes, b_dst = a_dst + kAStageBytes;
                    mbar_arrive_expect_tx(&B.full[s], (uint32_t)kStageBytes);
                    tma_load_2d(a_dst, &map_a, ks * kBK, mb * kBM, smem_addr(&B.full[s]));
                    tma_load_2d(b_dst, &map_b, ks * kBK, ncol0, smem_addr(&B.full[s]));
                    ++issued;
                }
            }
            if (*abort_flag) {
                // let every copy this thread issued land before the CTA goes
                for (int j = (issued > kStagesTc ? issued - kStagesTc : 0); j < issued; ++j)
                    mbar_wait_bounded(&B.full[j % kStagesTc], (uint32_t)(j / kStagesTc) & 1u, kWaitLimitNs);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            int it = 0;
            for (int t = 0; t < ntile && !*abort_flag; ++t) {
                const int b = t & 1;
                const uint32_t tph = (uint32_t)(t >> 1) & 1u;
                if (!tc_wait(&B.tempty[b], tph ^ 1u, abort_flag)) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * kBN);
                bool ok = true;
                for (int ks = 0; ks < k_slices; ++ks, ++it) {
                    const int s = it % kStagesTc;
                    const uint32_t ph = (uint32_t)(it / kStagesTc) & 1u;
                    if (!tc_wait(&B.full[s], ph, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_addr = base + s * kStageBytes, b_addr = a_addr + kAStageBytes;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk)  // four K = 16 MMAs, 32 bytes apart in the swizzle row
                        tc_mma(d, smem_desc_sw128(a_addr + 32u * kk), smem_desc_sw128(b_addr + 32u * kk), kIdesc,
                               (ks | kk) != 0 ? 1u : 0u);
                    tc_commit(smem_addr(&B.empty[s]));  // the stage is free once these MMAs are done
                }
                if (!ok) break;
                tc_commit(smem_addr(&B.tfull[b]));  // the accumulator is complete
            }
            // every MMA this thread issued has completed once this arrives
            tc_commit(smem_addr(&B.drain));
            mbar_wait_bounded(&B.drain, 0u, kWaitLimitNs);
        }
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w mod 4) .. + 31, one scene row per
        // thread; warps 2-5 take the first half of each tile's columns, 6-9 the second
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        constexpr int kChunks = kBN / 32 / 2;  // 32-column chunks per half tile
        float v[L];
        int ix[L];
#pragma unroll
        for (int q = 0; q < L; ++q) {
            v[q] = -FLT_MAX;
            ix[q] = INT_MAX;
        }
        float thr = -FLT_MAX;
        for (int t = 0; t < ntile; ++t) {
            const int b = t & 1;
            const uint32_t tph = (uint32_t)(t >> 1) & 1u;
            if (!tc_wait(&B.tfull[b], tph, abort_flag)) break;
            tc_fence_after();
            const int ncol0 = (t0 + t) * kBN + half * (kBN / 2);
            const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kBN + half * (kBN / 2));
            // the warp's whole share of the tile into registers with one wait, then
            // the buffer goes back to the MMA warp before any scanning
            uint32_t r[kChunks][32];
#pragma unroll
            for (int c = 0; c < kChunks; ++c) tc_ld32_issue(taddr + (uint32_t)(c * 32), r[c]);
            tc_wait_ld();
#pragma unroll
            for (int c = 0; c < kChunks; ++c) tc_pin(r[c]);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&B.tempty[b]);
#pragma unroll
            for (int c = 0; c < kChunks; ++c) {
                float x[32];
                const int j0 = ncol0 + c * 32;
                const int valid = n_model - j0;  // columns past the last model image hold zeros
#pragma unroll
                for (int u = 0; u < 32; ++u) x[u] = u < valid ? __uint_as_float(r[c][u]) : -FLT_MAX;
                // the list changes only where the chunk's maximum beats its k-th value; then
                // the maximum (the smallest column among equals) goes in and leaves the
                // chunk, and the next maximum is tried: one insertion site keeps the code small
                float mx = chunk_max(x);
                while (mx > thr) {
                    int pos = 31;
#pragma unroll
                    for (int u = 31; u >= 0; --u) pos = x[u] == mx ? u : pos;
                    thr = topk_push(v, ix, k, mx, j0 + pos);
#pragma unroll
                    for (int u = 0; u < 32; ++u) x[u] = u == pos ? -FLT_MAX : x[u];
                    mx = chunk_max(x);
                }
            }
        }
        const int grow = mb * kBM + row;
        if (grow < n_scene && !*abort_flag) {
            const int64_t o = ((int64_t)(2 * part + half) * n_scene + grow) * k;
#pragma unroll
            for (int q = 0; q < L; ++q)
                if (q < k) {
                    part_v[o + q] = v[q];
                    part_i[o + q] = ix[q];
                }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicOr(err, 1u);
}

// a before b: higher value, equal values by smaller index
__device__ __forceinline__ bool better_vi(float va, int ia, float vb, int ib) {
    return va > vb || (va == vb && ia < ib);
}

// One thread per scene row: the k best of the `parts` sorted lists.
__global__ void merge_parts_kernel(const float *__restrict__ part_v, const int *__restrict__ part_i, int n_scene,
                                   int parts, int k, const unsigned *err, int32_t *__restrict__ best_idx,
                                   float *__restrict__ best_val) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_scene) return;
    if (*err) {  // some CTA gave up a bounded wait: the call's lists are void
        for (int q = 0; q < k; ++q) {
            best_idx[(int64_t)r * k + q] = -2;
            best_val[(int64_t)r * k + q] = 0.0f;
        }
        return;
    }
    int head[2 * kMatchTcMaxParts];
    for (int p = 0; p < parts; ++p) head[p] = 0;
    for (int q = 0; q < k; ++q) {
        int bp = -1;
        float bv = 0.0f;
        int bi = INT_MAX;
        for (int p = 0; p < parts; ++p) {
            if (head[p] >= k) continue;
            const int64_t o = ((int64_t)p * n_scene + r) * k + head[p];
            const float x = part_v[o];
            const int xi = part_i[o];
            if (bp < 0 || better_vi(x, xi, bv, bi)) {
                bp = p;
                bv = x;
                bi = xi;
            }
        }
        ++head[bp];
        best_val[(int64_t)r * k + q] = bv;
        best_idx[(int64_t)r * k + q] = bi == INT_MAX ? -1 : bi;
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn(si_status *st) {
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
            *st = e != cudaSuccess ? cuda_fail(e, "cuTensorMapEncodeTiled entry point") : SI_ERR_CUDA;
            if (e == cudaSuccess) set_error("si_match: cuTensorMapEncodeTiled is not available");
            return nullptr;
        }
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    *st = SI_OK;
    return fn;
}

// Row-major BF16 [rows][kp] as a 2-D tensor map with (64 x box_rows) boxes.
si_status make_map(CUtensorMap *m, const void *ptr, int64_t rows, int kp, int box_rows) {
    si_status st;
    EncodeTiledFn fn = encode_fn(&st);
    if (!fn) return st;
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("si_match: cuTensorMapEncodeTiled failed (%d)", (int)r);
        return SI_ERR_CUDA;
    }
    return SI_OK;
}

}  // namespace

int match_tc_parts(int64_t n_scene, int64_t n_model, int sms) {
    const int64_t mblocks = (n_scene + kBM - 1) / kBM;
    const int64_t tiles = (n_model + kBN - 1) / kBN;
    // the smallest number of model parts (at most one per 4 tiles, at most
    // kMatchTcMaxParts) whose grid loses the least to a partly filled last wave
    int best = 1;
    double best_eff = -1.0;
    for (int p = 1; p <= kMatchTcMaxParts && (p == 1 || tiles / p >= 4); ++p) {
        const int64_t ctas = mblocks * p;
        const int64_t waves = (ctas + sms - 1) / sms;
        const double eff = (double)ctas / (double)(waves * sms);
        if (eff > best_eff + 1e-3) {
            best_eff = eff;
            best = p;
        }
        if (eff > 0.97) break;
    }
    return best;
}

si_status match_tc_launch(const __nv_bfloat16 *a, int64_t n_scene, const __nv_bfloat16 *b, int64_t n_model, int kp,
                          int k, int parts, float *part_v, int *part_i, unsigned *err, int32_t *best_idx,
                          float *best_val, cudaStream_t st) {
    if (kp % kBK != 0 || k < 1 || k > kMatchTcMaxK || parts < 1 || parts > kMatchTcMaxParts || n_scene < 1 ||
        n_model < 1 || n_scene > INT32_MAX || n_model > INT32_MAX) {
        set_error("si_match: internal tensor-core launch arguments");
        return SI_ERR_INVALID;
    }
    CUtensorMap ma, mbm;
    si_status s = make_map(&ma, a, n_scene, kp, kBM);
    if (s == SI_OK) s = make_map(&mbm, b, n_model, kp, kBN);
    if (s != SI_OK) return s;
    static std::mutex attr_mu;
    static bool attr_done[128] = {};
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(attr_mu);
        if (dev >= 0 && dev < 128 && !attr_done[dev]) {
            SI_CUDA(cudaFuncSetAttribute(match_tc_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
            SI_CUDA(cudaFuncSetAttribute(match_tc_kernel<kMatchTcMaxK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTcSmem));
            attr_done[dev] = true;
        }
    }
    const int64_t mblocks = (n_scene + kBM - 1) / kBM;
    const int tiles = (int)((n_model + kBN - 1) / kBN);
    auto kern = k <= 8 ? match_tc_kernel<8> : match_tc_kernel<kMatchTcMaxK>;
    // scene blocks per band: as many as leave L2 (129 MB) room for the model
    // stream, about 48 MB of scene operands (all blocks in BF16 mode at W <= 64)
    const int64_t a_block_bytes = (int64_t)kBM * kp * 2;
    const int band_m = (int)std::max<int64_t>(1, std::min<int64_t>(mblocks, (48ll << 20) / a_block_bytes));
    kern<<<(unsigned)(mblocks * parts), kTcThreads, kTcSmem, st>>>(ma, mbm, (int)n_scene, (int)n_model, kp / kBK,
                                                                  tiles, parts, band_m, k, part_v, part_i, err);
    note_launches(1);
    SI_CUDA(cudaGetLastError());
    // two lists per row and part: one per column half of the tiles
    merge_parts_kernel<<<(unsigned)((n_scene + 255) / 256), 256, 0, st>>>(part_v, part_i, (int)n_scene, 2 * parts,
                                                                          k, err, best_idx, best_val);
    note_launches(1);
    SI_CUDA(cudaGetLastError());
    return SI_OK;
}

}  // namespace si
