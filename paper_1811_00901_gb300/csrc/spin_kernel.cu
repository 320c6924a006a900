// spin_kernel.cu -- the persistent spin-image kernel (Algorithm 1's image loop
// as run by the workers of Algorithms 2-4, one GPU edition).
//
// Work decomposition
//   * The scheduled loop runs over image GROUPS: `S` consecutive query points
//     in grid (cell) order, generated together by one thread block against a
//     shared stream of candidate points.
//   * A block is a worker.  Under STATIC, block b runs step b (its block of
//     the loop, PSIA).  Under SS / GSS / FAC one thread claims the next step
//     with a global atomicAdd (the master's getChunk of Algorithm 3 is the
//     precomputed step table; the request/assign exchange is the atomic) and
//     broadcasts it through shared memory.
//   * For a group, the candidate points are the grid cells within the
//     candidate radius Rc of the group's bounding box, enumerated as
//     (z, y) rows of contiguous cells.  One thread streams them into a ring
//     of shared-memory tiles with 1-D bulk copies (TMA, mbarrier completion);
//     all threads consume the tiles.
//   * Lane l of a warp works on image slot (l mod S) against candidate
//     (l div S) of the warp's current step, so one candidate read is broadcast
//     to S lanes and the S images of a group are interleaved word by word in
//     shared memory (pixel p of slot q at word p*S + q): the 32 lanes of a
//     warp hit at most 32/S words per bank, whatever pixels they splat.
//   * Each lane evaluates two candidates per loop trip without branches (the
//     two chains interleave); only the splat of a contributing pair is
//     behind a branch.  Full tiles take a loop without per-lane range checks.
//
// Per pair (P = query, X = candidate, FP32, differences taken directly):
//   d = X - P; angle test n.n_X >= cos S; beta = n.d;
//   alpha^2 = |d - beta n|^2 (the part of d orthogonal to n: Algorithm 1's
//   |d|^2 - beta^2 for a unit n, without its cancellation near the normal
//   axis, where FP32 |d|^2 - beta^2 loses alpha to sqrt(eps) |d|);
//   u = W/2 - beta/B; v = alpha/B; support test 0 <= u < W-1 and, on the
//   fixed-point column V = rn(v 2^16), V < (W-1) 2^16 (v < W-1); fixed-point
//   bilinear splat of weight 65536 with four shared-memory int32 atomics.  The candidate cull
//   fl32(|d|^2) <= Rc2 is implied by the support test (every contributing
//   pair has |d|^2 < R^2 < Rc2), so only probes evaluate it.
// Images hold (W+1) x (W+1) words per slot: the extra row and column absorb
// the zero-weight corners of points whose coordinate rounds up onto W-1.
#include <atomic>

#include "device_common.cuh"
#include "internal.h"


namespace si {

namespace {

// Index checks of the SI_DEBUG_BOUNDS build: a failed check sets the item's
// kFlagBounds (si_get_stats reports it) and the access is skipped or pointed
// at valid memory; nothing traps.  In the normal build the checks are `true`
// and their conditions are not evaluated.
#ifdef SI_DEBUG_BOUNDS
__device__ __forceinline__ bool bounds_ok(bool c, unsigned *flags) {
    if (!c) atomicOr(flags, kFlagBounds);
    return c;
}
#define SI_IN_BOUNDS(cond, flags) bounds_ok((cond), (flags))
#else
#define SI_IN_BOUNDS(cond, flags) true
#endif

constexpr int kWarps = kThreads / 32;
// Two ways to run the tile ring, chosen per group shape:
//  * barrier mode (groups of 8+ images): every warp consumes; after each tile
//    a block barrier, then thread 0 refills the stage just drained;
//  * producer mode (groups of <= 4 images, where a tile is only a trip or two
//    per warp and the barrier would dominate): the last warp only produces,
//    in order, and the other warps release stages through "empty" mbarriers.
constexpr int kProdConsumers = kWarps - 1;

struct __align__(16) QueryInfo {
    float4 p;
    float4 n;
    int slot;
    int pad[3];
};

struct __align__(16) Header {
    uint64_t bar[kStages];
    int claim;
    int total;
    float gmin[3], gmax[3];
    int ylo, yhi, zlo, zhi;
    int warp_tmp[kWarps];
    unsigned long long grp_weight;
    unsigned long long grp_pix;
    uint64_t empty[kStages];  // producer mode: consumer warps release stages
    int fills[kStages];       // fills issued into each stage (both modes, whole kernel)
    int pfills[kStages];      // fills issued in producer mode (empty-barrier phases)
    int abort_flag;
    int slot_cnt[32];         // sliced groups: contributing pairs per image of this slice
    int cur_r, cur_o;          // barrier mode: producer row cursor
    unsigned long long t_step;  // heterogeneity emulation: start of a slow block's step
    unsigned long long t_trace; // claim trace: start of the current claim's work
    unsigned long long af_t_unit;  // adaptive factoring: start of the current unit
    // adaptive weighted factoring: this worker's claim and its measured rate
    int awf_lo, awf_hi;
    unsigned long long awf_t0;  // when the current chunk was claimed
    double awf_units, awf_ns;   // units done and time spent so far
    double awf_rate;            // awf_units / awf_ns (0: not measured yet)
    int awf_last;               // units of the current chunk
};

constexpr int kHeaderBytes = (sizeof(Header) + 127) / 128 * 128;
static_assert(sizeof(Header) <= kHeaderBytes, "header too large");
constexpr int kQueryBytes = 32 * sizeof(QueryInfo);
constexpr int kRowBytes = 3 * (kMaxRows + 4) * sizeof(int);
constexpr int kProbeBytes = 5 * 32 * sizeof(int);

// Shared-memory layout of a block: header, queries, stencil rows, probe
// counters, then per group the tile ring (kStages x tile) and the images.
constexpr int off_query() { return kHeaderBytes; }
constexpr int off_rows() { return off_query() + kQueryBytes; }
constexpr int off_probe() { return off_rows() + kRowBytes; }
constexpr int off_tiles() { return (off_probe() + kProbeBytes + 127) & ~127; }

constexpr int img_words_of(int W, int log2S) { return ((((W + 1) * (W + 1)) << log2S) + 3) & ~3; }
constexpr int shape_smem(int W, int log2S, int tn) {
    return off_tiles() + kStages * 32 * tn + 4 * img_words_of(W, log2S);
}

// Candidates per tile for a group shape.  Block-barrier shapes take the
// largest tile, a whole number of unrolled trips (2 x kWarps x 32/S
// candidates), that keeps SI_MIN_BLOCKS blocks per SM, else kTileMax.
// Producer-ring shapes (<= 4 images) take the largest tile in [kTileMin,
// kTileMax] that deals the same number of trips to every consumer warp, else
// kTileMax: a warp with a trip more than the others holds its stage back.
constexpr int tile_for_shape(int W, int log2S) {
    if (log2S <= 2) {
        const int unit = 2 * kProdConsumers * (32 >> log2S);
        for (int tn = kTileMax; tn >= kTileMin; tn -= 16)
            if (tn % unit == 0) return tn;
        return kTileMax;
    }
    const int unit = 2 * kWarps * (32 >> log2S);
    for (int tn = kTileMax; tn >= kTileMin; tn -= 16)
        if (tn % unit == 0 && shape_smem(W, log2S, tn) <= SI_SMEM_BUDGET_KB * 1024) return tn;
    return kTileMax;
}

// Exclusive scan of len[0..nr) into off[0..nr); returns the total to all threads.
__device__ int block_scan_rows(const int *len, int *off, int nr, Header &H) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = 2 * tid, i1 = 2 * tid + 1;
    const int a0 = i0 < nr ? len[i0] : 0;
    const int a1 = i1 < nr ? len[i1] : 0;
    const int s = a0 + a1;
    int incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) H.warp_tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = lane < kWarps ? H.warp_tmp[lane] : 0;
        int vi = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int o = __shfl_up_sync(0xffffffffu, vi, d);
            if (lane >= d) vi += o;
        }
        if (lane < kWarps) H.warp_tmp[lane] = vi - v;
        if (lane == kWarps - 1) H.total = vi;
    }
    __syncthreads();
    const int excl = H.warp_tmp[warp] + incl - s;
    if (i0 < nr) off[i0] = excl;
    if (i1 < nr) off[i1] = excl + a0;
    const int total = H.total;
    __syncthreads();
    return total;
}

// ---- the candidate stencil of a group (used by process_group and by the
// cost estimate of group_cost_kernel, so both see the same cells)

// Safety margin of the stencil: a few ulps of the coordinates and of the radius.
__device__ __forceinline__ float stencil_margin(const GridGeom &gg, float Rc) {
    return 1e-5f * (gg.mag + Rc + gg.cell_len) + 1e-30f;
}

// The y and z cell ranges within Rc (plus margin) of the box [lo, hi].
__device__ __forceinline__ void stencil_yz(float oy, float oz, float inv, int dy_, int dz_, float lo1, float lo2,
                                           float hi1, float hi2, float Rc, float margin, int &ylo, int &yhi,
                                           int &zlo, int &zhi) {
    const float r = Rc + margin;
    ylo = cell_coord(lo1 - r, oy, inv, dy_);
    yhi = cell_coord(hi1 + r, oy, inv, dy_);
    zlo = cell_coord(lo2 - r, oz, inv, dz_);
    zhi = cell_coord(hi2 + r, oz, inv, dz_);
}

// Cells [c0, c0 + n) of stencil row (y, z): the cells of the row within the
// candidate radius (Rc2, plus margin) of the box [gmin, gmax]; n = 0 when the
// row misses it.
__device__ __forceinline__ int stencil_row(float ox, float oy, float oz, float cell, float inv, int dx_, int dy_,
                                           const float *gmin, const float *gmax, float Rc2, float margin, int y,
                                           int z, int &c0) {
    const float sy0 = fmaf((float)y, cell, oy), sy1 = sy0 + cell;
    const float sz0 = fmaf((float)z, cell, oz), sz1 = sz0 + cell;
    const float gy = fmaxf(0.0f, fmaxf(sy0 - gmax[1], gmin[1] - sy1) - margin);
    const float gz = fmaxf(0.0f, fmaxf(sz0 - gmax[2], gmin[2] - sz1) - margin);
    const float rem = Rc2 - gy * gy - gz * gz;
    if (!(rem >= 0.0f)) return 0;
    const float rx = sqrtf(rem) + margin;
    const int x0 = cell_coord(gmin[0] - rx, ox, inv, dx_);
    const int x1 = cell_coord(gmax[0] + rx, ox, inv, dx_);
    c0 = (z * dy_ + y) * dx_ + x0;
    return x1 - x0 + 1;
}

// Query t of an item (in grid order): its output slot q, whether its index is
// valid, and its position in the grid's sorted points.
__device__ __forceinline__ int query_sorted_pos(const ItemDesc &it, int64_t t, int &q, bool &ok) {
    q = it.perm ? it.perm[t] : (int)t;
    int sp = (int)t;
    ok = true;
    if (!it.perm_is_grid) {
        const int src = it.query_idx ? it.query_idx[q] : q;
        ok = (unsigned)src < (unsigned)it.n_points;
        sp = ok ? it.sorted_pos[src] : 0;
    }
    return sp;
}

// Constants of one item that the pair evaluation needs (and, for the
// SI_DEBUG_BOUNDS build, the group's image words and the item's flags).
struct PairConsts {
    float Rc2, cosS, invB, halfW, umax, B;
    const int *img;
    int img_words;
    unsigned *flags;
};

// Shape of a group's images: compile-time when WT > 0, else runtime.
template <int WT, int LS>
struct Shape {
    int W_rt, LS_rt;
    __device__ __forceinline__ int W() const { return WT > 0 ? WT : W_rt; }
    __device__ __forceinline__ int log2S() const { return WT > 0 ? LS : LS_rt; }
    __device__ __forceinline__ int S() const { return 1 << log2S(); }
    __device__ __forceinline__ int row_words() const { return (W() + 1) << log2S(); }
};

// The distance part of a pair: d = X - P and, when D2, the candidate-set
// expression, exactly fl32(fma(dz,dz, fma(dy,dy, dx*dx))).
struct PairDist {
    float dx, dy, dz, d2;
};

template <bool D2>
__device__ __forceinline__ PairDist pair_dist(const float4 X, const float4 P) {
    PairDist r;
    r.dx = __fsub_rn(X.x, P.x);
    r.dy = __fsub_rn(X.y, P.y);
    r.dz = __fsub_rn(X.z, P.z);
    r.d2 = D2 ? __fmaf_rn(r.dz, r.dz, __fmaf_rn(r.dy, r.dy, __fmul_rn(r.dx, r.dx))) : 0.0f;
    return r;
}

// fl32(x + 2^23) for 0 <= x < 2^23 has the exponent field of 2^23; its top 16
// bits read kMagicHi + (rn(x) >> 16).
constexpr int kMagicHi = 0x4B00;

// Evaluates the rest of one (query, candidate) pair and splats it when it
// contributes.  Every contributing pair has |d|^2 < R^2 < Rc2, so the cull
// is not part of the support decision (`live` is the lane's range check).
// `img_adj` is the slot's pixel (0, 0) moved back by the exponent bias that
// the raw coordinate bits carry (kMagicHi rows and kMagicHi columns).
template <int WT, int LS, bool PROBE>
__device__ __forceinline__ void eval_pair(const PairDist &pd, const float4 NX, const bool live, const float4 N,
                                          const PairConsts &k, const Shape<WT, LS> sh, int *img_adj, int &cnt,
                                          int *pc_s) {
    const float dx = pd.dx, dy = pd.dy, dz = pd.dz;
    const float ca = fmaf(N.z, NX.z, fmaf(N.y, NX.y, N.x * NX.x));
    const float beta = fmaf(N.z, dz, fmaf(N.y, dy, N.x * dx));
    // alpha^2 from r = d - beta n: an error in beta moves r along n, which
    // changes |r|^2 only to second order, so alpha keeps ~1e-7 relative
    // accuracy even on the normal axis
    const float rx = fmaf(-beta, N.x, dx), ry = fmaf(-beta, N.y, dy), rz = fmaf(-beta, N.z, dz);
    const float a2 = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
    const float u = fmaf(-beta, k.invB, k.halfW);
    // 0 <= u < W-1 as one unsigned compare of the float bits: non-negative floats
    // order like their bits, negatives (sign bit) and NaN compare above umax; u
    // is never -0 (halfW - beta/B rounds an exact zero to +0)
    // alpha through the approximate square root (zero for a2 = 0, and a2 is a
    // sum of squares, never negative), whose last-bit error the 16-bit
    // quantisation absorbs.
    float alpha;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(alpha) : "f"(a2));
    // U = rn(u * 2^16): u * 2^16 is exact and below 2^23 (0 <= u < W - 1 <= 127
    // for a contributing pair), so adding 2^23 rounds it to an integer held in
    // the low 23 bits; the low 16 bits are the fraction, the top 16 the row
    // plus kMagicHi.  V = rn(alpha * (2^16 / B)) the same way.  For v >= 128
    // the sum leaves [2^23, 2^24) and its bits only grow (positive floats
    // order like their bits).
    const uint32_t Ub = __float_as_uint(fmaf(u, 65536.0f, 8388608.0f));
    const uint32_t Vb = __float_as_uint(fmaf(alpha, k.invB * 65536.0f, 8388608.0f));
    // The column test is V < (W - 1) 2^16 on those bits: the pair's last
    // corner column j + 1 = floor(V / 2^16) + 1 stays inside the image.  It
    // differs from the exact v < W - 1 only for v within 2^-17 of W - 1 or
    // within the square root's last-bit error of it, pairs well inside the
    // oracle's boundary band.
    const bool in = live & (ca >= k.cosS) & (__float_as_uint(u) < __float_as_uint(k.umax)) &
                    (Vb < 0x4B000000u + ((uint32_t)k.umax << 16));
    if (PROBE) {
        if (in) atomicAdd(pc_s, 1);
        if (live & (pd.d2 <= k.Rc2) & (ca >= k.cosS)) atomicAdd(pc_s + 96, 1);  // angle-passing candidates
    }
    const uint32_t A = Ub & 0xFFFFu, Bq = Vb & 0xFFFFu;
    const uint32_t w11 = (A * Bq + 32768u) >> 16;
    if (in) {
        const int rw = sh.row_words(), S = sh.S();
        int *p0 = img_adj + ((int)(Ub >> 16) * rw + (int)(Vb >> 16) * S);
        if (!SI_IN_BOUNDS(p0 >= k.img && p0 + rw + S < k.img + k.img_words, k.flags)) return;
        const uint32_t w01 = Bq - w11;
        atomicAdd(p0, (int)(65536u - A - w01));  // w00 = 2^16 - A - Bq + w11
        atomicAdd(p0 + rw, (int)(A - w11));
        atomicAdd(p0 + S, (int)w01);
        atomicAdd(p0 + rw + S, (int)w11);
        ++cnt;
    }
}

// Algorithm 1's own count (SI_BIN_NEAREST): pixel (ceil(u), ceil(v)) += 1 for
// 0 <= ceil(u), ceil(v) <= W-1, in IEEE FP32 with every rounding spelled out
// (the pixel index is decided by the rounded value):
//   angle n.n_X = fma(n.z, nX.z, fma(n.y, nX.y, n.x*nX.x)) >= cos S
//   beta = fma(n.z, dz, fma(n.y, dy, n.x*dx)); alpha = sqrt(max(fma(-beta, beta, |d|^2), 0))
//   u = W/2 - beta/B, v = alpha/B (correctly rounded divisions and square root).
// `img_q` is the slot's pixel (0, 0).
template <int WT, int LS, bool PROBE>
__device__ __forceinline__ void eval_pair_nearest(const PairDist &pd, const float4 NX, const bool live,
                                                  const float4 N, const PairConsts &k, const Shape<WT, LS> sh,
                                                  int *img_q, int &cnt, int *pc_s) {
    const float ca = __fmaf_rn(N.z, NX.z, __fmaf_rn(N.y, NX.y, __fmul_rn(N.x, NX.x)));
    const float beta = __fmaf_rn(N.z, pd.dz, __fmaf_rn(N.y, pd.dy, __fmul_rn(N.x, pd.dx)));
    const float a2 = __fmaf_rn(-beta, beta, pd.d2);
    const float alpha = __fsqrt_rn(a2 > 0.0f ? a2 : 0.0f);
    const float u = __fsub_rn(k.halfW, __fdiv_rn(beta, k.B));
    const float v = __fdiv_rn(alpha, k.B);
    const float kr = ceilf(u), lc = ceilf(v);
    const bool in = live & (ca >= k.cosS) & (kr >= 0.0f) & (kr <= k.umax) & (lc >= 0.0f) & (lc <= k.umax);
    if (PROBE) {
        if (in) atomicAdd(pc_s, 1);
        if (live & (ca >= k.cosS)) atomicAdd(pc_s + 96, 1);  // live is the cull here: angle-passing candidates
    }
    if (in) {
        int *p = img_q + (int)kr * sh.row_words() + ((int)lc << sh.log2S());
        if (!SI_IN_BOUNDS(p >= k.img && p < k.img + k.img_words, k.flags)) return;
        atomicAdd(p, 1);
        ++cnt;
    }
}

// One warp trip: two candidates per lane, at p0 and p1 (position, normal).
template <int WT, int LS, bool PROBE, bool NB>
__device__ __forceinline__ void trip(const float4 *p0, const float4 *p1, const bool l0, const bool l1,
                                     const float4 P, const float4 N, const PairConsts &k, const Shape<WT, LS> sh,
                                     int *img_adj, int &cnt, int *pc_c, int *pc_s, unsigned *pc_h) {
    const float4 X0 = p0[0], X1 = p1[0];
    // |d|^2: the nearest-bin count's spelled-out alpha and the probes' cull need it
    constexpr bool kD2 = PROBE || NB;
    const PairDist d0 = pair_dist<kD2>(X0, P), d1 = pair_dist<kD2>(X1, P);
    const bool near0 = l0 & (d0.d2 <= k.Rc2), near1 = l1 & (d1.d2 <= k.Rc2);
    if (PROBE) {
        if (near0) {
            atomicAdd(pc_c, 1);
            atomicAdd(pc_h, fmix32(__float_as_uint(X0.w)));
        }
        if (near1) {
            atomicAdd(pc_c, 1);
            atomicAdd(pc_h, fmix32(__float_as_uint(X1.w)));
        }
    }
    const float4 N0 = p0[1], N1 = p1[1];
    if constexpr (NB) {
        // img_adj is the slot's pixel (0, 0) for the nearest-bin count
        eval_pair_nearest<WT, LS, PROBE>(d0, N0, near0, N, k, sh, img_adj, cnt, pc_s);
        eval_pair_nearest<WT, LS, PROBE>(d1, N1, near1, N, k, sh, img_adj, cnt, pc_s);
    } else {
        eval_pair<WT, LS, PROBE>(d0, N0, l0, N, k, sh, img_adj, cnt, pc_s);
        eval_pair<WT, LS, PROBE>(d1, N1, l1, N, k, sh, img_adj, cnt, pc_s);
    }
}

// Whether a full tile (TN candidates) of this shape takes a path without
// per-lane range checks: compile-time shapes only.
template <int WT, int LS, int NCONS, int TN>
constexpr bool has_full_path() {
    return WT > 0 && TN > 0 && TN % (2 * (NCONS == kWarps ? NCONS : 1) * (32 >> LS)) == 0;
}

// Consumes one staged tile: every lane pairs its slot's query with its
// candidates; two candidates per lane per trip.  With FULL the tile holds
// TN candidates and every trip is in range:
//  * all warps consuming (NCONS == kWarps): warp w takes trips at candidate
//    w*cpw + 2*NCONS*cpw*t (a compile-time count, unrolled);
//  * NCONS consumer warps: trip t covers candidates [2*cpw*t, 2*cpw*(t+1)),
//    dealt round-robin (unrolled when every warp gets the same number of
//    trips, which the producer-ring tile sizes are chosen for).
template <int WT, int LS, bool PROBE, bool NB, int NCONS, int TN, bool FULL>
__device__ __forceinline__ void consume_tile(const float4 *__restrict__ tile, const int len, const int warp,
                                             const int lane, const bool active, const float4 P, const float4 N,
                                             const PairConsts &k, const Shape<WT, LS> sh, int *img_adj, int &cnt,
                                             int *pc_c, int *pc_s, unsigned *pc_h) {
    const int l2 = sh.log2S();
    const int cpw = 32 >> l2;      // candidates per warp step
    const int sub = lane >> l2;
    const int stride = NCONS * cpw;
    if constexpr (FULL && NCONS == kWarps) {
        constexpr int kStride = NCONS * (32 >> LS);
        constexpr int kTrips = TN / (2 * kStride);
        const float4 *t0 = tile + 2 * (warp * cpw + sub);
#pragma unroll
        for (int tr = 0; tr < kTrips; ++tr)
            trip<WT, LS, PROBE, NB>(t0 + 4 * tr * kStride, t0 + 4 * tr * kStride + 2 * kStride, active, active, P, N,
                                k, sh, img_adj, cnt, pc_c, pc_s, pc_h);
    } else if constexpr (FULL) {
        constexpr int kCpw = 32 >> LS;
        constexpr int kTrips = TN / (2 * kCpw);
        const float4 *t0 = tile + 2 * sub;
        if constexpr (kTrips % NCONS == 0) {
#pragma unroll
            for (int i = 0; i < kTrips / NCONS; ++i) {
                const int tr = warp + i * NCONS;
                trip<WT, LS, PROBE, NB>(t0 + 4 * tr * kCpw, t0 + 4 * tr * kCpw + 2 * kCpw, active, active, P, N, k,
                                        sh, img_adj, cnt, pc_c, pc_s, pc_h);
            }
        } else {
            for (int tr = warp; tr < kTrips; tr += NCONS)
                trip<WT, LS, PROBE, NB>(t0 + 4 * tr * kCpw, t0 + 4 * tr * kCpw + 2 * kCpw, active, active, P, N, k,
                                        sh, img_adj, cnt, pc_c, pc_s, pc_h);
        }
    } else {
        for (int cb = warp * cpw; cb < len; cb += 2 * stride) {
            const int c0 = cb + sub, c1 = cb + stride + sub;
            const bool l0 = active & (c0 < len), l1 = active & (c1 < len);
            const int i0 = l0 ? c0 : 0, i1 = l1 ? c1 : 0;
            trip<WT, LS, PROBE, NB>(tile + 2 * i0, tile + 2 * i1, l0, l1, P, N, k, sh, img_adj, cnt, pc_c, pc_s, pc_h);
        }
    }
}

// Consumes a tile, through the range-check-free path when it holds TN
// candidates (TN = 0: shapes known only at run time, no such path).
template <int WT, int LS, bool PROBE, bool NB, int NCONS, int TN>
__device__ __forceinline__ void consume_any(const float4 *__restrict__ tile, const int len, const int warp,
                                            const int lane, const bool active, const float4 P, const float4 N,
                                            const PairConsts &k, const Shape<WT, LS> sh, int *img_adj, int &cnt,
                                            int *pc_c, int *pc_s, unsigned *pc_h) {
    if constexpr (has_full_path<WT, LS, NCONS, TN>()) {
        if (len == TN) {
            consume_tile<WT, LS, PROBE, NB, NCONS, TN, true>(tile, len, warp, lane, active, P, N, k, sh, img_adj, cnt, pc_c,
                                                     pc_s, pc_h);
            return;
        }
    }
    consume_tile<WT, LS, PROBE, NB, NCONS, TN, false>(tile, len, warp, lane, active, P, N, k, sh, img_adj, cnt, pc_c, pc_s,
                                              pc_h);
}

struct SmemView {
    Header *H;
    QueryInfo *Q;
    int *row_start, *row_len, *row_off;
    int *pc_culled, *pc_support, *pc_examined, *pc_angle;
    unsigned *pc_hash;
    float4 *tiles;
    uint32_t dyn_bytes;  // dynamic shared memory of the launch
};

// Row and offset of flat candidate position `first` in a row list with
// exclusive offsets row_off[0..nr): the last row starting at or before it.
__device__ __forceinline__ void row_cursor(const int *row_off, int nr, int first, int &cr, int &co) {
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= first)
            lo = mid;
        else
            hi = mid - 1;
    }
    cr = lo;
    co = first - row_off[lo];
}

// Generates the images of one unit u of item `it` (a group, or one slice of
// a group's candidate stream).  Returns false when a bounded wait gave up
// (the block then stops).
template <int WT, int LS, bool PROBE, bool PMODE, bool NB = false>
__device__ bool process_group(const ItemDesc &it, const int u, const int step, const SmemView &sv,
                              uint32_t &phase_bits) {
    Header &H = *sv.H;
    QueryInfo *Q = sv.Q;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const Shape<WT, LS> sh{it.W, it.log2S};
    const int S = sh.S(), W = sh.W(), W1 = W + 1;
    const int64_t m = it.m;
    const float4 *__restrict__ pn = it.pn;
    const int *__restrict__ cstart = it.cell_start;
    const GridGeom &gg = *it.geom;
    const float ox = gg.origin[0], oy = gg.origin[1], oz = gg.origin[2];
    const float cell = gg.cell_len, inv = gg.inv_cell;
    const int dx_ = gg.dims[0], dy_ = gg.dims[1], dz_ = gg.dims[2];
    PairConsts k{it.Rc2, it.cosS, it.invB, it.halfW, it.umax, it.B, nullptr, 0, it.flags};
    const float Rc = it.Rc;
    const float margin = stencil_margin(gg, Rc);
    const int slot = lane & (S - 1);
    // candidates per tile: a compile-time constant for the specialised shapes
    constexpr int TNC = WT > 0 ? tile_for_shape(WT, LS) : 0;
    const int TN = WT > 0 ? TNC : tile_for_shape(W, sh.log2S());
    int *const img = reinterpret_cast<int *>(sv.tiles + (size_t)kStages * TN * 2);
    if ((uint32_t)shape_smem(W, sh.log2S(), TN) > sv.dyn_bytes) {
        // the launch's shared memory does not hold this shape (an internal error)
        if (tid == 0) atomicOr(it.flags, kFlagLaunch);
        return true;
    }
    const int img_words_pad = ((S * W1 * W1) + 3) & ~3;
    k.img = img;
    k.img_words = img_words_pad;

    // unit u = slice `sl` of group `g`: with K slices per group, K blocks share
    // the group's candidate stream and add their partial images into `out`
    // (with a cost order, loop position gi holds group gorder[gi])
    const int K = it.slices > 1 ? it.slices : 1;
    const int gi = K == 1 ? u : u / K;
    const int sl = K == 1 ? 0 : u - gi * K;
    const int g = it.gorder ? it.gorder[gi] : gi;
    const int64_t t0 = (int64_t)g * S;
    const int nq = (int)(m - t0 < (int64_t)S ? m - t0 : (int64_t)S);
    if (K > 1 && tid < 32) H.slot_cnt[tid] = 0;
    // ---- queries of the group
    if (tid < S) {
        if (tid < nq) {
            const int64_t t = t0 + tid;
            int q;
            bool ok;
            int sp = query_sorted_pos(it, t, q, ok);
            if (!ok) atomicOr(it.flags, kFlagBadQuery);
            if (!SI_IN_BOUNDS((unsigned)sp < (unsigned)it.n_points, it.flags)) sp = 0;
            Q[tid].p = pn[2 * (int64_t)sp];
            Q[tid].n = pn[2 * (int64_t)sp + 1];
            Q[tid].slot = ok ? q : -1;
        } else {
            Q[tid].slot = -1;
        }
    }
    if (PROBE && tid < 32) {
        sv.pc_culled[tid] = 0;
        sv.pc_support[tid] = 0;
        sv.pc_hash[tid] = 0;
        sv.pc_examined[tid] = 0;
        sv.pc_angle[tid] = 0;
    }
    {
        int4 *z4 = reinterpret_cast<int4 *>(img);
        for (int w = tid; w < img_words_pad / 4; w += kThreads) z4[w] = make_int4(0, 0, 0, 0);
    }
    __syncthreads();
    // ---- bounding box of the group and the stencil's y/z cell range
    if (warp == 0) {
        float lo0 = INFINITY, lo1 = INFINITY, lo2 = INFINITY;
        float hi0 = -INFINITY, hi1 = -INFINITY, hi2 = -INFINITY;
        if (lane < nq) {
            const float4 p = Q[lane].p;
            lo0 = hi0 = p.x;
            lo1 = hi1 = p.y;
            lo2 = hi2 = p.z;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, d));
            lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, d));
            lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, d));
            hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, d));
            hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, d));
            hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, d));
        }
        if (lane == 0) {
            H.gmin[0] = lo0;
            H.gmin[1] = lo1;
            H.gmin[2] = lo2;
            H.gmax[0] = hi0;
            H.gmax[1] = hi1;
            H.gmax[2] = hi2;
            stencil_yz(oy, oz, inv, dy_, dz_, lo1, lo2, hi1, hi2, Rc, margin, H.ylo, H.yhi, H.zlo, H.zhi);
        }
    }
    __syncthreads();
    const float4 qP = Q[slot].p;
    const float4 qN = Q[slot].n;
    const bool active = slot < nq;
    int cnt = 0;
    // bilinear: pixel (0, 0) of the slot moved back by the coordinates' exponent
    // bias; nearest bin: pixel (0, 0) itself
    int *img_adj = NB ? img + slot : img + slot - kMagicHi * (sh.row_words() + S);
    const int ylo = H.ylo, zlo = H.zlo;
    const int ny = H.yhi - ylo + 1, nz = H.zhi - zlo + 1;
    const int nrows_total = ny * nz;
    bool ok_all = true;

    for (int rb = 0; rb < nrows_total && ok_all; rb += kMaxRows) {
        const int nr = min(kMaxRows, nrows_total - rb);
        // ---- candidate rows: for each (z, y) the x range of cells within Rc
        for (int r = tid; r < nr; r += kThreads) {
            const int rr = rb + r;
            const int y = ylo + rr % ny, z = zlo + rr / ny;
            int c0 = 0;
            const int ncx = stencil_row(ox, oy, oz, cell, inv, dx_, dy_, H.gmin, H.gmax, k.Rc2, margin, y, z, c0);
            int start = 0, len = 0;
            if (ncx > 0 && SI_IN_BOUNDS(c0 >= 0 && c0 + ncx <= gg.ncell, it.flags)) {
                start = cstart[c0];
                len = cstart[c0 + ncx] - start;
            }
            sv.row_start[r] = start;
            sv.row_len[r] = len;
        }
        __syncthreads();
        const int total = block_scan_rows(sv.row_len, sv.row_off, nr, H);
        const int ntiles = (total + TN - 1) / TN;
        // this unit's share of the tiles: [tlo, tlo + nt)
        const int tlo = (int)((int64_t)ntiles * sl / K);
        const int nt = (int)((int64_t)ntiles * (sl + 1) / K) - tlo;
        if constexpr (PMODE) {
        volatile int *abort_flag = &H.abort_flag;
        if (warp == kWarps - 1) {
            // ---- producer warp: fills every tile in order with a running row cursor,
            // reusing a stage once all consumer warps have released its last tile
            if (lane == 0) {
                int cr = 0, co = 0;
                if (nt > 0) row_cursor(sv.row_off, nr, tlo * TN, cr, co);
                for (int tt = 0; tt < nt; ++tt) {
                    const int b = tt % kStages;
                    const int t = tlo + tt;
                    const int j = H.pfills[b];
                    if (j > 0) {
                        const uint32_t par = (uint32_t)(j - 1) & 1u;
                        bool ok = mbar_try_wait(&H.empty[b], par);
                        const uint64_t t_start = global_ns();
                        while (!ok && !*abort_flag && global_ns() - t_start <= kWaitLimitNs)
                            ok = mbar_try_wait(&H.empty[b], par);
                        if (!ok) {
                            atomicOr(&H.abort_flag, 1);
                            break;
                        }
                    }
                    const int need = min(TN, total - t * TN);
                    float4 *dst = sv.tiles + (size_t)b * TN * 2;
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&H.bar[b], (uint32_t)need * 32u);
                    int done = 0;
                    while (done < need && cr < nr) {
                        const int avail = sv.row_len[cr] - co;
                        if (avail <= 0) {
                            ++cr;
                            co = 0;
                            continue;
                        }
                        const int take = min(need - done, avail);
                        int src0 = sv.row_start[cr] + co;
                        if (!SI_IN_BOUNDS(done + take <= TN && src0 >= 0 && src0 + take <= it.n_points, it.flags))
                            src0 = 0;  // keep the copy (its bytes complete the stage) inside the mesh
                        bulk_copy_g2s(dst + 2 * done, pn + 2 * (int64_t)src0, (uint32_t)take * 32u, &H.bar[b]);
                        done += take;
                        co += take;
                    }
                    H.pfills[b] = j + 1;
                    H.fills[b] += 1;
                }
            }
            __syncwarp();
            // keep this warp's view of the full-barrier phases in step with the consumers
            if (!*abort_flag)
                for (int tt = 0; tt < nt; ++tt) phase_bits ^= 1u << (tt % kStages);
        } else {
            // ---- consumer warps
            for (int tt = 0; tt < nt; ++tt) {
                const int b = tt % kStages;
                const int t = tlo + tt;
                const uint32_t par = (phase_bits >> b) & 1u;
                bool ok = mbar_try_wait(&H.bar[b], par);
                if (!ok) {
                    const uint64_t t_start = global_ns();
                    while (!ok && !*abort_flag && global_ns() - t_start <= kWaitLimitNs)
                        ok = mbar_try_wait(&H.bar[b], par);
                }
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) atomicOr(&H.abort_flag, 1);
                    break;
                }
                phase_bits ^= 1u << b;
                const int len = min(TN, total - t * TN);
                if (PROBE && tid < nq) sv.pc_examined[tid] += len;
                consume_any<WT, LS, PROBE, NB, kProdConsumers, TNC>(sv.tiles + (size_t)b * TN * 2, len, warp, lane,
                                                           active, qP, qN, k, sh, img_adj, cnt, sv.pc_culled + slot,
                                                           sv.pc_support + slot, sv.pc_hash + slot);
                __syncwarp();
                if (lane == 0) mbar_arrive(&H.empty[b]);
            }
        }
        __syncthreads();
        if (*abort_flag) ok_all = false;
        __syncthreads();
        } else {
        // ---- producer state (thread 0): row cursor
        if (tid == 0) {
            int cr0 = 0, co0 = 0;
            if (nt > 0) row_cursor(sv.row_off, nr, tlo * TN, cr0, co0);
            H.cur_r = cr0;
            H.cur_o = co0;
        }
        auto fill = [&](int tt) {
            int cr = H.cur_r, co = H.cur_o;
            const int b = tt % kStages;
            const int t = tlo + tt;
            const int need = min(TN, total - t * TN);
            float4 *dst = sv.tiles + (size_t)b * TN * 2;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&H.bar[b], (uint32_t)need * 32u);
            int done = 0;
            while (done < need && cr < nr) {
                const int avail = sv.row_len[cr] - co;
                if (avail <= 0) {
                    ++cr;
                    co = 0;
                    continue;
                }
                const int take = min(need - done, avail);
                int src0 = sv.row_start[cr] + co;
                if (!SI_IN_BOUNDS(done + take <= TN && src0 >= 0 && src0 + take <= it.n_points, it.flags))
                    src0 = 0;  // keep the copy (its bytes complete the stage) inside the mesh
                bulk_copy_g2s(dst + 2 * done, pn + 2 * (int64_t)src0, (uint32_t)take * 32u, &H.bar[b]);
                done += take;
                co += take;
            }
            H.cur_r = cr;
            H.cur_o = co;
            H.fills[b] += 1;
        };
        if (tid == 0) {
            for (int tt = 0; tt < kStages && tt < nt; ++tt) fill(tt);
        }
        for (int tt = 0; tt < nt; ++tt) {
            const int b = tt % kStages;
            const bool ok = mbar_wait_bounded(&H.bar[b], (phase_bits >> b) & 1u, kWaitLimitNs);
            if (ok) {
                phase_bits ^= 1u << b;
                const int len = min(TN, total - (tlo + tt) * TN);
                if (PROBE && tid < nq) sv.pc_examined[tid] += len;
                consume_any<WT, LS, PROBE, NB, kWarps, TNC>(sv.tiles + (size_t)b * TN * 2, len, warp, lane, active, qP,
                                                   qN, k, sh, img_adj, cnt, sv.pc_culled + slot, sv.pc_support + slot,
                                                   sv.pc_hash + slot);
            }
            if (__syncthreads_or(!ok)) {
                ok_all = false;
                break;
            }
            if (tid == 0 && tt + kStages < nt) fill(tt + kStages);
        }
        }
    }
    if (!ok_all) {
        if (tid == 0) {
            atomicOr(it.flags, kFlagTimeout);
            // drain this block's copies still in flight before leaving
            for (int b = 0; b < kStages; ++b)
                if (H.fills[b] > 0) mbar_wait_bounded(&H.bar[b], (uint32_t)(H.fills[b] - 1) & 1u, kWaitLimitNs);
        }
        return false;
    }
    __syncthreads();
    // ---- write-out: pixel (i, j) of slot q lives at ((i*(W+1) + j) * S + q).
    // A thread moves up to four images of one pixel with one shared read; the
    // threads of a warp take consecutive quads of a pixel, then consecutive
    // pixels, so the shared reads stay conflict-free and each warp store
    // writes min(32, 128 / S) consecutive pixels of each image it touches:
    // whole 32-byte sectors for groups of up to 16 images, half sectors for
    // 32 (a partial sector costs a transfer of its own when the output is host
    // memory).
    long long pix = 0;
    const int npix = W * W;
    int32_t *__restrict__ out = it.out;
    const int lv = sh.log2S() < 2 ? sh.log2S() : 2;  // log2 of the images per read
    const int lq = sh.log2S() - lv;                   // log2 of the reads per pixel
    const int nvq = (nq + (1 << lv) - 1) >> lv;       // reads per pixel that hold live images
    for (int e = tid; e < (npix << lq); e += kThreads) {
        const int c = e & ((1 << lq) - 1);
        if (c >= nvq) continue;
        const int p = e >> lq;
        const int i = p / W, j = p - i * W;
        const int *src = img + (i * W1 + j) * S + (c << lv);
        int v[4];
        if (lv == 2) {
            const int4 x = *reinterpret_cast<const int4 *>(src);
            v[0] = x.x, v[1] = x.y, v[2] = x.z, v[3] = x.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = k < (1 << lv) ? src[k] : 0;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int q = (c << lv) + k;
            if (k >= (1 << lv) || q >= nq) continue;
            const int qs = Q[q].slot;
            if (qs >= 0 && SI_IN_BOUNDS(qs < m && p < npix, it.flags)) {
                if (K == 1)
                    __stcs(out + (int64_t)qs * npix + p, v[k]);
                else if (v[k] != 0)
                    atomicAdd(out + (int64_t)qs * npix + p, v[k]);  // partial image of one slice
            }
            pix += v[k];
        }
    }
    if (K > 1) {
        // contributing pairs per image, summed over slices for the exact
        // overflow check that runs after the kernel
        if (active && cnt) atomicAdd(&H.slot_cnt[slot], cnt);
        __syncthreads();
        if (tid < nq && Q[tid].slot >= 0 && H.slot_cnt[tid]) atomicAdd(&it.counts[Q[tid].slot], H.slot_cnt[tid]);
    }
    // ---- exact overflow check of the group: the written pixels (int32 read
    // as signed) sum to 65536 x pairs unless a pixel wrapped
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        pix += __shfl_xor_sync(0xffffffffu, pix, d);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, d);
    }
    if (lane == 0) {
        atomicAdd(&H.grp_pix, (unsigned long long)pix);
        atomicAdd(&H.grp_weight, (unsigned long long)cnt * (NB ? 1ull : 65536ull));
    }
    if (PROBE && tid < nq && Q[tid].slot >= 0) {
        const int q = Q[tid].slot;
        if (it.p_culled) it.p_culled[q] = sv.pc_culled[tid];
        if (it.p_hash) it.p_hash[q] = sv.pc_hash[tid];
        if (it.p_support) it.p_support[q] = sv.pc_support[tid];
        if (it.p_worker) it.p_worker[q] = (int)blockIdx.x;
        if (it.p_examined) it.p_examined[q] = sv.pc_examined[tid];
        if (it.p_angle) it.p_angle[q] = sv.pc_angle[tid];
        if (it.p_step) it.p_step[q] = step;
    }
    __syncthreads();
    if (tid == 0) {
        if (H.grp_pix != H.grp_weight) atomicOr(it.flags, kFlagOverflow);
        H.grp_pix = 0;
        H.grp_weight = 0;
    }
    return true;
}

// Adaptive weighted factoring, the request half of getChunk run on the device
// by thread 0 of a worker: fold the chunk just finished into the worker's
// rate, take the batch chunk (FAC2 on the units that remain, the first batch
// at half size), scale it by the worker's weight (its rate over the mean of
// the measured rates) and take that many units from the shared cursor.  Sets H.claim (the claim index), H.awf_lo and
// H.awf_hi.
__device__ void awf_claim(const LaunchArgs &a, Header &H, const int claim_iter, const bool first_slow) {
    const uint64_t now = global_ns();
    if (claim_iter > 0 && H.awf_last > 0) {
        H.awf_units += (double)H.awf_last;
        H.awf_ns += (double)(now - H.awf_t0);
        const double rate = H.awf_units / fmax(H.awf_ns, 1.0);
        atomicAdd(&a.ctr->awf_rate_sum, rate - H.awf_rate);
        if (H.awf_rate == 0.0) atomicAdd(&a.ctr->awf_rated, 1u);
        H.awf_rate = rate;
    }
    // slow workers (heterogeneity emulation) request first: claim k is slow worker k's
    const unsigned long long s =
        first_slow ? (unsigned long long)blockIdx.x
                   : (unsigned long long)a.slow_workers + atomicAdd(&a.ctr->awf_claims, 1ull);
    const unsigned long long j = s / gridDim.x;
    // the batch chunk: FAC2 on what remains now, ceil(R / (2P)); the first batch
    // (claims 0 .. P-1, made before any rate exists) at half that, so a slow
    // worker's first chunk cannot set the makespan on its own
    const unsigned long long cur = *(volatile unsigned long long *)&a.ctr->awf_next;
    const long long rem = cur >= (unsigned long long)a.total_units ? 0 : (long long)a.total_units - (long long)cur;
    const long long div = 2ll * gridDim.x * (j == 0 ? 2 : 1);
    const int batch = (int)max((long long)a.min_chunk, (rem + div - 1) / div);
    double w = 1.0;
    const unsigned rated = *(volatile unsigned *)&a.ctr->awf_rated;
    const double sum = *(volatile double *)&a.ctr->awf_rate_sum;
    if (H.awf_rate > 0.0 && rated > 0 && sum > 0.0) w = fmin(fmax(H.awf_rate * (double)rated / sum, 0.05), 20.0);
    const int chunk = max(a.min_chunk, (int)(w * (double)batch + 0.5));
    const unsigned long long lo = atomicAdd(&a.ctr->awf_next, (unsigned long long)chunk);
    const int total = a.total_units;
    H.awf_lo = lo >= (unsigned long long)total ? total : (int)lo;
    H.awf_hi = lo >= (unsigned long long)total ? total : (int)min(lo + (unsigned long long)chunk,
                                                                   (unsigned long long)total);
    H.awf_last = H.awf_hi - H.awf_lo;
    H.awf_t0 = now;
    H.claim = (int)s;
}

// ---- cost order of the groups (si_schedule.order = 1)

// One warp per group of the concatenated group space: the group's stencil
// (its queries' bounding box, the rows and their cell ranges, exactly as
// process_group builds it) and the number of candidates it streams, bucketed
// as round(32 log2(candidates)) and stored as kCostBuckets - 1 - bucket, so
// that an ascending pass over the keys visits the costliest groups first.
__global__ void group_cost_kernel(const ItemDesc *__restrict__ items, const int *__restrict__ ord_items,
                                  const int *__restrict__ gbase, int n_ord, int total_groups, uint16_t *key,
                                  int *hist) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int G = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; G < total_groups; G += warps) {
        int lo = 0, hi = n_ord - 1;  // the ordered item whose range holds G
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (gbase[mid] <= G)
                lo = mid;
            else
                hi = mid - 1;
        }
        const ItemDesc &it = items[ord_items[lo]];
        const int g = G - gbase[lo];
        const int S = 1 << it.log2S;
        const int64_t t0 = (int64_t)g * S;
        const int nq = (int)(it.m - t0 < (int64_t)S ? it.m - t0 : (int64_t)S);
        float lo0 = INFINITY, lo1 = INFINITY, lo2 = INFINITY, hi0 = -INFINITY, hi1 = -INFINITY, hi2 = -INFINITY;
        if (lane < nq) {
            int q;
            bool ok;
            int sp = query_sorted_pos(it, t0 + lane, q, ok);
            if ((unsigned)sp >= (unsigned)it.n_points) sp = 0;
            const float4 p = it.pn[2 * (int64_t)sp];
            lo0 = hi0 = p.x;
            lo1 = hi1 = p.y;
            lo2 = hi2 = p.z;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            lo0 = fminf(lo0, __shfl_xor_sync(0xffffffffu, lo0, d));
            lo1 = fminf(lo1, __shfl_xor_sync(0xffffffffu, lo1, d));
            lo2 = fminf(lo2, __shfl_xor_sync(0xffffffffu, lo2, d));
            hi0 = fmaxf(hi0, __shfl_xor_sync(0xffffffffu, hi0, d));
            hi1 = fmaxf(hi1, __shfl_xor_sync(0xffffffffu, hi1, d));
            hi2 = fmaxf(hi2, __shfl_xor_sync(0xffffffffu, hi2, d));
        }
        const GridGeom &gg = *it.geom;
        const float ox = gg.origin[0], oy = gg.origin[1], oz = gg.origin[2];
        const float cell = gg.cell_len, inv = gg.inv_cell;
        const int dx_ = gg.dims[0], dy_ = gg.dims[1], dz_ = gg.dims[2];
        const float margin = stencil_margin(gg, it.Rc);
        int ylo, yhi, zlo, zhi;
        stencil_yz(oy, oz, inv, dy_, dz_, lo1, lo2, hi1, hi2, it.Rc, margin, ylo, yhi, zlo, zhi);
        const float gmin[3] = {lo0, lo1, lo2}, gmax[3] = {hi0, hi1, hi2};
        const int ny = yhi - ylo + 1, nrows = ny * (zhi - zlo + 1);
        long long cand = 0;
        for (int r = lane; r < nrows; r += 32) {
            const int y = ylo + r % ny, z = zlo + r / ny;
            int c0 = 0;
            const int ncx = stencil_row(ox, oy, oz, cell, inv, dx_, dy_, gmin, gmax, it.Rc2, margin, y, z, c0);
            if (ncx > 0 && c0 >= 0 && c0 + ncx <= gg.ncell) cand += it.cell_start[c0 + ncx] - it.cell_start[c0];
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) cand += __shfl_xor_sync(0xffffffffu, cand, d);
        if (lane == 0) {
            const int b = cand > 0 ? min(kCostBuckets - 1, __float2int_rn(32.0f * __log2f((float)cand))) : 0;
            const int kb = kCostBuckets - 1 - b;
            key[G] = (uint16_t)kb;
            atomicAdd(hist + (int64_t)lo * kCostBuckets + kb, 1);
        }
    }
}

// One block per ordered item: the exclusive scan of its bucket counts, offset
// by the item's first group, in place.
__global__ void group_cost_scan_kernel(const int *__restrict__ gbase, int *hist) {
    __shared__ int part[kCostBuckets];
    int *h = hist + (int64_t)blockIdx.x * kCostBuckets;
    const int t = threadIdx.x;  // blockDim.x == kCostBuckets
    part[t] = h[t];
    __syncthreads();
    for (int d = 1; d < kCostBuckets; d <<= 1) {
        const int v = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    h[t] = gbase[blockIdx.x] + part[t] - h[t];
}

// One thread per group: its rank in decreasing cost order (groups of one
// bucket in the order they claim it), dealt over the chunks of its deal
// batch, gives its loop position.
__global__ void group_cost_scatter_kernel(const int *__restrict__ gbase, const int *__restrict__ dbase,
                                          const int *__restrict__ deal, int n_ord, int total_groups,
                                          const uint16_t *__restrict__ key, int *hist, int *gorder) {
    for (int G = blockIdx.x * blockDim.x + threadIdx.x; G < total_groups; G += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_ord - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (gbase[mid] <= G)
                lo = mid;
            else
                hi = mid - 1;
        }
        const int r = atomicAdd(hist + (int64_t)lo * kCostBuckets + key[G], 1) - gbase[lo];
        int pos = r;
        for (int b = dbase[lo]; b < dbase[lo + 1]; ++b) {
            const int s0 = deal[3 * b], nc = deal[3 * b + 1], c = deal[3 * b + 2];
            if (r >= s0 && r - s0 < nc * c) {
                const int off = r - s0;
                pos = s0 + (off % nc) * c + off / nc;
                break;
            }
        }
        gorder[gbase[lo] + pos] = G - gbase[lo];
    }
}

// Adaptive factoring (Banicescu and Liu's AF rule), the request half of
// getChunk run on the device by thread 0 of a worker.  The chunk just
// finished is folded into the worker's statistics of its per-unit time: each
// unit time is scaled by the chunk's wall time over its summed unit times, so
// the claim overhead and a slow worker's idle count as the worker's own.  The
// worker then publishes sigma^2 / mu and 1 / mu into launch-wide sums and takes
//   x_i = (D + 2 E R - sqrt(D^2 + 4 D E R)) / (2 mu_i),
//   D = sum_j sigma_j^2 / mu_j,  E = 1 / sum_j 1 / mu_j,
// units, R being the units that remain; the sums run over the workers
// measured so far, scaled to all P.  x_i mu_i = T is the smaller root of
// T + sqrt(D T) = E R: the chunk's expected time plus a deviation allowance
// equals a worker's share of what remains.  Before a worker has measured a
// chunk (and before any worker has) it takes AWF's first chunk, half of
// FAC2's, ceil(R / (4P)).  Chunks are at least min_chunk.  Sets H.claim,
// H.awf_lo and H.awf_hi.
__device__ void af_claim(const LaunchArgs &a, Header &H, const int claim_iter, const bool first_slow) {
    const uint64_t now = global_ns();
    AfWorker &w = a.af_workers[blockIdx.x];
    if (claim_iter > 0 && w.cn > 0) {
        const double wall = (double)(now - H.awf_t0);
        const double f = w.cs > 0.0 ? fmax(wall / w.cs, 1.0) : 1.0;
        w.sum += f * w.cs;
        w.sumsq += f * f * w.cs2;
        w.n += w.cn;
        w.cs = 0.0;
        w.cs2 = 0.0;
        w.cn = 0;
        const double mu = fmax(w.sum / (double)w.n, 1.0);
        const double var =
            w.n > 1 ? fmax(w.sumsq / (double)w.n - mu * mu, 0.0) * ((double)w.n / (double)(w.n - 1)) : 0.0;
        const double d = var / mu, e = 1.0 / mu;
        atomicAdd(&a.ctr->af_d_sum, d - w.d);
        atomicAdd(&a.ctr->af_e_sum, e - w.e);
        if (w.e == 0.0) atomicAdd(&a.ctr->awf_rated, 1u);
        w.d = d;
        w.e = e;
    }
    const unsigned long long s =
        first_slow ? (unsigned long long)blockIdx.x
                   : (unsigned long long)a.slow_workers + atomicAdd(&a.ctr->awf_claims, 1ull);
    const unsigned long long cur = *(volatile unsigned long long *)&a.ctr->awf_next;
    const long long rem = cur >= (unsigned long long)a.total_units ? 0 : (long long)a.total_units - (long long)cur;
    const double P = (double)gridDim.x;
    long long chunk;
    const unsigned rated = *(volatile unsigned *)&a.ctr->awf_rated;
    const double dsum = *(volatile double *)&a.ctr->af_d_sum, esum = *(volatile double *)&a.ctr->af_e_sum;
    if (w.e > 0.0 && rated > 0 && esum > 0.0) {
        const double scale = P / (double)rated;
        const double D = fmax(dsum, 0.0) * scale, E = 1.0 / (esum * scale), R = (double)rem;
        const double x = (D + 2.0 * E * R - sqrt(D * D + 4.0 * D * E * R)) / (2.0 / w.e);
        chunk = (long long)ceil(fmax(x, 0.0));
    } else {
        const long long div = 4ll * gridDim.x;
        chunk = (rem + div - 1) / div;
    }
    chunk = max((long long)a.min_chunk, min(chunk, max(rem, 1ll)));
    const unsigned long long lo = atomicAdd(&a.ctr->awf_next, (unsigned long long)chunk);
    const int total = a.total_units;
    H.awf_lo = lo >= (unsigned long long)total ? total : (int)lo;
    H.awf_hi = lo >= (unsigned long long)total ? total : (int)min(lo + (unsigned long long)chunk,
                                                                   (unsigned long long)total);
    H.awf_last = H.awf_hi - H.awf_lo;
    H.awf_t0 = now;
    H.claim = (int)s;
}

// MODES: the paths compiled in (kModeBarrier | kModeProducer | kModeNearest),
// plus kModeWide for a mixed launch that runs two blocks per SM;
// a launch whose groups all use one discipline runs the instance without the
// other, whose registers are then allocated for its own loop alone.  Groups
// in producer mode hold >= 67 KB of images, so at most two blocks fit on an
// SM: that instance may use the registers of two blocks.
template <int MODES>
constexpr int min_blocks_for() {
    return MODES == kModeProducer || (MODES & kModeWide) ? 2 : SI_MIN_BLOCKS;
}

template <bool PROBE, int MODES>
__global__ void __launch_bounds__(kThreads, min_blocks_for<MODES>()) spin_kernel(LaunchArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    SmemView sv;
    sv.H = reinterpret_cast<Header *>(smem);
    sv.Q = reinterpret_cast<QueryInfo *>(smem + off_query());
    sv.row_start = reinterpret_cast<int *>(smem + off_rows());
    sv.row_len = sv.row_start + (kMaxRows + 4);
    sv.row_off = sv.row_len + (kMaxRows + 4);
    sv.pc_culled = reinterpret_cast<int *>(smem + off_probe());
    sv.pc_support = sv.pc_culled + 32;
    sv.pc_hash = reinterpret_cast<unsigned *>(sv.pc_support + 32);
    sv.pc_examined = sv.pc_support + 64;
    sv.pc_angle = sv.pc_support + 96;  // probe counters: the slot's support counter + 96
    sv.tiles = reinterpret_cast<float4 *>(smem + off_tiles());
    Header &H = *sv.H;
    const int tid = threadIdx.x;

    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(sv.dyn_bytes));

    if (tid == 0) {
        for (int b = 0; b < kStages; ++b) {
            mbar_init(&H.bar[b], 1);
            mbar_init(&H.empty[b], kProdConsumers);
            H.fills[b] = 0;
            H.pfills[b] = 0;
        }
        H.abort_flag = 0;
        fence_mbar_init();
        H.grp_weight = 0;
        H.grp_pix = 0;
    }
    __syncthreads();

    uint32_t phase_bits = 0;  // expected parity per stage (every thread tracks it)
    bool alive = true;
    int claim_iter = 0;
    // heterogeneity emulation: slow blocks (index < a.slow_workers) take the
    // first steps, one each, and the shared counter hands out the steps after
    // them; H.t_step holds the start of a slow block's current step
    if (tid == 0) {
        H.awf_units = 0.0;
        H.awf_ns = 0.0;
        H.awf_rate = 0.0;
        if (a.af) a.af_workers[blockIdx.x] = AfWorker{};
    }

    // generates units [u0, u1) of item `item`; `step` is the claim they came from
    auto run = [&](const int item, const int u0, const int u1, const int step) {
        const ItemDesc &it = a.items[item];
        const int key = it.W * 8 + it.log2S;
        for (int u = u0; u < u1 && alive; ++u) {
            if (a.af && tid == 0) H.af_t_unit = global_ns();
            // specialised shapes for the common widths, a runtime one otherwise
            // (the nearest-bin count: W = 32 in groups of 16, else the runtime shape)
            if ((MODES & kModeNearest) != 0 && it.binning == SI_BIN_NEAREST) {
                if constexpr ((MODES & kModeNearest) != 0) {
                    if (key == 32 * 8 + 4)
                        alive = process_group<32, 4, PROBE, false, true>(it, u, step, sv, phase_bits);
                    else if (it.log2S <= 2)
                        alive = process_group<0, 0, PROBE, true, true>(it, u, step, sv, phase_bits);
                    else
                        alive = process_group<0, 0, PROBE, false, true>(it, u, step, sv, phase_bits);
                }
            } else if (it.log2S <= 2) {
                if constexpr ((MODES & kModeProducer) != 0) {
                    switch (key) {
                        case 64 * 8 + 1:
                            alive = process_group<64, 1, PROBE, true>(it, u, step, sv, phase_bits);
                            break;
                        case 64 * 8 + 2:
                            alive = process_group<64, 2, PROBE, true>(it, u, step, sv, phase_bits);
                            break;
                        default:
                            alive = process_group<0, 0, PROBE, true>(it, u, step, sv, phase_bits);
                            break;
                    }
                }
            } else {
                if constexpr ((MODES & kModeBarrier) != 0) {
                    switch (key) {
                        case 16 * 8 + 5:
                            alive = process_group<16, 5, PROBE, false>(it, u, step, sv, phase_bits);
                            break;
                        case 32 * 8 + 4:
                            alive = process_group<32, 4, PROBE, false>(it, u, step, sv, phase_bits);
                            break;
                        case 32 * 8 + 3:
                            alive = process_group<32, 3, PROBE, false>(it, u, step, sv, phase_bits);
                            break;
                        default:
                            alive = process_group<0, 0, PROBE, false>(it, u, step, sv, phase_bits);
                            break;
                    }
                }
            }
            if (a.af && tid == 0) {
                // process_group ends on a block barrier: the unit's work is done
                AfWorker &aw = a.af_workers[blockIdx.x];
                const double t = (double)(global_ns() - H.af_t_unit);
                aw.cs += t;
                aw.cs2 += t * t;
                ++aw.cn;
            }
        }
    };

    while (alive) {
        __syncthreads();
        if (tid == 0) {
            const bool first_slow = (int)blockIdx.x < a.slow_workers && claim_iter == 0;
            if (a.af) {
                af_claim(a, H, claim_iter, first_slow);
            } else if (a.awf) {
                awf_claim(a, H, claim_iter, first_slow);
            } else {
                int s;
                if (a.is_static)
                    s = claim_iter == 0 ? (int)blockIdx.x : a.nsteps;
                else if (first_slow)
                    s = (int)blockIdx.x;
                else
                    s = a.slow_workers + (int)atomicAdd(&a.ctr->step, 1ull);
                H.claim = s;
            }
            if ((int)blockIdx.x < a.slow_workers) H.t_step = global_ns();
            if (a.trace) H.t_trace = global_ns();
        }
        __syncthreads();
        const int step = H.claim;
        ++claim_iter;
        // the claim as ranges of one item each: the step's pieces, or (AWF) the
        // units [H.awf_lo, H.awf_hi) of the concatenated unit space
        int pi = 0, pend = 0, g = 0, ghi = 0;
        if (a.awf) {
            g = H.awf_lo;
            ghi = H.awf_hi;
            if (g >= ghi) break;
        } else {
            if (step >= a.nsteps) break;
            pi = a.step_piece[step];
            pend = a.step_piece[step + 1];
        }
        while (alive) {
            int item, u0, u1;
            if (a.awf) {
                if (g >= ghi) break;
                int lo_k = 0, hi_k = a.nitems - 1;  // the last item whose first unit is <= g
                while (lo_k < hi_k) {
                    const int mid = (lo_k + hi_k + 1) >> 1;
                    if (a.unit_base[mid] <= g)
                        lo_k = mid;
                    else
                        hi_k = mid - 1;
                }
                const int base = a.unit_base[lo_k], end = min(ghi, a.unit_base[lo_k + 1]);
                item = lo_k;
                u0 = g - base;
                u1 = end - base;
                g = end;
            } else {
                if (pi >= pend) break;
                const Piece pc = a.pieces[pi++];
                item = pc.item;
                u0 = pc.u0;
                u1 = pc.u1;
            }
            run(item, u0, u1, step);
        }
        if ((int)blockIdx.x < a.slow_workers && alive && tid == 0) {
            // a slow worker idles (slowdown - 1) x the time of its step, at most
            // kSlowIdleCapNs; the other threads wait at the next claim's barrier
            const uint64_t took = global_ns() - H.t_step;
            uint64_t idle = (uint64_t)((double)took * (double)(a.slowdown - 1.0f));
            if (idle > kSlowIdleCapNs) idle = kSlowIdleCapNs;
            const uint64_t until = global_ns() + idle;
            while (global_ns() < until) __nanosleep(2000);
        }
        if (a.trace && tid == 0 && alive) {
            // the claim's entry: worker, step, start and end of its work (a slow
            // worker's idle included: it stands for the slower processor)
            const unsigned long long e = atomicAdd(a.trace_count, 1ull);
            if ((int64_t)e < a.trace_cap) {
                int64_t *t = a.trace + 4 * (int64_t)e;
                t[0] = blockIdx.x;
                t[1] = step;
                t[2] = (int64_t)H.t_trace;
                t[3] = (int64_t)global_ns();
            }
        }
    }
    // ---- the last block to finish resets the dynamic step counter for the next launch
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned long long prev = atomicAdd(&a.ctr->done_blocks, 1ull);
        if (prev == gridDim.x - 1) {
            atomicExch(&a.ctr->step, 0ull);
            atomicExch(&a.ctr->awf_next, 0ull);
            atomicExch(&a.ctr->awf_claims, 0ull);
            atomicExch(reinterpret_cast<unsigned long long *>(&a.ctr->awf_rate_sum), 0ull);  // +0.0
            atomicExch(&a.ctr->awf_rated, 0u);
            atomicExch(reinterpret_cast<unsigned long long *>(&a.ctr->af_d_sum), 0ull);
            atomicExch(reinterpret_cast<unsigned long long *>(&a.ctr->af_e_sum), 0ull);
            atomicExch(&a.ctr->done_blocks, 0ull);
        }
    }
}

}  // namespace

size_t image_words(int W, int log2S) {
    size_t w = (size_t)(W + 1) * (W + 1) << log2S;
    return (w + 3) & ~size_t(3);
}

size_t spin_smem_bytes(int W, int log2S) { return (size_t)shape_smem(W, log2S, tile_for_shape(W, log2S)); }

constexpr int kModeAll = kModeBarrier | kModeProducer | kModeNearest;
constexpr int kModeMixedWide = kModeBarrier | kModeProducer | kModeWide;

cudaError_t setup_spin_kernel_attributes(size_t smem_bytes) {
    // the attribute belongs to each device's context: remember it per device
    constexpr int kMaxDevices = 128;
    static std::atomic<size_t> done_per_device[kMaxDevices];
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return de;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::atomic<size_t> &done_ref = done_per_device[dev];
    if (smem_bytes <= done_ref.load()) return cudaSuccess;
    const int bytes = (int)smem_bytes;
    const cudaFuncAttribute attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(spin_kernel<false, kModeBarrier | kModeProducer>, attr, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spin_kernel<false, kModeBarrier>, attr, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spin_kernel<false, kModeProducer>, attr, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spin_kernel<false, kModeMixedWide>, attr, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spin_kernel<false, kModeAll>, attr, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(spin_kernel<true, kModeAll>, attr, bytes);
    if (e == cudaSuccess) {
        size_t prev = done_ref.load();
        while (prev < smem_bytes && !done_ref.compare_exchange_weak(prev, smem_bytes)) {
        }
    }
    return e;
}

int blocks_per_sm_for(size_t smem_bytes, int modes) {
    int n = 0;
    if (setup_spin_kernel_attributes(smem_bytes) != cudaSuccess) return 0;
    cudaError_t e;
    if (modes == kModeBarrier)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, spin_kernel<false, kModeBarrier>, kThreads, smem_bytes);
    else if (modes == kModeProducer)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, spin_kernel<false, kModeProducer>, kThreads,
                                                          smem_bytes);
    else if (modes == (kModeBarrier | kModeProducer))
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, spin_kernel<false, kModeBarrier | kModeProducer>,
                                                          kThreads, smem_bytes);
    else if (modes == kModeMixedWide)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, spin_kernel<false, kModeMixedWide>, kThreads,
                                                          smem_bytes);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, spin_kernel<false, kModeAll>, kThreads, smem_bytes);
    return e == cudaSuccess ? n : 0;
}

si_status enqueue_group_order(const ItemDesc *items, const int *ord_items, const int *gbase, const int *dbase,
                              const int *deal, int n_ord, int total_groups, uint16_t *key, int *hist, int *gorder,
                              cudaStream_t st, int *kernels) {
    *kernels = 0;
    if (n_ord <= 0 || total_groups <= 0) return SI_OK;
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * (size_t)n_ord * kCostBuckets, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(cost histogram)");
    const int warp_blocks = (int)std::min<int64_t>(((int64_t)total_groups + 7) / 8, 65535);
    group_cost_kernel<<<warp_blocks, 256, 0, st>>>(items, ord_items, gbase, n_ord, total_groups, key, hist);
    group_cost_scan_kernel<<<n_ord, kCostBuckets, 0, st>>>(gbase, hist);
    const int blocks = (int)std::min<int64_t>(((int64_t)total_groups + 255) / 256, 65535);
    group_cost_scatter_kernel<<<blocks, 256, 0, st>>>(gbase, dbase, deal, n_ord, total_groups, key, hist, gorder);
    *kernels = 3;
    e = cudaGetLastError();
    return e == cudaSuccess ? SI_OK : cuda_fail(e, "group cost order");
}

void launch_spin_kernel(const LaunchArgs &a, int blocks, size_t smem, cudaStream_t stream) {
    // a.modes is launch_modes(...) of the call
    if (a.probe)
        spin_kernel<true, kModeAll><<<blocks, kThreads, smem, stream>>>(a);
    else if (a.modes == kModeBarrier)
        spin_kernel<false, kModeBarrier><<<blocks, kThreads, smem, stream>>>(a);
    else if (a.modes == kModeProducer)
        spin_kernel<false, kModeProducer><<<blocks, kThreads, smem, stream>>>(a);
    else if (a.modes == (kModeBarrier | kModeProducer))
        spin_kernel<false, kModeBarrier | kModeProducer><<<blocks, kThreads, smem, stream>>>(a);
    else if (a.modes == kModeMixedWide)
        spin_kernel<false, kModeMixedWide><<<blocks, kThreads, smem, stream>>>(a);
    else
        spin_kernel<false, kModeAll><<<blocks, kThreads, smem, stream>>>(a);
}

// Shared memory of a block that leaves room for two blocks per SM (228 KB per
// SM, of which the system reserves 1 KB per block).
constexpr size_t kTwoBlockSmem = (size_t)113 * 1024;

// Largest group (power of two, <= 32, or the requested one) whose images fit
// next to the fixed shared-memory layout within the build's per-block budget.
int choose_log2_group(int W, int requested_group) {
    if (requested_group > 0) {
        int l = 0;
        while ((1 << l) < requested_group && l < 5) ++l;
        return l;
    }
    const size_t budget = (size_t)SI_SMEM_BUDGET_KB * 1024;
    int l = 0;
    for (int c = 5; c > 0; --c)
        if (spin_smem_bytes(W, c) <= budget) {
            l = c;
            break;
        }
    // wide images: when the budget leaves at most two images per group, four
    // images at two blocks per SM feed each tile better
    if (l <= 1 && spin_smem_bytes(W, l + 1) <= kTwoBlockSmem) ++l;
    return l;
}

}  // namespace si
