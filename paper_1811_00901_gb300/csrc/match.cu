// match.cu -- spin-image matching: every scene image against every model
// image by the linear correlation coefficient over all W x W bins, and each
// scene image's k best model images.
//
// Over all bins the correlation of p and q is the dot product of the centred,
// unit-length images, so the all-pairs step is one dense contraction
// [scene x W^2] . [W^2 x model].  Both precisions run it on the tensor cores
// through this library's tcgen05 kernel with the top-k in its epilogue
// (match_tc.cu):
//   * SI_MATCH_BF16: the centred images rounded to BF16, FP32 accumulation;
//   * SI_MATCH_FP32: each centred value split into three BF16 terms,
//     x = x1 + x2 + x3 (24 significant bits), and the six products that reach
//     FP32 accuracy -- x1y1, x1y2, x2y1, x1y3, x2y2, x3y1 -- laid out along K
//     (scene [x1 | x1 | x2 | x1 | x2 | x3], model [y1 | y2 | y1 | y3 | y2 |
//     y1]), so one BF16 GEMM over 6K sums them.
// The images are centred here (centre4_kernel for even W, centre_kernel
// otherwise), with K padded to a multiple of the kernel's 64-element slices.
#include <cuda_bf16.h>

#include <cmath>

#include "internal.h"
#include "match_tc.h"

namespace si {
namespace {

// ---------------------------------------------------------------- kernels --
// One warp per image: (x - mean) / |x - mean| (0 for an image without
// variance), without FP64 arithmetic per pixel: the pixel sum is exact in
// int64, m = the nearest integer to the mean and f = mean - m (|f| <= 1/2);
// the centred values are (x - m) - f, their squared norm
// sum (x - m)^2 - K f^2 with the per-lane sums in FP32 (32 terms each for
// K = 1024, relative error ~2e-6) and the lanes' totals in FP64; the
// output is FP32 ((x - m) - f) times the reciprocal norm.
// Operand layouts: one BF16 term per value (SPLIT = 0), or the three-term
// split laid out for the scene (SPLIT = 1: x1 x1 x2 x1 x2 x3) or the model
// (SPLIT = 2: y1 y2 y1 y3 y2 y1), each segment `kp` long.
template <int SPLIT>
__device__ __forceinline__ void put(__nv_bfloat16 *o, int kp, int k, float x) {
    const __nv_bfloat16 t1 = __float2bfloat16_rn(x);
    if (SPLIT == 0) {
        o[k] = t1;
        return;
    }
    const float r1 = x - __bfloat162float(t1);  // exact: x and t1 agree in their leading 8 bits
    const __nv_bfloat16 t2 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 t3 = __float2bfloat16_rn(r1 - __bfloat162float(t2));
    const __nv_bfloat16 seq1[6] = {t1, t1, t2, t1, t2, t3};
    const __nv_bfloat16 seq2[6] = {t1, t2, t1, t3, t2, t1};
#pragma unroll
    for (int s = 0; s < 6; ++s) o[s * kp + k] = SPLIT == 1 ? seq1[s] : seq2[s];
}

template <int SPLIT>
__global__ void centre_kernel(const int32_t *__restrict__ img, int64_t n, int K, __nv_bfloat16 *__restrict__ out,
                              int kp) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int32_t *x = img + r * K;
        long long s = 0;
        for (int k = lane; k < K; k += 32) s += x[k];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        // m = round(s / K), halves away from zero; f = s / K - m
        const long long m = s >= 0 ? (2 * s + K) / (2 * (long long)K) : -((-2 * s + K) / (2 * (long long)K));
        const double fd = (double)(s - m * (long long)K) / (double)K;
        const float f = (float)fd;
        float ssf = 0.0f;
        for (int k = lane; k < K; k += 32) {
            const float c = (float)(int)(x[k] - (int)m);
            ssf = fmaf(c, c, ssf);
        }
        double ss = (double)ssf;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, d);
        ss -= (double)K * fd * fd;
        const float inv = ss > 0.0 ? (float)(1.0 / sqrt(ss)) : 0.0f;
        __nv_bfloat16 *o = out + r * (int64_t)kp * (SPLIT ? 6 : 1);
        for (int k = lane; k < K; k += 32) put<SPLIT>(o, kp, k, ((float)(int)(x[k] - (int)m) - f) * inv);
        for (int k = K + lane; k < kp; k += 32) put<SPLIT>(o, kp, k, 0.0f);  // zero padding of K
    }
}

// The same centring with 16-byte loads and 8-byte stores: four pixels of an
// image per lane per step (K % 4 == 0 and 16-byte aligned images, i.e. even W).
// Each output segment row is kp BF16 long (a multiple of 64), so a lane's four
// values are one aligned 8-byte store per segment.
template <int SPLIT>
__device__ __forceinline__ void put4(__nv_bfloat16 *o, int kp, int k, const float (&x)[4]) {
    __nv_bfloat16 t1[4], t2[4], t3[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        t1[i] = __float2bfloat16_rn(x[i]);
        if (SPLIT) {
            const float r1 = x[i] - __bfloat162float(t1[i]);  // exact, as in put()
            t2[i] = __float2bfloat16_rn(r1);
            t3[i] = __float2bfloat16_rn(r1 - __bfloat162float(t2[i]));
        }
    }
    auto pack = [](const __nv_bfloat16 (&t)[4]) {
        uint2 v;
        v.x = (uint32_t)__bfloat16_as_ushort(t[0]) | ((uint32_t)__bfloat16_as_ushort(t[1]) << 16);
        v.y = (uint32_t)__bfloat16_as_ushort(t[2]) | ((uint32_t)__bfloat16_as_ushort(t[3]) << 16);
        return v;
    };
    if (SPLIT == 0) {
        *reinterpret_cast<uint2 *>(o + k) = pack(t1);
        return;
    }
    const uint2 p1 = pack(t1), p2 = pack(t2), p3 = pack(t3);
    const uint2 seq1[6] = {p1, p1, p2, p1, p2, p3};
    const uint2 seq2[6] = {p1, p2, p1, p3, p2, p1};
#pragma unroll
    for (int s = 0; s < 6; ++s) *reinterpret_cast<uint2 *>(o + s * kp + k) = SPLIT == 1 ? seq1[s] : seq2[s];
}

template <int SPLIT>
__global__ void centre4_kernel(const int32_t *__restrict__ img, int64_t n, int K, __nv_bfloat16 *__restrict__ out,
                               int kp) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int K4 = K >> 2;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int4 *x = reinterpret_cast<const int4 *>(img + r * K);
        long long s = 0;
        for (int v = lane; v < K4; v += 32) {
            const int4 a = x[v];
            s += (long long)a.x + a.y + a.z + a.w;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        const long long m = s >= 0 ? (2 * s + K) / (2 * (long long)K) : -((-2 * s + K) / (2 * (long long)K));
        const double fd = (double)(s - m * (long long)K) / (double)K;
        const float f = (float)fd;
        const int mi = (int)m;
        float ssf = 0.0f;
        for (int v = lane; v < K4; v += 32) {
            const int4 a = x[v];
            const float c0 = (float)(a.x - mi), c1 = (float)(a.y - mi), c2 = (float)(a.z - mi), c3 = (float)(a.w - mi);
            ssf = fmaf(c3, c3, fmaf(c2, c2, fmaf(c1, c1, fmaf(c0, c0, ssf))));
        }
        double ss = (double)ssf;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, d);
        ss -= (double)K * fd * fd;
        const float inv = ss > 0.0 ? (float)(1.0 / sqrt(ss)) : 0.0f;
        __nv_bfloat16 *o = out + r * (int64_t)kp * (SPLIT ? 6 : 1);
        for (int v = lane; v < K4; v += 32) {
            const int4 a = x[v];
            const float y[4] = {((float)(a.x - mi) - f) * inv, ((float)(a.y - mi) - f) * inv,
                                ((float)(a.z - mi) - f) * inv, ((float)(a.w - mi) - f) * inv};
            put4<SPLIT>(o, kp, 4 * v, y);
        }
        const float zero[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int k = K + 4 * lane; k < kp; k += 128) put4<SPLIT>(o, kp, k, zero);  // zero padding of K
    }
}

template <int SPLIT>
void launch_centre(const int32_t *img, int64_t n, int K, __nv_bfloat16 *out, int kp, int blocks, cudaStream_t st) {
    if (K % 4 == 0 && reinterpret_cast<uintptr_t>(img) % 16 == 0)
        centre4_kernel<SPLIT><<<blocks, 256, 0, st>>>(img, n, K, out, kp);
    else
        centre_kernel<SPLIT><<<blocks, 256, 0, st>>>(img, n, K, out, kp);
}

constexpr int kMatchMaxK = kMatchTcMaxK;

// Centred operands (padded, split for FP32), one tensor-core launch with the
// top-k in its epilogue, and a merge of the model ranges.
si_status match_tc(const int32_t *scene, int64_t n_scene, const int32_t *model, int64_t n_model, int W, int k,
                   bool split, int32_t *best_idx, float *best_corr, cudaStream_t st, int dev) {
    const int K = W * W;
    const int kp = (K + 63) / 64 * 64;
    const int kk = split ? 6 * kp : kp;  // K of the GEMM
    const int parts = match_tc_parts(n_scene, n_model, num_sms(dev));
    __nv_bfloat16 *a = nullptr, *b = nullptr;
    float *pv = nullptr;
    int *pi = nullptr;
    unsigned *err = nullptr;
    si_status s = dev_alloc((void **)&a, sizeof(__nv_bfloat16) * (size_t)n_scene * kk, st);
    if (s == SI_OK) s = dev_alloc((void **)&b, sizeof(__nv_bfloat16) * (size_t)n_model * kk, st);
    if (s == SI_OK) s = dev_alloc((void **)&pv, sizeof(float) * (size_t)2 * parts * n_scene * k, st);
    if (s == SI_OK) s = dev_alloc((void **)&pi, sizeof(int) * (size_t)2 * parts * n_scene * k, st);
    if (s == SI_OK) s = dev_alloc((void **)&err, sizeof(unsigned), st);
    cudaError_t e = cudaSuccess;
    if (s == SI_OK) {
        const int blocks = num_sms(dev) * 8;
        e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) {
            if (split) {
                launch_centre<2>(model, n_model, K, b, kp, blocks, st);
                launch_centre<1>(scene, n_scene, K, a, kp, blocks, st);
            } else {
                launch_centre<0>(model, n_model, K, b, kp, blocks, st);
                launch_centre<0>(scene, n_scene, K, a, kp, blocks, st);
            }
            note_launches(2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            s = match_tc_launch(a, n_scene, b, n_model, kk, k, parts, pv, pi, err, best_idx, best_corr, st);
    }
    if (e != cudaSuccess && s == SI_OK) s = cuda_fail(e, "si_match");
    dev_free(a, st);
    dev_free(b, st);
    dev_free(pv, st);
    dev_free(pi, st);
    dev_free(err, st);
    return s;
}

}  // namespace
}  // namespace si

using namespace si;

extern "C" si_status si_match(const int32_t *scene, int64_t n_scene, const int32_t *model, int64_t n_model,
                              int32_t W, int32_t k, int32_t precision, int32_t *best_idx, float *best_corr,
                              si_stream stream) {
    if (n_scene < 0 || n_model < 1 || n_model > INT32_MAX || n_scene > INT32_MAX || W < 2 || W > kMaxW || k < 1 ||
        k > kMatchMaxK || k > n_model || (precision != SI_MATCH_FP32 && precision != SI_MATCH_BF16) ||
        (n_scene > 0 && (!scene || !best_idx || !best_corr)) || !model) {
        set_error("si_match: bad arguments (1 <= k <= min(%d, n_model), W in [2, %d], precision 0 or 1)",
                  kMatchMaxK, kMaxW);
        return SI_ERR_INVALID;
    }
    if (n_scene == 0) return SI_OK;
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    return match_tc(scene, n_scene, model, n_model, W, k, precision == SI_MATCH_FP32, best_idx, best_corr,
                    (cudaStream_t)stream, dev);
}
