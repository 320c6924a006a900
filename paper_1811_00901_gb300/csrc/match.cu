// match.cu -- spin-image matching: every scene image against every model
// image by the linear correlation coefficient over all W x W bins, and each
// scene image's k best model images.
//
// Over all bins the correlation of p and q is the dot product of the centred,
// unit-length images, so the all-pairs step is one dense contraction
// [scene x W^2] . [W^2 x model]: it runs as a GEMM on the tensor cores (BF16
// operands, FP32 accumulation) or as an FP32 GEMM, through cuBLAS, which this
// file loads at first use (no link-time dependency).  Centring/normalising the
// images and the top-k selection are this library's kernels.  Scene images are
// processed in row blocks whose correlation tile fits a scratch bound.
#include <cuda_bf16.h>
#include <cublas_v2.h>
#include <dlfcn.h>

#include <cmath>
#include <mutex>

#include "internal.h"
#include "match_tc.h"

namespace si {
namespace {

// ---------------------------------------------------------------- cuBLAS --
struct Blas {
    bool tried = false;
    void *lib = nullptr;
    decltype(&cublasCreate_v2) create = nullptr;
    decltype(&cublasSetStream_v2) set_stream = nullptr;
    cublasStatus_t (*gemm)(cublasHandle_t, cublasOperation_t, cublasOperation_t, int, int, int, const void *,
                           const void *, cudaDataType, int, const void *, cudaDataType, int, const void *, void *,
                           cudaDataType, int, cublasComputeType_t, cublasGemmAlgo_t) = nullptr;
    decltype(&cublasSetMathMode) set_math = nullptr;
    cublasHandle_t handle[128] = {};
};
Blas g_blas;
std::mutex g_blas_mu;

// Resolves cuBLAS and this device's handle; nullptr with the error set if not possible.
cublasHandle_t blas_handle(int dev) {
    std::lock_guard<std::mutex> lk(g_blas_mu);
    Blas &b = g_blas;
    if (!b.tried) {
        b.tried = true;
        const char *names[] = {"libcublas.so.13", "libcublas.so", "/usr/local/cuda/lib64/libcublas.so.13"};
        for (const char *n : names)
            if ((b.lib = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (b.lib) {
            b.create = reinterpret_cast<decltype(b.create)>(dlsym(b.lib, "cublasCreate_v2"));
            b.set_stream = reinterpret_cast<decltype(b.set_stream)>(dlsym(b.lib, "cublasSetStream_v2"));
            b.gemm = reinterpret_cast<decltype(b.gemm)>(dlsym(b.lib, "cublasGemmEx"));
            b.set_math = reinterpret_cast<decltype(b.set_math)>(dlsym(b.lib, "cublasSetMathMode"));
        }
    }
    if (!b.create || !b.set_stream || !b.gemm || !b.set_math) {
        set_error("si_match: cuBLAS could not be loaded");
        return nullptr;
    }
    if (dev < 0 || dev >= 128) {
        set_error("si_match: device %d out of range", dev);
        return nullptr;
    }
    if (!b.handle[dev]) {
        cublasHandle_t h = nullptr;
        if (b.create(&h) != CUBLAS_STATUS_SUCCESS) {
            set_error("si_match: cublasCreate failed");
            return nullptr;
        }
        b.handle[dev] = h;
    }
    return b.handle[dev];
}

// ---------------------------------------------------------------- kernels --
// One warp per image: (x - mean) / |x - mean| (0 for an image without
// variance), without FP64 arithmetic per pixel: the pixel sum is exact in
// int64, m = the nearest integer to the mean and f = mean - m (|f| <= 1/2);
// the centred values are (x - m) - f, their squared norm
// sum (x - m)^2 - K f^2 with the per-lane sums in FP32 (32 terms each for
// K = 1024, relative error ~2e-6) and the lanes' totals in FP64; the
// output is FP32 ((x - m) - f) times the reciprocal norm.
template <typename T>
__device__ __forceinline__ T to_out(float x);
template <>
__device__ __forceinline__ float to_out<float>(float x) {
    return x;
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16>(float x) {
    return __float2bfloat16_rn(x);
}

template <typename T>
__global__ void centre_kernel(const int32_t *__restrict__ img, int64_t n, int K, T *__restrict__ out,
                              int out_stride) {
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
        T *o = out + r * out_stride;
        for (int k = lane; k < K; k += 32) o[k] = to_out<T>(((float)(int)(x[k] - (int)m) - f) * inv);
        for (int k = K + lane; k < out_stride; k += 32) o[k] = to_out<T>(0.0f);  // zero padding of K
    }
}

// a before b: higher value, equal values by smaller index
__device__ __forceinline__ bool better(float va, int ia, float vb, int ib) {
    return va > vb || (va == vb && ia < ib);
}

// A thread's k best so far, highest first (kept in local memory: insertions
// are rare once the list holds high values).
struct TopList {
    float v[16];
    int ix[16];
};

// Inserts (x, xi) into a sorted list of k, dropping the last; returns the new k-th.
__device__ __noinline__ void topk_insert(TopList &t, const int k, float x, int xi, float &thr_v, int &thr_i) {
    for (int q = 0; q < k; ++q) {
        if (better(x, xi, t.v[q], t.ix[q])) {
            const float tv = t.v[q];
            const int ti = t.ix[q];
            t.v[q] = x;
            t.ix[q] = xi;
            x = tv;
            xi = ti;
        }
    }
    thr_v = t.v[k - 1];
    thr_i = t.ix[k - 1];
}

// One block per scene row of the correlation tile.  Each thread scans its
// strided share with eight loads in flight, offering a value to its list only
// when it beats the list's k-th; then each warp merges its 32 lists by k warp
// arg-max rounds, and thread 0 picks the k best of the warps' lists.
constexpr int kTopThreads = 256;

__global__ void __launch_bounds__(kTopThreads) topk_kernel(const float *__restrict__ C, int rows, int cols, int k,
                                                            int64_t row0, int32_t *__restrict__ best_idx,
                                                            float *__restrict__ best_val) {
    __shared__ float sv[kTopThreads / 32][16];
    __shared__ int si_[kTopThreads / 32][16];
    __shared__ float mv[kTopThreads];
    __shared__ int mi[kTopThreads];
    __shared__ float tv_s;
    __shared__ int ti_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kU = 8;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const float *c = C + (int64_t)r * cols;
        // pass 1: each thread's best; the k-th best of these 256 bounds the
        // row's k-th best from below, so nothing worse can make the list
        float bv = -INFINITY;
        int bi = INT_MAX;
        {
            int j0 = threadIdx.x;
            for (; j0 + kTopThreads * (kU - 1) < cols; j0 += kTopThreads * kU) {
                float x[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) x[u] = c[j0 + kTopThreads * u];
#pragma unroll
                for (int u = 0; u < kU; ++u)
                    if (better(x[u], j0 + kTopThreads * u, bv, bi)) {
                        bv = x[u];
                        bi = j0 + kTopThreads * u;
                    }
            }
            for (int j = j0; j < cols; j += kTopThreads) {
                const float x = c[j];
                if (better(x, j, bv, bi)) {
                    bv = x;
                    bi = j;
                }
            }
        }
        mv[threadIdx.x] = bv;
        mi[threadIdx.x] = bi;
        __syncthreads();
        int rank = 0;
        for (int o = 0; o < kTopThreads; ++o) rank += better(mv[o], mi[o], bv, bi) ? 1 : 0;
        if (rank == k - 1) {  // ranks of distinct (value, index) pairs are distinct
            tv_s = bv;
            ti_s = bi;
        }
        __syncthreads();
        // pass 2: lists of the values not worse than that bound
        TopList t;
        for (int q = 0; q < k; ++q) {
            t.v[q] = -INFINITY;
            t.ix[q] = INT_MAX;
        }
        const float bound_v = tv_s;
        const int bound_i = ti_s;
        float thr_v = -INFINITY;
        int thr_i = INT_MAX;
        auto wanted = [&](float x, int j) {
            return !better(bound_v, bound_i, x, j) && better(x, j, thr_v, thr_i);
        };
        int j0 = threadIdx.x;
        for (; j0 + kTopThreads * (kU - 1) < cols; j0 += kTopThreads * kU) {
            float x[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) x[u] = __ldcs(c + j0 + kTopThreads * u);
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (wanted(x[u], j0 + kTopThreads * u)) topk_insert(t, k, x[u], j0 + kTopThreads * u, thr_v, thr_i);
        }
        for (int j = j0; j < cols; j += kTopThreads) {
            const float x = __ldcs(c + j);
            if (wanted(x, j)) topk_insert(t, k, x, j, thr_v, thr_i);
        }
        // warp merge: k rounds of arg-max over the lanes' list heads
        int head = 0;
        for (int q = 0; q < k; ++q) {
            float bv = head < k ? t.v[head] : -INFINITY;
            int bi = head < k ? t.ix[head] : INT_MAX, bl = lane;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                const float ov = __shfl_xor_sync(0xffffffffu, bv, d);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, d);
                const int ol = __shfl_xor_sync(0xffffffffu, bl, d);
                if (better(ov, oi, bv, bi)) {
                    bv = ov;
                    bi = oi;
                    bl = ol;
                }
            }
            if (lane == bl) ++head;
            if (lane == 0) {
                sv[warp][q] = bv;
                si_[warp][q] = bi;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int hw[kTopThreads / 32] = {};
            for (int q = 0; q < k; ++q) {
                // k picks from 8 lists of k: some list always has an entry left
                int bw = -1;
                for (int w = 0; w < kTopThreads / 32; ++w) {
                    if (hw[w] >= k) continue;
                    if (bw < 0 || better(sv[w][hw[w]], si_[w][hw[w]], sv[bw][hw[bw]], si_[bw][hw[bw]])) bw = w;
                }
                best_val[(row0 + r) * k + q] = sv[bw][hw[bw]];
                best_idx[(row0 + r) * k + q] = si_[bw][hw[bw]] == INT_MAX ? -1 : si_[bw][hw[bw]];
                ++hw[bw];
            }
        }
        __syncthreads();
    }
}

constexpr int kMatchMaxK = 16;
constexpr size_t kTileBytes = (size_t)1 << 30;  // correlation tile scratch bound

// BF16: centred images padded to a multiple of 64 in K, one tensor-core
// launch with the top-k in its epilogue, a merge of the model ranges.
si_status match_bf16_tc(const int32_t *scene, int64_t n_scene, const int32_t *model, int64_t n_model, int W, int k,
                        int32_t *best_idx, float *best_corr, cudaStream_t st, int dev) {
    const int K = W * W;
    const int kp = (K + 63) / 64 * 64;
    const int parts = match_tc_parts(n_scene, n_model, num_sms(dev));
    __nv_bfloat16 *a = nullptr, *b = nullptr;
    float *pv = nullptr;
    int *pi = nullptr;
    unsigned *err = nullptr;
    si_status s = dev_alloc((void **)&a, sizeof(__nv_bfloat16) * (size_t)n_scene * kp, st);
    if (s == SI_OK) s = dev_alloc((void **)&b, sizeof(__nv_bfloat16) * (size_t)n_model * kp, st);
    if (s == SI_OK) s = dev_alloc((void **)&pv, sizeof(float) * (size_t)parts * n_scene * k, st);
    if (s == SI_OK) s = dev_alloc((void **)&pi, sizeof(int) * (size_t)parts * n_scene * k, st);
    if (s == SI_OK) s = dev_alloc((void **)&err, sizeof(unsigned), st);
    cudaError_t e = cudaSuccess;
    if (s == SI_OK) {
        const int blocks = num_sms(dev) * 8;
        e = cudaMemsetAsync(err, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) {
            centre_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(model, n_model, K, b, kp);
            centre_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(scene, n_scene, K, a, kp);
            note_launches(2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            s = match_tc_launch(a, n_scene, b, n_model, kp, k, parts, pv, pi, err, best_idx, best_corr, st);
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
    if (n_scene < 0 || n_model < 1 || n_model > INT32_MAX || W < 2 || W > kMaxW || k < 1 || k > kMatchMaxK ||
        k > n_model || (precision != SI_MATCH_FP32 && precision != SI_MATCH_BF16) ||
        (n_scene > 0 && (!scene || !best_idx || !best_corr)) || !model) {
        set_error("si_match: bad arguments (1 <= k <= min(%d, n_model), W in [2, %d], precision 0 or 1)",
                  kMatchMaxK, kMaxW);
        return SI_ERR_INVALID;
    }
    if (n_scene == 0) return SI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    if (precision == SI_MATCH_BF16) return match_bf16_tc(scene, n_scene, model, n_model, W, k, best_idx, best_corr, st, dev);
    cublasHandle_t h = blas_handle(dev);
    const int K = W * W;
    const bool bf16 = precision == SI_MATCH_BF16;
    const size_t esz = bf16 ? sizeof(__nv_bfloat16) : sizeof(float);
    // scene rows per tile: the correlation tile holds rows x n_model floats
    const int64_t rows = std::max<int64_t>(1, std::min<int64_t>(n_scene, (int64_t)(kTileBytes / (4 * (size_t)n_model))));
    void *a = nullptr, *b = nullptr;
    float *ct = nullptr;
    si_status s = dev_alloc(&a, esz * (size_t)rows * K, st);
    if (s == SI_OK) s = dev_alloc(&b, esz * (size_t)n_model * K, st);
    if (s == SI_OK) s = dev_alloc((void **)&ct, sizeof(float) * (size_t)rows * n_model, st);
    cudaError_t e = cudaSuccess;
    if (s == SI_OK) {
        const int blocks = num_sms(dev) * 8;
        if (bf16)
            centre_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(model, n_model, K, (__nv_bfloat16 *)b, K);
        else
            centre_kernel<float><<<blocks, 256, 0, st>>>(model, n_model, K, (float *)b, K);
        note_launches(1);
        e = cudaGetLastError();
    }
    std::lock_guard<std::mutex> lk(g_blas_mu);  // the handle's stream is per call
    if (s == SI_OK && e == cudaSuccess) {
        if (g_blas.set_stream(h, st) != CUBLAS_STATUS_SUCCESS ||
            g_blas.set_math(h, bf16 ? CUBLAS_DEFAULT_MATH : CUBLAS_PEDANTIC_MATH) != CUBLAS_STATUS_SUCCESS) {
            set_error("si_match: cuBLAS stream / math mode");
            s = SI_ERR_CUDA;
        }
    }
    const cudaDataType_t dt = bf16 ? CUDA_R_16BF : CUDA_R_32F;
    for (int64_t r0 = 0; r0 < n_scene && s == SI_OK && e == cudaSuccess; r0 += rows) {
        const int nr = (int)std::min<int64_t>(rows, n_scene - r0);
        const int blocks = num_sms(dev) * 8;
        if (bf16)
            centre_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(scene + r0 * K, nr, K, (__nv_bfloat16 *)a, K);
        else
            centre_kernel<float><<<blocks, 256, 0, st>>>(scene + r0 * K, nr, K, (float *)a, K);
        note_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        // row-major C[nr][n_model] = A[nr][K] . B[n_model][K]^T, i.e. column-major
        // C^T (n_model x nr) = B (op T of the K x n_model column-major B^T) . A^T
        const float one = 1.0f, zero = 0.0f;
        if (g_blas.gemm(h, CUBLAS_OP_T, CUBLAS_OP_N, (int)n_model, nr, K, &one, b, dt, K, a, dt, K, &zero, ct,
                        CUDA_R_32F, (int)n_model, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT) != CUBLAS_STATUS_SUCCESS) {
            set_error("si_match: cublasGemmEx failed");
            s = SI_ERR_CUDA;
            break;
        }
        note_launches(1);
        topk_kernel<<<nr, kTopThreads, 0, st>>>(ct, nr, (int)n_model, k, r0, best_idx, best_corr);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess && s == SI_OK) s = cuda_fail(e, "si_match");
    dev_free(a, st);
    dev_free(b, st);
    dev_free(ct, st);
    return s;
}
