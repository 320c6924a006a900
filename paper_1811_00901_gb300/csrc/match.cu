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
// One warp per image: mean, centred norm (FP64 sums), then (x - mean) / norm
// (0 for an image without variance).
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
__global__ void centre_kernel(const int32_t *__restrict__ img, int64_t n, int K, T *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int32_t *x = img + r * K;
        double s = 0.0;
        for (int k = lane; k < K; k += 32) s += (double)x[k];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        const double mean = s / K;
        double ss = 0.0;
        for (int k = lane; k < K; k += 32) {
            const double c = (double)x[k] - mean;
            ss += c * c;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, d);
        const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
        T *o = out + r * K;
        for (int k = lane; k < K; k += 32) o[k] = to_out<T>((float)(((double)x[k] - mean) * inv));
    }
}

// a before b: higher value, equal values by smaller index
__device__ __forceinline__ bool better(float va, int ia, float vb, int ib) {
    return va > vb || (va == vb && ia < ib);
}

// One warp per scene row of the correlation tile: each lane keeps its k best
// (sorted, in registers), then the warp merges them k times by a warp arg-max.
template <int KMAX>
__global__ void topk_kernel(const float *__restrict__ C, int rows, int cols, int k, int64_t row0,
                            int32_t *__restrict__ best_idx, float *__restrict__ best_val) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += warps) {
        const float *c = C + (int64_t)r * cols;
        float v[KMAX];
        int ix[KMAX];
#pragma unroll
        for (int t = 0; t < KMAX; ++t) {
            v[t] = -INFINITY;
            ix[t] = INT_MAX;
        }
        for (int j = lane; j < cols; j += 32) {
            float x = c[j];
            int xi = j;
            // insert (x, xi) into the sorted list, dropping the last
#pragma unroll
            for (int t = 0; t < KMAX; ++t) {
                if (t < k && better(x, xi, v[t], ix[t])) {
                    const float tv = v[t];
                    const int ti = ix[t];
                    v[t] = x;
                    ix[t] = xi;
                    x = tv;
                    xi = ti;
                }
            }
        }
        int head = 0;
        for (int t = 0; t < k; ++t) {
            float hv = -INFINITY;
            int hi = INT_MAX;
#pragma unroll
            for (int q = 0; q < KMAX; ++q)
                if (q == head) {
                    hv = v[q];
                    hi = ix[q];
                }
            float bv = hv;
            int bi = hi, bl = lane;
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
                best_idx[(row0 + r) * k + t] = bi == INT_MAX ? -1 : bi;
                best_val[(row0 + r) * k + t] = bv;
            }
        }
    }
}

constexpr int kMatchMaxK = 16;
constexpr size_t kTileBytes = (size_t)1 << 30;  // correlation tile scratch bound

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
    cublasHandle_t h = blas_handle(dev);
    if (!h) return SI_ERR_CUDA;
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
            centre_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(model, n_model, K, (__nv_bfloat16 *)b);
        else
            centre_kernel<float><<<blocks, 256, 0, st>>>(model, n_model, K, (float *)b);
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
            centre_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(scene + r0 * K, nr, K, (__nv_bfloat16 *)a);
        else
            centre_kernel<float><<<blocks, 256, 0, st>>>(scene + r0 * K, nr, K, (float *)a);
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
        topk_kernel<kMatchMaxK><<<(nr + 7) / 8, 256, 0, st>>>(ct, nr, (int)n_model, k, r0, best_idx, best_corr);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess && s == SI_OK) s = cuda_fail(e, "si_match");
    dev_free(a, st);
    dev_free(b, st);
    dev_free(ct, st);
    return s;
}
