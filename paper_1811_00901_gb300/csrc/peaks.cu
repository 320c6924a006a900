// peaks.cu -- measured throughput of shared-memory int32 atomic adds on this
// device: the denominator of the spin kernel's shared-atomic roofline (no
// vendor figure exists for it).  Every lane adds to a word in its own bank
// (conflict-free), or, in the second mode, to words spread like the spin
// kernel's splats over one 33 x 33 image per lane group.
#include "internal.h"

namespace si {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakWords = 8192;  // 32 KB of shared memory per block

__global__ void __launch_bounds__(kPeakThreads) smem_atomic_kernel(int iters, int mode, int *sink) {
    __shared__ int buf[kPeakWords];
    for (int k = threadIdx.x; k < kPeakWords; k += kPeakThreads) buf[k] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    unsigned h = 2654435761u * (threadIdx.x + 1) + blockIdx.x;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            int addr;
            if (mode == 0) {
                addr = ((warp * 8 + u + it) & (kPeakWords / 32 - 1)) * 32 + lane;  // bank = lane
            } else {
                h = h * 1664525u + 1013904223u;  // LCG (Numerical Recipes constants)
                addr = (int)((h >> 8) % 1089u) * 4 + (lane & 3);  // 4 images x 33 x 33, interleaved
            }
            atomicAdd(&buf[addr], 1);
        }
    }
    __syncthreads();
    int s = 0;
    for (int k = threadIdx.x; k < kPeakWords; k += kPeakThreads) s += buf[k];
    atomicAdd(sink, s);
}

}  // namespace
}  // namespace si

using namespace si;

extern "C" si_status si_peak_smem_atomics(int32_t mode, double *atomics_per_s, si_stream stream) {
    if (!atomics_per_s || (mode != 0 && mode != 1)) {
        set_error("si_peak_smem_atomics: bad arguments");
        return SI_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    int per_sm = 0;
    SI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, smem_atomic_kernel, kPeakThreads, 0));
    const int blocks = num_sms(dev) * std::max(1, per_sm);
    int *sink = nullptr;
    si_status s = dev_alloc((void **)&sink, sizeof(int), st);
    if (s != SI_OK) return s;
    const int iters = 4096;
    cudaEvent_t e0, e1;
    SI_CUDA(cudaEventCreate(&e0));
    SI_CUDA(cudaEventCreate(&e1));
    smem_atomic_kernel<<<blocks, kPeakThreads, 0, st>>>(64, mode, sink);  // warm-up
    cudaEventRecord(e0, st);
    smem_atomic_kernel<<<blocks, kPeakThreads, 0, st>>>(iters, mode, sink);
    cudaEventRecord(e1, st);
    note_launches(2);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(sink, st);
    if (e != cudaSuccess) return cuda_fail(e, "si_peak_smem_atomics");
    *atomics_per_s = (double)blocks * kPeakThreads * iters * 8 / (ms / 1e3);
    return SI_OK;
}
