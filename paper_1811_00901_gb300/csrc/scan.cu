// scan.cu -- exclusive prefix sums of int32 counts (grid cell starts, query
// sort offsets).  Three-phase: block-local scans of 4096 elements, a
// recursive scan of the block totals, and a uniform add.
#include "internal.h"
#include "scan.h"

namespace si {

namespace {
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanBlock = kScanThreads * kScanPer;  // 4096

__global__ void __launch_bounds__(kScanThreads)
scan_block_kernel(const int *__restrict__ in, int *__restrict__ out, int *__restrict__ block_sums, int64_t n) {
    __shared__ int buf[kScanBlock];
    __shared__ int warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    const int tid = threadIdx.x;
    for (int k = tid; k < kScanBlock; k += kScanThreads) {
        int64_t g = base + k;
        buf[k] = g < n ? in[g] : 0;
    }
    __syncthreads();
    int local[kScanPer];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        local[k] = s;
        s += buf[tid * kScanPer + k];
    }
    // inclusive warp scan of the per-thread totals
    const int lane = tid & 31, warp = tid >> 5;
    int incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int vi = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int o = __shfl_up_sync(0xffffffffu, vi, d);
            if (lane >= d) vi += o;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = vi - v;  // exclusive
    }
    __syncthreads();
    const int offset = warp_tot[warp] + incl - s;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) buf[tid * kScanPer + k] = local[k] + offset;
    if (block_sums && tid == kScanThreads - 1) block_sums[blockIdx.x] = offset + s;
    __syncthreads();
    for (int k = tid; k < kScanBlock; k += kScanThreads) {
        int64_t g = base + k;
        if (g < n) out[g] = buf[k];
    }
}

__global__ void scan_add_kernel(int *__restrict__ out, const int *__restrict__ block_off, int64_t n) {
    const int64_t base = (int64_t)blockIdx.x * kScanBlock;
    const int add = block_off[blockIdx.x];
    for (int k = threadIdx.x; k < kScanBlock; k += blockDim.x) {
        int64_t g = base + k;
        if (g < n) out[g] += add;
    }
}
}  // namespace

si_status scan_exclusive(const int *in, int *out, int64_t n, cudaStream_t stream) {
    if (n <= 0) return SI_OK;
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 1) {
        scan_block_kernel<<<1, kScanThreads, 0, stream>>>(in, out, nullptr, n);
        note_launches(1);
        SI_CUDA(cudaGetLastError());
        return SI_OK;
    }
    int *sums = nullptr;
    si_status st = dev_alloc((void **)&sums, sizeof(int) * nb, stream);
    if (st != SI_OK) return st;
    scan_block_kernel<<<(unsigned)nb, kScanThreads, 0, stream>>>(in, out, sums, n);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        dev_free(sums, stream);
        return cuda_fail(e, "scan_block_kernel");
    }
    st = scan_exclusive(sums, sums, nb, stream);
    if (st == SI_OK) {
        scan_add_kernel<<<(unsigned)nb, kScanThreads, 0, stream>>>(out, sums, n);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "scan_add_kernel");
    }
    dev_free(sums, stream);
    return st;
}

}  // namespace si
