// selfcheck.cu -- a self-check of the bounded device waits that every
// mbarrier wait of the spin kernel uses (mbar_wait_bounded): a block waits on
// an mbarrier that nothing ever arrives at, with a short limit, and must give
// up, report it through a flag and leave the context usable.  It exercises the
// failure path of the spin kernel's waits without a fault or a hang.
#include <cstring>

#include "device_common.cuh"
#include "internal.h"

namespace si {
namespace {

__global__ void bounded_wait_kernel(uint64_t limit_ns, unsigned *flag, unsigned long long *waited_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint64_t t0 = global_ns();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);  // phase 0 never completes
    const uint64_t t1 = global_ns();
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!ok) atomicOr(flag, kFlagTimeout);
        atomicMax(waited_ns, (unsigned long long)(t1 - t0));
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"((uint32_t)__cvta_generic_to_shared(&bar))
                     : "memory");
    }
}

}  // namespace
}  // namespace si

using namespace si;

extern "C" si_status si_check_bounded_wait(int32_t limit_ms, int32_t *timed_out, double *waited_ms,
                                           si_stream stream) {
    if (!timed_out || limit_ms < 1 || limit_ms > 1000) {
        set_error("si_check_bounded_wait: need 1 <= limit_ms <= 1000 and an output");
        return SI_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned *d = nullptr;
    si_status s = dev_alloc((void **)&d, 16, st);
    if (s != SI_OK) return s;
    unsigned host[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemsetAsync(d, 0, 16, st);
    if (e == cudaSuccess) {
        bounded_wait_kernel<<<2, 64, 0, st>>>((uint64_t)limit_ms * 1000000ull, d,
                                              reinterpret_cast<unsigned long long *>(d + 2));
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, d, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(d, st);
    if (e != cudaSuccess) return cuda_fail(e, "si_check_bounded_wait");
    *timed_out = (host[0] & kFlagTimeout) ? 1 : 0;
    unsigned long long ns = 0;
    std::memcpy(&ns, host + 2, sizeof(ns));
    if (waited_ms) *waited_ms = (double)ns / 1e6;
    return SI_OK;
}
