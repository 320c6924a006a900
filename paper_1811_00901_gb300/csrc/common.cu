// common.cu -- error reporting, stream-ordered allocation, the pinned staging
// ring for host->device uploads, and device queries.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>

#include "internal.h"

namespace si {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

si_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SI_ERR_OOM : SI_ERR_CUDA;
}

// ------------------------------------------------------------ allocation --
// Device memory comes from the device's default memory pool through
// cudaMallocAsync: stream ordered, cached by the pool (release threshold
// raised once per device), and capturable in CUDA graphs.
static std::mutex g_pool_mu;
static bool g_pool_ready[64] = {false};

static void ensure_pool(int dev) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64 || g_pool_ready[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    g_pool_ready[dev] = true;
}

// Accounting and host-side failure injection: every device allocation of the
// library goes through dev_alloc, which counts it and, while an injection is
// armed, lets `g_inject_skip` more allocations through and then fails the next
// `g_inject_fail` as if the device were out of memory.
static std::atomic<int64_t> g_alloc_calls{0};
static std::mutex g_inject_mu;
static int64_t g_inject_skip = 0, g_inject_fail = 0;
static std::atomic<bool> g_inject_armed{false};

static bool injected_failure() {
    if (!g_inject_armed.load()) return false;
    std::lock_guard<std::mutex> lk(g_inject_mu);
    if (g_inject_fail <= 0) return false;
    if (g_inject_skip > 0) {
        --g_inject_skip;
        return false;
    }
    if (--g_inject_fail == 0) g_inject_armed.store(false);
    return true;
}

si_status dev_alloc(void **p, size_t bytes, cudaStream_t stream) {
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    ensure_pool(dev);
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    g_alloc_calls.fetch_add(1);
    if (injected_failure()) {
        set_error("device allocation of %zu bytes failed: injected failure (si_debug_fail_allocs)", bytes);
        return SI_ERR_OOM;
    }
    cudaError_t e = cudaMallocAsync(p, bytes, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        return SI_ERR_OOM;
    }
    return SI_OK;
}

void dev_free(void *p, cudaStream_t stream) {
    if (p) cudaFreeAsync(p, stream);
}

// ----------------------------------------------------------- staging ring --
// Small host->device uploads (descriptor tables, chunk tables) go through a
// pinned ring: bytes are copied into the ring, a cudaMemcpyAsync is enqueued
// and an event marks when that region may be reused.  The ring never blocks
// unless a region is still in flight after a full lap.
namespace {
struct Ring {
    char *base = nullptr;
    size_t cap = 0, head = 0;
    struct Region {
        size_t off, len;
        cudaEvent_t ev;
    };
    std::vector<Region> inflight;
    std::mutex mu;
};
std::map<int, Ring *> g_rings;
std::mutex g_rings_mu;

Ring *ring_for(int dev) {
    std::lock_guard<std::mutex> lk(g_rings_mu);
    auto it = g_rings.find(dev);
    if (it != g_rings.end()) return it->second;
    Ring *r = new Ring();
    g_rings[dev] = r;
    return r;
}
}  // namespace

si_status stage_upload(void *dev_dst, const void *src, size_t bytes, cudaStream_t stream) {
    if (bytes == 0) return SI_OK;
    int dev = 0;
    SI_CUDA(cudaGetDevice(&dev));
    Ring *r = ring_for(dev);
    std::lock_guard<std::mutex> lk(r->mu);
    size_t need = (bytes + 255) & ~size_t(255);
    if (r->base == nullptr || need > r->cap) {
        // (re)create a ring large enough; wait for the old one to drain
        for (auto &g : r->inflight) {
            cudaEventSynchronize(g.ev);
            cudaEventDestroy(g.ev);
        }
        r->inflight.clear();
        if (r->base) cudaFreeHost(r->base);
        size_t cap = std::max<size_t>(need * 2, size_t(8) << 20);
        cudaError_t e = cudaHostAlloc((void **)&r->base, cap, cudaHostAllocPortable);
        if (e != cudaSuccess) {
            r->base = nullptr;
            r->cap = 0;
            return cuda_fail(e, "cudaHostAlloc(staging ring)");
        }
        r->cap = cap;
        r->head = 0;
    }
    if (r->head + need > r->cap) r->head = 0;
    size_t off = r->head;
    // retire regions that overlap [off, off + need)
    for (size_t k = 0; k < r->inflight.size();) {
        auto &g = r->inflight[k];
        bool overlap = g.off < off + need && off < g.off + g.len;
        if (overlap || cudaEventQuery(g.ev) == cudaSuccess) {
            if (overlap) cudaEventSynchronize(g.ev);
            cudaEventDestroy(g.ev);
            r->inflight.erase(r->inflight.begin() + k);
        } else {
            ++k;
        }
    }
    std::memcpy(r->base + off, src, bytes);
    SI_CUDA(cudaMemcpyAsync(dev_dst, r->base + off, bytes, cudaMemcpyHostToDevice, stream));
    cudaEvent_t ev;
    SI_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    SI_CUDA(cudaEventRecord(ev, stream));
    r->inflight.push_back({off, need, ev});
    r->head = off + need;
    return SI_OK;
}

// ---------------------------------------------------------------- devices --
int num_sms(int device) {
    static int cache[64] = {0};
    if (device >= 0 && device < 64 && cache[device]) return cache[device];
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    if (v <= 0) v = 1;
    if (device >= 0 && device < 64) cache[device] = v;
    return v;
}

static std::atomic<int> g_timing{0};
bool timing_enabled() { return g_timing.load() != 0; }

static std::atomic<long long> g_launches{0};
void note_launches(int k) { g_launches.fetch_add(k); }

}  // namespace si

extern "C" {

const char *si_last_error(void) { return si::g_err; }

const char *si_version(void) { return "spin-gb300 0.1 (sm_103a)"; }

void si_set_timing(int32_t enabled) { si::g_timing.store(enabled ? 1 : 0); }

int64_t si_kernel_launches(void) { return (int64_t)si::g_launches.load(); }

}  // extern "C"

extern "C" si_status si_alloc_stats(int64_t *calls, int64_t *pool_used, int64_t *pool_reserved) {
    if (calls) *calls = si::g_alloc_calls.load();
    if (pool_used || pool_reserved) {
        int dev = 0;
        SI_CUDA(cudaGetDevice(&dev));
        cudaMemPool_t pool;
        SI_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
        uint64_t v = 0;
        if (pool_used) {
            SI_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v));
            *pool_used = (int64_t)v;
        }
        if (pool_reserved) {
            SI_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v));
            *pool_reserved = (int64_t)v;
        }
    }
    return SI_OK;
}

extern "C" si_status si_debug_fail_allocs(int64_t skip, int64_t count) {
    if (skip < 0 || count < 0) {
        si::set_error("si_debug_fail_allocs: skip and count must be >= 0");
        return SI_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(si::g_inject_mu);
    si::g_inject_skip = skip;
    si::g_inject_fail = count;
    si::g_inject_armed.store(count > 0);
    return SI_OK;
}
