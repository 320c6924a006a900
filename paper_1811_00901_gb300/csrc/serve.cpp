// serve.cpp -- serving with continuous batching.
//
// A server keeps meshes resident (the paper's replicated input, Sec. 3) and
// runs spin-image requests as they arrive.  One host thread owns the GPU side:
//   * admission: requests wait in FIFO order until an in-flight slot and
//     enough of the memory budget (server-allocated output + scratch) are free;
//   * batching: every admitted request waiting at that moment is packed into
//     ONE batched persistent launch (si_generate_batched's path), each item
//     with its own mesh, W, bin size, angle, queries and output;
//   * overlap: consecutive batches go to different streams, so a batch can
//     start while the previous one drains;
//   * completion: an event per batch; when it fires, every request of the
//     batch completes (latency = submit to the host seeing the event).
// Requests arriving while batches run join the next batch as soon as memory
// and slots free up.  Integer accumulation makes a request's images the same
// alone and in any mix.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "internal.h"

namespace si {

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket;
    si_batch_item item;
    size_t bytes;        // budget charged while in flight (scratch + owned output)
    size_t out_bytes;    // server-owned output bytes (kept until release)
    bool own_out;
    Clock::time_point submit;
    Clock::time_point done_at;
    bool done = false;
    si_status status = SI_OK;
};

struct Batch {
    std::vector<Request *> reqs;
    cudaEvent_t done;
    cudaStream_t stream;
};

constexpr int kServeStreams = 4;
constexpr int kMaxBatchItems = 256;

}  // namespace

struct Server {
    int device = 0;
    size_t budget = 0, used = 0;
    int max_inflight = 1, inflight = 0;
    std::vector<si_mesh_t> meshes;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    std::vector<Batch> running;
    cudaStream_t streams[kServeStreams] = {};
    int next_stream = 0;
    uint64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    si_status fatal = SI_OK;

    void run();
    bool admit_and_launch(std::unique_lock<std::mutex> &lk);
    void reap(bool block);
};

// Budget charged for a request's call scratch: query permutation and sort
// histogram (an estimate; the grid itself belongs to the mesh).
static size_t request_scratch_bytes(const si_batch_item &it) {
    return sizeof(int) * (2 * (size_t)it.m + 65536) + 8192;
}

bool Server::admit_and_launch(std::unique_lock<std::mutex> &lk) {
    // called with mu held; releases it while enqueueing
    std::vector<Request *> take;
    size_t add = 0;
    while (!queue.empty() && inflight + (int)take.size() < max_inflight && (int)take.size() < kMaxBatchItems) {
        Request *r = queue.front();
        if (used + add + r->bytes > budget) break;  // FIFO: the head waits for memory
        add += r->bytes;
        take.push_back(r);
        queue.pop_front();
    }
    if (take.empty()) return false;
    used += add;
    inflight += (int)take.size();
    Batch b;
    b.stream = streams[next_stream];
    next_stream = (next_stream + 1) % kServeStreams;
    b.reqs = take;
    lk.unlock();  // submit/poll stay responsive while the batch is enqueued
    std::vector<si_batch_item> items;
    std::vector<si_schedule> scheds;
    std::vector<const si_probe *> probes;
    si_status st = SI_OK;
    for (Request *r : take) {
        if (r->own_out && r->item.out == nullptr) {
            void *p = nullptr;
            st = dev_alloc(&p, r->out_bytes, b.stream);
            if (st != SI_OK) break;
            r->item.out = reinterpret_cast<int32_t *>(p);
        }
        items.push_back(r->item);
        si_schedule s{SI_SCHED_GSS, 1, 0, 0, 0};
        const Mesh *m = reinterpret_cast<const Mesh *>(r->item.mesh);
        if (si_tune_lookup(r->item.W, m->n, r->item.m, &s) != SI_OK) s = si_schedule{SI_SCHED_GSS, 1, 0, 0, 0};
        s.num_workers = 0;
        scheds.push_back(s);
    }
    if (st == SI_OK) st = enqueue_batch(items, scheds, probes, b.stream, 0);
    cudaError_t e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(b.done, b.stream);
    if (e != cudaSuccess && st == SI_OK) st = cuda_fail(e, "serve batch event");
    lk.lock();
    for (Request *r : take) r->status = st;
    running.push_back(b);
    return true;
}

void Server::reap(bool block) {
    // called with mu held
    for (size_t k = 0; k < running.size();) {
        Batch &b = running[k];
        cudaError_t q = cudaEventQuery(b.done);
        if (q == cudaErrorNotReady && block) {
            mu.unlock();
            cudaEventSynchronize(b.done);
            mu.lock();
            q = cudaEventQuery(b.done);
        }
        if (q == cudaErrorNotReady) {
            ++k;
            continue;
        }
        const auto now = Clock::now();
        for (Request *r : b.reqs) {
            if (q != cudaSuccess && r->status == SI_OK) r->status = cuda_fail(q, "serve batch");
            r->done = true;
            r->done_at = now;
            used -= (r->bytes - r->out_bytes);  // scratch back; owned output stays charged until release
            --inflight;
        }
        cudaEventDestroy(b.done);
        running.erase(running.begin() + k);
        cv_done.notify_all();
    }
}

void Server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        reap(false);
        bool launched = admit_and_launch(lk);
        if (stop && queue.empty() && running.empty()) break;
        if (launched) continue;
        if (running.empty()) {
            cv_work.wait_for(lk, std::chrono::milliseconds(5));
        } else {
            // poll completions at a fine grain without holding the lock
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace si

using namespace si;

extern "C" {

si_status si_serve_create(size_t mem_budget_bytes, int32_t max_inflight, si_server_t *out) {
    if (!out || max_inflight < 1 || mem_budget_bytes == 0) {
        set_error("si_serve_create: need a budget > 0, max_inflight >= 1 and an output handle");
        return SI_ERR_INVALID;
    }
    Server *s = new Server();
    SI_CUDA(cudaGetDevice(&s->device));
    s->budget = mem_budget_bytes;
    s->max_inflight = max_inflight;
    for (int k = 0; k < kServeStreams; ++k) {
        cudaError_t e = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (int j = 0; j < k; ++j) cudaStreamDestroy(s->streams[j]);
            delete s;
            return cuda_fail(e, "cudaStreamCreate(server)");
        }
    }
    s->worker = std::thread([s] { s->run(); });
    *out = reinterpret_cast<si_server_t>(s);
    return SI_OK;
}

si_status si_serve_add_mesh(si_server_t sv, si_mesh_t mesh, int32_t *mesh_slot) {
    if (!sv || !mesh) {
        set_error("si_serve_add_mesh: NULL argument");
        return SI_ERR_INVALID;
    }
    Server *s = reinterpret_cast<Server *>(sv);
    std::lock_guard<std::mutex> lk(s->mu);
    s->meshes.push_back(mesh);
    if (mesh_slot) *mesh_slot = (int32_t)s->meshes.size() - 1;
    return SI_OK;
}

si_status si_serve_submit(si_server_t sv, const si_batch_item *req, uint64_t *ticket) {
    if (!sv || !req || !ticket) {
        set_error("si_serve_submit: NULL argument");
        return SI_ERR_INVALID;
    }
    Server *s = reinterpret_cast<Server *>(sv);
    bool known = false;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (si_mesh_t m : s->meshes) known |= (m == req->mesh);
    }
    if (!known) {
        set_error("si_serve_submit: mesh was not added to this server");
        return SI_ERR_INVALID;
    }
    si_batch_item it = *req;
    const bool own = it.out == nullptr;
    // validate now (synchronous argument errors); a placeholder output pointer
    // stands in for a server-allocated one
    si_batch_item chk = it;
    if (own) chk.out = reinterpret_cast<int32_t *>(16);
    si_schedule sc{SI_SCHED_GSS, 1, 0, 0, 0};
    si_status st = check_item(chk, sc, s->device);
    if (st != SI_OK) return st;
    Request *r = new Request();
    r->item = it;
    r->own_out = own;
    r->out_bytes = own ? sizeof(int32_t) * (size_t)it.m * it.W * it.W : 0;
    r->bytes = r->out_bytes + request_scratch_bytes(it);
    r->submit = Clock::now();
    if (r->bytes > s->budget) {
        set_error("si_serve_submit: request needs %zu bytes, the whole budget is %zu", r->bytes, s->budget);
        delete r;
        return SI_ERR_BUSY;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return SI_OK;
}

si_status si_serve_poll(si_server_t sv, uint64_t ticket, int32_t *done) {
    if (!sv || !done) {
        set_error("si_serve_poll: NULL argument");
        return SI_ERR_INVALID;
    }
    Server *s = reinterpret_cast<Server *>(sv);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        set_error("si_serve_poll: unknown ticket");
        return SI_ERR_INVALID;
    }
    *done = it->second->done ? 1 : 0;
    return it->second->done ? it->second->status : SI_OK;
}

si_status si_serve_wait(si_server_t sv, uint64_t ticket, int32_t timeout_ms) {
    if (!sv) {
        set_error("si_serve_wait: NULL server");
        return SI_ERR_INVALID;
    }
    Server *s = reinterpret_cast<Server *>(sv);
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        set_error("si_serve_wait: unknown ticket");
        return SI_ERR_INVALID;
    }
    Request *r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, pred);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        set_error("si_serve_wait: ticket %llu not done after %d ms", (unsigned long long)ticket, timeout_ms);
        return SI_ERR_TIMEOUT;
    }
    return r->status;
}

si_status si_serve_result(si_server_t sv, uint64_t ticket, int32_t **out, double *latency_us) {
    if (!sv) {
        set_error("si_serve_result: NULL server");
        return SI_ERR_INVALID;
    }
    Server *s = reinterpret_cast<Server *>(sv);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end() || !it->second->done) {
        set_error("si_serve_result: ticket unknown or not complete");
        return SI_ERR_INVALID;
    }
    Request *r = it->second;
    if (out) *out = r->item.out;
    if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(r->done_at - r->submit).count();
    return r->status;
}

si_status si_serve_release(si_server_t sv, uint64_t ticket) {
    if (!sv) {
        set_error("si_serve_release: NULL server");
        return SI_ERR_INVALID;
    }
    Server *s = reinterpret_cast<Server *>(sv);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end() || !it->second->done) {
        set_error("si_serve_release: ticket unknown or not complete");
        return SI_ERR_INVALID;
    }
    Request *r = it->second;
    if (r->own_out && r->item.out) cudaFreeAsync(r->item.out, s->streams[0]);
    s->used -= r->out_bytes;
    s->all.erase(it);
    delete r;
    s->cv_work.notify_one();
    return SI_OK;
}

si_status si_serve_destroy(si_server_t sv) {
    if (!sv) {
        set_error("si_serve_destroy: NULL server");
        return SI_ERR_INVALID;
    }
    Server *s = reinterpret_cast<Server *>(sv);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    for (auto &kv : s->all) {
        Request *r = kv.second;
        if (r->own_out && r->item.out) cudaFreeAsync(r->item.out, s->streams[0]);
        delete r;
    }
    for (int k = 0; k < kServeStreams; ++k) {
        cudaStreamSynchronize(s->streams[k]);
        cudaStreamDestroy(s->streams[k]);
    }
    delete s;
    return SI_OK;
}

}  // extern "C"
