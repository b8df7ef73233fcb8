// Serving runtime: continuous batching of evaluation requests on one device.
//
// Requests (a problem, its branch lengths and host outputs) queue in arrival order.  One worker
// thread admits the oldest ones while a slot (a CUDA stream, its completion event and a pinned
// result buffer) and room in the device arena are free: the problem is laid out in an arena range,
// copied on the slot's stream, evaluated there (the same launches as pg_eval_async, so a result is
// bit-identical whether the request runs alone or among others) and its logL, gradient, Hessian
// diagonal and device status are copied back into the slot's pinned buffer.  The worker retires a
// request when its event has completed, frees its range and admits the next; requests that
// arrive meanwhile join as soon as a slot and memory free up, so the streams of different requests
// overlap on the device.  The arena is one device allocation with a first-fit sub-allocator, so
// admission never calls cudaMalloc or cudaFree (both would wait for the whole device).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pg_host.h"

using pg::host::fail;

namespace {

constexpr size_t kGranule = 256;

// First-fit sub-allocator over one device range; free ranges are kept by offset and coalesce.
class Arena {
  public:
    bool init(size_t bytes) {
        bytes = (bytes / kGranule) * kGranule;
        if (bytes == 0 || cudaMalloc(&base_, bytes) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return false;
        }
        total_ = bytes;
        free_[0] = bytes;
        return true;
    }
    void destroy() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    void *alloc(size_t n) {
        n = (n + kGranule - 1) / kGranule * kGranule;
        last_request_ = n;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            const size_t off = it->first, rest = it->second - n;
            free_.erase(it);
            if (rest) free_[off + n] = rest;
            used_[off] = n;
            return static_cast<char *>(base_) + off;
        }
        return nullptr;
    }
    void release(void *p) {
        const size_t off = static_cast<size_t>(static_cast<char *>(p) - static_cast<char *>(base_));
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t start = off, len = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && next->first == start + len) {
            len += next->second;
            free_.erase(next);
        }
        auto prev = free_.lower_bound(start);
        if (prev != free_.begin()) {
            --prev;
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
    }
    size_t total() const { return total_; }
    size_t last_request() const { return last_request_; }

  private:
    void *base_ = nullptr;
    size_t total_ = 0, last_request_ = 0;
    std::map<size_t, size_t> free_;               // offset -> bytes
    std::unordered_map<size_t, size_t> used_;     // offset -> bytes
};

void *arena_alloc(void *self, size_t n) { return static_cast<Arena *>(self)->alloc(n); }
void arena_release(void *self, void *p) { static_cast<Arena *>(self)->release(p); }

enum { kPending = 0, kRunning = 1, kDone = 2 };

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    char *pinned = nullptr;   // logL, grad [n], hess [n], status
    size_t cap = 0;
};

struct Request {
    uint64_t ticket = 0;
    pg_request rq{};
    int state = kPending;
    pg_status status = PG_OK;
    std::string error;
    pg_handle *h = nullptr;
    void *block = nullptr;
    int slot = -1;
    int n = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
};

}  // namespace

struct pg_server {
    pg_ctx *ctx = nullptr;
    Arena arena;
    std::vector<Slot> slots;
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::vector<Request *> running;
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

size_t result_bytes(int n) { return sizeof(double) * (1 + 2 * (size_t)n) + 16; }

// copy the request in, evaluate, copy the results out, all on the slot's stream
pg_status admit(pg_server *S, Request *r, int si) {
    Slot &sl = S->slots[si];
    pg::host::Placement pl;
    pl.alloc = arena_alloc;
    pl.release = arena_release;
    pl.self = &S->arena;
    pl.stream = sl.stream;
    pg_handle *h = nullptr;
    pg_status st = pg::host::upload(S->ctx, r->rq.problem, &h, &pl);
    if (st != PG_OK) return st;
    void *block = h->block;
    auto drop = [&](pg_status why) {   // undo the upload once the stream has let go of the range
        cudaStreamSynchronize(sl.stream);
        pg_free(h);
        S->arena.release(block);
        return why;
    };
    const int n = h->n_user;   // the caller's nodes (a multifurcating tree's added nodes stay internal)
    if (sl.cap < result_bytes(n)) {   // grow the slot's pinned buffer (rare)
        cudaStreamSynchronize(sl.stream);
        if (sl.pinned) cudaFreeHost(sl.pinned);
        sl.pinned = nullptr;
        sl.cap = 0;
        if (cudaMallocHost(reinterpret_cast<void **>(&sl.pinned), result_bytes(n)) != cudaSuccess) {
            cudaGetLastError();
            return drop(fail(PG_ERR_OOM, "pinned host allocation failed"));
        }
        sl.cap = result_bytes(n);
    }
    r->h = h;
    r->block = block;
    r->n = n;
    double *pin = reinterpret_cast<double *>(sl.pinned);
    cudaError_t e = cudaMemcpyAsync(h->io_b, r->rq.b, sizeof(double) * n, cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess) {
        st = pg::host::enqueue(h, 0, h->io_b, h->io_logL, r->rq.grad ? h->io_grad : nullptr,
                               r->rq.hess ? h->io_hess : nullptr, nullptr, nullptr, sl.stream);
        if (st != PG_OK) return drop(st);
        e = cudaMemcpyAsync(pin, h->io_logL, sizeof(double), cudaMemcpyDeviceToHost, sl.stream);
    }
    if (e == cudaSuccess && r->rq.grad)
        e = cudaMemcpyAsync(pin + 1, h->io_grad, sizeof(double) * n, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess && r->rq.hess)
        e = cudaMemcpyAsync(pin + 1 + n, h->io_hess, sizeof(double) * n, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pin + 1 + 2 * (size_t)n, h->desc.status, sizeof(int), cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
    if (e != cudaSuccess) return drop(fail(PG_ERR_CUDA, "serving copies: %s", cudaGetErrorString(e)));
    return PG_OK;
}

// the slot's event has completed: hand the results to the caller and free the request's memory
void retire(pg_server *S, Request *r, cudaError_t q) {
    Slot &sl = S->slots[r->slot];
    const double *pin = reinterpret_cast<const double *>(sl.pinned);
    const int n = r->n;
    if (q != cudaSuccess) {
        r->status = PG_ERR_CUDA;
        r->error = cudaGetErrorString(q);
    } else {
        int dev_status = 0;
        std::memcpy(&dev_status, pin + 1 + 2 * (size_t)n, sizeof(int));
        if (r->rq.logL) *r->rq.logL = pin[0];
        if (r->rq.grad) std::memcpy(r->rq.grad, pin + 1, sizeof(double) * n);
        if (r->rq.hess) std::memcpy(r->rq.hess, pin + 1 + n, sizeof(double) * n);
        if (dev_status & pg::kStatusBadLength) r->status = PG_ERR_INVALID;
        else if (dev_status & pg::kStatusNumeric) r->status = PG_ERR_NUMERIC;
        else if (dev_status & pg::kStatusTimeout) r->status = PG_ERR_TIMEOUT;
        else r->status = PG_OK;
    }
    pg_free(r->h);
    S->arena.release(r->block);
    r->h = nullptr;
    r->block = nullptr;
    S->free_slots.push_back(r->slot);
    r->slot = -1;
    r->state = kDone;
    r->t_done = S->now();
}

void worker(pg_server *S) {
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progress = false;
        for (size_t i = 0; i < S->running.size();) {
            Request *r = S->running[i];
            const cudaError_t q = cudaEventQuery(S->slots[r->slot].done);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            retire(S, r, q);
            S->running.erase(S->running.begin() + (long)i);
            progress = true;
            S->cv_done.notify_all();
        }
        while (!S->pending.empty() && !S->free_slots.empty()) {
            Request *r = S->pending.front();
            const int si = S->free_slots.back();
            lk.unlock();
            const pg_status st = admit(S, r, si);
            const std::string err = st == PG_OK ? std::string() : pg::host::g_err;
            lk.lock();
            // no room in the arena yet: wait for running requests to free theirs
            if (st == PG_ERR_OOM && !S->running.empty() && S->arena.last_request() <= S->arena.total()) break;
            S->pending.pop_front();
            if (st != PG_OK) {
                r->state = kDone;
                r->status = st;
                r->error = err;
                r->t_start = r->t_done = S->now();
                S->cv_done.notify_all();
                continue;
            }
            S->free_slots.pop_back();
            r->slot = si;
            r->state = kRunning;
            r->t_start = S->now();
            S->running.push_back(r);
            progress = true;
        }
        if (S->stop && S->pending.empty() && S->running.empty()) break;
        if (S->pending.empty() && S->running.empty()) {
            S->cv_work.wait(lk);
            continue;
        }
        if (!progress) {   // poll the running requests' events again shortly
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

}  // namespace

extern "C" {

pg_status pg_server_create(pg_ctx *ctx, const pg_server_options *opt, pg_server **out) {
    if (!ctx || !out) return fail(PG_ERR_INVALID, "NULL argument");
    *out = nullptr;
    pg_server_options o{};
    if (opt) o = *opt;
    if (o.max_inflight < 0) return fail(PG_ERR_INVALID, "max_inflight = %d", o.max_inflight);
    const int slots = o.max_inflight ? o.max_inflight : 4;
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(PG_ERR_CUDA, "cannot select device %d", ctx->device);
    size_t bytes = o.arena_bytes;
    if (bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(PG_ERR_CUDA, "cudaMemGetInfo failed");
        bytes = fr / 10 * 6;
    }
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (ctx->budget && ctx->used + bytes > ctx->budget)
            return fail(PG_ERR_OOM, "arena of %zu bytes exceeds the context's budget", bytes);
    }
    pg_server *S = new (std::nothrow) pg_server;
    if (!S) return fail(PG_ERR_OOM, "host allocation failed");
    S->ctx = ctx;
    S->t0 = std::chrono::steady_clock::now();
    if (!S->arena.init(bytes)) {
        delete S;
        if (prev >= 0) cudaSetDevice(prev);
        return fail(PG_ERR_OOM, "cannot allocate a serving arena of %zu bytes", bytes);
    }
    S->slots.resize(slots);
    for (int i = 0; i < slots; ++i) {
        Slot &sl = S->slots[i];
        bool ok = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess &&
                  cudaMallocHost(reinterpret_cast<void **>(&sl.pinned), result_bytes(16384)) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            for (auto &x : S->slots) {
                if (x.stream) cudaStreamDestroy(x.stream);
                if (x.done) cudaEventDestroy(x.done);
                if (x.pinned) cudaFreeHost(x.pinned);
            }
            S->arena.destroy();
            delete S;
            if (prev >= 0) cudaSetDevice(prev);
            return fail(PG_ERR_CUDA, "cannot create the serving streams");
        }
        sl.cap = result_bytes(16384);
        S->free_slots.push_back(slots - 1 - i);
    }
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->used += S->arena.total();
    }
    S->worker = std::thread(worker, S);
    if (prev >= 0) cudaSetDevice(prev);
    *out = S;
    return PG_OK;
}

pg_status pg_server_submit(pg_server *S, const pg_request *rq, uint64_t *ticket) {
    if (!S || !rq || !rq->problem || !rq->b || !ticket) return fail(PG_ERR_INVALID, "NULL argument");
    Request *r = new (std::nothrow) Request;
    if (!r) return fail(PG_ERR_OOM, "host allocation failed");
    r->rq = *rq;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) {
            delete r;
            return fail(PG_ERR_INVALID, "the server is shutting down");
        }
        r->ticket = S->next_ticket++;
        r->t_submit = S->now();
        S->reqs[r->ticket] = r;
        S->pending.push_back(r);
        *ticket = r->ticket;
    }
    S->cv_work.notify_one();
    return PG_OK;
}

pg_status pg_server_wait(pg_server *S, uint64_t ticket, pg_request_info *info) {
    if (!S) return fail(PG_ERR_INVALID, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(PG_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    S->cv_done.wait(lk, [&] { return r->state == kDone; });
    const pg_status st = r->status;
    if (info) {
        info->status = st;
        info->reserved = 0;
        info->submit_s = r->t_submit;
        info->start_s = r->t_start;
        info->done_s = r->t_done;
    }
    if (st != PG_OK) pg::host::set_error(r->error);
    S->reqs.erase(it);
    delete r;
    return st;
}

pg_status pg_server_destroy(pg_server *S) {
    if (!S) return PG_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->reqs) delete kv.second;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->ctx->device);
    for (auto &sl : S->slots) {
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
        cudaFreeHost(sl.pinned);
    }
    {
        std::lock_guard<std::mutex> g(S->ctx->mu);
        S->ctx->used -= S->arena.total();
    }
    S->arena.destroy();
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
    return PG_OK;
}

}  // extern "C"
