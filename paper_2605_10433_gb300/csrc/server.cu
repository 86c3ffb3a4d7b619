// Serving loop: continuous batching of syndrome-decoding requests from several codes.
//
// Requests (a code, a batch of syndromes and priors in host memory, host output buffers)
// arrive at any time through sagms_server_submit.  A scheduler thread admits them in
// arrival order as device memory and in-flight slots free up: memory comes from one
// device arena allocated at creation (first fit with coalescing), so admission is gated by
// free memory and no request allocates.  Each admitted request gets its own stream: copy
// in, decode, copy out, completion event.  In continuous mode several requests are on the
// GPU at once and each decode's grid is capped at about one CTA per `shots_per_cta` shots,
// so its CTAs retire as they finish and the CTAs of newer requests take the freed SMs
// (inside a CTA the continuous-batching kernels refill their slots or groups shot by shot).  Plain mode is the
// baseline the loop is measured against: one request at a time on one stream, each decode
// with the full persistent grid.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using sagms_internal::Plan;

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit allocator over [0, size) with coalescing free blocks (offsets, host side).
class Arena {
  public:
    explicit Arena(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
  private:
    std::map<size_t, size_t> free_;
    size_t used_ = 0;
};

enum State { kQueued, kRunning, kDone, kCancelled, kFailed };

struct Request {
    uint64_t id;
    int code_id;
    int64_t shots;
    const uint32_t* h_syn;
    const float* h_L0;
    uint32_t* h_err;
    uint8_t* h_conv;
    int32_t* h_iters;
    size_t bytes = 0, off = 0;
    int slot = -1;
    State state = kQueued;
    int rc = SAGMS_OK;
    int64_t t_submit = 0, t_done = 0;
};

struct CodeEntry {
    const sagms_code* code;
    sagms_params params;
    int m, n;
};

}  // namespace

struct sagms_server {
    int device = 0;
    int mode = SAGMS_SERVE_CONTINUOUS;
    int shots_per_cta = 16;
    size_t budget = 0;
    unsigned char* arena_base = nullptr;
    int* counters = nullptr;   // per slot: chunk counters of its launches
    std::unique_ptr<Arena> arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<uint64_t> slot_req;   // request id per in-flight slot (0 = free)
    std::vector<CodeEntry> codes;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    uint64_t next_id = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    std::atomic<int64_t> admitted{0}, completed{0};

    void run();
    void launch_request(Request& r, int slot);
};

namespace {

constexpr int kCountersPerSlot = 64;

size_t request_bytes(const CodeEntry& c, int64_t shots, bool per_qubit) {
    const size_t mw = (c.m + 31) / 32, nw = (c.n + 31) / 32;
    return align_up((size_t)shots * mw * 4, 256) + align_up((per_qubit ? (size_t)c.n : (size_t)shots) * 4, 256) +
           align_up((size_t)shots * nw * 4, 256) + align_up((size_t)shots, 256) + align_up((size_t)shots * 4, 256);
}

}  // namespace

void sagms_server::launch_request(Request& r, int slot) {
    const sagms_internal::NvtxRange nvtx("sagms_server_request");
    const CodeEntry& c = codes[r.code_id];
    const bool per_qubit = (c.params.flags & SAGMS_FLAG_L0_PER_QUBIT) != 0;
    const size_t mw = (c.m + 31) / 32, nw = (c.n + 31) / 32;
    unsigned char* p = arena_base + r.off;
    uint32_t* d_syn = reinterpret_cast<uint32_t*>(p);
    p += align_up((size_t)r.shots * mw * 4, 256);
    float* d_L0 = reinterpret_cast<float*>(p);
    const size_t l0_bytes = (per_qubit ? (size_t)c.n : (size_t)r.shots) * 4;
    p += align_up(l0_bytes, 256);
    uint32_t* d_err = reinterpret_cast<uint32_t*>(p);
    p += align_up((size_t)r.shots * nw * 4, 256);
    uint8_t* d_conv = p;
    p += align_up((size_t)r.shots, 256);
    int32_t* d_iters = reinterpret_cast<int32_t*>(p);
    cudaStream_t st = streams[slot];
    cudaError_t ce = cudaMemcpyAsync(d_syn, r.h_syn, (size_t)r.shots * mw * 4, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_L0, r.h_L0, l0_bytes, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) { r.rc = sagms_internal::cuda_error(ce, "server copy-in"); return; }
    Plan plan;
    plan.work = counters + slot * kCountersPerSlot;
    if (mode == SAGMS_SERVE_CONTINUOUS)
        plan.max_grid = std::max<long long>(1, (r.shots + shots_per_cta - 1) / shots_per_cta);
    r.rc = sagms_internal::launch(c.code, &c.params, r.shots, d_syn, d_L0, d_err, d_conv, d_iters, st, &plan);
    if (r.rc != SAGMS_OK) return;
    ce = cudaMemcpyAsync(r.h_err, d_err, (size_t)r.shots * nw * 4, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(r.h_conv, d_conv, (size_t)r.shots, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(r.h_iters, d_iters, (size_t)r.shots * 4, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaEventRecord(events[slot], st);
    if (ce != cudaSuccess) r.rc = sagms_internal::cuda_error(ce, "server copy-out");
}

void sagms_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // completions
        bool any_running = false;
        for (size_t k = 0; k < slot_req.size(); ++k) {
            if (!slot_req[k]) continue;
            Request& r = *reqs[slot_req[k]];
            const cudaError_t q = cudaEventQuery(events[k]);
            if (q == cudaErrorNotReady) { any_running = true; continue; }
            r.rc = (q == cudaSuccess) ? SAGMS_OK : sagms_internal::cuda_error(q, "server decode");
            r.state = (q == cudaSuccess) ? kDone : kFailed;
            r.t_done = now_ns();
            arena->release(r.off, r.bytes);
            slot_req[k] = 0;
            completed++;
            cv_done.notify_all();
        }
        // admissions in arrival order, gated by a free slot and arena memory
        while (!queue.empty()) {
            const auto it = reqs.find(queue.front());
            if (it == reqs.end() || it->second->state == kCancelled) { queue.pop_front(); continue; }
            Request& r = *it->second;
            int slot = -1;
            for (size_t k = 0; k < slot_req.size(); ++k)
                if (!slot_req[k]) { slot = (int)k; break; }
            if (slot < 0) break;
            size_t off = 0;
            if (!arena->alloc(r.bytes, &off)) break;   // head-of-line: wait for memory
            queue.pop_front();
            r.off = off;
            r.slot = slot;
            launch_request(r, slot);
            if (r.rc != SAGMS_OK) {
                cudaStreamSynchronize(streams[slot]);   // copies already queued must finish first
                arena->release(off, r.bytes);
                r.state = kFailed;
                r.t_done = now_ns();
                cv_done.notify_all();
                continue;
            }
            r.state = kRunning;
            slot_req[slot] = r.id;
            admitted++;
            any_running = true;
        }
        if (stop && !any_running && queue.empty()) break;
        if (!any_running && queue.empty()) {
            cv_work.wait(lk);
        } else {
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        }
    }
}

extern "C" {

int sagms_server_create(size_t mem_budget, int32_t max_inflight, int32_t mode, int32_t shots_per_cta,
                        sagms_server** out) {
    using sagms_internal::set_error;
    if (!out) return set_error(SAGMS_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (mode != SAGMS_SERVE_CONTINUOUS && mode != SAGMS_SERVE_PLAIN) return set_error(SAGMS_ERR_ARG, "unknown serving mode");
    if (mem_budget < 4096 || max_inflight < 1 || max_inflight > 256 || shots_per_cta < 1)
        return set_error(SAGMS_ERR_ARG, "need mem_budget >= 4096, 1 <= max_inflight <= 256, shots_per_cta >= 1");
    auto s = std::make_unique<sagms_server>();
    cudaError_t ce = cudaGetDevice(&s->device);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "cudaGetDevice");
    s->mode = mode;
    s->shots_per_cta = shots_per_cta;
    s->budget = mem_budget;
    const int slots = (mode == SAGMS_SERVE_PLAIN) ? 1 : max_inflight;
    ce = cudaMalloc(&s->arena_base, mem_budget);
    if (ce != cudaSuccess) return sagms_internal::cuda_error(ce, "server arena");
    ce = cudaMalloc(&s->counters, (size_t)slots * kCountersPerSlot * sizeof(int));
    if (ce != cudaSuccess) {
        cudaFree(s->arena_base);
        return sagms_internal::cuda_error(ce, "server counters");
    }
    s->arena = std::make_unique<Arena>(mem_budget);
    for (int k = 0; k < slots; ++k) {
        cudaStream_t st;
        cudaEvent_t ev;
        ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (ce != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            for (auto x : s->events) cudaEventDestroy(x);
            cudaFree(s->arena_base);
            cudaFree(s->counters);
            return sagms_internal::cuda_error(ce, "server streams");
        }
        s->streams.push_back(st);
        s->events.push_back(ev);
    }
    s->slot_req.assign(slots, 0);
    sagms_server* raw = s.release();
    raw->worker = std::thread([raw] { raw->run(); });
    *out = raw;
    return SAGMS_OK;
}

int sagms_server_add_code(sagms_server* s, const sagms_code* code, const sagms_params* params, int32_t* code_id) {
    using sagms_internal::set_error;
    if (!s || !code || !params || !code_id) return set_error(SAGMS_ERR_ARG, "NULL argument");
    const int rc = sagms_check_params(params);
    if (rc != SAGMS_OK) return rc;
    int32_t m = 0, n = 0;
    sagms_code_info(code, &m, &n, nullptr, nullptr);
    std::lock_guard<std::mutex> lk(s->mu);
    s->codes.push_back(CodeEntry{code, *params, m, n});
    *code_id = (int32_t)s->codes.size() - 1;
    return SAGMS_OK;
}

int sagms_server_submit(sagms_server* s, int32_t code_id, int64_t shots, const uint32_t* h_syn, const float* h_L0,
                        uint32_t* h_err, uint8_t* h_conv, int32_t* h_iters, uint64_t* ticket) {
    using sagms_internal::set_error;
    if (!s || !ticket) return set_error(SAGMS_ERR_ARG, "NULL argument");
    if (shots < 1) return set_error(SAGMS_ERR_ARG, "a request needs at least one shot");
    if (!h_syn || !h_L0 || !h_err || !h_conv || !h_iters) return set_error(SAGMS_ERR_ARG, "NULL host buffer");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return set_error(SAGMS_ERR_BUSY, "server is shutting down");
    if (code_id < 0 || code_id >= (int32_t)s->codes.size()) return set_error(SAGMS_ERR_ARG, "unknown code id");
    const CodeEntry& c = s->codes[code_id];
    const size_t need = request_bytes(c, shots, (c.params.flags & SAGMS_FLAG_L0_PER_QUBIT) != 0);
    if (need > s->budget) return set_error(SAGMS_ERR_SIZE, "request needs more device memory than the server budget");
    auto r = std::make_unique<Request>();
    r->id = s->next_id++;
    r->code_id = code_id;
    r->shots = shots;
    r->h_syn = h_syn; r->h_L0 = h_L0; r->h_err = h_err; r->h_conv = h_conv; r->h_iters = h_iters;
    r->bytes = need;
    r->t_submit = now_ns();
    *ticket = r->id;
    s->queue.push_back(r->id);
    s->reqs[r->id] = std::move(r);
    s->cv_work.notify_one();
    return SAGMS_OK;
}

int sagms_server_poll(sagms_server* s, uint64_t ticket, int64_t timeout_us) {
    using sagms_internal::set_error;
    if (!s) return set_error(SAGMS_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(SAGMS_ERR_ARG, "unknown ticket");
    Request* r = it->second.get();
    auto finished = [&] { return r->state == kDone || r->state == kFailed || r->state == kCancelled; };
    if (!finished()) {
        if (timeout_us <= 0) return set_error(SAGMS_ERR_TIMEOUT, "request not finished");
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), finished);
        if (!finished()) return set_error(SAGMS_ERR_TIMEOUT, "request not finished within the timeout");
    }
    if (r->state == kCancelled) return set_error(SAGMS_ERR_CANCELLED, "request was cancelled");
    return r->rc;
}

int sagms_server_cancel(sagms_server* s, uint64_t ticket) {
    using sagms_internal::set_error;
    if (!s) return set_error(SAGMS_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(SAGMS_ERR_ARG, "unknown ticket");
    Request& r = *it->second;
    if (r.state != kQueued) return set_error(SAGMS_ERR_BUSY, "request already admitted or finished");
    r.state = kCancelled;
    r.t_done = now_ns();
    // out of the admission queue now, so a release right after the cancel leaves no stale id
    const auto q = std::find(s->queue.begin(), s->queue.end(), ticket);
    if (q != s->queue.end()) s->queue.erase(q);
    s->cv_done.notify_all();
    return SAGMS_OK;
}

int sagms_server_times(sagms_server* s, uint64_t ticket, int64_t* submit_ns, int64_t* done_ns) {
    using sagms_internal::set_error;
    if (!s) return set_error(SAGMS_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(SAGMS_ERR_ARG, "unknown ticket");
    if (submit_ns) *submit_ns = it->second->t_submit;
    if (done_ns) *done_ns = it->second->t_done;
    return SAGMS_OK;
}

int sagms_server_release(sagms_server* s, uint64_t ticket) {
    using sagms_internal::set_error;
    if (!s) return set_error(SAGMS_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(SAGMS_ERR_ARG, "unknown ticket");
    const State st = it->second->state;
    if (st == kQueued || st == kRunning) return set_error(SAGMS_ERR_BUSY, "request not finished");
    s->reqs.erase(it);
    return SAGMS_OK;
}

int sagms_server_destroy(sagms_server* s) {
    if (!s) return SAGMS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (uint64_t id : s->queue) {
            const auto it = s->reqs.find(id);
            if (it != s->reqs.end() && it->second->state == kQueued) {
                it->second->state = kCancelled;
                it->second->t_done = now_ns();
            }
        }
        s->queue.clear();
        s->cv_work.notify_all();
        s->cv_done.notify_all();
    }
    s->worker.join();
    for (auto x : s->streams) cudaStreamDestroy(x);
    for (auto x : s->events) cudaEventDestroy(x);
    cudaFree(s->arena_base);
    cudaFree(s->counters);
    delete s;
    return SAGMS_OK;
}

int sagms_server_replay(sagms_server* s, int32_t n, const int32_t* code_ids, const int64_t* shots,
                        const int64_t* arrival_ns, const uint32_t* const* h_syn, const float* const* h_L0,
                        uint32_t* const* h_err, uint8_t* const* h_conv, int32_t* const* h_iters, uint64_t* tickets) {
    using sagms_internal::set_error;
    if (!s || n < 0 || (n > 0 && (!code_ids || !shots || !arrival_ns || !h_syn || !h_L0 || !h_err || !h_conv ||
                                  !h_iters || !tickets)))
        return set_error(SAGMS_ERR_ARG, "bad replay arguments");
    const int64_t t0 = now_ns();
    for (int i = 0; i < n; ++i) {
        while (now_ns() - t0 < arrival_ns[i]) {
        }
        const int rc = sagms_server_submit(s, code_ids[i], shots[i], h_syn[i], h_L0[i], h_err[i], h_conv[i],
                                           h_iters[i], &tickets[i]);
        if (rc != SAGMS_OK) return rc;
    }
    return SAGMS_OK;
}

}  // extern "C"
