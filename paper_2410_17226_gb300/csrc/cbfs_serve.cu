// libcbfs.so, part 4: the distance-query server (continuous batching).
//
// The labels of Section 4.2 stay resident on the device; requests (arrays of
// vertex pairs of any size, in host memory) arrive at any time.  A
// dispatcher thread packs waiting requests, in arrival order, into batches of
// at most max_batch pairs and launches each batch on one of `slots` CUDA
// streams as soon as a slot is free and the batch's device bytes fit the
// budget: page-locked staging -> H2D copy -> the query kernel
// (cbfs_query_distance) -> D2H copy -> event.  Batches launched while others
// are on the device overlap with them.  Each slot has its own waiter thread,
// which blocks on that slot's event, scatters the answers into the
// requests' host buffers and marks requests complete -- so a batch that
// finishes early is never held behind an earlier, larger one.
//
// Memory: at creation the server takes its batch buffers (device pairs and
// answers, 10 bytes per pair, slots x max_batch pairs) within a device budget
// (the caller's, or a quarter of the device memory free at creation); a
// batch is admitted when the bytes of the batches in flight plus its own fit
// the budget.  A request's answers do not depend on what else is in flight:
// every pair is answered independently by the same kernel.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cbfs_internal.cuh"

namespace {

constexpr int64_t kPairBytes = 8 + 2;  // int32 pair + uint16 answer on the device

using Clock = std::chrono::steady_clock;

struct Request {
    const int32_t* pairs;  // caller's host memory, [q][2]
    uint16_t* out;         // caller's host memory, [q]
    int64_t q = 0;
    bool pinned_pairs = false;  // page-locked: copied by DMA straight into the batch
    bool pinned_out = false;    // page-locked: answers copied by DMA straight out of the batch
    int64_t packed = 0;     // pairs handed to batches so far
    int64_t remaining = 0;  // pairs not yet answered
    int status = CBFS_OK;
    bool done = false;
    Clock::time_point t_arrival, t_done;
};

struct Part {
    Request* req;
    int64_t req_off, batch_off, count;
};

struct Slot {
    cudaStream_t stream = nullptr;
    int32_t* h_pairs = nullptr;
    uint16_t* h_out = nullptr;
    int32_t* d_pairs = nullptr;
    uint16_t* d_out = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<Part> parts;
    int64_t count = 0;
    int64_t bytes = 0;
    bool launched = false;
    int launch_status = CBFS_OK;
    std::thread waiter;
};

}  // namespace

struct cbfs_server_s {
    cbfs_labels_t labels = nullptr;
    int device = 0;
    int64_t max_batch = 0;
    int64_t budget = 0;
    int64_t used = 0;
    std::vector<Slot*> slots;
    std::deque<Slot*> free_slots;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> tickets;
    uint64_t next_ticket = 1;
    std::mutex mu;
    std::condition_variable cv_dispatch;  // pending work, a free slot or budget, or stop
    std::condition_variable cv_done;      // a request completed
    std::condition_variable cv_slot;      // a slot was launched (waiters)
    bool stop = false;
    bool dispatcher_done = false;  // set by the dispatcher as it exits: no slot will be launched again
    std::thread dispatcher;
    // statistics
    uint64_t batches = 0, pairs_done = 0;
    std::vector<double> latency_ms;
};

namespace {

void run_waiter(cbfs_server_s* S, Slot* sl) {
    cudaSetDevice(S->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_slot.wait(lk, [&] { return sl->launched || S->dispatcher_done; });
            if (!sl->launched) return;  // stopping, and nothing in flight on this slot
        }
        int st = sl->launch_status;
        if (st == CBFS_OK && cudaEventSynchronize(sl->ev) != cudaSuccess) st = CBFS_E_CUDA;
        const Clock::time_point now = Clock::now();
        std::vector<Request*> finished;
        for (const Part& p : sl->parts) {
            if (st != CBFS_OK)
                p.req->status = st;
            else if (!p.req->pinned_out)  // page-locked outputs were written by DMA
                std::memcpy(p.req->out + p.req_off, sl->h_out + p.batch_off, sizeof(uint16_t) * (size_t)p.count);
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (const Part& p : sl->parts) {
                p.req->remaining -= p.count;
                if (p.req->remaining == 0) {
                    p.req->done = true;
                    p.req->t_done = now;
                    finished.push_back(p.req);
                }
            }
            for (Request* r : finished)
                S->latency_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_arrival).count());
            S->batches += 1;
            S->pairs_done += (uint64_t)sl->count;
            S->used -= sl->bytes;
            sl->parts.clear();
            sl->count = 0;
            sl->bytes = 0;
            sl->launched = false;
            S->free_slots.push_back(sl);
        }
        S->cv_done.notify_all();
        S->cv_dispatch.notify_all();
    }
}

void run_dispatcher(cbfs_server_s* S) {
    cudaSetDevice(S->device);
    for (;;) {
        Slot* sl = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_dispatch.wait(lk, [&] {
                return (S->stop && S->pending.empty()) ||
                       (!S->pending.empty() && !S->free_slots.empty() && S->used + kPairBytes <= S->budget);
            });
            if (S->pending.empty()) break;  // stopping, nothing left to launch
            sl = S->free_slots.front();
            S->free_slots.pop_front();
            // pack waiting requests in arrival order until the batch or the budget is full
            const int64_t room = std::min(S->max_batch, (S->budget - S->used) / kPairBytes);
            while (!S->pending.empty() && sl->count < room) {
                Request* r = S->pending.front();
                const int64_t take = std::min(r->q - r->packed, room - sl->count);
                sl->parts.push_back({r, r->packed, sl->count, take});
                sl->count += take;
                r->packed += take;
                if (r->packed == r->q) S->pending.pop_front();
            }
            sl->bytes = sl->count * kPairBytes;
            S->used += sl->bytes;
        }
        // staging and launch outside the lock (the parts' requests stay alive:
        // a request is released only after it is done).  Page-locked request
        // buffers are copied by DMA directly; the others through the slot's
        // page-locked staging, one host memcpy each way.
        // The staged parts go in one copy of the batch range they span, which
        // may include page-locked parts; those are copied after it on the same
        // stream, so their own pairs overwrite whatever the range carried.
        int st = CBFS_OK;
        int64_t staged_lo = -1, staged_hi = -1;  // batch range of the staged parts
        for (const Part& p : sl->parts) {
            if (p.req->pinned_pairs) continue;
            std::memcpy(sl->h_pairs + 2 * p.batch_off, p.req->pairs + 2 * p.req_off, sizeof(int32_t) * 2 * (size_t)p.count);
            if (staged_lo < 0) staged_lo = p.batch_off;
            staged_hi = p.batch_off + p.count;
        }
        if (staged_lo >= 0 &&
            cudaMemcpyAsync(sl->d_pairs + 2 * staged_lo, sl->h_pairs + 2 * staged_lo,
                            sizeof(int32_t) * 2 * (size_t)(staged_hi - staged_lo), cudaMemcpyHostToDevice,
                            sl->stream) != cudaSuccess)
            st = CBFS_E_CUDA;
        for (const Part& p : sl->parts) {
            if (st != CBFS_OK) break;
            if (p.req->pinned_pairs &&
                cudaMemcpyAsync(sl->d_pairs + 2 * p.batch_off, p.req->pairs + 2 * p.req_off,
                                sizeof(int32_t) * 2 * (size_t)p.count, cudaMemcpyHostToDevice, sl->stream) != cudaSuccess)
                st = CBFS_E_CUDA;
        }
        if (st == CBFS_OK) st = cbfs_query_distance(S->labels, sl->d_pairs, sl->count, sl->d_out, sl->stream);
        int64_t out_lo = -1, out_hi = -1;
        for (const Part& p : sl->parts) {
            if (st != CBFS_OK) break;
            if (p.req->pinned_out) {
                if (cudaMemcpyAsync(p.req->out + p.req_off, sl->d_out + p.batch_off, sizeof(uint16_t) * (size_t)p.count,
                                    cudaMemcpyDeviceToHost, sl->stream) != cudaSuccess)
                    st = CBFS_E_CUDA;
                continue;
            }
            if (out_lo < 0) out_lo = p.batch_off;
            out_hi = p.batch_off + p.count;
        }
        if (st == CBFS_OK && out_lo >= 0 &&
            cudaMemcpyAsync(sl->h_out + out_lo, sl->d_out + out_lo, sizeof(uint16_t) * (size_t)(out_hi - out_lo),
                            cudaMemcpyDeviceToHost, sl->stream) != cudaSuccess)
            st = CBFS_E_CUDA;
        if (st == CBFS_OK && cudaEventRecord(sl->ev, sl->stream) != cudaSuccess) st = CBFS_E_CUDA;
        if (st != CBFS_OK) cudaGetLastError();
        {
            std::lock_guard<std::mutex> lk(S->mu);
            sl->launch_status = st;
            sl->launched = true;
        }
        S->cv_slot.notify_all();
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->dispatcher_done = true;
    }
    S->cv_slot.notify_all();
}

// True for page-locked host memory (cudaHostAlloc / cudaHostRegister).
bool is_page_locked(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

void free_slot(Slot* sl) {
    if (sl->stream) cudaStreamDestroy(sl->stream);
    if (sl->ev) cudaEventDestroy(sl->ev);
    if (sl->h_pairs) cudaFreeHost(sl->h_pairs);
    if (sl->h_out) cudaFreeHost(sl->h_out);
    if (sl->d_pairs) cudaFree(sl->d_pairs);
    if (sl->d_out) cudaFree(sl->d_out);
    delete sl;
}

}  // namespace

extern "C" {

int cbfs_server_create(cbfs_labels_t L, int64_t max_batch, int slots, size_t device_budget_bytes,
                       cbfs_server_t* out) {
    if (!L || !out || max_batch < 1 || slots < 1 || slots > 64) return CBFS_E_INVALID;
    *out = nullptr;
    cbfs_server_s* S = new (std::nothrow) cbfs_server_s();
    if (!S) return CBFS_E_NOMEM;
    cudaGetDevice(&S->device);
    S->labels = L;
    int64_t budget = (int64_t)device_budget_bytes;
    if (budget == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            delete S;
            return CBFS_E_CUDA;
        }
        budget = (int64_t)(free_b / 4);
    }
    // the batch buffers come out of the budget: fewer or smaller slots if it is tight
    S->max_batch = std::min<int64_t>(max_batch, budget / (kPairBytes * slots));
    if (S->max_batch < 1) {
        delete S;
        return CBFS_E_NOMEM;
    }
    S->budget = S->max_batch * kPairBytes * slots;
    for (int i = 0; i < slots; ++i) {
        Slot* sl = new (std::nothrow) Slot();
        if (!sl) break;
        S->slots.push_back(sl);
        const size_t np = (size_t)S->max_batch;
        if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc((void**)&sl->h_pairs, sizeof(int32_t) * 2 * np, cudaHostAllocPortable) != cudaSuccess ||
            cudaHostAlloc((void**)&sl->h_out, sizeof(uint16_t) * np, cudaHostAllocPortable) != cudaSuccess ||
            cudaMalloc((void**)&sl->d_pairs, sizeof(int32_t) * 2 * np) != cudaSuccess ||
            cudaMalloc((void**)&sl->d_out, sizeof(uint16_t) * np) != cudaSuccess) {
            cudaGetLastError();
            for (Slot* x : S->slots) free_slot(x);
            delete S;
            return CBFS_E_NOMEM;
        }
        S->free_slots.push_back(sl);
    }
    if ((int)S->slots.size() != slots) {
        for (Slot* x : S->slots) free_slot(x);
        delete S;
        return CBFS_E_NOMEM;
    }
    for (Slot* sl : S->slots) sl->waiter = std::thread(run_waiter, S, sl);
    S->dispatcher = std::thread(run_dispatcher, S);
    *out = S;
    return CBFS_OK;
}

int cbfs_server_submit(cbfs_server_t S, const int32_t* host_pairs, int64_t q, uint16_t* host_out, uint64_t* ticket) {
    if (!S || !ticket || q < 0 || (q > 0 && (!host_pairs || !host_out))) return CBFS_E_INVALID;
    Request* r = new (std::nothrow) Request();
    if (!r) return CBFS_E_NOMEM;
    r->pairs = host_pairs;
    r->out = host_out;
    r->q = q;
    if (q > 0) {
        r->pinned_pairs = is_page_locked(host_pairs);
        r->pinned_out = is_page_locked(host_out);
    }
    r->remaining = q;
    r->t_arrival = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete r;
            return CBFS_E_INVALID;
        }
        *ticket = S->next_ticket++;
        S->tickets[*ticket] = r;
        if (q == 0) {
            r->done = true;
            r->t_done = r->t_arrival;
            S->latency_ms.push_back(0.0);
        } else {
            S->pending.push_back(r);
        }
    }
    if (q > 0) S->cv_dispatch.notify_one();
    return CBFS_OK;
}

int cbfs_server_wait(cbfs_server_t S, uint64_t ticket, double timeout_s) {
    if (!S) return CBFS_E_INVALID;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return CBFS_E_INVALID;
    Request* r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
        return CBFS_E_TIMEOUT;  // not answered yet; the ticket stays valid
    }
    const int st = r->status;
    S->tickets.erase(it);
    delete r;
    return st;
}

int cbfs_server_stats(cbfs_server_t S, uint64_t* host_counts, double* host_latency_ms, int64_t cap,
                      int64_t* host_n_latency) {
    if (!S) return CBFS_E_INVALID;
    std::lock_guard<std::mutex> lk(S->mu);
    if (host_counts) {
        host_counts[0] = (uint64_t)S->latency_ms.size();
        host_counts[1] = S->batches;
        host_counts[2] = S->pairs_done;
        host_counts[3] = (uint64_t)S->max_batch;
        host_counts[4] = (uint64_t)S->budget;
    }
    if (host_n_latency) *host_n_latency = (int64_t)S->latency_ms.size();
    if (host_latency_ms && cap > 0) {
        const int64_t m = std::min<int64_t>(cap, (int64_t)S->latency_ms.size());
        std::memcpy(host_latency_ms, S->latency_ms.data(), sizeof(double) * (size_t)m);
    }
    return CBFS_OK;
}

int cbfs_server_destroy(cbfs_server_t S) {
    if (!S) return CBFS_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_dispatch.notify_all();
    if (S->dispatcher.joinable()) S->dispatcher.join();  // launches what is pending, then returns
    S->cv_slot.notify_all();
    for (Slot* sl : S->slots)
        if (sl->waiter.joinable()) sl->waiter.join();  // each finishes its batch in flight
    for (Slot* sl : S->slots) free_slot(sl);
    for (auto& kv : S->tickets) delete kv.second;  // answered or not, nobody can wait any more
    delete S;
    return CBFS_OK;
}

}  // extern "C"
