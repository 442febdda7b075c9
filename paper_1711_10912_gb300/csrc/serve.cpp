// serve.cpp -- request contexts: admission against a memory budget and
// continuous batching of ttv / ttm / entrywise requests over several streams.
//
// tl_batch_submit validates a request's operations, copies their descriptors
// and queues it; a worker thread owned by the context
//   1. retires launched batches whose completion event has fired (recording
//      each request's submission-to-completion latency and returning its
//      bytes to the budget),
//   2. admits queued requests in arrival order while their operand + output
//      bytes fit in the budget, and
//   3. launches everything admitted as one batch on a free stream slot: one
//      persistent launch (TL_CTX_PERSISTENT) or one launch per operation.
// Requests that arrive while earlier batches run are admitted as soon as a
// slot and budget free up, so work from different requests overlaps on the
// device.  Nothing here waits on the GPU while holding the context lock.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.h"
#include "runtime.h"

namespace tl {
namespace {

using Clock = std::chrono::steady_clock;

// A tl_tensor with its own copies of the n / pi / w arrays.
struct OwnedTensor {
    std::vector<int64_t> n, w;
    std::vector<uint32_t> pi;
    tl_tensor t{};
    void copy(const tl_tensor& src)
    {
        t = src;
        if (src.n && src.p) {
            n.assign(src.n, src.n + src.p);
            t.n = n.data();
        }
        if (src.pi && src.p) {
            pi.assign(src.pi, src.pi + src.p);
            t.pi = pi.data();
        } else {
            t.pi = nullptr;
        }
        if (src.w && src.p) {
            w.assign(src.w, src.w + src.p);
            t.w = w.data();
        } else {
            t.w = nullptr;
        }
    }
};

struct OwnedOp {
    tl_op op{};
    OwnedTensor A, B, C;
    void copy(const tl_op& src)
    {
        op = src;
        A.copy(src.A);
        B.copy(src.B);
        C.copy(src.C);
        op.A = A.t;
        op.B = B.t;
        op.C = C.t;
    }
};

struct Request {
    uint64_t ticket = 0;
    std::vector<std::unique_ptr<OwnedOp>> ops;
    size_t bytes = 0;
    Clock::time_point t_submit;
    int32_t status = TL_PENDING;
    double latency_ms = 0.0;
    bool cancelled = false;
};

struct SlotState {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    Slot* table = nullptr;
    bool busy = false;
    std::vector<Request*> reqs;
};

}  // namespace
}  // namespace tl

struct tl_ctx {
    int device = 0;
    int32_t flags = 0;
    size_t budget = 0;
    size_t inflight_bytes = 0;
    std::vector<tl::SlotState> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<tl::Request*> pending;
    std::unordered_map<uint64_t, std::unique_ptr<tl::Request>> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    int32_t failure = TL_OK;
    size_t max_inflight = 0;
    uint64_t batches = 0;
    uint64_t completed = 0;
    std::thread worker;
};

namespace tl {
namespace {

constexpr size_t kSlotCapacity = 8192;     // operations per persistent launch

void run_worker(tl_ctx* c)
{
    cudaSetDevice(c->device);
    std::vector<const tl_op*> batch_ops;
    std::unique_lock<std::mutex> lk(c->mu);
    while (!c->stop) {
        bool progress = false;
        // 1. retire completed batches
        for (SlotState& s : c->slots) {
            if (!s.busy) continue;
            cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            const auto now = Clock::now();
            for (Request* r : s.reqs) {
                r->status = (q == cudaSuccess) ? TL_OK : TL_ECUDA;
                r->latency_ms = std::chrono::duration<double, std::milli>(now - r->t_submit).count();
                c->inflight_bytes -= r->bytes;
                c->completed++;
            }
            if (q != cudaSuccess) cudaGetLastError();
            s.reqs.clear();
            s.busy = false;
            progress = true;
        }
        if (progress) c->cv.notify_all();
        // 2. admit queued requests onto a free slot
        SlotState* free_slot = nullptr;
        for (SlotState& s : c->slots)
            if (!s.busy) { free_slot = &s; break; }
        if (free_slot && !c->pending.empty()) {
            std::vector<Request*> take;
            size_t ops = 0;
            while (!c->pending.empty()) {
                Request* r = c->pending.front();
                if (r->cancelled) {
                    c->pending.pop_front();
                    continue;
                }
                if (c->inflight_bytes + r->bytes > c->budget && !take.empty()) break;
                if (c->inflight_bytes + r->bytes > c->budget && c->inflight_bytes > 0) break;
                if (ops + r->ops.size() > kSlotCapacity && !take.empty()) break;
                c->pending.pop_front();
                c->inflight_bytes += r->bytes;
                ops += r->ops.size();
                take.push_back(r);
            }
            if (!take.empty()) {
                if (c->inflight_bytes > c->max_inflight) c->max_inflight = c->inflight_bytes;
                c->batches++;
                free_slot->busy = true;
                free_slot->reqs = take;
                batch_ops.clear();
                for (Request* r : take)
                    for (auto& o : r->ops) batch_ops.push_back(&o->op);
                // 3. launch without holding the lock
                lk.unlock();
                NvtxRange nvtx_range("tl_ctx_batch_launch");
                int rc;
                if (c->flags & TL_CTX_PERSISTENT) {
                    rc = slot_launch(free_slot->table, batch_ops.data(), batch_ops.size(),
                                     free_slot->stream);
                } else {
                    rc = TL_OK;
                    for (const tl_op* o : batch_ops) {
                        const tl_op* ops1[1] = {o};
                        // a capacity-0 table sends every operation to its own kernel
                        rc = slot_launch(nullptr, ops1, 1, free_slot->stream);
                        if (rc) break;
                    }
                }
                if (rc == TL_OK && cudaEventRecord(free_slot->done, free_slot->stream) != cudaSuccess)
                    rc = TL_ECUDA;
                lk.lock();
                if (rc != TL_OK) {
                    // the launch failed on the host: the requests fail, the slot frees
                    cudaStreamSynchronize(free_slot->stream);
                    cudaGetLastError();
                    for (Request* r : take) {
                        r->status = rc;
                        r->latency_ms = std::chrono::duration<double, std::milli>(
                                            Clock::now() - r->t_submit).count();
                        c->inflight_bytes -= r->bytes;
                    }
                    free_slot->reqs.clear();
                    free_slot->busy = false;
                    c->cv.notify_all();
                }
                continue;
            }
        }
        bool any_busy = false;
        for (SlotState& s : c->slots) any_busy |= s.busy;
        // sleep until a submission arrives, or briefly while batches run
        c->cv.wait_for(lk, any_busy ? std::chrono::microseconds(20) : std::chrono::milliseconds(2));
    }
}

}  // namespace
}  // namespace tl

using namespace tl;

extern "C" {

int tl_ctx_create(size_t budget_bytes, int32_t streams, int32_t flags, tl_ctx** out)
{
    if (!out || streams < 1 || streams > 64 || budget_bytes == 0) return TL_EINVAL;
    *out = nullptr;
    auto* c = new tl_ctx();
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return TL_ECUDA;
    }
    c->flags = flags;
    c->budget = budget_bytes;
    c->slots.resize(streams);
    for (SlotState& s : c->slots) {
        bool ok = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) == cudaSuccess;
        if (ok && (flags & TL_CTX_PERSISTENT)) {
            s.table = slot_create(kSlotCapacity);
            ok = s.table != nullptr;
        }
        if (!ok) {
            cudaGetLastError();
            tl_ctx_destroy(c);
            return TL_ENOMEM;
        }
    }
    c->worker = std::thread(run_worker, c);
    *out = c;
    return TL_OK;
}

int tl_ctx_destroy(tl_ctx* c)
{
    if (!c) return TL_OK;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
    }
    c->cv.notify_all();
    if (c->worker.joinable()) c->worker.join();
    for (SlotState& s : c->slots) {
        if (s.stream) cudaStreamSynchronize(s.stream);
        if (s.table) slot_destroy(s.table);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    delete c;
    return TL_OK;
}

int tl_batch_submit(tl_ctx* c, const tl_op* ops, size_t count, uint64_t* ticket)
{
    if (!c || !ops || !count || !ticket) return TL_EINVAL;
    auto r = std::make_unique<Request>();
    for (size_t i = 0; i < count; ++i) {
        long long b = op_bytes(ops[i]);
        if (b < 0) return (int)b;
        r->bytes += (size_t)b;
        auto o = std::make_unique<OwnedOp>();
        o->copy(ops[i]);
        r->ops.push_back(std::move(o));
    }
    if (r->bytes > c->budget) return TL_ENOMEM;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(c->mu);
        r->ticket = c->next_ticket++;
        *ticket = r->ticket;
        c->pending.push_back(r.get());
        c->reqs.emplace(r->ticket, std::move(r));
    }
    c->cv.notify_all();
    return TL_OK;
}

int tl_poll(tl_ctx* c, uint64_t ticket, int32_t* status, double* latency_ms)
{
    if (!c || !status) return TL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->reqs.find(ticket);
    if (it == c->reqs.end()) return TL_EINVAL;
    *status = it->second->status;
    if (latency_ms) *latency_ms = it->second->latency_ms;
    if (*status != TL_PENDING) c->reqs.erase(it);     // final status reported once
    return TL_OK;
}

int tl_wait(tl_ctx* c, uint64_t ticket, double timeout_ms, int32_t* status, double* latency_ms)
{
    if (!c) return TL_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    auto it = c->reqs.find(ticket);
    if (it == c->reqs.end()) return TL_EINVAL;
    Request* r = it->second.get();
    const auto deadline = Clock::now() + std::chrono::microseconds((long long)(timeout_ms * 1000));
    while (r->status == TL_PENDING) {
        if (c->cv.wait_until(lk, deadline) == std::cv_status::timeout && r->status == TL_PENDING) {
            if (status) *status = TL_PENDING;
            return TL_ETIMEOUT;
        }
    }
    if (status) *status = r->status;
    if (latency_ms) *latency_ms = r->latency_ms;
    c->reqs.erase(ticket);                               // final status reported once
    return TL_OK;
}

int tl_ctx_stats(tl_ctx* c, size_t* max_inflight_bytes, uint64_t* batches, uint64_t* completed)
{
    if (!c) return TL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    if (max_inflight_bytes) *max_inflight_bytes = c->max_inflight;
    if (batches) *batches = c->batches;
    if (completed) *completed = c->completed;
    return TL_OK;
}

int tl_cancel(tl_ctx* c, uint64_t ticket)
{
    if (!c) return TL_EINVAL;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->reqs.find(ticket);
    if (it == c->reqs.end()) return TL_EINVAL;
    Request* r = it->second.get();
    if (r->status != TL_PENDING) return r->status;
    for (auto p = c->pending.begin(); p != c->pending.end(); ++p) {
        if (*p == r) {
            c->pending.erase(p);
            r->cancelled = true;
            r->status = TL_ECANCELED;
            c->cv.notify_all();
            return TL_OK;
        }
    }
    return TL_PENDING;   // already launched: it runs to completion
}

}  // extern "C"
