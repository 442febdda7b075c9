// serve.cpp -- request contexts: admission against a memory budget and
// continuous batching of ttv / ttm / entrywise requests over several streams.
//
// tl_batch_submit validates a request's operations, copies their descriptors
// and queues it; a worker thread owned by the context
//   1. retires launched batches whose completion event has fired (recording
//      each request's submission-to-completion latency and returning its
//      bytes to the budget),
//   2. admits queued requests in arrival order while their operand + output
//      bytes fit in the budget, grouped into batches of bounded size (a large
//      request is a batch of its own), and
//   3. launches each batch on a free stream slot: one persistent launch
//      (TL_CTX_PERSISTENT) or one launch per operation.
// Requests that arrive while earlier batches run are admitted as soon as a
// slot and budget free up, so work from different requests overlaps on the
// device.  While batches are in flight, and for a few milliseconds after the
// last one, the worker polls without sleeping, so completions and new
// requests are seen within microseconds; when idle longer it sleeps until a
// submission.  Nothing here waits on the GPU while
// holding the context lock.
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
// Batch formation: a request of kLargeBytes or more runs as a batch of its own
// (on its own stream, so small requests keep flowing on the others); small
// requests are grouped up to kBatchOps operations and kBatchBytes, so that a
// batch completes (and releases its requests) within tens of microseconds
// instead of holding every queued request until the whole queue is done.
constexpr size_t kLargeBytes = size_t(16) << 20;
constexpr size_t kBatchBytes = size_t(64) << 20;
constexpr size_t kBatchOps = 256;
// After the last request completes the worker keeps polling this long before
// it sleeps (one host core busy while requests keep arriving).
constexpr int kSpinMs = 5;

// Marks every request of a retired slot complete; returns true if any was.
bool retire(tl_ctx* c)
{
    bool progress = false;
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
    return progress;
}

// Takes the next batch off the queue in arrival order, admitting each taken
// request against the budget.  large_lane: the first large request (one of
// kLargeBytes or more) alone.  Otherwise: consecutive small requests within
// the batch caps, passing over large requests, which wait for the large lane.
// Empty when nothing can be admitted.
std::vector<Request*> take_batch(tl_ctx* c, bool large_lane)
{
    std::vector<Request*> take;
    size_t ops = 0, bytes = 0;
    for (auto it = c->pending.begin(); it != c->pending.end();) {
        Request* r = *it;
        if (r->cancelled) {
            it = c->pending.erase(it);
            continue;
        }
        const bool large = r->bytes >= kLargeBytes;
        if (large != large_lane) {
            // the large lane looks for the first large request; a batch of
            // small requests passes over large ones (they wait for the lane)
            ++it;
            continue;
        }
        if (c->inflight_bytes + r->bytes > c->budget && c->inflight_bytes > 0) break;
        if (!take.empty() && (ops + r->ops.size() > kBatchOps || bytes + r->bytes > kBatchBytes))
            break;
        it = c->pending.erase(it);
        c->inflight_bytes += r->bytes;
        ops += r->ops.size();
        bytes += r->bytes;
        take.push_back(r);
        if (large) break;
    }
    return take;
}

void run_worker(tl_ctx* c)
{
    cudaSetDevice(c->device);
    std::vector<const tl_op*> batch_ops;
    std::unique_lock<std::mutex> lk(c->mu);
    auto last_active = Clock::now();
    while (!c->stop) {
        // 1. retire completed batches
        if (retire(c)) c->cv.notify_all();
        // 2. admit queued requests onto every free slot: the last slot is the
        //    large-request lane (low stream priority, one request at a time),
        //    the others take batches of small requests (high priority)
        for (;;) {
            SlotState* free_slot = nullptr;
            std::vector<Request*> take;
            SlotState& lane = c->slots.back();
            if (!lane.busy && !c->pending.empty()) {
                take = take_batch(c, true);
                if (!take.empty()) free_slot = &lane;
            }
            if (take.empty()) {
                for (size_t i = 0; i + 1 < c->slots.size(); ++i)
                    if (!c->slots[i].busy) { free_slot = &c->slots[i]; break; }
                if (!free_slot || c->pending.empty()) break;
                take = take_batch(c, false);
            }
            if (take.empty()) break;
            if (c->inflight_bytes > c->max_inflight) c->max_inflight = c->inflight_bytes;
            c->batches++;
            free_slot->busy = true;
            free_slot->reqs = take;
            batch_ops.clear();
            for (Request* r : take)
                for (auto& o : r->ops) batch_ops.push_back(&o->op);
            // 3. launch without holding the lock
            lk.unlock();
            int rc;
            {
                NvtxRange nvtx_range("tl_ctx_batch_launch");
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
            }
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
        }
        bool any_busy = false;
        for (SlotState& s : c->slots) any_busy |= s.busy;
        const auto now = Clock::now();
        if (any_busy || !c->pending.empty()) last_active = now;
        if (now - last_active < std::chrono::milliseconds(kSpinMs)) {
            // work in flight, or some in the last few milliseconds: poll
            // without sleeping (letting submitters take the lock between
            // polls), so a finished batch or a new request is seen within
            // microseconds rather than after a thread wake-up
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        } else {
            // idle: sleep until a submission arrives
            c->cv.wait_for(lk, std::chrono::milliseconds(2));
        }
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
    // `streams` slots for batches of small requests at the highest stream
    // priority, plus one lane for large requests at the lowest, so that
    // small work is scheduled first whenever SMs free up
    c->slots.resize((size_t)streams + 1);
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    for (size_t i = 0; i < c->slots.size(); ++i) {
        SlotState& s = c->slots[i];
        const int prio = i + 1 == c->slots.size() ? least : greatest;
        bool ok = cudaStreamCreateWithPriority(&s.stream, cudaStreamNonBlocking, prio) == cudaSuccess &&
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
