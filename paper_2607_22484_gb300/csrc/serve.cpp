// Batches and serving for libsvt (host code).
//
// svt_batch: every matrix gets its own plan at its own offset of the workspace;
// the solves are issued round-robin over the context's worker streams, so the
// independent matrices overlap on the device, and the caller's stream waits on
// all of them.
//
// Serving: a scheduler thread owns an admission queue. Each tick it
//   * retires requests whose completion event has fired (their workspace range
//     goes back to the arena, their status is read from the pinned copy),
//   * admits queued requests in arrival order while a slot is free and their
//     workspace fits in a free range of the context's workspace (first fit),
//     and enqueues each admitted request's whole solve on a worker stream.
// Requests that arrive while others run are admitted as soon as slots and
// memory free up, and their kernels overlap with the running ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "plan.h"

using namespace svt;

namespace {

constexpr int kStreams = 8;
constexpr int kSlots = 16;
constexpr size_t kQueueLimit = 1 << 16;

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) in kAlign units.
struct Arena {
    size_t size = 0;
    std::map<size_t, size_t> free_;  // offset -> length
    void reset(size_t s)
    {
        size = s;
        free_.clear();
        if (s)
            free_[0] = s;
    }
    bool alloc(size_t len, size_t *off)
    {
        len = align_up(len, kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *off = it->first;
                size_t rest = it->second - len;
                size_t roff = it->first + len;
                free_.erase(it);
                if (rest)
                    free_[roff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t len)
    {
        len = align_up(len, kAlign);
        auto it = free_.emplace(off, len).first;
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
};

struct Request {
    uint64_t ticket = 0;
    svt_matrix m;
    Resolved opt;
    size_t ws_len = 0, ws_off = 0;
    int slot = -1;
    double t_submit = 0, t_done = 0;
    int state = 0;  // 0 queued, 1 running, 2 done
    svt_status result = SVT_OK;
};

} // namespace

struct ServeState {
    std::mutex mu;
    std::condition_variable cv;
    std::thread thread;
    bool stop = false;
    bool started = false;
    uint64_t next_ticket = 1;
    std::deque<Request *> queue;
    std::list<Request *> active;
    std::map<uint64_t, Request *> tickets;
    Arena arena;
    cudaStream_t streams[kStreams] = {};
    cudaEvent_t events[kSlots] = {};
    int *h_status = nullptr;  // pinned, one int per slot
    bool slot_used[kSlots] = {};
    int rr = 0;
};

namespace svt {

namespace {

svt_status start_workers(svt_ctx *ctx, ServeState *s)
{
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    for (int i = 0; i < kStreams; ++i)
        if (!s->streams[i] && cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess)
            return SVT_ERR_CUDA;
    for (int i = 0; i < kSlots; ++i)
        if (!s->events[i] && cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming) != cudaSuccess)
            return SVT_ERR_CUDA;
    if (!s->h_status && cudaMallocHost(reinterpret_cast<void **>(&s->h_status), sizeof(int) * kSlots) != cudaSuccess)
        return SVT_ERR_CUDA;
    return SVT_OK;
}

ServeState *state_of(svt_ctx *ctx)
{
    if (!ctx->serve)
        ctx->serve = new ServeState();
    return ctx->serve;
}

// One scheduler tick under s->mu. Returns true if anything happened.
bool tick(svt_ctx *ctx, ServeState *s)
{
    bool progress = false;
    // Retire.
    for (auto it = s->active.begin(); it != s->active.end();) {
        Request *r = *it;
        cudaError_t q = cudaEventQuery(s->events[r->slot]);
        if (q == cudaErrorNotReady) {
            ++it;
            continue;
        }
        r->t_done = now_ms();
        r->result = (q == cudaSuccess) ? (svt_status)s->h_status[r->slot] : SVT_ERR_CUDA;
        r->state = 2;
        s->arena.release(r->ws_off, r->ws_len);
        s->slot_used[r->slot] = false;
        it = s->active.erase(it);
        progress = true;
    }
    // Admit in arrival order.
    while (!s->queue.empty() && (int)s->active.size() < kSlots) {
        Request *r = s->queue.front();
        size_t off;
        if (!s->arena.alloc(r->ws_len, &off))
            break;
        s->queue.pop_front();
        int slot = 0;
        while (s->slot_used[slot])
            ++slot;
        s->slot_used[slot] = true;
        r->slot = slot;
        r->ws_off = off;
        cudaStream_t st = s->streams[s->rr++ % kStreams];
        Plan *plan = nullptr;
        svt_status e;
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            if (ctx->plans.size() > 512)
                ctx->plans.clear();
            e = get_plan(ctx, r->m.m, r->m.n, r->opt, off, ctx->ws_bytes - off, &plan);
            if (e == SVT_OK) {
                CallArgs a{r->m.A, r->m.lda, r->m.tau, r->m.Y, r->m.ldy, r->m.d_status};
                e = run_plan(ctx, *plan, a, st);
            }
            if (e == SVT_OK)
                e = plan_status_copy(ctx, *plan, &s->h_status[slot], st);
        }
        if (e == SVT_OK && cudaEventRecord(s->events[slot], st) != cudaSuccess)
            e = SVT_ERR_CUDA;
        if (e != SVT_OK) {
            r->result = e;
            r->state = 2;
            r->t_done = now_ms();
            s->arena.release(off, r->ws_len);
            s->slot_used[slot] = false;
        } else {
            r->state = 1;
            s->active.push_back(r);
        }
        progress = true;
    }
    return progress;
}

void scheduler(svt_ctx *ctx, ServeState *s)
{
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool progress = tick(ctx, s);
        if (progress)
            continue;
        if (s->active.empty())
            s->cv.wait_for(lk, std::chrono::milliseconds(5));
        else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

} // namespace

void serve_shutdown(svt_ctx *ctx)
{
    ServeState *s = ctx->serve;
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->thread.joinable())
        s->thread.join();
    for (int i = 0; i < kStreams; ++i)
        if (s->streams[i]) {
            cudaStreamSynchronize(s->streams[i]);
            cudaStreamDestroy(s->streams[i]);
        }
    for (int i = 0; i < kSlots; ++i)
        if (s->events[i])
            cudaEventDestroy(s->events[i]);
    if (s->h_status)
        cudaFreeHost(s->h_status);
    for (auto &kv : s->tickets)
        delete kv.second;
    for (Request *r : s->queue)
        if (!s->tickets.count(r->ticket))
            delete r;
    delete s;
    ctx->serve = nullptr;
}

bool serve_busy(svt_ctx *ctx)
{
    ServeState *s = ctx->serve;
    if (!s)
        return false;
    std::lock_guard<std::mutex> g(s->mu);
    return !s->queue.empty() || !s->active.empty();
}

} // namespace svt

extern "C" {

svt_status svt_batch_workspace_bytes(const svt_matrix *mats, int count, size_t *out)
{
    if (!out || count < 0 || (count > 0 && !mats))
        return SVT_ERR_INVALID;
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        size_t b = 0;
        svt_status st = svt_workspace_bytes_ex(mats[i].m, mats[i].n, &mats[i].opt, &b);
        if (st != SVT_OK)
            return st;
        total += align_up(b, kAlign);
    }
    *out = total;
    return SVT_OK;
}

svt_status svt_batch(svt_ctx_t ctx, const svt_matrix *mats, int count, void *stream)
{
    if (!ctx || count < 0 || (count > 0 && !mats))
        return SVT_ERR_INVALID;
    if (serve_busy(ctx))
        return SVT_ERR_BUSY;
    std::vector<Resolved> res(count);
    size_t total = 0;
    std::vector<size_t> off(count);
    for (int i = 0; i < count; ++i) {
        const svt_matrix &m = mats[i];
        svt_status st = validate(m.A, m.m, m.n, m.lda, m.tau, m.Y, m.ldy);
        if (st != SVT_OK)
            return st;
        if (!resolve(&m.opt, &res[i]))
            return SVT_ERR_INVALID;
        if (res[i].prec == SVT_FP64 && (m.m > kF64MaxDim || m.n > kF64MaxDim))
            return SVT_ERR_UNSUPPORTED;
        off[i] = total;
        total += align_up(make_layout(m.m, m.n, res[i]).total, kAlign);
    }
    if (total > ctx->ws_bytes)
        return SVT_ERR_OOM;
    ServeState *s = state_of(ctx);
    if (start_workers(ctx, s) != SVT_OK)
        return SVT_ERR_CUDA;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> g(ctx->mu);
    // Worker streams start after everything already queued on the caller's stream.
    cudaEvent_t ev = s->events[0];
    if (cudaEventRecord(ev, cs) != cudaSuccess)
        return SVT_ERR_CUDA;
    for (int i = 0; i < kStreams; ++i)
        if (cudaStreamWaitEvent(s->streams[i], ev, 0) != cudaSuccess)
            return SVT_ERR_CUDA;
    for (int i = 0; i < count; ++i) {
        const svt_matrix &m = mats[i];
        Plan *plan = nullptr;
        svt_status st = get_plan(ctx, m.m, m.n, res[i], off[i], ctx->ws_bytes - off[i], &plan);
        if (st != SVT_OK)
            return st;
        CallArgs a{m.A, m.lda, m.tau, m.Y, m.ldy, m.d_status};
        st = run_plan(ctx, *plan, a, s->streams[i % kStreams]);
        if (st != SVT_OK)
            return st;
    }
    // The caller's stream waits for all worker streams.
    for (int i = 0; i < kStreams; ++i) {
        if (cudaEventRecord(s->events[1 + i], s->streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(cs, s->events[1 + i], 0) != cudaSuccess)
            return SVT_ERR_CUDA;
    }
    return SVT_OK;
}

svt_status svt_serve_submit(svt_ctx_t ctx, const svt_matrix *req, uint64_t *ticket)
{
    if (!ctx || !req || !ticket)
        return SVT_ERR_INVALID;
    svt_status st = validate(req->A, req->m, req->n, req->lda, req->tau, req->Y, req->ldy);
    if (st != SVT_OK)
        return st;
    Resolved r;
    if (!resolve(&req->opt, &r))
        return SVT_ERR_INVALID;
    if (r.prec == SVT_FP64 && (req->m > kF64MaxDim || req->n > kF64MaxDim))
        return SVT_ERR_UNSUPPORTED;
    size_t need = align_up(make_layout(req->m, req->n, r).total, kAlign);
    if (need > ctx->ws_bytes)
        return SVT_ERR_OOM;
    ServeState *s;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        s = state_of(ctx);
    }
    std::lock_guard<std::mutex> g(s->mu);
    if (!s->started) {
        if (start_workers(ctx, s) != SVT_OK)
            return SVT_ERR_CUDA;
        s->arena.reset(ctx->ws_bytes);
        s->thread = std::thread(scheduler, ctx, s);
        s->started = true;
    }
    if (s->queue.size() >= kQueueLimit)
        return SVT_ERR_BUSY;
    auto *q = new Request();
    q->ticket = s->next_ticket++;
    q->m = *req;
    q->opt = r;
    q->ws_len = need;
    q->t_submit = now_ms();
    s->queue.push_back(q);
    s->tickets[q->ticket] = q;
    *ticket = q->ticket;
    s->cv.notify_all();
    return SVT_OK;
}

svt_status svt_serve_poll(svt_ctx_t ctx, uint64_t ticket, double *latency_ms)
{
    if (!ctx || !ctx->serve)
        return SVT_ERR_INVALID;
    ServeState *s = ctx->serve;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end())
        return SVT_ERR_INVALID;
    Request *r = it->second;
    if (r->state != 2)
        return SVT_ERR_NOT_READY;
    if (latency_ms)
        *latency_ms = r->t_done - r->t_submit;
    return r->result;
}

svt_status svt_serve_release(svt_ctx_t ctx, uint64_t ticket)
{
    if (!ctx || !ctx->serve)
        return SVT_ERR_INVALID;
    ServeState *s = ctx->serve;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end())
        return SVT_ERR_INVALID;
    if (it->second->state != 2)
        return SVT_ERR_NOT_READY;
    delete it->second;
    s->tickets.erase(it);
    return SVT_OK;
}

} // extern "C"
