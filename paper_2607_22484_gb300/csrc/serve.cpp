// Batches and serving for libsvt (host code).
//
// svt_batch: every matrix gets its own plan at its own offset of the workspace.
// When all matrices share one option set (the usual case), their solves are
// merged into ONE persistent launch of the product kernel: its problem table
// (tensor maps included, in device memory) lists every product of every matrix,
// stage by stage, and each problem waits on device-side counters only for the
// earlier products of its own matrix, so independent matrices fill each other's
// waits. The memory-bound steps run as grouped kernels over all matrices. The whole launch sequence is captured once
// per batch shape signature into a CUDA graph; a call uploads the per-matrix
// pointers and thresholds (the call table) and replays the graph on the caller's
// stream. Batches whose matrices differ in options fall back to per-matrix
// solves spread over the context's worker streams.
//
// Serving (continuous batching at stage granularity): a scheduler thread owns an
// admission queue. Each tick it
//   * retires requests whose last op has completed (their workspace range goes
//     back to the arena, their status is read from the pinned copy),
//   * admits queued requests in arrival order while a slot is free and their
//     workspace fits in a free range of the context's workspace (first fit),
//   * issues one window on its stream: grouped ingest of the newly admitted,
//     ONE grouped product launch per tile width that carries the next stage of
//     every active request (both polar chains of each), and grouped finalize of
//     requests at their last op.
// A request therefore joins the very next window after memory frees up, and
// its stages share launches with whatever else is running.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "arena.h"
#include "plan.h"

using namespace svt;

namespace {

constexpr int kStreams = 8;
constexpr int kSlots = 16;
// Two lanes share the SMs. Requests of at least kLargeElems elements take the large
// lane; smaller ones advance stage by stage in windows (the small lane), whose grids
// shrink to kSmallSms while large work runs. A large solve is issued as consecutive
// launches over parts of its product table (plan_segments) of about kSegmentWork
// tensor flops each, a few milliseconds, at most two in flight; each takes every SM
// while the small lane is idle and leaves kSmallSms free while it has work. Up to
// kMaxLarge large requests are admitted at once, and each launch goes to the admitted
// one with the least work left (shortest remaining work first): a 4096 x 2048 request
// does not wait for a 200 ms FP32-tier 8192^2 solve to finish, and a small request
// waits at most for the launch in progress, never for a whole large solve. The large
// lane, which carries nearly all of the work, keeps the whole GPU while it runs alone.
constexpr int64_t kLargeElems = (int64_t)8 << 20;
constexpr int kSmallSms = 32;
constexpr double kSegmentWork = 6e12;
constexpr int kMaxLarge = 4;
constexpr size_t kQueueLimit = 1 << 16;

// Optional scheduler trace: with SVT_SERVE_TRACE=<file> in the environment, one line
// per scheduler event (time in ms, event, ticket, detail) is appended to the file.
FILE *trace_file()
{
    static FILE *f = [] {
        const char *p = std::getenv("SVT_SERVE_TRACE");
        return p && *p ? std::fopen(p, "a") : nullptr;
    }();
    return f;
}

double now_ms();

void trace(const char *ev, uint64_t ticket, long long detail)
{
    if (FILE *f = trace_file())
        std::fprintf(f, "%.3f %s %llu %lld\n", now_ms(), ev, (unsigned long long)ticket, detail);
}

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t ticket = 0;
    svt_matrix m;
    Resolved opt;
    size_t ws_len = 0, ws_off = 0;
    int slot = -1;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int state = 0;  // 0 queued, 1 running (ops being issued), 4 large solve between
                    // launches, 3 all issued, 2 done
    bool cancel = false;     // svt_serve_cancel on a running request: drop before next window
    bool cancelled = false;  // retire as SVT_ERR_CANCELLED once its issued work is done
    svt_status result = SVT_OK;
    Plan *plan = nullptr;
    std::shared_ptr<Plan> plan_ref;  // keeps the plan alive while ops are in flight
    size_t pc = 0;          // next op of the plan to issue
    bool grouped = false;   // ops limited to the kinds the grouped kernels cover
    bool large = false;     // large lane
    double est_work = 0.0;  // large lane: m n min(m, n), times 3 in the FP32 tier
    Segments seg;           // large lane: the solve's launches (plan_segments)
    int seg_next = 0;       // next of them to issue
    double seg_total = 0.0;
    double remaining() const  // estimated work not yet issued
    {
        if (seg.count() <= 0 || seg_total <= 0.0)
            return seg_next > 0 ? 0.0 : est_work;
        double left = 0.0;
        for (int k = seg_next; k < seg.count(); ++k)
            left += seg.work[k];
        return est_work * left / seg_total;
    }
};

// Device tables of one serving window live in a ring of slots at the end of the
// workspace; each slot is staged from its own pinned host buffer.
constexpr int kRing = 8;
constexpr size_t kRingSlotBytes = 128 << 10;
constexpr size_t kRingBytes = kRing * kRingSlotBytes;

// Grouped batch: the stage-merged launch sequence of `count` same-option solves.
struct BatchPlan {
    int count = 0;
    size_t tables_off = 0;           // device tables, at this workspace offset
    std::vector<TcLaunch> launches;  // grouped product launches (device pointers set)
    std::vector<int> tiles, bns;
    AuxRec *d_aux = nullptr;
    CallRec *d_calls = nullptr;
    int blocks_reduce = 0, blocks_split = 0;
    CallRec *h_calls = nullptr;      // pinned staging of the call table
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t uploaded = nullptr;  // the previous replay consumed h_calls
    bool pending = false;
    int kernels_per_call = 0;
    int *counters = nullptr;         // fused launch: done[] and tile counter (zeroed per call)
    size_t counter_bytes = 0;
    // Host images of the device tables, re-uploaded when another user of the
    // workspace has overwritten them since this plan last ran.
    std::vector<std::pair<void *, std::vector<uint8_t>>> tables;
    ~BatchPlan()
    {
        if (exec)
            cudaGraphExecDestroy(exec);
        if (uploaded)
            cudaEventDestroy(uploaded);
        if (h_calls)
            cudaFreeHost(h_calls);
    }
};

struct BatchKey {
    std::vector<int64_t> shapes;     // m0, n0, m1, n1, ...
    Resolved r;
    int bn = 0;                      // product tile width of the grouped launch
    bool operator<(const BatchKey &o) const
    {
        auto tie_r = [](const Resolved &x) {
            return std::tie(x.iters, x.prec, x.schedule, x.norm, x.ell0, x.delta, x.polish, x.mode,
                            x.hp_steps);
        };
        if (shapes != o.shapes)
            return shapes < o.shapes;
        if (bn != o.bn)
            return bn < o.bn;
        return tie_r(r) < tie_r(o.r);
    }
};

// Upper bound on the device table bytes of a grouped batch.
size_t batch_table_bytes(int count, const Resolved &r)
{
    const size_t n_tc = 1 + 3 * (size_t)std::max(0, r.iters) + 2 + 1;
    const size_t nprob = n_tc * 2 * (size_t)count;
    return align_up(sizeof(AuxRec) * count, kAlign) + align_up(sizeof(CallRec) * count, kAlign) +
           align_up(sizeof(TcProblem) * nprob, kAlign) + 2 * align_up(sizeof(int) * (nprob + 1), kAlign);
}

bool same_options(const Resolved &a, const Resolved &b)
{
    return a.iters == b.iters && a.prec == b.prec && a.schedule == b.schedule && a.norm == b.norm &&
           a.ell0 == b.ell0 && a.delta == b.delta && a.polish == b.polish && a.mode == b.mode &&
           a.hp_steps == b.hp_steps;
}

} // namespace

struct ServeState {
    std::mutex mu;
    std::condition_variable cv;
    std::thread thread;
    bool stop = false;
    bool started = false;
    uint64_t next_ticket = 1;
    std::deque<Request *> queue;   // small lane, arrival order
    std::deque<Request *> bigq;    // large lane, arrival order
    std::vector<Request *> bigs;   // admitted large requests, launches being issued or in flight
    cudaStream_t big_stream = nullptr;
    cudaEvent_t seg_ev[2] = {};    // the large lane's launch k done (slot k % 2)
    uint64_t big_issued = 0;       // large-lane launches issued
    std::list<Request *> active;
    std::map<uint64_t, Request *> tickets;
    Arena arena;
    cudaStream_t streams[kStreams] = {};
    cudaEvent_t events[kSlots] = {};
    int *h_status = nullptr;  // pinned, one int per slot
    bool slot_used[kSlots] = {};
    int rr = 0;
    std::map<BatchKey, std::unique_ptr<BatchPlan>> batches;
    cudaStream_t capture = nullptr;
    // windowed serving
    cudaStream_t win = nullptr;       // all windows are issued in order on this stream
    uint8_t *h_ring = nullptr;        // pinned, kRing x kRingSlotBytes
    cudaEvent_t ring_ev[kRing] = {};  // slot k's window has been consumed
    bool ring_busy[kRing] = {};
    int ring_next = 0;
    uint64_t windows = 0;
    FILE *metrics = nullptr;          // per-request JSON lines (svt_serve_metrics)
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
    if (!s->win && cudaStreamCreateWithFlags(&s->win, cudaStreamNonBlocking) != cudaSuccess)
        return SVT_ERR_CUDA;
    if (!s->big_stream && cudaStreamCreateWithFlags(&s->big_stream, cudaStreamNonBlocking) != cudaSuccess)
        return SVT_ERR_CUDA;
    for (int i = 0; i < 2; ++i)
        if (!s->seg_ev[i] && cudaEventCreateWithFlags(&s->seg_ev[i], cudaEventDisableTiming) != cudaSuccess)
            return SVT_ERR_CUDA;
    if (!s->h_ring && cudaMallocHost(reinterpret_cast<void **>(&s->h_ring), kRingBytes) != cudaSuccess)
        return SVT_ERR_CUDA;
    for (int i = 0; i < kRing; ++i)
        if (!s->ring_ev[i] && cudaEventCreateWithFlags(&s->ring_ev[i], cudaEventDisableTiming) != cudaSuccess)
            return SVT_ERR_CUDA;
    return SVT_OK;
}

ServeState *state_of(svt_ctx *ctx)
{
    if (!ctx->serve)
        ctx->serve = new ServeState();
    return ctx->serve;
}

bool grouped_kinds(const Plan &P)
{
    for (const Op &op : P.ops)
        if (op.kind != OP_MEMSET && op.kind != OP_REDUCE && op.kind != OP_SPLIT &&
            op.kind != OP_TC && op.kind != OP_FINAL)
            return false;
    return true;
}

const char *prec_name(int p)
{
    return p == SVT_FP64 ? "fp64" : (p == SVT_FP32 ? "fp32" : (p == SVT_BF16 ? "bf16" : "fp8"));
}

// One JSON line per retired request (svt_serve_metrics), under s->mu.
void record(ServeState *s, const Request *r)
{
    if (!s->metrics)
        return;
    const double admit = r->t_admit > 0 ? r->t_admit : r->t_done;
    std::fprintf(s->metrics,
                 "{\"ticket\": %llu, \"m\": %lld, \"n\": %lld, \"prec\": \"%s\", \"tau\": %.9g, "
                 "\"iters\": %d, \"lane\": \"%s\", \"queue_ms\": %.4f, \"run_ms\": %.4f, "
                 "\"latency_ms\": %.4f, \"status\": \"%s\"}\n",
                 (unsigned long long)r->ticket, (long long)r->m.m, (long long)r->m.n,
                 prec_name(r->opt.prec), (double)r->m.tau, r->opt.iters, r->large ? "large" : "small",
                 admit - r->t_submit, r->t_done - admit, r->t_done - r->t_submit,
                 svt_status_str(r->result));
    std::fflush(s->metrics);
}

void finish(ServeState *s, Request *r, svt_status st)
{
    r->plan = nullptr;
    r->plan_ref.reset();
    r->result = st;
    r->state = 2;
    r->t_done = now_ms();
    s->arena.release(r->ws_off, r->ws_len);
    s->slot_used[r->slot] = false;
    record(s, r);
}

// Serving admits a request no earlier than the debug admission delay after its submission.
bool admissible(const svt_ctx *ctx, const Request *r, double now)
{
    return ctx->dbg_admit_delay_us <= 0 || now >= r->t_submit + 1e-3 * (double)ctx->dbg_admit_delay_us;
}

// One serving window: grouped ingest of newly admitted requests, one grouped
// product launch per tile width holding the next product stage of every active
// request, grouped finalize of requests that reached their last op.
svt_status issue_window(svt_ctx *ctx, ServeState *s, int sms)
{
    // Ring slot for this window's tables.
    const int k = s->ring_next;
    if (s->ring_busy[k]) {
        cudaError_t q = cudaEventQuery(s->ring_ev[k]);
        if (q == cudaErrorNotReady)
            return SVT_ERR_NOT_READY;  // the device is a full ring behind: try next tick
        if (q != cudaSuccess)
            return SVT_ERR_CUDA;
        s->ring_busy[k] = false;
    }
    ctx->table_owner = nullptr;
    uint8_t *h = s->h_ring + (size_t)k * kRingSlotBytes;
    uint8_t *d = ctx->ws + (ctx->ws_bytes - kRingBytes) + (size_t)k * kRingSlotBytes;
    size_t used = 0;
    auto take = [&](size_t bytes) -> size_t {
        size_t o = used;
        used = align_up(used + bytes, kAlign);
        return o;
    };
    std::vector<Request *> ingest, tc, fin, single;
    for (Request *r : s->active) {
        if (r->state != 1)
            continue;
        if (!r->grouped) {
            single.push_back(r);
            continue;
        }
        const Op &op = r->plan->ops[r->pc];
        if (op.kind == OP_MEMSET)
            ingest.push_back(r);
    }
    // Ingest: MEMSET, REDUCE, SPLIT are the first three ops of a grouped plan.
    std::vector<AuxRec> aux;
    std::vector<CallRec> calls;
    auto call_of = [](const Request *r) {
        CallRec c;
        c.A = r->m.A;
        c.Y = r->m.Y;
        c.lda = r->m.lda;
        c.ldy = r->m.ldy;
        c.tau = r->m.tau;
        c.pad = 0;
        c.d_status = r->m.d_status;
        return c;
    };
    auto aux_of = [&](const Request *r, int br, int bs) {
        const Plan &P = *r->plan;
        const Layout &L = P.lay;
        uint8_t *base = ctx->ws + P.ws_base;
        AuxRec a;
        std::memset(&a, 0, sizeof(a));
        a.m = P.m;
        a.n = P.n;
        a.wide = P.wide ? 1 : 0;
        a.scal = reinterpret_cast<double *>(base + L.scal);
        a.status = reinterpret_cast<int *>(base + L.status);
        a.colnorm = reinterpret_cast<double *>(base + L.colnorm);
        a.zero_words = (int64_t)((L.colnorm + (size_t)L.N * sizeof(double) - L.scal) / 8);
        const Buf &same = P.wide ? L.Xt[0] : L.X[0];
        const Buf &tran = P.wide ? L.X[0] : L.Xt[0];
        a.xs_hi = base + same.hi;
        a.xs_lo = same.has_lo ? base + same.lo : nullptr;
        a.ld_s = same.ld;
        a.xt_hi = base + tran.hi;
        a.xt_lo = tran.has_lo ? base + tran.lo : nullptr;
        a.ld_t = tran.ld;
        if (P.opt.prec == SVT_BF16) {
            if (P.wide)
                a.xs_lo = base + L.XtLo0.hi;
            else
                a.xt_lo = base + L.XtLo0.hi;
        }
        a.blk_reduce = br;
        a.blk_split = bs;
        return a;
    };
    int blk_r = 0, blk_s = 0;
    for (Request *r : ingest) {
        aux.push_back(aux_of(r, blk_r, blk_s));
        calls.push_back(call_of(r));
        blk_r += grouped_reduce_blocks(r->plan->m, r->plan->n, aux.back().wide);
        blk_s += grouped_split_blocks(r->plan->m, r->plan->n);
        r->pc += 3;
    }
    // Product stage of every grouped request (including the ones just ingested).
    std::vector<TcProblem> probs[2];
    std::vector<int> starts[2];
    int tiles[2] = {0, 0};
    for (Request *r : s->active) {
        if (r->state != 1 || !r->grouped)
            continue;
        Plan &P = *r->plan;
        const Op &op = P.ops[r->pc];
        if (op.kind != OP_TC)
            continue;
        const int g = (op.bn == 256) ? 1 : 0;
        const TcLaunch &l = P.tc[op.idx];
        for (int q = 0; q < l.nprob; ++q) {
            TcProblem tp = l.p[q];
            for (const PatchRec &pr : P.patches)
                if (pr.kind == OP_TC && pr.launch == op.idx && pr.prob == q) {
                    if (pr.flags & PT_C_IS_A) {
                        tp.ep.c0 = r->m.A;
                        tp.ep.ldc = r->m.lda;
                    }
                    if (pr.flags & PT_O_IS_Y) {
                        tp.ep.o0 = r->m.Y;
                        tp.ep.ldo = r->m.ldy;
                        attach_store_maps(tp);
                    }
                    if (pr.flags & PT_ALPHA_NEG_TAU)
                        tp.ep.alpha = -(double)r->m.tau;
                }
            tp.patch = 0;
            starts[g].push_back(tiles[g]);
            tiles[g] += tc_num_tiles(tp, op.bn);
            probs[g].push_back(tp);
        }
        r->pc += 1;
        if (P.ops[r->pc].kind == OP_FINAL)
            fin.push_back(r);
    }
    // Finalize records.
    std::vector<AuxRec> faux;
    std::vector<CallRec> fcalls;
    for (Request *r : fin) {
        faux.push_back(aux_of(r, 0, 0));
        fcalls.push_back(call_of(r));
    }
    // Stage the tables.
    size_t o_aux = take(sizeof(AuxRec) * aux.size()), o_calls = take(sizeof(CallRec) * calls.size());
    size_t o_faux = take(sizeof(AuxRec) * faux.size()), o_fcalls = take(sizeof(CallRec) * fcalls.size());
    size_t o_p[2], o_s[2];
    for (int g = 0; g < 2; ++g) {
        starts[g].push_back(tiles[g]);
        o_p[g] = take(sizeof(TcProblem) * probs[g].size());
        o_s[g] = take(sizeof(int) * starts[g].size());
    }
    if (used > kRingSlotBytes)
        return SVT_ERR_OOM;
    std::memcpy(h + o_aux, aux.data(), sizeof(AuxRec) * aux.size());
    std::memcpy(h + o_calls, calls.data(), sizeof(CallRec) * calls.size());
    std::memcpy(h + o_faux, faux.data(), sizeof(AuxRec) * faux.size());
    std::memcpy(h + o_fcalls, fcalls.data(), sizeof(CallRec) * fcalls.size());
    for (int g = 0; g < 2; ++g) {
        std::memcpy(h + o_p[g], probs[g].data(), sizeof(TcProblem) * probs[g].size());
        std::memcpy(h + o_s[g], starts[g].data(), sizeof(int) * starts[g].size());
    }
    cudaStream_t st = s->win;
    if (used && cudaMemcpyAsync(d, h, used, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SVT_ERR_CUDA;
    auto A = [&](size_t o) { return reinterpret_cast<AuxRec *>(d + o); };
    auto C = [&](size_t o) { return reinterpret_cast<CallRec *>(d + o); };
    int launched = 0;
    if (!ingest.empty()) {
        const int n = (int)ingest.size();
        if (grouped_zero_launch(A(o_aux), n, st) != cudaSuccess ||
            grouped_reduce_launch(A(o_aux), C(o_calls), n, blk_r, st) != cudaSuccess ||
            grouped_split_launch(A(o_aux), C(o_calls), n, blk_s, st) != cudaSuccess)
            return SVT_ERR_CUDA;
        launched += 3;
    }
    for (int g = 0; g < 2; ++g) {
        if (probs[g].empty())
            continue;
        TcLaunch L;
        std::memset(&L, 0, sizeof(L));
        L.gtab = reinterpret_cast<const TcProblem *>(d + o_p[g]);
        L.gstart = reinterpret_cast<const int *>(d + o_s[g]);
        L.gcount = (int)probs[g].size();
        L.dep_wait_ns = ctx->dbg_wait_ns;
        if (tc_gemm_launch_grouped(L, g ? 256 : 128, tiles[g], sms, st) != cudaSuccess)
            return SVT_ERR_CUDA;
        ++launched;
    }
    // Requests outside the grouped kinds advance one op with ordinary launches.
    for (Request *r : single) {
        CallArgs a{r->m.A, r->m.lda, r->m.tau, r->m.Y, r->m.ldy, r->m.d_status};
        size_t last = r->pc + 1;
        if (r->plan->ops[r->pc].kind == OP_MEMSET)
            last = r->pc + 3;  // memset, reduce, split together
        svt_status e;
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            e = run_ops(ctx, *r->plan, a, st, r->pc, last, sms);
        }
        if (e != SVT_OK)
            return e;
        r->pc = last;
        if (r->pc >= r->plan->ops.size()) {
            if (plan_status_copy(ctx, *r->plan, &s->h_status[r->slot], st) != SVT_OK ||
                cudaEventRecord(s->events[r->slot], st) != cudaSuccess)
                return SVT_ERR_CUDA;
            r->state = 3;
        }
    }
    if (!fin.empty()) {
        if (grouped_finalize_launch(A(o_faux), C(o_fcalls), (int)fin.size(), st) != cudaSuccess)
            return SVT_ERR_CUDA;
        ++launched;
        for (Request *r : fin) {
            r->pc += 1;
            if (plan_status_copy(ctx, *r->plan, &s->h_status[r->slot], st) != SVT_OK ||
                cudaEventRecord(s->events[r->slot], st) != cudaSuccess)
                return SVT_ERR_CUDA;
            r->state = 3;
        }
    }
    if (cudaEventRecord(s->ring_ev[k], st) != cudaSuccess)
        return SVT_ERR_CUDA;
    s->ring_busy[k] = true;
    s->ring_next = (k + 1) % kRing;
    ctx->launches += (uint64_t)launched;
    ++s->windows;
    return SVT_OK;
}

// One scheduler tick under s->mu. Returns true if anything happened.
bool tick(svt_ctx *ctx, ServeState *s)
{
    bool progress = false;
    // Retire requests whose last op has completed on the device.
    for (auto it = s->active.begin(); it != s->active.end();) {
        Request *r = *it;
        if (r->state != 3) {
            ++it;
            continue;
        }
        cudaError_t q = cudaEventQuery(s->events[r->slot]);
        if (q == cudaErrorNotReady) {
            ++it;
            continue;
        }
        finish(s, r, q != cudaSuccess ? SVT_ERR_CUDA
                                      : (r->cancelled ? SVT_ERR_CANCELLED
                                                      : (svt_status)s->h_status[r->slot]));
        trace("done", r->ticket, (long long)r->result);
        if (r->large)
            s->bigs.erase(std::remove(s->bigs.begin(), s->bigs.end(), r), s->bigs.end());
        it = s->active.erase(it);
        progress = true;
    }
    // Large lane admission: the queued large request with the least work (the oldest of
    // equals) once fewer than kMaxLarge run and its workspace fits. While it waits for
    // workspace no new small request is admitted (the running ones free theirs within
    // milliseconds).
    bool hold_small = false;
    const double t_tick = now_ms();
    while ((int)s->bigs.size() < kMaxLarge && !s->bigq.empty() && (int)s->active.size() < kSlots) {
        auto pick = s->bigq.end();
        for (auto it = s->bigq.begin(); it != s->bigq.end(); ++it)
            if (admissible(ctx, *it, t_tick) && (pick == s->bigq.end() || (*it)->est_work < (*pick)->est_work))
                pick = it;
        if (pick == s->bigq.end())
            break;
        Request *r = *pick;
        size_t off;
        if (!s->arena.alloc(r->ws_len, &off)) {
            hold_small = s->bigs.empty();
            trace("hold", r->ticket, (long long)r->ws_len);
            break;
        }
        s->bigq.erase(pick);
        const double t0 = trace_file() ? now_ms() : 0.0;
        int slot = 0;
        while (s->slot_used[slot])
            ++slot;
        s->slot_used[slot] = true;
        r->slot = slot;
        r->ws_off = off;
        r->t_admit = now_ms();
        Plan *plan = nullptr;
        svt_status e;
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            NvtxRange nvtx("svt serve large admit");
            evict_plans(ctx, 512);
            e = get_plan(ctx, r->m.m, r->m.n, r->opt, off, ctx->ws_bytes - kRingBytes - off, &plan, 0,
                         &r->plan_ref);
            if (e == SVT_OK) {
                r->seg = plan_segments(*plan, kSegmentWork);
                r->seg_next = 0;
                r->seg_total = 0.0;
                for (double w : r->seg.work)
                    r->seg_total += w;
            }
        }
        trace("large_admit", r->ticket, trace_file() ? (long long)((now_ms() - t0) * 1e3) : 0);
        if (e != SVT_OK) {
            finish(s, r, e);
        } else {
            r->plan = plan;
            r->state = 4;
            s->active.push_back(r);
            s->bigs.push_back(r);
        }
        progress = true;
    }
    // Large lane launches: at most two in flight; each to the admitted request with the
    // least work left; every SM while no small request waits or runs.
    for (;;) {
        Request *r = nullptr;
        for (Request *q : s->bigs)
            if (q->state == 4 && q->cancel) {  // dropped before its next launch
                if (cudaEventRecord(s->events[q->slot], s->big_stream) != cudaSuccess)
                    continue;  // retried next tick
                q->state = 3;
                q->cancelled = true;
                trace("cancel", q->ticket, (long long)q->seg_next);
                progress = true;
            }
        for (Request *q : s->bigs)
            if (q->state == 4 && (!r || q->remaining() < r->remaining()))
                r = q;
        if (!r)
            break;
        const uint64_t k = s->big_issued;
        if (k >= 2 && cudaEventQuery(s->seg_ev[k % 2]) == cudaErrorNotReady)
            break;
        bool small_busy = !s->queue.empty();
        for (Request *q : s->active)
            small_busy = small_busy || !q->large;
        const int width = small_busy ? ctx->num_sms - kSmallSms : ctx->num_sms;
        const int part = r->seg_next;
        const bool last = part == r->seg.count() - 1;
        svt_status e;
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            NvtxRange nvtx("svt serve large launch");
            CallArgs a{r->m.A, r->m.lda, r->m.tau, r->m.Y, r->m.ldy, r->m.d_status};
            e = run_plan_segment(ctx, *r->plan, a, s->big_stream, r->seg, part, width);
            if (e == SVT_OK && cudaEventRecord(s->seg_ev[k % 2], s->big_stream) != cudaSuccess)
                e = SVT_ERR_CUDA;
            if (e == SVT_OK && last) {
                e = plan_status_copy(ctx, *r->plan, &s->h_status[r->slot], s->big_stream);
                if (e == SVT_OK && cudaEventRecord(s->events[r->slot], s->big_stream) != cudaSuccess)
                    e = SVT_ERR_CUDA;
            }
        }
        trace("large_launch", r->ticket, (long long)part * 1000 + width);
        progress = true;
        s->big_issued = k + 1;
        if (e != SVT_OK) {
            cudaStreamSynchronize(s->big_stream);
            s->active.remove(r);
            s->bigs.erase(std::remove(s->bigs.begin(), s->bigs.end(), r), s->bigs.end());
            finish(s, r, e);
            continue;
        }
        r->seg_next = part + 1;
        if (last)
            r->state = 3;
    }
    // Small lane: admit in arrival order while a slot and workspace are free.
    while (!hold_small && !s->queue.empty() && (int)s->active.size() < kSlots &&
           admissible(ctx, s->queue.front(), t_tick)) {
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
        r->t_admit = now_ms();
        Plan *plan = nullptr;
        svt_status e;
        const double t0 = trace_file() ? now_ms() : 0.0;
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            evict_plans(ctx, 512);  // plans of active requests stay alive through plan_ref
            e = get_plan(ctx, r->m.m, r->m.n, r->opt, off, ctx->ws_bytes - kRingBytes - off, &plan,
                         0, &r->plan_ref);
        }
        trace("admit", r->ticket, trace_file() ? (long long)((now_ms() - t0) * 1e3) : 0);
        if (e != SVT_OK) {
            finish(s, r, e);
            progress = true;
            continue;
        }
        r->plan = plan;
        r->pc = 0;
        r->grouped = grouped_kinds(*plan);
        r->state = 1;
        s->active.push_back(r);
        progress = true;
    }
    // Cancelled requests whose stages were being issued: no further windows; they retire
    // once the work already issued (in order on the window stream) has finished.
    for (Request *r : s->active)
        if (r->state == 1 && r->cancel) {
            if (cudaEventRecord(s->events[r->slot], s->win) != cudaSuccess)
                continue;  // retried next tick
            r->state = 3;
            r->cancelled = true;
            trace("cancel", r->ticket, (long long)r->pc);
            progress = true;
        }
    // Issue one window if any request has ops left to issue.
    bool any = false;
    for (Request *r : s->active)
        if (r->state == 1)
            any = true;
    if (any) {
        const double t0 = trace_file() ? now_ms() : 0.0;
        NvtxRange nvtx("svt serve window");
        svt_status e = issue_window(ctx, s, s->bigs.empty() ? ctx->num_sms : kSmallSms);
        if (e == SVT_ERR_NOT_READY)
            return progress;
        trace("window", s->windows, trace_file() ? (long long)((now_ms() - t0) * 1e3) : 0);
        if (e != SVT_OK) {
            for (auto it = s->active.begin(); it != s->active.end();) {
                Request *r = *it;
                if (r->state == 1) {
                    cudaStreamSynchronize(s->win);
                    finish(s, r, e);
                    it = s->active.erase(it);
                } else {
                    ++it;
                }
            }
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
        if (progress) {
            lk.unlock();  // let submit / poll in between windows
            std::this_thread::yield();
            lk.lock();
            continue;
        }
        if (s->active.empty())
            s->cv.wait_for(lk, std::chrono::milliseconds(5));
        else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

// Merge the per-matrix plans stage by stage into grouped launches, upload the
// device tables and capture the launch sequence in a CUDA graph.
svt_status build_batch(svt_ctx *ctx, ServeState *s, const svt_matrix *mats, int count,
                       const Resolved &r_in, const std::vector<size_t> &off, size_t tables_off,
                       int bn, BatchPlan *bp)
{
    Resolved r = r_in;
    r.fuse = 0;  // grouped launches take the per-stage problems
    std::vector<Plan *> plans(count);
    for (int i = 0; i < count; ++i) {
        svt_status st = get_plan(ctx, mats[i].m, mats[i].n, r, off[i], ctx->ws_bytes - off[i],
                                 &plans[i], bn);
        if (st != SVT_OK)
            return st;
    }
    // Structure check: same op kinds in the same order.
    const Plan &p0 = *plans[0];
    for (int i = 1; i < count; ++i) {
        if (plans[i]->ops.size() != p0.ops.size())
            return SVT_ERR_UNSUPPORTED;
        for (size_t k = 0; k < p0.ops.size(); ++k)
            if (plans[i]->ops[k].kind != p0.ops[k].kind)
                return SVT_ERR_UNSUPPORTED;
    }
    for (const Op &op : p0.ops)
        if (op.kind != OP_MEMSET && op.kind != OP_REDUCE && op.kind != OP_SPLIT &&
            op.kind != OP_TC && op.kind != OP_FINAL)
            return SVT_ERR_UNSUPPORTED;
    bp->count = count;
    bp->tables_off = tables_off;
    uint8_t *tbase = ctx->ws + tables_off;
    size_t toff = 0;
    auto take = [&](size_t bytes) {
        size_t o = toff;
        toff = align_up(toff + bytes, kAlign);
        return o;
    };
    // Per-matrix records of the memory-bound steps.
    std::vector<AuxRec> aux(count);
    int blk_r = 0, blk_s = 0;
    for (int i = 0; i < count; ++i) {
        const Plan &P = *plans[i];
        const Layout &L = P.lay;
        uint8_t *base = ctx->ws + P.ws_base;
        AuxRec &a = aux[i];
        std::memset(&a, 0, sizeof(a));
        a.m = P.m;
        a.n = P.n;
        a.wide = P.wide ? 1 : 0;
        a.f64 = (r.prec == SVT_FP64) ? 1 : 0;
        a.scal = reinterpret_cast<double *>(base + L.scal);
        a.status = reinterpret_cast<int *>(base + L.status);
        a.colnorm = reinterpret_cast<double *>(base + L.colnorm);
        a.zero_words = (int64_t)((L.colnorm + (size_t)L.N * sizeof(double) - L.scal) / 8);
        const Buf &same = P.wide ? L.Xt[0] : L.X[0];
        const Buf &tran = P.wide ? L.X[0] : L.Xt[0];
        a.xs_hi = base + same.hi;
        a.xs_lo = same.has_lo ? base + same.lo : nullptr;
        a.ld_s = same.ld;
        a.xt_hi = base + tran.hi;
        a.xt_lo = tran.has_lo ? base + tran.lo : nullptr;
        a.ld_t = tran.ld;
        if (r.prec == SVT_BF16) {  // lo part of X0^T only, for the Gram
            if (P.wide)
                a.xs_lo = base + L.XtLo0.hi;
            else
                a.xt_lo = base + L.XtLo0.hi;
        }
        a.blk_reduce = blk_r;
        a.blk_split = blk_s;
        blk_r += grouped_reduce_blocks(P.m, P.n, a.wide);
        blk_s += grouped_split_blocks(P.m, P.n);
    }
    bp->blocks_reduce = blk_r;
    bp->blocks_split = blk_s;
    bp->d_aux = reinterpret_cast<AuxRec *>(tbase + take(sizeof(AuxRec) * count));
    bp->d_calls = reinterpret_cast<CallRec *>(tbase + take(sizeof(CallRec) * count));
    bp->tables.emplace_back(bp->d_aux, std::vector<uint8_t>(
                                           reinterpret_cast<uint8_t *>(aux.data()),
                                           reinterpret_cast<uint8_t *>(aux.data() + count)));
    // One persistent launch for every product of every matrix: stage-major order
    // (stage k of all matrices, then stage k + 1), each problem depending on the
    // previous problem of its matrix's chain (the combine on both chains).
    std::vector<TcProblem> probs;
    std::vector<int> starts, valid;
    std::vector<std::array<int, 2>> lastp(count, std::array<int, 2>{-1, -1});
    std::vector<std::vector<int>> chain_base(count);
    for (int i = 0; i < count; ++i) {
        const Plan &P = *plans[i];
        int acc = 0;
        for (const TcLaunch &l : P.tc) {
            chain_base[i].push_back(acc);
            acc += l.nprob;
        }
    }
    int total = 0;
    for (size_t k = 0; k < p0.ops.size(); ++k) {
        if (p0.ops[k].kind != OP_TC)
            continue;
        for (int i = 0; i < count; ++i) {
            const Plan &P = *plans[i];
            const int li = P.ops[k].idx;
            const TcLaunch &l = P.tc[li];
            for (int q = 0; q < l.nprob; ++q) {
                TcProblem tp = l.p[q];
                const int chain = P.tc_chain[chain_base[i][li] + q];
                tp.patch = 0;
                for (const PatchRec &pr : P.patches)
                    if (pr.kind == OP_TC && pr.launch == li && pr.prob == q)
                        tp.patch |= pr.flags;
                tp.call_idx = i;
                if (tp.patch & PT_O_IS_Y)
                    tp.o_tma = 0;  // per-call output: plain stores
                tp.pid = (int)probs.size();
                tp.dep[0] = tp.dep[1] = -1;
                tp.dep_target[0] = tp.dep_target[1] = 0;
                if (chain < 2) {
                    tp.dep[0] = lastp[i][chain];
                } else {
                    tp.dep[0] = lastp[i][0];
                    tp.dep[1] = lastp[i][1];
                }
                for (int d = 0; d < 2; ++d)
                    if (tp.dep[d] >= 0)
                        tp.dep_target[d] = kEpiWarpsPublic * valid[tp.dep[d]];
                starts.push_back(total);
                total += tc_num_tiles(tp, bn);
                valid.push_back(tc_valid_ctas(tp, bn));
                if (chain < 2)
                    lastp[i][chain] = tp.pid;
                else
                    lastp[i][0] = lastp[i][1] = tp.pid;
                probs.push_back(tp);
            }
        }
    }
    starts.push_back(total);
    TcProblem *dp = reinterpret_cast<TcProblem *>(tbase + take(sizeof(TcProblem) * probs.size()));
    int *ds = reinterpret_cast<int *>(tbase + take(sizeof(int) * starts.size()));
    int *counters = reinterpret_cast<int *>(tbase + take(sizeof(int) * (probs.size() + 1)));
    if (toff > batch_table_bytes(count, r))
        return SVT_ERR_OOM;
    bp->tables.emplace_back(dp, std::vector<uint8_t>(
                                    reinterpret_cast<uint8_t *>(probs.data()),
                                    reinterpret_cast<uint8_t *>(probs.data() + probs.size())));
    bp->tables.emplace_back(ds, std::vector<uint8_t>(
                                    reinterpret_cast<uint8_t *>(starts.data()),
                                    reinterpret_cast<uint8_t *>(starts.data() + starts.size())));
    {
        TcLaunch L;
        std::memset(&L, 0, sizeof(L));
        L.gtab = dp;
        L.gstart = ds;
        L.gcount = (int)probs.size();
        L.calls = bp->d_calls;
        L.dep_wait_ns = ctx->dbg_wait_ns;
        L.done = counters;
        L.tile_counter = counters + probs.size();
        bp->launches.push_back(L);
        bp->tiles.push_back(total);
        bp->bns.push_back(bn);
        bp->counters = counters;
        bp->counter_bytes = sizeof(int) * (probs.size() + 1);
    }
    if (cudaMallocHost(reinterpret_cast<void **>(&bp->h_calls), sizeof(CallRec) * count) != cudaSuccess)
        return SVT_ERR_CUDA;
    if (cudaEventCreateWithFlags(&bp->uploaded, cudaEventDisableTiming) != cudaSuccess)
        return SVT_ERR_CUDA;
    // Capture: calls upload, zero, reduce, split, grouped products, finalize.
    if (!s->capture && cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking) != cudaSuccess)
        return SVT_ERR_CUDA;
    for (size_t k = 0; k < bp->launches.size(); ++k)  // set function attributes before capture
        if (tc_gemm_launch_fused(bp->launches[k], bp->bns[k], 0, ctx->num_sms, s->capture) !=
            cudaSuccess)
            return SVT_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    cudaStream_t cs = s->capture;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return SVT_ERR_CUDA;
    bool ok = cudaMemcpyAsync(bp->d_calls, bp->h_calls, sizeof(CallRec) * count,
                              cudaMemcpyHostToDevice, cs) == cudaSuccess;
    ok = ok && cudaMemsetAsync(bp->counters, 0, bp->counter_bytes, cs) == cudaSuccess;
    ok = ok && grouped_zero_launch(bp->d_aux, count, cs) == cudaSuccess;
    ok = ok && grouped_reduce_launch(bp->d_aux, bp->d_calls, count, bp->blocks_reduce, cs) == cudaSuccess;
    ok = ok && grouped_split_launch(bp->d_aux, bp->d_calls, count, bp->blocks_split, cs) == cudaSuccess;
    for (size_t k = 0; ok && k < bp->launches.size(); ++k)
        ok = tc_gemm_launch_fused(bp->launches[k], bp->bns[k], bp->tiles[k], ctx->num_sms, cs) ==
             cudaSuccess;
    ok = ok && grouped_finalize_launch(bp->d_aux, bp->d_calls, count, cs) == cudaSuccess;
    cudaError_t ec = cudaStreamEndCapture(cs, &graph);
    if (!ok || ec != cudaSuccess || !graph) {
        if (graph)
            cudaGraphDestroy(graph);
        return SVT_ERR_CUDA;
    }
    cudaError_t ei = cudaGraphInstantiate(&bp->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess)
        return SVT_ERR_CUDA;
    bp->kernels_per_call = 4 + (int)bp->launches.size();
    return SVT_OK;
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
    s->batches.clear();
    if (s->capture)
        cudaStreamDestroy(s->capture);
    if (s->win) {
        cudaStreamSynchronize(s->win);
        cudaStreamDestroy(s->win);
    }
    if (s->big_stream) {
        cudaStreamSynchronize(s->big_stream);
        cudaStreamDestroy(s->big_stream);
    }
    for (int i = 0; i < kRing; ++i)
        if (s->ring_ev[i])
            cudaEventDestroy(s->ring_ev[i]);
    for (int i = 0; i < 2; ++i)
        if (s->seg_ev[i])
            cudaEventDestroy(s->seg_ev[i]);
    if (s->h_ring)
        cudaFreeHost(s->h_ring);
    if (s->metrics)
        std::fclose(s->metrics);
    // Every request lives in `tickets` from submission until its release (queued and
    // active ones included), so the ticket map owns them all.
    s->queue.clear();
    s->bigq.clear();
    s->active.clear();
    for (auto &kv : s->tickets)
        delete kv.second;
    s->tickets.clear();
    delete s;
    ctx->serve = nullptr;
}

bool serve_busy(svt_ctx *ctx)
{
    ServeState *s = ctx->serve;
    if (!s)
        return false;
    std::lock_guard<std::mutex> g(s->mu);
    return !s->queue.empty() || !s->bigq.empty() || !s->active.empty();
}

} // namespace svt

namespace {

// Tile width of a grouped batch: the one with less padded tensor work over the
// matrices' largest products (M x N), 128-wide tiles weighted as ~15 % less
// efficient per flop.
int batch_bn(const svt_matrix *mats, int count)
{
    double a128 = 0, a256 = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t M = std::max(mats[i].m, mats[i].n), N = std::min(mats[i].m, mats[i].n);
        const double tm = (double)((M + kBM - 1) / kBM);
        a128 += tm * (double)((N + 127) / 128) * 128.0 / 0.85;
        a256 += tm * (double)((N + 255) / 256) * 256.0;
    }
    return a128 < a256 ? 128 : 256;
}

// Options of all matrices resolved: SVT_OK, or the first matrix's option status.
svt_status resolve_all(const svt_matrix *mats, int count, std::vector<Resolved> &res, bool *same)
{
    res.resize(count);
    *same = true;
    for (int i = 0; i < count; ++i) {
        if (svt_status st = resolve_status(&mats[i].opt, &res[i]))
            return st;
        if (i > 0 && !same_options(res[i], res[0]))
            *same = false;
    }
    if (count > 0 && res[0].prec == SVT_FP64)
        *same = false;  // the FP64 tier runs per-matrix launches
    if (count > 0 && (!res[0].polish || res[0].mode != SVT_MODE_SVT))
        *same = false;  // grouped kernels cover the default pipeline
    return SVT_OK;
}

} // namespace

extern "C" {

svt_status svt_batch_workspace_bytes(const svt_matrix *mats, int count, size_t *out)
{
    if (!out || count < 0 || (count > 0 && !mats))
        return SVT_ERR_INVALID;
    std::vector<Resolved> res;
    bool same = false;
    if (svt_status rs = resolve_all(mats, count, res, &same))
        return rs;
    size_t total = 0;
    for (int i = 0; i < count; ++i) {
        if (mats[i].m <= 0 || mats[i].n <= 0)
            return SVT_ERR_INVALID;
        total += align_up(make_layout(mats[i].m, mats[i].n, res[i]).total, kAlign);
    }
    if (same && count > 0)
        total += batch_table_bytes(count, res[0]);
    *out = total;
    return SVT_OK;
}

svt_status svt_batch(svt_ctx_t ctx, const svt_matrix *mats, int count, void *stream)
{
    if (!ctx || count < 0 || (count > 0 && !mats))
        return SVT_ERR_INVALID;
    if (count == 0)
        return SVT_OK;
    if (serve_busy(ctx))
        return SVT_ERR_BUSY;
    std::vector<Resolved> res;
    bool same = false;
    if (svt_status rs = resolve_all(mats, count, res, &same))
        return rs;
    size_t total = 0;
    std::vector<size_t> off(count);
    for (int i = 0; i < count; ++i) {
        const svt_matrix &m = mats[i];
        svt_status st = validate(m.A, m.m, m.n, m.lda, m.tau, m.Y, m.ldy);
        if (st != SVT_OK)
            return st;
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

    // Grouped path: one launch per stage for all matrices, replayed from a CUDA graph.
    if (same && total + batch_table_bytes(count, res[0]) <= ctx->ws_bytes) {
        BatchKey key;
        key.r = res[0];
        key.bn = (res[0].tile == 128 || res[0].tile == 256) ? res[0].tile : batch_bn(mats, count);
        for (int i = 0; i < count; ++i) {
            key.shapes.push_back(mats[i].m);
            key.shapes.push_back(mats[i].n);
        }
        BatchPlan *bp = nullptr;
        auto it = s->batches.find(key);
        if (it != s->batches.end()) {
            bp = it->second.get();
        } else {
            if (s->batches.size() > 16)
                s->batches.clear();
            auto nb = std::make_unique<BatchPlan>();
            svt_status st = build_batch(ctx, s, mats, count, res[0], off, total, key.bn, nb.get());
            if (st == SVT_OK) {
                bp = nb.get();
                s->batches[key] = std::move(nb);
            } else if (st != SVT_ERR_UNSUPPORTED) {
                return st;
            }
        }
        if (bp) {
            if (bp->pending && cudaEventSynchronize(bp->uploaded) != cudaSuccess)
                return SVT_ERR_CUDA;
            if (ctx->table_owner != bp) {
                for (auto &t : bp->tables)
                    if (cudaMemcpyAsync(t.first, t.second.data(), t.second.size(),
                                        cudaMemcpyHostToDevice, cs) != cudaSuccess)
                        return SVT_ERR_CUDA;
                ctx->table_owner = bp;
            }
            for (int i = 0; i < count; ++i) {
                CallRec &c = bp->h_calls[i];
                c.A = mats[i].A;
                c.Y = mats[i].Y;
                c.lda = mats[i].lda;
                c.ldy = mats[i].ldy;
                c.tau = mats[i].tau;
                c.pad = 0;
                c.d_status = mats[i].d_status;
            }
            if (cudaGraphLaunch(bp->exec, cs) != cudaSuccess ||
                cudaEventRecord(bp->uploaded, cs) != cudaSuccess)
                return SVT_ERR_CUDA;
            bp->pending = true;
            ctx->launches += (uint64_t)bp->kernels_per_call;
            return SVT_OK;
        }
    }

    // Per-matrix solves over the worker streams (mixed options, FP64 tier).
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
    for (int i = 0; i < kStreams; ++i) {
        if (cudaEventRecord(s->events[1 + i], s->streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(cs, s->events[1 + i], 0) != cudaSuccess)
            return SVT_ERR_CUDA;
    }
    return SVT_OK;
}

svt_status svt_autotune_batch(svt_ctx_t ctx, const svt_matrix *mats, int count, int reps,
                              void *stream, int *tile_out, double *ms_out)
{
    if (!ctx || !mats || count <= 0 || reps < 1 || !tile_out)
        return SVT_ERR_INVALID;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    std::vector<svt_matrix> m(mats, mats + count);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0)
            cudaEventDestroy(e0);
        return SVT_ERR_CUDA;
    }
    svt_status st = SVT_OK;
    int best = 0;
    float best_ms = 0.0f;
    for (int bn : {128, 256}) {
        for (svt_matrix &x : m)
            x.opt.tile = bn;
        // one untimed call builds and records the batch's launches
        if ((st = svt_batch(ctx, m.data(), count, stream)) != SVT_OK)
            break;
        if (cudaEventRecord(e0, cs) != cudaSuccess) {
            st = SVT_ERR_CUDA;
            break;
        }
        for (int r = 0; r < reps && st == SVT_OK; ++r)
            st = svt_batch(ctx, m.data(), count, stream);
        float ms = 0.0f;
        if (st != SVT_OK || cudaEventRecord(e1, cs) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            if (st == SVT_OK)
                st = SVT_ERR_CUDA;
            break;
        }
        ms /= (float)reps;
        if (!best || ms < best_ms) {
            best = bn;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SVT_OK)
        return st;
    *tile_out = best;
    if (ms_out)
        *ms_out = best_ms;
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
    if ((st = resolve_status(&req->opt, &r)) != SVT_OK)
        return st;
    if (r.prec == SVT_FP64 && (req->m > kF64MaxDim || req->n > kF64MaxDim))
        return SVT_ERR_UNSUPPORTED;
    // Large requests: one fused solve; small ones: per-stage problems grouped in windows.
    const bool large = req->m * req->n >= kLargeElems && r.prec != SVT_FP64;
    r.fuse = large ? 1 : 0;
    size_t need = align_up(make_layout(req->m, req->n, r).total, kAlign);
    if (ctx->ws_bytes < kRingBytes || need > ctx->ws_bytes - kRingBytes)
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
        if (!s->metrics) {
            const char *mp = std::getenv("SVT_SERVE_METRICS");
            if (mp && *mp)
                s->metrics = std::fopen(mp, "a");
        }
        s->arena.reset(ctx->ws_bytes - kRingBytes);
        s->thread = std::thread(scheduler, ctx, s);
        s->started = true;
    }
    if (s->queue.size() + s->bigq.size() >= kQueueLimit)
        return SVT_ERR_BUSY;
    auto *q = new Request();
    q->ticket = s->next_ticket++;
    q->m = *req;
    q->opt = r;
    q->ws_len = need;
    q->t_submit = now_ms();
    q->large = large;
    q->est_work = (double)req->m * (double)req->n * (double)std::min(req->m, req->n) *
                  (r.prec == SVT_FP32 ? 3.0 : 1.0);
    (large ? s->bigq : s->queue).push_back(q);
    trace("submit", q->ticket, large ? 1 : 0);
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

svt_status svt_serve_cancel(svt_ctx_t ctx, uint64_t ticket)
{
    if (!ctx || !ctx->serve)
        return SVT_ERR_INVALID;
    ServeState *s = ctx->serve;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end())
        return SVT_ERR_INVALID;
    Request *r = it->second;
    switch (r->state) {
    case 0: {  // still queued: nothing of it reached the device
        auto &q = r->large ? s->bigq : s->queue;
        q.erase(std::remove(q.begin(), q.end(), r), q.end());
        r->result = SVT_ERR_CANCELLED;
        r->state = 2;
        r->t_done = now_ms();
        trace("cancel", r->ticket, -1);
        record(s, r);
        return SVT_OK;
    }
    case 1:  // stages being issued: the scheduler drops it before its next window
    case 4:  // large solve between launches: dropped before its next launch
        r->cancel = true;
        s->cv.notify_all();
        return SVT_OK;
    case 3:  // everything it needs is on the device already
        return r->cancelled ? SVT_OK : SVT_ERR_BUSY;
    default:
        return SVT_ERR_INVALID;
    }
}

svt_status svt_serve_metrics(svt_ctx_t ctx, const char *path)
{
    if (!ctx)
        return SVT_ERR_INVALID;
    FILE *f = nullptr;
    if (path && !(f = std::fopen(path, "a")))
        return SVT_ERR_INVALID;
    ServeState *s;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        s = state_of(ctx);
    }
    std::lock_guard<std::mutex> g(s->mu);
    if (s->metrics)
        std::fclose(s->metrics);
    s->metrics = f;
    return SVT_OK;
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
