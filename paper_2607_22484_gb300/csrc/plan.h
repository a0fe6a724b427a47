// Host-side plan structures of libsvt, shared by svt_api.cu and serve.cpp.
//
// A plan is the launch sequence of one solve for a fixed shape, option set and
// workspace offset: the tensor maps and static epilogue parameters are built
// once; per call only the input/output pointers and tau are patched in.
#pragma once

#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "svt_internal.h"

namespace svt {

// Host-side NVTX range for the duration of a scope (a profiler shows the library's
// stages: solves, plan builds, serving windows, batches); free when no tool listens.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int64_t kF64MaxDim = 4096;
constexpr size_t kAlign = 256;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int64_t ld_of(int64_t cols) { return (cols + 63) / 64 * 64; }

// Options with defaults applied.
struct Resolved {
    int iters;
    int prec;
    int schedule;   // SVT_SCHED_PE5 or SVT_SCHED_NS3
    int norm;       // SVT_NORM_FRO or SVT_NORM_GRAM
    double ell0, delta;
    int polish;
    int mode;
    int hp_steps;   // leading S-chain steps in the FP32-class tier (BF16 tier)
    int fuse;       // one persistent launch for all products of a solve
    int tile;       // requested tile-width code (0 automatic); read by svt_polar_ex only
    int out64 = 0;  // FP64 tier only: the result is stored as FP64 (svt_polar_f64)
    // FP8 experiment (BF16 tier only): bit t of fp8_p -- the P chain's Y^2 product of
    // step t on e4m3 copies of Y; bit t of fp8_s -- the S chain's step t (a BF16 step)
    // on e4m3 operands, all three products, or only Y^2 when fp8_s_y2.
    uint64_t fp8_p = 0, fp8_s = 0;
    int fp8_s_y2 = 0;
};

bool resolve(const svt_options *in, Resolved *r);
// resolve() as a status: SVT_ERR_UNSUPPORTED for the reserved FP8 tier, SVT_ERR_INVALID
// for any other option outside its range.
svt_status resolve_status(const svt_options *in, Resolved *r);

// A matrix buffer in the workspace: hi part and (FP32-class pairs) lo part.
struct Buf {
    size_t hi = 0, lo = 0;   // byte offsets (lo == 0: absent)
    int64_t rows = 0, cols = 0, ld = 0;
    bool has_lo = false;
};

struct Layout {
    int64_t M = 0, N = 0, ldM = 0, ldN = 0;
    size_t esz = 2;          // element size of matrix buffers (2 BF16, 8 FP64)
    size_t scal = 0, status = 0, counters = 0, colnorm = 0;
    size_t strips = 0, strips_bytes = 0;  // fused solves: strip counters (at the end)
    int max_strips = 0;                   // strip counters per problem
    int max_problems = 0;    // capacity of the fused counters / table
    size_t fused_tab = 0, fused_tab_bytes = 0;
    Buf X[2], Xt[2], XtLo0, S[2], Yp, Zp, Ys, Zs, ZPp, ZSp, B, Sp;
    Buf Yp8, S8[2], Ys8, Zs8;  // e4m3 copies (FP8 experiment), 1-byte elements
    size_t total = 0;
};

Layout make_layout(int64_t m, int64_t n, const Resolved &r);

// ------------------------------------------------------------ plan

enum OpKind { OP_MEMSET, OP_REDUCE, OP_SPLIT, OP_TC, OP_F64, OP_PREP, OP_FINAL };

struct Op {
    int kind;
    int idx;      // index into tc / f64 arrays
    int bn;       // TC tile width
};

struct PatchRec {
    int kind;     // OP_TC / OP_F64
    int launch, prob, flags;
};

struct Plan {
    int64_t m, n;
    bool wide;
    Resolved opt;
    Layout lay;
    size_t ws_base;
    std::vector<double> coef;
    std::vector<double> lo;         // lower end of each step's design interval
    int hp_steps_s = 0;             // leading S steps in the FP32-class tier
    bool final_s_pair = false;      // final S iterate carries a lo part
    std::vector<Op> ops;
    std::vector<TcLaunch> tc;
    std::vector<F64Launch> f64;
    std::vector<PatchRec> patches;
    std::vector<double> tc_flops;   // algorithmic flops of each tensor-core launch
    // flops the tensor cores execute for each launch: every hi/lo segment, whole tiles
    // (padding, the diagonal tiles of symmetric products), K rounded up to 64
    std::vector<double> tc_tensor_flops;
    double fused_tensor_flops = 0.0;
    std::vector<int> tc_chain;      // per problem of each launch: 0 P chain, 1 S chain, 2 both
    // Per problem of each launch: the buffers it reads and writes (device addresses of
    // their hi parts; null = none or the caller's), for the fused solve's dependencies.
    struct ProbIO {
        const void *l, *r, *c, *o, *t;
        int o_trans;
        const double *theta_src, *norm_acc;
        const void *f;  // the e4m3 copy written (FP8 experiment), null: none
    };
    std::vector<ProbIO> tc_io;
    bool uses_strips = false;       // the fused launch waits on strip counters
    // Fused execution: one launch for every product (table and counters in the workspace).
    bool fused = false;
    TcLaunch fused_launch;
    int fused_tiles = 0, fused_bn = 0;
    double fused_flops = 0.0;
    // Table order of the fused solve: first tile of each problem, then the tile count;
    // the tensor flops of each problem; the op range of the products in `ops`.
    std::vector<int> fused_starts;
    std::vector<double> fused_work;
    size_t fused_first_op = 0, fused_last_op = 0;
    // The fused table lives in the shared workspace, which other solves overwrite:
    // it is copied from this immutable pinned host image before every fused launch.
    uint8_t *h_fused = nullptr;
    size_t fused_bytes = 0;
    ~Plan()
    {
        if (h_fused)
            cudaFreeHost(h_fused);
    }
    int tc_launches_per_solve = 0;
    int kernel_launches = 0;
    int force_bn = 0;               // 0: tile width per launch; 128 / 256: fixed (grouped batches);
                                    // -1: per-launch widths from bn_choice (autotuned)
    std::vector<int> bn_choice;     // tile width of each product launch (autotuned plans)
};

// Autotuned tile widths of one (shape, options): one entry per product launch.
struct TuneKey {
    int64_t m, n;
    int iters, prec, schedule, norm, polish, mode, hp_steps;
    double ell0, delta;
    int fuse;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(m, n, iters, prec, schedule, norm, polish, mode, hp_steps, ell0, delta,
                        fuse) <
               std::tie(o.m, o.n, o.iters, o.prec, o.schedule, o.norm, o.polish, o.mode,
                        o.hp_steps, o.ell0, o.delta, o.fuse);
    }
};
inline TuneKey tune_key(int64_t m, int64_t n, const Resolved &r)
{
    return TuneKey{m, n, r.iters, r.prec, r.schedule, r.norm, r.polish, r.mode, r.hp_steps,
                   r.ell0, r.delta, r.fuse};
}

struct Key {
    int64_t m, n;
    int iters, prec, schedule, norm, polish, mode, hp_steps;
    double ell0, delta;
    size_t ws_base;
    int force_bn;
    int fuse;
    int out64;
    uint64_t fp8_p, fp8_s;
    int fp8_s_y2;
    bool operator<(const Key &o) const
    {
        return std::tie(m, n, iters, prec, schedule, norm, polish, mode, hp_steps, ell0, delta,
                        ws_base, force_bn, fuse, out64, fp8_p, fp8_s, fp8_s_y2) <
               std::tie(o.m, o.n, o.iters, o.prec, o.schedule, o.norm, o.polish, o.mode,
                        o.hp_steps, o.ell0, o.delta, o.ws_base, o.force_bn, o.fuse, o.out64,
                        o.fp8_p, o.fp8_s, o.fp8_s_y2);
    }
};


struct CallArgs {
    const float *A;
    int64_t lda;
    float tau;
    float *Y;
    int64_t ldy;
    svt_status *d_status;
    // Launches recorded into a CUDA graph body: no fused-table upload (the caller
    // uploads it before launching the graph), no event records, no launch count.
    bool in_graph = false;
};

svt_status validate(const float *A, int64_t m, int64_t n, int64_t lda, float tau, const float *Y,
                    int64_t ldy);
// The same checks for an output of ysz-byte elements (svt_polar_f64: FP64).
svt_status validate_out(const float *A, int64_t m, int64_t n, int64_t lda, float tau,
                        const void *Y, int64_t ldy, size_t ysz);

// Whether the byte ranges [a, a + abytes) and [b, b + bbytes) intersect.
inline bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes)
{
    const char *a0 = static_cast<const char *>(a), *b0 = static_cast<const char *>(b);
    return a0 < b0 + bbytes && b0 < a0 + abytes;
}

struct CompletionGraph;  // completion.cu

} // namespace svt

// Serving state of a context (serve.cpp).
struct ServeState;

struct svt_ctx {
    int device = 0;
    int num_sms = 0;
    uint8_t *ws = nullptr;
    size_t ws_bytes = 0;
    uint64_t launches = 0;
    std::map<svt::Key, std::shared_ptr<svt::Plan>> plans;  // users may hold their own reference
    std::mutex mu;
    ServeState *serve = nullptr;
    // Optional per-launch timing of the tensor-core kernel (svt_ctx_profile).
    bool profile = false;
    std::vector<cudaEvent_t> prof_pool;
    struct ProfRec { cudaEvent_t a, b; double flops, tensor_flops; };
    std::vector<ProfRec> prof_pending;
    size_t prof_next = 0;
    std::map<svt::TuneKey, std::vector<int>> tuning;  // svt_autotune results
    // Which grouped-batch plan's device tables are intact in the workspace (any
    // other use of the workspace resets it; the batch then re-uploads its tables).
    const void *table_owner = nullptr;
    // Cached device-resident completion loops (completion.cu), most recent last.
    std::vector<svt::CompletionGraph *> completion_graphs;
    cudaStream_t capture_stream = nullptr;  // private stream for graph capture
    char gpu_name[256] = {};                // device name (autotune cache key)
    // Debug settings (svt_ctx_debug): plan builds until one fails (0: off), serving
    // admission delay, device dependency-wait limit (0: default).
    int64_t dbg_fail_plan = 0;
    int64_t dbg_admit_delay_us = 0;
    uint64_t dbg_wait_ns = 0;
};

namespace svt {
// Look up or build the plan of a solve (under ctx->mu). `keep` (nullable) receives
// a reference that keeps the plan alive across cache evictions.
svt_status get_plan(svt_ctx *ctx, int64_t m, int64_t n, const Resolved &r, size_t ws_base,
                    size_t ws_avail, Plan **out, int force_bn = 0,
                    std::shared_ptr<Plan> *keep = nullptr);
// Drop cached plans nobody else holds once the cache exceeds max_entries (under ctx->mu).
void evict_plans(svt_ctx *ctx, size_t max_entries);
// sms: SMs the product launches may use (0 = all of the device).
svt_status run_plan(svt_ctx *ctx, Plan &P, const CallArgs &a, cudaStream_t s, int sms = 0);
// Ops [first, last) of a plan only (the serving loop advances requests op by op).
svt_status run_ops(svt_ctx *ctx, Plan &P, const CallArgs &a, cudaStream_t s, size_t first,
                   size_t last, int sms = 0);
// Read the plan's internal status word back to host memory (async on s).
svt_status plan_status_copy(svt_ctx *ctx, const Plan &P, int *host_dst, cudaStream_t s);
// The plan a solve of this shape and these options uses (tuned, explicit or automatic
// tile width), as svt_polar_ex looks it up (under ctx->mu).
svt_status plan_for_solve(svt_ctx *ctx, int64_t m, int64_t n, const Resolved &r, Plan **out,
                          std::shared_ptr<Plan> *keep = nullptr);
// Refresh the plan's fused-launch table in the workspace from its host image (async on s).
svt_status upload_fused_table(svt_ctx *ctx, Plan &P, cudaStream_t s);
// A solve split into consecutive parts of about `target` tensor flops each (at most
// kMaxFusedSegments). A fused plan splits its product table into contiguous problem
// ranges (`bounds`: the first problem of each part, then the problem count), each part
// one launch of the fused kernel over its tiles; a plan issued launch by launch splits
// its op list (`bounds`: op indices). `work`: the tensor flops of each part.
struct Segments {
    bool fused = false;
    std::vector<int> bounds;
    std::vector<double> work;
    int count() const { return (int)bounds.size() - 1; }
};
Segments plan_segments(const Plan &P, double target);
// Issues part k of a solve split by plan_segments on stream s with grids of `sms` SMs.
// Fused: with k == 0 first the ops before the products (scratch reset, ingest) and the
// table upload, then the launch over the part's tiles, and with the last part the ops
// after the products. Parts must be issued in order, each after the previous one on the
// same stream: the dependency counters carry over between them.
svt_status run_plan_segment(svt_ctx *ctx, Plan &P, const CallArgs &a, cudaStream_t s,
                            const Segments &seg, int k, int sms);
// Release the context's cached completion graphs (after the device is idle).
void completion_release(svt_ctx *ctx);
void serve_shutdown(svt_ctx *ctx);
bool serve_busy(svt_ctx *ctx);
} // namespace svt
