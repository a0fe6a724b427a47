// One proximal-gradient step of nuclear-norm regularised matrix completion,
// the use of singular value soft-thresholding that Section 2 names (SVT as the
// proximal operator of the nuclear norm inside proximal gradient methods):
//
//   minimise F(X) = 1/2 || P_Omega(X - M) ||_F^2 + lambda ||X||_*
//   step:    Z = X + h P_Omega(M - X)         (gradient step on the smooth part)
//            X <- A_{h lambda}(Z)             (Eq. 1, through the library's solve)
//
// The gradient of the smooth part is P_Omega(X - M), whose Lipschitz constant
// is 1, so any step h in (0, 1] does not increase F. The masked gradient step
// is one memory-bound kernel (one pass over X, M, the mask and Z); the
// thresholding is svt_polar_ex on Z with tau = h lambda, written into X.
//
// svt_complete runs the same steps as a device-resident loop with lambda
// continuation: a CUDA graph with one conditional WHILE node per stage, whose body
// is the masked step (also saving X), the solve, an FP64 reduction of the step's
// change and a one-thread kernel that decides whether the body runs again.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "plan.h"

namespace {

// Z = X + h P_Omega(M - X), one CTA per row at a time; float4 accesses where the
// row's addresses allow them (checked on the real addresses), scalar otherwise.
// COPY: also Xprev = X (the device-resident loop measures the step's change).
template <bool COPY>
__global__ void __launch_bounds__(256) prox_grad_kernel(const float *X, int64_t ldx, const float *M,
                                                        int64_t ldm, const uint8_t *W, int64_t ldw,
                                                        float *Z, int64_t ldz, int64_t m, int64_t n,
                                                        float h, float *Xprev, int64_t ldp)
{
    const bool unit = (h == 1.0f);  // observed entries become M exactly
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        const float *x = X + i * ldx;
        const float *mm = M + i * ldm;
        const uint8_t *w = W + i * ldw;
        float *z = Z + i * ldz;
        float *xp = COPY ? Xprev + i * ldp : nullptr;
        const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(mm) |
                           reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(xp)) &
                          15u) == 0 &&
                         (reinterpret_cast<uintptr_t>(w) & 3u) == 0;
        int64_t j0 = 0;
        if (vec) {
            const int64_t n4 = n >> 2;
            for (int64_t q = threadIdx.x; q < n4; q += blockDim.x) {
                const float4 xv = reinterpret_cast<const float4 *>(x)[q];
                const float4 mv = reinterpret_cast<const float4 *>(mm)[q];
                const uchar4 wv = reinterpret_cast<const uchar4 *>(w)[q];
                float4 zv;
                zv.x = wv.x ? (unit ? mv.x : fmaf(h, mv.x - xv.x, xv.x)) : xv.x;
                zv.y = wv.y ? (unit ? mv.y : fmaf(h, mv.y - xv.y, xv.y)) : xv.y;
                zv.z = wv.z ? (unit ? mv.z : fmaf(h, mv.z - xv.z, xv.z)) : xv.z;
                zv.w = wv.w ? (unit ? mv.w : fmaf(h, mv.w - xv.w, xv.w)) : xv.w;
                reinterpret_cast<float4 *>(z)[q] = zv;
                if (COPY)
                    reinterpret_cast<float4 *>(xp)[q] = xv;
            }
            j0 = n4 << 2;
        }
        for (int64_t j = j0 + threadIdx.x; j < n; j += blockDim.x) {
            const float xv = x[j];
            z[j] = w[j] ? (unit ? mm[j] : fmaf(h, mm[j] - xv, xv)) : xv;
            if (COPY)
                xp[j] = xv;
        }
    }
}

// Block sum of v over 256 threads, added into *acc by thread 0.
__device__ __forceinline__ void block_add(double v, double *acc)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ double part[8];
    if ((threadIdx.x & 31) == 0)
        part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < 8; ++w)
            a += part[w];
        atomicAdd(acc, a);
    }
}

// ||X - Xprev||_F^2 in FP64, added into *acc; 256 threads, one CTA per row at a
// time, float4 loads where both rows are 16-byte aligned.
__global__ void __launch_bounds__(256) change_kernel(const float *X, int64_t ldx, const float *P,
                                                     int64_t ldp, int64_t m, int64_t n, double *acc)
{
    double d2 = 0.0;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        const float *x = X + i * ldx;
        const float *p = P + i * ldp;
        int64_t j0 = 0;
        if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(p)) & 15u) == 0) {
            const int64_t n4 = n >> 2;
            for (int64_t q = threadIdx.x; q < n4; q += blockDim.x) {
                const float4 xv = reinterpret_cast<const float4 *>(x)[q];
                const float4 pv = reinterpret_cast<const float4 *>(p)[q];
                const double e0 = (double)xv.x - pv.x, e1 = (double)xv.y - pv.y;
                const double e2 = (double)xv.z - pv.z, e3 = (double)xv.w - pv.w;
                d2 += e0 * e0 + e1 * e1 + e2 * e2 + e3 * e3;
            }
            j0 = n4 << 2;
        }
        for (int64_t j = j0 + threadIdx.x; j < n; j += blockDim.x) {
            const double e = (double)x[j] - p[j];
            d2 += e * e;
        }
    }
    block_add(d2, acc);
}

// ||P_Omega(M)||_F^2 in FP64, added into *acc (the scale of the relative change).
__global__ void __launch_bounds__(256) data_norm_kernel(const float *M, int64_t ldm,
                                                        const uint8_t *W, int64_t ldw, int64_t m,
                                                        int64_t n, double *acc)
{
    double s2 = 0.0;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x)
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
            if (W[i * ldw + j]) {
                const double v = M[i * ldm + j];
                s2 += v * v;
            }
    block_add(s2, acc);
}

__global__ void loop_init_kernel(svt_completion_stats *st)
{
    st->steps = 0;
    st->stages = 0;
    st->stage_steps = 0;
    st->status = SVT_OK;
    st->solve_status = SVT_OK;
    st->reserved = 0;
    st->lambda = 0.0;
    st->rel_change = 0.0;
    st->diff2 = 0.0;
    st->data2 = 0.0;
}

// Before a stage's WHILE node: run its body at least once unless the run is over.
__global__ void stage_enter_kernel(svt_completion_stats *st, cudaGraphConditionalHandle h,
                                   int max_steps, double lambda)
{
    const bool go = st->status == SVT_OK && st->steps < max_steps;
    if (go) {
        st->stages += 1;
        st->stage_steps = 0;
        st->lambda = lambda;
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

// End of a body: count the step, turn the reduction into the relative change, take
// the solve's status, and decide whether the body runs again.
__global__ void step_decide_kernel(svt_completion_stats *st, cudaGraphConditionalHandle h,
                                   int max_steps, int stage_cap, double tol)
{
    st->steps += 1;
    st->stage_steps += 1;
    const double d2 = st->diff2, s2 = st->data2;
    st->diff2 = 0.0;
    const double rho = s2 > 0.0 ? sqrt(d2 / s2) : (d2 > 0.0 ? INFINITY : 0.0);
    st->rel_change = rho;
    if (st->status == SVT_OK && st->solve_status != SVT_OK)
        st->status = st->solve_status;
    if (st->status == SVT_OK && !isfinite(d2))
        st->status = SVT_ERR_DIVERGED;
    const bool go = st->status == SVT_OK && st->steps < max_steps &&
                    (stage_cap <= 0 || st->stage_steps < stage_cap) && !(rho <= tol);
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

} // namespace

extern "C" svt_status svt_prox_grad_step(svt_ctx_t ctx, float *X, int64_t ldx, const float *M,
                                         int64_t ldm, const uint8_t *mask, int64_t ldw, float *Z,
                                         int64_t ldz, int64_t m, int64_t n, float step,
                                         float lambda, const svt_options *opt,
                                         svt_status *d_status, void *stream)
{
    if (!ctx || !X || !M || !mask || !Z || m <= 0 || n <= 0 || ldx < n || ldm < n || ldw < n ||
        ldz < n)
        return SVT_ERR_INVALID;
    if (!std::isfinite(step) || !(step > 0.0f) || !std::isfinite(lambda) || lambda < 0.0f ||
        !std::isfinite(step * lambda))
        return SVT_ERR_INVALID;
    // Z is written before X is read back by the solve: it may alias none of the inputs.
    const size_t zb = (size_t)((m - 1) * ldz + n) * sizeof(float);
    if (svt::overlaps(Z, zb, X, (size_t)((m - 1) * ldx + n) * sizeof(float)) ||
        svt::overlaps(Z, zb, M, (size_t)((m - 1) * ldm + n) * sizeof(float)) ||
        svt::overlaps(Z, zb, mask, (size_t)((m - 1) * ldw + n)))
        return SVT_ERR_INVALID;
    // Everything the solve checks (sizes, options, workspace) before any launch.
    svt::Resolved r;
    svt_status st = svt::resolve_status(opt, &r);
    if (st != SVT_OK)
        return st;
    st = svt::validate(Z, m, n, ldz, step * lambda, X, ldx);
    if (st != SVT_OK)
        return st;
    if (r.prec == SVT_FP64 && (m > svt::kF64MaxDim || n > svt::kF64MaxDim))
        return SVT_ERR_UNSUPPORTED;
    size_t need = 0;
    if (svt_workspace_bytes_ex(m, n, opt, &need) != SVT_OK)
        return SVT_ERR_INVALID;
    if (need > ctx->ws_bytes)
        return SVT_ERR_OOM;
    if (svt::serve_busy(ctx))
        return SVT_ERR_BUSY;
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t want = (int64_t)ctx->num_sms * 8;
    const int grid = (int)(m < want ? m : want);
    prox_grad_kernel<false><<<grid, 256, 0, s>>>(X, ldx, M, ldm, mask, ldw, Z, ldz, m, n, step,
                                                  nullptr, 0);
    if (cudaGetLastError() != cudaSuccess)
        return SVT_ERR_CUDA;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->launches += 1;
    }
    return svt_polar_ex(ctx, Z, m, n, ldz, step * lambda, opt, X, ldx, d_status, stream);
}

namespace svt {

// Everything a recorded loop depends on; compared bytewise.
struct CompletionKey {
    const void *X, *M, *mask, *Z, *Xprev, *stats, *plan;
    int64_t ldx, ldm, ldw, ldz, ldp, m, n;
    svt_completion_params p;
};

struct CompletionGraph {
    CompletionKey key;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;  // recorded after the latest launch
    std::shared_ptr<Plan> plan;  // keeps the plan's host table alive
};

namespace {

constexpr size_t kMaxCompletionGraphs = 4;
constexpr int kMaxStages = 64;

void destroy_graph(CompletionGraph *g)
{
    if (g->exec)
        cudaGraphExecDestroy(g->exec);
    if (g->done)
        cudaEventDestroy(g->done);
    delete g;
}

struct LoopArgs {
    float *X;
    int64_t ldx;
    const float *M;
    int64_t ldm;
    const uint8_t *mask;
    int64_t ldw;
    float *Z;
    int64_t ldz;
    float *Xprev;
    int64_t ldp;
    int64_t m, n;
    svt_completion_params p;
    svt_completion_stats *stats;
};

// Record the loop: init, then per stage an enter kernel and a WHILE node whose body
// is captured from the step's launches on the context's private stream.
svt_status record_loop(svt_ctx *ctx, Plan &P, const LoopArgs &a, const std::vector<double> &lams,
                       cudaGraphExec_t *exec_out)
{
    if (!ctx->capture_stream &&
        cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
        return SVT_ERR_CUDA;
    cudaStream_t cs = ctx->capture_stream;
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess)
        return SVT_ERR_CUDA;
    svt_status st = SVT_OK;
    cudaGraphNode_t prev = nullptr;
    auto add_kernel = [&](void *fn, void **args, int grid_x = 1, int block_x = 1) -> bool {
        cudaKernelNodeParams kp;
        std::memset(&kp, 0, sizeof(kp));
        kp.func = fn;
        kp.gridDim = dim3(grid_x);
        kp.blockDim = dim3(block_x);
        kp.kernelParams = args;
        cudaGraphNode_t node = nullptr;
        if (cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp) !=
            cudaSuccess)
            return false;
        prev = node;
        return true;
    };
    svt_completion_stats *stats = a.stats;
    int max_steps = a.p.max_steps;
    const int64_t want = (int64_t)ctx->num_sms * 8;
    const int grid = (int)(a.m < want ? a.m : want);
    const int cgrid = (int)(a.m < (int64_t)ctx->num_sms * 4 ? a.m : (int64_t)ctx->num_sms * 4);
    const float *Mp = a.M;
    const uint8_t *Wp = a.mask;
    int64_t ldm = a.ldm, ldw = a.ldw, mm = a.m, nn = a.n;
    double *data2 = &stats->data2;
    void *init_args[] = {&stats};
    void *norm_args[] = {&Mp, &ldm, &Wp, &ldw, &mm, &nn, &data2};
    if (!add_kernel(reinterpret_cast<void *>(loop_init_kernel), init_args) ||
        !add_kernel(reinterpret_cast<void *>(data_norm_kernel), norm_args, cgrid, 256))
        st = SVT_ERR_CUDA;
    for (size_t k = 0; k < lams.size() && st == SVT_OK; ++k) {
        cudaGraphConditionalHandle h = 0;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 0, 0);
        if (e != cudaSuccess) {
            st = (e == cudaErrorNotSupported) ? SVT_ERR_UNSUPPORTED : SVT_ERR_CUDA;
            break;
        }
        double lam = lams[k];
        void *enter_args[] = {&stats, &h, &max_steps, &lam};
        if (!add_kernel(reinterpret_cast<void *>(stage_enter_kernel), enter_args)) {
            st = SVT_ERR_CUDA;
            break;
        }
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t cn = nullptr;
        e = cudaGraphAddNode(&cn, g, &prev, nullptr, 1, &np);
        if (e != cudaSuccess) {
            st = (e == cudaErrorNotSupported) ? SVT_ERR_UNSUPPORTED : SVT_ERR_CUDA;
            break;
        }
        prev = cn;
        cudaGraph_t body = np.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = SVT_ERR_CUDA;
            break;
        }
        const float tau = (float)((double)a.p.step * lam);
        const bool last = (k + 1 == lams.size());
        const int cap = last ? 0 : a.p.stage_steps;
        prox_grad_kernel<true><<<grid, 256, 0, cs>>>(a.X, a.ldx, a.M, a.ldm, a.mask, a.ldw, a.Z,
                                                     a.ldz, a.m, a.n, a.p.step, a.Xprev, a.ldp);
        bool ok = cudaGetLastError() == cudaSuccess;
        if (ok) {
            CallArgs ca{a.Z, a.ldz, tau, a.X, a.ldx,
                        reinterpret_cast<svt_status *>(&stats->solve_status), true};
            ok = run_plan(ctx, P, ca, cs) == SVT_OK;
        }
        if (ok) {
            change_kernel<<<cgrid, 256, 0, cs>>>(a.X, a.ldx, a.Xprev, a.ldp, a.m, a.n,
                                                 &stats->diff2);
            step_decide_kernel<<<1, 1, 0, cs>>>(stats, h, max_steps, cap, (double)a.p.tol);
            ok = cudaGetLastError() == cudaSuccess;
        }
        cudaGraph_t captured = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cs, &captured);
        if (!ok || ee != cudaSuccess)
            st = SVT_ERR_CUDA;
    }
    if (st == SVT_OK && cudaGraphInstantiate(exec_out, g, 0) != cudaSuccess)
        st = SVT_ERR_CUDA;
    cudaGraphDestroy(g);
    cudaGetLastError();  // a failed capture leaves its error sticky for this thread only
    return st;
}

} // namespace

void completion_release(svt_ctx *ctx)
{
    for (CompletionGraph *g : ctx->completion_graphs)
        destroy_graph(g);
    ctx->completion_graphs.clear();
    if (ctx->capture_stream) {
        cudaStreamDestroy(ctx->capture_stream);
        ctx->capture_stream = nullptr;
    }
}

} // namespace svt

extern "C" svt_status svt_complete(svt_ctx_t ctx, float *X, int64_t ldx, const float *M,
                                   int64_t ldm, const uint8_t *mask, int64_t ldw, float *Z,
                                   int64_t ldz, float *Xprev, int64_t ldp, int64_t m, int64_t n,
                                   const svt_completion_params *p, const svt_options *opt,
                                   svt_completion_stats *d_stats, void *stream)
{
    using namespace svt;
    if (!ctx || !X || !M || !mask || !Z || !Xprev || !p || !d_stats || m <= 0 || n <= 0 ||
        ldx < n || ldm < n || ldw < n || ldz < n || ldp < n ||
        (reinterpret_cast<uintptr_t>(d_stats) & 7u) != 0)
        return SVT_ERR_INVALID;
    const svt_completion_params q = *p;
    auto fin = [](float v) { return std::isfinite(v); };
    if (!fin(q.lambda) || q.lambda < 0.0f || !fin(q.lambda0) || q.lambda0 < q.lambda ||
        !fin(q.step) || !(q.step > 0.0f) || !fin(q.step * q.lambda0) || !fin(q.tol) ||
        q.tol < 0.0f || q.max_steps < 0 || q.stage_steps < 0)
        return SVT_ERR_INVALID;
    if (q.lambda0 > q.lambda && !(fin(q.eta) && q.eta > 0.0f && q.eta < 1.0f))
        return SVT_ERR_INVALID;
    // Stage lambdas: lambda0 eta^k while above lambda, then lambda.
    std::vector<double> lams;
    if (q.lambda0 > q.lambda) {
        double l = q.lambda0;
        while (l > (double)q.lambda && (int)lams.size() < kMaxStages) {
            lams.push_back(l);
            l *= (double)q.eta;
        }
    }
    if ((int)lams.size() >= kMaxStages)
        return SVT_ERR_INVALID;
    lams.push_back(q.lambda);
    // Buffers written by the run (Z, Xprev, the statistics) alias nothing else.
    const size_t xb = (size_t)((m - 1) * ldx + n) * sizeof(float);
    const size_t mb = (size_t)((m - 1) * ldm + n) * sizeof(float);
    const size_t wb = (size_t)((m - 1) * ldw + n);
    const size_t zb = (size_t)((m - 1) * ldz + n) * sizeof(float);
    const size_t pb = (size_t)((m - 1) * ldp + n) * sizeof(float);
    const size_t sb = sizeof(svt_completion_stats);
    struct Span {
        const void *p;
        size_t b;
    } spans[6] = {{X, xb}, {M, mb}, {mask, wb}, {Z, zb}, {Xprev, pb}, {d_stats, sb}};
    for (int i = 0; i < 6; ++i)
        for (int j = std::max(i + 1, 3); j < 6; ++j)
            if (overlaps(spans[i].p, spans[i].b, spans[j].p, spans[j].b))
                return SVT_ERR_INVALID;
    Resolved r;
    svt_status st = resolve_status(opt, &r);
    if (st != SVT_OK)
        return st;
    st = validate(Z, m, n, ldz, q.step * q.lambda0, X, ldx);
    if (st != SVT_OK)
        return st;
    if (r.prec == SVT_FP64 && (m > kF64MaxDim || n > kF64MaxDim))
        return SVT_ERR_UNSUPPORTED;
    size_t need = 0;
    if (svt_workspace_bytes_ex(m, n, opt, &need) != SVT_OK)
        return SVT_ERR_INVALID;
    if (need > ctx->ws_bytes)
        return SVT_ERR_OOM;
    if (serve_busy(ctx))
        return SVT_ERR_BUSY;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    Plan *plan = nullptr;
    std::shared_ptr<Plan> keep;
    st = plan_for_solve(ctx, m, n, r, &plan, &keep);
    if (st != SVT_OK)
        return st;
    CompletionKey key;
    std::memset(&key, 0, sizeof(key));
    key.X = X;
    key.M = M;
    key.mask = mask;
    key.Z = Z;
    key.Xprev = Xprev;
    key.stats = d_stats;
    key.plan = plan;
    key.ldx = ldx;
    key.ldm = ldm;
    key.ldw = ldw;
    key.ldz = ldz;
    key.ldp = ldp;
    key.m = m;
    key.n = n;
    key.p = q;
    auto &cache = ctx->completion_graphs;
    CompletionGraph *cg = nullptr;
    for (size_t i = 0; i < cache.size(); ++i)
        if (std::memcmp(&cache[i]->key, &key, sizeof(key)) == 0) {
            cg = cache[i];
            cache.erase(cache.begin() + (long)i);
            break;
        }
    if (!cg) {
        LoopArgs la{X, ldx, M, ldm, mask, ldw, Z, ldz, Xprev, ldp, m, n, q, d_stats};
        cudaGraphExec_t exec = nullptr;
        st = record_loop(ctx, *plan, la, lams, &exec);
        if (st != SVT_OK)
            return st;
        cg = new CompletionGraph();
        cg->key = key;
        cg->exec = exec;
        cg->plan = keep;
        if (cudaEventCreateWithFlags(&cg->done, cudaEventDisableTiming) != cudaSuccess) {
            destroy_graph(cg);
            return SVT_ERR_CUDA;
        }
        while (cache.size() >= kMaxCompletionGraphs) {
            cudaEventSynchronize(cache.front()->done);
            destroy_graph(cache.front());
            cache.erase(cache.begin());
        }
    }
    cache.push_back(cg);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (upload_fused_table(ctx, *plan, s) != SVT_OK || cudaGraphLaunch(cg->exec, s) != cudaSuccess ||
        cudaEventRecord(cg->done, s) != cudaSuccess)
        return SVT_ERR_CUDA;
    ctx->launches += 1;
    return SVT_OK;
}
