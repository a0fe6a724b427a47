// Iteration-schedule autotuning: the fewest polynomial steps (and the first design
// interval's lower end ell0) whose solve stays within a target deviation of a
// reference solve of the same input. The paper leaves the count open (Section 4's
// maxIts; more steps reach smaller singular values, Section 3's Fig. 1), so the
// count is measured per input class and tier rather than fixed.
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "plan.h"

namespace {

// acc[0] += ||Y - R||_F^2, acc[1] += ||R||_F^2, acc[2] += ||A||_F^2 (A may be null):
// FP64 sums, 256 threads, one CTA per row at a time.
__global__ void __launch_bounds__(256) deviation_kernel(const float *Y, int64_t ldy,
                                                        const float *R, int64_t ldr,
                                                        const float *A, int64_t lda, int64_t m,
                                                        int64_t n, double *acc)
{
    double d2 = 0.0, r2 = 0.0, a2 = 0.0;
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x)
        for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
            const double y = Y[i * ldy + j], r = R[i * ldr + j];
            d2 += (y - r) * (y - r);
            r2 += r * r;
            if (A) {
                const double a = A[i * lda + j];
                a2 += a * a;
            }
        }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
        r2 += __shfl_down_sync(0xffffffffu, r2, o);
        a2 += __shfl_down_sync(0xffffffffu, a2, o);
    }
    __shared__ double part[3][8];
    if ((threadIdx.x & 31) == 0) {
        part[0][threadIdx.x >> 5] = d2;
        part[1][threadIdx.x >> 5] = r2;
        part[2][threadIdx.x >> 5] = a2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w)
            t += part[threadIdx.x][w];
        atomicAdd(acc + threadIdx.x, t);
    }
}

} // namespace

extern "C" svt_status svt_autotune_schedule(svt_ctx_t ctx, const float *A, int64_t m, int64_t n,
                                            int64_t lda, float tau, const svt_options *opt,
                                            double target, int max_iters, float *Y, int64_t ldy,
                                            float *Yref, int64_t ldr, int *iters_out,
                                            double *ell0_out, double *dev_out, void *stream)
{
    using namespace svt;
    if (!ctx || !Y || !Yref || !iters_out || !ell0_out || !dev_out || !std::isfinite(target) ||
        !(target > 0.0) || max_iters < 2 || max_iters > 32 || ldr < n)
        return SVT_ERR_INVALID;
    svt_status st = validate(A, m, n, lda, tau, Y, ldy);
    if (st != SVT_OK)
        return st;
    if ((st = validate(A, m, n, lda, tau, Yref, ldr)) != SVT_OK)
        return st;
    if (overlaps(Y, (size_t)((m - 1) * ldy + n) * sizeof(float), Yref,
                 (size_t)((m - 1) * ldr + n) * sizeof(float)))
        return SVT_ERR_INVALID;
    svt_options base;
    svt_options_default(&base);
    if (opt)
        base = *opt;
    Resolved r;
    if ((st = resolve_status(&base, &r)) != SVT_OK)
        return st;
    if (r.prec == SVT_FP64)
        return SVT_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    svt_options ref = base;
    ref.prec = SVT_FP32;
    ref.iters = 32;
    ref.ell0 = 1e-3;
    ref.schedule = SVT_SCHED_PE5;
    ref.hp_steps = -1;
    if ((st = svt_polar_ex(ctx, A, m, n, lda, tau, &ref, Yref, ldr, nullptr, stream)) != SVT_OK)
        return st;
    double *acc = nullptr;
    if (cudaMalloc(&acc, 3 * sizeof(double)) != cudaSuccess)
        return SVT_ERR_OOM;
    const int grid = (int)std::min<int64_t>(m, (int64_t)ctx->num_sms * 4);
    double a2 = -1.0;  // ||A||_F^2, taken with the first candidate
    auto deviation = [&](double *dev) -> svt_status {
        if (cudaMemsetAsync(acc, 0, 3 * sizeof(double), s) != cudaSuccess)
            return SVT_ERR_CUDA;
        deviation_kernel<<<grid, 256, 0, s>>>(Y, ldy, Yref, ldr, a2 < 0.0 ? A : nullptr, lda, m,
                                              n, acc);
        double h[3];
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return SVT_ERR_CUDA;
        if (a2 < 0.0)
            a2 = h[2];
        const double den = h[1] > 0.0 ? h[1] : a2;
        *dev = den > 0.0 ? std::sqrt(h[0] / den) : (h[0] > 0.0 ? INFINITY : 0.0);
        return SVT_OK;
    };
    static const int kSteps[] = {2, 3, 4, 5, 6, 8, 10, 12, 14, 16, 20, 24, 28, 32};
    static const double kEll0[] = {1e-3, 1e-2};
    int best_k = -1;
    double best_l = 1e-3, best_dev = INFINITY;
    for (double l0 : kEll0) {
        for (int k : kSteps) {
            if (k > max_iters || (best_k > 0 && k >= best_k))
                break;
            svt_options o = base;
            o.iters = k;
            o.ell0 = l0;
            o.schedule = SVT_SCHED_PE5;
            double dev = 0.0;
            if ((st = svt_polar_ex(ctx, A, m, n, lda, tau, &o, Y, ldy, nullptr, stream)) != SVT_OK ||
                (st = deviation(&dev)) != SVT_OK) {
                cudaFree(acc);
                return st;
            }
            if (dev <= target) {
                best_k = k;
                best_l = l0;
                best_dev = dev;
                break;
            }
        }
    }
    if (best_k < 0) {  // nothing reached the target: the most steps allowed
        svt_options o = base;
        o.iters = max_iters;
        o.ell0 = 1e-3;
        o.schedule = SVT_SCHED_PE5;
        if ((st = svt_polar_ex(ctx, A, m, n, lda, tau, &o, Y, ldy, nullptr, stream)) != SVT_OK ||
            (st = deviation(&best_dev)) != SVT_OK) {
            cudaFree(acc);
            return st;
        }
        best_k = max_iters;
        best_l = 1e-3;
    }
    cudaFree(acc);
    *iters_out = best_k;
    *ell0_out = best_l;
    *dev_out = best_dev;
    return SVT_OK;
}
