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
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "plan.h"

namespace {

// Z = X + h P_Omega(M - X), one CTA per row at a time; float4 accesses where the
// row's addresses allow them (checked on the real addresses), scalar otherwise.
__global__ void __launch_bounds__(256) prox_grad_kernel(const float *X, int64_t ldx, const float *M,
                                                        int64_t ldm, const uint8_t *W, int64_t ldw,
                                                        float *Z, int64_t ldz, int64_t m, int64_t n,
                                                        float h)
{
    const bool unit = (h == 1.0f);  // observed entries become M exactly
    for (int64_t i = blockIdx.x; i < m; i += gridDim.x) {
        const float *x = X + i * ldx;
        const float *mm = M + i * ldm;
        const uint8_t *w = W + i * ldw;
        float *z = Z + i * ldz;
        const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(mm) |
                           reinterpret_cast<uintptr_t>(z)) & 15u) == 0 &&
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
            }
            j0 = n4 << 2;
        }
        for (int64_t j = j0 + threadIdx.x; j < n; j += blockDim.x) {
            const float xv = x[j];
            z[j] = w[j] ? (unit ? mm[j] : fmaf(h, mm[j] - xv, xv)) : xv;
        }
    }
}

bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes)
{
    const char *a0 = static_cast<const char *>(a), *b0 = static_cast<const char *>(b);
    return a0 < b0 + bbytes && b0 < a0 + abytes;
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
    if (overlaps(Z, zb, X, (size_t)((m - 1) * ldx + n) * sizeof(float)) ||
        overlaps(Z, zb, M, (size_t)((m - 1) * ldm + n) * sizeof(float)) ||
        overlaps(Z, zb, mask, (size_t)((m - 1) * ldw + n)))
        return SVT_ERR_INVALID;
    // Everything the solve checks (sizes, options, workspace) before any launch.
    svt::Resolved r;
    if (!svt::resolve(opt, &r))
        return SVT_ERR_INVALID;
    svt_status st = svt::validate(Z, m, n, ldz, step * lambda, X, ldx);
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
    prox_grad_kernel<<<grid, 256, 0, s>>>(X, ldx, M, ldm, mask, ldw, Z, ldz, m, n, step);
    if (cudaGetLastError() != cudaSuccess)
        return SVT_ERR_CUDA;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->launches += 1;
    }
    return svt_polar_ex(ctx, Z, m, n, ldz, step * lambda, opt, X, ldx, d_status, stream);
}
