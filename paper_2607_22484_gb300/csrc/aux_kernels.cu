// Memory-bound kernels around the tensor-core products, and the FP64 SIMT tier.
//
//  * ingest_reduce: FP64 norms of the input (||A||_F^2 and the Gram diagonal,
//    i.e. the squared column norms of the tall matrix) and the finiteness check.
//  * ingest_split: X0 = A / alpha with alpha an exact power of two near ||A||_F,
//    written in the same orientation and transposed, as BF16 hi (+ lo) parts or
//    FP64, through a shared-memory transpose so both writes are coalesced.
//  * f64_gemm: D = L R^T in FP64 with the same fused epilogue as the tensor-core
//    kernel; the correctness tier for small inputs.
//  * finalize: output-norm divergence check and status hand-off.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "svt_internal.h"

namespace svt {

namespace {

__device__ __forceinline__ void set_status(int *status, svt_status s)
{
    if (status)
        atomicCAS(status, 0, (int)s);
}

// alpha = 2^e with e = round(log2 ||A||_F) (1 for a zero matrix): dividing by it is exact.
__device__ __forceinline__ double pow2_alpha(double nrm2)
{
    if (!(nrm2 > 0.0) || !isfinite(nrm2))
        return 1.0;
    int e;
    double f = frexp(sqrt(nrm2), &e);  // sqrt = f 2^e, f in [0.5, 1)
    if (f < 0.70710678118654752)
        e -= 1;
    return ldexp(1.0, e);
}

// ---- ingest: column (or row) norms and the split into scaled copies
//
// The same block functions serve the single-matrix kernels and the grouped
// kernels of batches, so that a matrix is ingested identically either way. Rows
// are read with 16-byte loads where A and lda allow (vec), with the same thread
// mapping and summation order otherwise. Squares are summed in FP32 over four
// values and in FP64 beyond; the FP64 tier (F64SUM) sums every square in FP64.

constexpr int kColRows4 = 128;  // rows per block of the column norms

// Column norms (tall input): 256 threads; block (bx, by) covers 128 columns (32
// lanes x 4) and kColRows4 rows, warp w taking rows r0 + w, r0 + w + 8, ...
template <bool F64SUM>
__device__ __forceinline__ void colnorm4_block(const float *__restrict__ A, int64_t m, int64_t n,
                                               int64_t lda, double *colnorm2, double *scal,
                                               int *status, int bx, int by, bool vec)
{
    __shared__ double part[8][129];
    __shared__ double wsum[4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t c0 = (int64_t)bx * 128 + lane * 4;
    const int64_t r0 = (int64_t)by * kColRows4;
    const int64_t r1 = (m < r0 + kColRows4) ? m : r0 + kColRows4;
    const bool full = vec && c0 + 3 < n;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    bool finite = true;
    if (c0 < n) {
        for (int64_t r = r0 + w; r < r1; r += 32) {
            float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t rr = r + 8 * u;
                if (rr < r1) {
                    const float *a = A + rr * lda + c0;
                    float4 v;
                    if (full) {
                        v = *reinterpret_cast<const float4 *>(a);
                    } else {
                        v.x = a[0];
                        v.y = c0 + 1 < n ? a[1] : 0.f;
                        v.z = c0 + 2 < n ? a[2] : 0.f;
                        v.w = c0 + 3 < n ? a[3] : 0.f;
                    }
                    finite &= isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
                    if (F64SUM) {
                        s0 += (double)v.x * v.x;
                        s1 += (double)v.y * v.y;
                        s2 += (double)v.z * v.z;
                        s3 += (double)v.w * v.w;
                    } else {
                        p0 = fmaf(v.x, v.x, p0);
                        p1 = fmaf(v.y, v.y, p1);
                        p2 = fmaf(v.z, v.z, p2);
                        p3 = fmaf(v.w, v.w, p3);
                    }
                }
            }
            if (!F64SUM) {
                s0 += p0;
                s1 += p1;
                s2 += p2;
                s3 += p3;
            }
        }
    }
    if (!finite)
        set_status(status, SVT_ERR_NONFINITE);
    part[w][lane * 4 + 0] = s0;
    part[w][lane * 4 + 1] = s1;
    part[w][lane * 4 + 2] = s2;
    part[w][lane * 4 + 3] = s3;
    __syncthreads();
    if (threadIdx.x < 128) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i)
            t += part[i][threadIdx.x];
        const int64_t col = (int64_t)bx * 128 + threadIdx.x;
        if (col < n && t != 0.0)
            atomicAdd(&colnorm2[col], t);
        for (int o = 16; o > 0; o >>= 1)
            t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0)
            wsum[w] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double b = wsum[0] + wsum[1] + wsum[2] + wsum[3];
        if (b != 0.0)
            atomicAdd(&scal[SC_NRM_A2], b);
    }
}

// Row norms (wide input): one warp per row, rows 8 bx .. 8 bx + 7 (256 threads).
template <bool F64SUM>
__device__ __forceinline__ void rownorm4_block(const float *__restrict__ A, int64_t m, int64_t n,
                                               int64_t lda, double *colnorm2, double *scal,
                                               int *status, int bx, bool vec)
{
    __shared__ double wsum[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t row = (int64_t)bx * 8 + w;
    double s = 0.0;
    if (row < m) {
        const float *a = A + row * lda;
        bool finite = true;
        const int64_t n4 = n >> 2;
        for (int64_t q = lane; q < n4; q += 32) {
            float4 v;
            if (vec) {
                v = reinterpret_cast<const float4 *>(a)[q];
            } else {
                v.x = a[4 * q];
                v.y = a[4 * q + 1];
                v.z = a[4 * q + 2];
                v.w = a[4 * q + 3];
            }
            finite &= isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w);
            if (F64SUM)
                s += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
            else
                s += (double)fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, v.w * v.w)));
        }
        for (int64_t c = (n4 << 2) + lane; c < n; c += 32) {
            const float v = a[c];
            finite &= isfinite(v);
            s += (double)v * (double)v;
        }
        if (!finite)
            set_status(status, SVT_ERR_NONFINITE);
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0)
            colnorm2[row] = s;
    }
    if (lane == 0)
        wsum[w] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < 8; ++i)
            b += wsum[i];
        if (b != 0.0)
            atomicAdd(&scal[SC_NRM_A2], b);
    }
}

// Four consecutive values of row `row` from column `col` as BF16 (hi, and lo = the
// rounding remainder when lo is non-null); one 8-byte store each where the four
// elements are in range and 8-byte aligned.
__device__ __forceinline__ void store4_bf16(void *hi, void *lo, int64_t row, int64_t col,
                                            int64_t ld, int64_t ncols, bool aligned,
                                            const float (&v)[4])
{
    __nv_bfloat16 h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        h[e] = __float2bfloat16_rn(v[e]);
        l[e] = __float2bfloat16_rn(v[e] - __bfloat162float(h[e]));
    }
    const int64_t off = row * ld + col;
    __nv_bfloat16 *ph = static_cast<__nv_bfloat16 *>(hi) + off;
    __nv_bfloat16 *pl = lo ? static_cast<__nv_bfloat16 *>(lo) + off : nullptr;
    if (aligned && col + 3 < ncols) {
        uint2 uh, ul;
        uh.x = (uint32_t)__bfloat16_as_ushort(h[0]) | ((uint32_t)__bfloat16_as_ushort(h[1]) << 16);
        uh.y = (uint32_t)__bfloat16_as_ushort(h[2]) | ((uint32_t)__bfloat16_as_ushort(h[3]) << 16);
        *reinterpret_cast<uint2 *>(ph) = uh;
        if (pl) {
            ul.x = (uint32_t)__bfloat16_as_ushort(l[0]) | ((uint32_t)__bfloat16_as_ushort(l[1]) << 16);
            ul.y = (uint32_t)__bfloat16_as_ushort(l[2]) | ((uint32_t)__bfloat16_as_ushort(l[3]) << 16);
            *reinterpret_cast<uint2 *>(pl) = ul;
        }
        return;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (col + e < ncols) {
            ph[e] = h[e];
            if (pl)
                pl[e] = l[e];
        }
}

__device__ __forceinline__ void store4_f64(void *out, int64_t row, int64_t col, int64_t ld,
                                           int64_t ncols, const float (&v)[4])
{
    double *p = static_cast<double *>(out) + row * ld + col;
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (col + e < ncols)
            p[e] = (double)v[e];
}

// 64 x 64 tile (bx, by) of A -> same-orientation and transposed copies of A / alpha
// (BF16 hi and optional lo parts, or FP64). 256 threads: thread t loads rows
// (t >> 4) + 16 k, columns 4 (t & 15) .. + 3, and stores the transposed tile the same
// way from shared memory. vec_in: A's rows 16-byte aligned; st_al: BF16 outputs
// 8-byte aligned at columns that are multiples of 4.
template <bool F64>
__device__ __forceinline__ void split64_block(const float *__restrict__ A, int64_t m, int64_t n,
                                              int64_t lda, float tau, void *xs_hi, void *xs_lo,
                                              int64_t ld_s, void *xt_hi, void *xt_lo, int64_t ld_t,
                                              double *scal, int bx, int by, bool vec_in, bool st_al)
{
    __shared__ float tile[64][65];
    const double nrm2 = scal[SC_NRM_A2];
    const double alpha = pow2_alpha(nrm2);
    const float inv_alpha = (float)(1.0 / alpha);  // exact power of two
    if (bx == 0 && by == 0 && threadIdx.x == 0) {
        scal[SC_ALPHA] = alpha;
        scal[SC_INV_ALPHA2] = 1.0 / (alpha * alpha);
        scal[SC_TAU2_SCALED] = ((double)tau * (double)tau) / (alpha * alpha);
        scal[SC_NRM_X0] = nrm2 / (alpha * alpha);
    }
    const int t = threadIdx.x, cq = t & 15, rr = t >> 4;
    const int64_t i0 = (int64_t)by * 64, j0 = (int64_t)bx * 64;
    const bool full_in = vec_in && i0 + 64 <= m && j0 + 64 <= n;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int li = rr + 16 * k;
        const int64_t i = i0 + li, j = j0 + 4 * cq;
        float v[4];
        if (full_in) {
            const float4 q = *reinterpret_cast<const float4 *>(A + i * lda + j);
            v[0] = q.x;
            v[1] = q.y;
            v[2] = q.z;
            v[3] = q.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                v[e] = (i < m && j + e < n) ? A[i * lda + j + e] : 0.0f;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            v[e] *= inv_alpha;
            tile[li][4 * cq + e] = v[e];
        }
        if (xs_hi && i < m && j < n) {
            if (F64)
                store4_f64(xs_hi, i, j, ld_s, n, v);
            else
                store4_bf16(xs_hi, xs_lo, i, j, ld_s, n, st_al, v);
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int lj = rr + 16 * k;
        const int64_t j = j0 + lj, i = i0 + 4 * cq;  // output row j, columns i .. i + 3
        float v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            v[e] = tile[4 * cq + e][lj];
        if (xt_hi && j < n && i < m) {
            if (F64)
                store4_f64(xt_hi, j, i, ld_t, m, v);
            else
                store4_bf16(xt_hi, xt_lo, j, i, ld_t, m, st_al, v);
        }
    }
}

__device__ __forceinline__ bool rows_vec(const float *A, int64_t lda)
{
    return (reinterpret_cast<uintptr_t>(A) & 15u) == 0 && (lda & 3) == 0;
}

__device__ __forceinline__ bool bf16_outs_aligned(const void *a, const void *b, const void *c,
                                                  const void *d, int64_t ld_s, int64_t ld_t)
{
    const uintptr_t u = reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
                        reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(d);
    return (u & 7u) == 0 && (ld_s & 3) == 0 && (ld_t & 3) == 0;
}

template <bool F64SUM>
__global__ void __launch_bounds__(256) ingest_reduce_kernel(const float *__restrict__ A, int64_t m,
                                                            int64_t n, int64_t lda, int wide,
                                                            double *colnorm2, double *scal,
                                                            int *status)
{
    const bool vec = rows_vec(A, lda);
    if (!wide)
        colnorm4_block<F64SUM>(A, m, n, lda, colnorm2, scal, status, blockIdx.x, blockIdx.y, vec);
    else
        rownorm4_block<F64SUM>(A, m, n, lda, colnorm2, scal, status, blockIdx.x, vec);
}

template <bool F64>
__global__ void __launch_bounds__(256) ingest_split_kernel(const float *__restrict__ A, int64_t m,
                                                           int64_t n, int64_t lda, float tau,
                                                           void *xs_hi, void *xs_lo, int64_t ld_s,
                                                           void *xt_hi, void *xt_lo, int64_t ld_t,
                                                           double *scal)
{
    split64_block<F64>(A, m, n, lda, tau, xs_hi, xs_lo, ld_s, xt_hi, xt_lo, ld_t, scal, blockIdx.x,
                       blockIdx.y, rows_vec(A, lda),
                       bf16_outs_aligned(xs_hi, xs_lo, xt_hi, xt_lo, ld_s, ld_t));
}

__global__ void finalize_kernel(double *scal, int *status, svt_status *user)
{
    double nrm = scal[SC_NRM_OUT];
    if (!isfinite(nrm))
        atomicCAS(status, 0, (int)SVT_ERR_DIVERGED);
    if (user)
        *reinterpret_cast<int *>(user) = *status;
}

// ------------------------------------------------------------ grouped (batches)

__device__ __forceinline__ int find_rec(const AuxRec *recs, int count, int b, bool split)
{
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        int start = split ? recs[mid].blk_split : recs[mid].blk_reduce;
        if (start <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void grouped_zero_kernel(const AuxRec *recs)
{
    const AuxRec &r = recs[blockIdx.x];
    for (int64_t i = threadIdx.x; i < r.zero_words; i += blockDim.x)
        reinterpret_cast<unsigned long long *>(r.scal)[i] = 0ull;
}

__global__ void __launch_bounds__(256) grouped_reduce_kernel(const AuxRec *recs,
                                                             const CallRec *calls, int count)
{
    const int i = find_rec(recs, count, blockIdx.x, false);
    const AuxRec &r = recs[i];
    const CallRec &c = calls[i];
    const int lb = blockIdx.x - r.blk_reduce;
    const bool vec = rows_vec(c.A, c.lda);
    if (!r.wide) {
        const int gx = (int)((r.n + 127) / 128);
        if (r.f64)
            colnorm4_block<true>(c.A, r.m, r.n, c.lda, r.colnorm, r.scal, r.status, lb % gx,
                                 lb / gx, vec);
        else
            colnorm4_block<false>(c.A, r.m, r.n, c.lda, r.colnorm, r.scal, r.status, lb % gx,
                                  lb / gx, vec);
    } else {
        if (r.f64)
            rownorm4_block<true>(c.A, r.m, r.n, c.lda, r.colnorm, r.scal, r.status, lb, vec);
        else
            rownorm4_block<false>(c.A, r.m, r.n, c.lda, r.colnorm, r.scal, r.status, lb, vec);
    }
}

__global__ void __launch_bounds__(256) grouped_split_kernel(const AuxRec *recs,
                                                            const CallRec *calls, int count)
{
    const int i = find_rec(recs, count, blockIdx.x, true);
    const AuxRec &r = recs[i];
    const CallRec &c = calls[i];
    const int lb = blockIdx.x - r.blk_split;
    const int gx = (int)((r.n + 63) / 64);
    const bool vec = rows_vec(c.A, c.lda);
    if (r.f64)
        split64_block<true>(c.A, r.m, r.n, c.lda, c.tau, r.xs_hi, nullptr, r.ld_s, r.xt_hi, nullptr,
                            r.ld_t, r.scal, lb % gx, lb / gx, vec, false);
    else
        split64_block<false>(c.A, r.m, r.n, c.lda, c.tau, r.xs_hi, r.xs_lo, r.ld_s, r.xt_hi,
                             r.xt_lo, r.ld_t, r.scal, lb % gx, lb / gx, vec,
                             bf16_outs_aligned(r.xs_hi, r.xs_lo, r.xt_hi, r.xt_lo, r.ld_s, r.ld_t));
}

__global__ void grouped_finalize_kernel(const AuxRec *recs, const CallRec *calls, int count)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count)
        return;
    const AuxRec &r = recs[i];
    if (!isfinite(r.scal[SC_NRM_OUT]))
        atomicCAS(r.status, 0, (int)SVT_ERR_DIVERGED);
    if (calls[i].d_status)
        *reinterpret_cast<int *>(calls[i].d_status) = *r.status;
}

// ------------------------------------------------------------ FP64 tier

constexpr int kF64Tile = 64;
constexpr int kF64K = 16;

__device__ __forceinline__ double f64_load_c(const Epi &e, int64_t r, int64_t c)
{
    int64_t off = e.c_trans ? c * e.ldc + r : r * e.ldc + c;
    if (e.c_kind == C_F64)
        return static_cast<const double *>(e.c0)[off];
    if (e.c_kind == C_F32)
        return (double)static_cast<const float *>(e.c0)[off];
    return 0.0;
}

__device__ __forceinline__ void f64_store(int kind, void *p, int64_t off, double v)
{
    if (kind == O_F64)
        static_cast<double *>(p)[off] = v;
    else if (kind == O_F32)
        static_cast<float *>(p)[off] = (float)v;
}

// D = L R^T, 64 x 64 tile per block of 256 threads, 4 x 4 outputs per thread.
__global__ void __launch_bounds__(256) f64_gemm_kernel(const __grid_constant__ F64Launch l)
{
    const F64Problem &P = l.p[blockIdx.z];
    const int tm = blockIdx.y, tn = blockIdx.x;
    if ((int64_t)tm * kF64Tile >= P.M || (int64_t)tn * kF64Tile >= P.N)
        return;
    if (P.sym && tm > tn)
        return;
    __shared__ double sL[kF64K][kF64Tile + 1];
    __shared__ double sR[kF64K][kF64Tile + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < P.K; k0 += kF64K) {
        for (int idx = threadIdx.x; idx < kF64Tile * kF64K; idx += 256) {
            int rr = idx / kF64K, kk = idx % kF64K;
            int64_t gr = (int64_t)tm * kF64Tile + rr, gk = k0 + kk;
            sL[kk][rr] = (gr < P.M && gk < P.K) ? P.L[gr * P.ldl + gk] : 0.0;
            int64_t gc = (int64_t)tn * kF64Tile + rr;
            sR[kk][rr] = (gc < P.N && gk < P.K) ? P.R[gc * P.ldr + gk] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kF64K; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = sL[kk][ty + 16 * i];
                b[i] = sR[kk][tx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    const Epi &e = P.ep;
    double al = e.alpha, be = e.beta, ga = e.gamma;
    if (e.theta_src) {
        double theta = pow(*e.theta_src, e.theta_pow);
        if (theta > 0.0 && isfinite(theta)) {
            al *= pow(theta, -e.ea);
            be *= pow(theta, -e.eb);
            ga *= pow(theta, -e.eg);
        } else if (!isfinite(theta)) {
            set_status(e.status, SVT_ERR_DIVERGED);
        }  // theta == 0: the chain's matrix is zero; nothing to scale
    }
    double nrm = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t r = (int64_t)tm * kF64Tile + ty + 16 * i;
            int64_t c = (int64_t)tn * kF64Tile + tx + 16 * j;
            if (r >= P.M || c >= P.N || (P.sym && r > c))
                continue;
            double x = al * acc[i][j];
            if (e.c_kind != C_NONE)
                x += be * f64_load_c(e, r, c);
            if (r == c) {
                x += ga;
                if (e.diag)
                    x = e.diag[r] * e.dss[0] - e.dss[1];
            }
            if (e.norm_acc)
                nrm += (P.sym && r != c) ? 2.0 * x * x : x * x;
            f64_store(e.o_kind, e.o0, e.o_trans ? c * e.ldo + r : r * e.ldo + c, x);
            if (P.sym && r != c)
                f64_store(e.o_kind, e.o0, c * e.ldo + r, x);
            if (e.t_kind != O_NONE)
                f64_store(e.t_kind, e.t0, c * e.ldt + r, x);
        }
    if (e.norm_acc) {
        for (int o = 16; o > 0; o >>= 1)
            nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        if ((threadIdx.x & 31) == 0 && nrm != 0.0)
            atomicAdd(e.norm_acc, nrm);
    }
}

} // namespace

cudaError_t ingest_reduce_launch(const float *A, int64_t m, int64_t n, int64_t lda, int wide,
                                 int f64, double *colnorm2, double *scal, int *status,
                                 cudaStream_t s)
{
    dim3 grid = wide ? dim3((unsigned)((m + 7) / 8))
                     : dim3((unsigned)((n + 127) / 128), (unsigned)((m + kColRows4 - 1) / kColRows4));
    if (f64)
        ingest_reduce_kernel<true><<<grid, 256, 0, s>>>(A, m, n, lda, wide, colnorm2, scal, status);
    else
        ingest_reduce_kernel<false><<<grid, 256, 0, s>>>(A, m, n, lda, wide, colnorm2, scal, status);
    return cudaGetLastError();
}

cudaError_t ingest_split_launch(const float *A, int64_t m, int64_t n, int64_t lda, float tau,
                                int f64, void *xs_hi, void *xs_lo, int64_t ld_s, void *xt_hi,
                                void *xt_lo, int64_t ld_t, double *scal, int *status,
                                cudaStream_t s)
{
    (void)status;
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((m + 63) / 64));
    if (f64)
        ingest_split_kernel<true><<<grid, 256, 0, s>>>(A, m, n, lda, tau, xs_hi, nullptr, ld_s,
                                                       xt_hi, nullptr, ld_t, scal);
    else
        ingest_split_kernel<false><<<grid, 256, 0, s>>>(A, m, n, lda, tau, xs_hi, xs_lo, ld_s,
                                                        xt_hi, xt_lo, ld_t, scal);
    return cudaGetLastError();
}

int grouped_reduce_blocks(int64_t m, int64_t n, int wide)
{
    if (!wide)
        return (int)(((n + 127) / 128) * ((m + kColRows4 - 1) / kColRows4));
    return (int)((m + 7) / 8);
}

int grouped_split_blocks(int64_t m, int64_t n) { return (int)(((n + 63) / 64) * ((m + 63) / 64)); }

cudaError_t grouped_zero_launch(const AuxRec *recs, int count, cudaStream_t s)
{
    if (count <= 0)
        return cudaSuccess;
    grouped_zero_kernel<<<count, 256, 0, s>>>(recs);
    return cudaGetLastError();
}

cudaError_t grouped_reduce_launch(const AuxRec *recs, const CallRec *calls, int count,
                                  int blocks_reduce, cudaStream_t s)
{
    if (count <= 0 || blocks_reduce <= 0)
        return cudaSuccess;
    grouped_reduce_kernel<<<blocks_reduce, 256, 0, s>>>(recs, calls, count);
    return cudaGetLastError();
}

cudaError_t grouped_split_launch(const AuxRec *recs, const CallRec *calls, int count,
                                 int blocks_split, cudaStream_t s)
{
    if (count <= 0 || blocks_split <= 0)
        return cudaSuccess;
    grouped_split_kernel<<<blocks_split, 256, 0, s>>>(recs, calls, count);
    return cudaGetLastError();
}

cudaError_t grouped_finalize_launch(const AuxRec *recs, const CallRec *calls, int count,
                                    cudaStream_t s)
{
    if (count <= 0)
        return cudaSuccess;
    grouped_finalize_kernel<<<(count + 255) / 256, 256, 0, s>>>(recs, calls, count);
    return cudaGetLastError();
}

cudaError_t finalize_launch(double *scal, int *status, svt_status *user_status, cudaStream_t s)
{
    finalize_kernel<<<1, 1, 0, s>>>(scal, status, user_status);
    return cudaGetLastError();
}

cudaError_t f64_gemm_launch(const F64Launch &l, cudaStream_t s)
{
    int tm = 0, tn = 0;
    for (int i = 0; i < l.nprob; ++i) {
        tm = max(tm, (l.p[i].M + kF64Tile - 1) / kF64Tile);
        tn = max(tn, (l.p[i].N + kF64Tile - 1) / kF64Tile);
    }
    if (tm == 0 || tn == 0)
        return cudaSuccess;
    f64_gemm_kernel<<<dim3(tn, tm, l.nprob), 256, 0, s>>>(l);
    return cudaGetLastError();
}

} // namespace svt
