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

// Column norms (wide = 0): block (32, 8) covers 32 columns and kRowsPerBlock rows.
constexpr int kRowsPerBlock = 256;

// Block (bx, by) of the column-norm reduction; threads (tx, ty) in 32 x 8.
__device__ __forceinline__ void colnorm_block(const float *__restrict__ A, int64_t m, int64_t n,
                                              int64_t lda, double *colnorm2, double *scal,
                                              int *status, int bx, int by, int tx, int ty)
{
    __shared__ double part[8][33];
    const int64_t col = (int64_t)bx * 32 + tx;
    const int64_t r0 = (int64_t)by * kRowsPerBlock;
    const int64_t r1 = (m < r0 + kRowsPerBlock) ? m : r0 + kRowsPerBlock;
    double s = 0.0;
    bool finite = true;
    if (col < n) {
        for (int64_t r = r0 + ty; r < r1; r += 8) {
            float a = A[r * lda + col];
            finite &= isfinite(a);
            s += (double)a * (double)a;
        }
    }
    if (!finite)
        set_status(status, SVT_ERR_NONFINITE);
    part[ty][tx] = s;
    __syncthreads();
    if (ty == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i)
            t += part[i][tx];
        if (col < n)
            atomicAdd(&colnorm2[col], t);
        // block total for ||A||_F^2
        for (int o = 16; o > 0; o >>= 1)
            t += __shfl_xor_sync(0xffffffffu, t, o);
        if (tx == 0)
            atomicAdd(&scal[SC_NRM_A2], t);
    }
}

__global__ void ingest_colnorm_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                      int64_t lda, double *colnorm2, double *scal, int *status)
{
    colnorm_block(A, m, n, lda, colnorm2, scal, status, blockIdx.x, blockIdx.y, threadIdx.x,
                  threadIdx.y);
}

// Row norms (wide = 1): one warp per row.
// Row norms of rows 8 bx .. 8 bx + 7 (one warp per row, 256 threads).
__device__ __forceinline__ void rownorm_block(const float *__restrict__ A, int64_t m, int64_t n,
                                              int64_t lda, double *colnorm2, double *scal,
                                              int *status, int bx, int tid)
{
    const int64_t row = (int64_t)bx * 8 + tid / 32;
    const int lane = tid & 31;
    if (row >= m)
        return;
    double s = 0.0;
    bool finite = true;
    for (int64_t c = lane; c < n; c += 32) {
        float a = A[row * lda + c];
        finite &= isfinite(a);
        s += (double)a * (double)a;
    }
    if (!finite)
        set_status(status, SVT_ERR_NONFINITE);
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        colnorm2[row] = s;
        atomicAdd(&scal[SC_NRM_A2], s);
    }
}

__global__ void ingest_rownorm_kernel(const float *__restrict__ A, int64_t m, int64_t n,
                                      int64_t lda, double *colnorm2, double *scal, int *status)
{
    rownorm_block(A, m, n, lda, colnorm2, scal, status, blockIdx.x, threadIdx.x);
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

// 32 x 32 tile of A -> same-orientation and transposed copies of A / alpha.
template <bool F64>
__device__ __forceinline__ void split_block(const float *__restrict__ A, int64_t m, int64_t n,
                                            int64_t lda, float tau, void *xs_hi, void *xs_lo,
                                            int64_t ld_s, void *xt_hi, void *xt_lo, int64_t ld_t,
                                            double *scal, int bx, int by, int tx, int ty)
{
    __shared__ float tile[32][33];
    const double nrm2 = scal[SC_NRM_A2];
    const double alpha = pow2_alpha(nrm2);
    const float inv_alpha = (float)(1.0 / alpha);  // exact power of two
    if (bx == 0 && by == 0 && tx == 0 && ty == 0) {
        scal[SC_ALPHA] = alpha;
        scal[SC_INV_ALPHA2] = 1.0 / (alpha * alpha);
        scal[SC_TAU2_SCALED] = ((double)tau * (double)tau) / (alpha * alpha);
        scal[SC_NRM_X0] = nrm2 / (alpha * alpha);
    }
    const int64_t i0 = (int64_t)by * 32, j0 = (int64_t)bx * 32;
    for (int k = ty; k < 32; k += 8) {
        const int64_t i = i0 + k, j = j0 + tx;
        float x = (i < m && j < n) ? A[i * lda + j] * inv_alpha : 0.0f;
        tile[k][tx] = x;
        if (i < m && j < n && xs_hi) {
            if (F64) {
                static_cast<double *>(xs_hi)[i * ld_s + j] = (double)x;
            } else {
                __nv_bfloat16 hi = __float2bfloat16_rn(x);
                static_cast<__nv_bfloat16 *>(xs_hi)[i * ld_s + j] = hi;
                if (xs_lo)
                    static_cast<__nv_bfloat16 *>(xs_lo)[i * ld_s + j] =
                        __float2bfloat16_rn(x - __bfloat162float(hi));
            }
        }
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t j = j0 + k, i = i0 + tx;  // transposed element (j, i)
        if (i < m && j < n && xt_hi) {
            float x = tile[tx][k];
            if (F64) {
                static_cast<double *>(xt_hi)[j * ld_t + i] = (double)x;
            } else {
                __nv_bfloat16 hi = __float2bfloat16_rn(x);
                static_cast<__nv_bfloat16 *>(xt_hi)[j * ld_t + i] = hi;
                if (xt_lo)
                    static_cast<__nv_bfloat16 *>(xt_lo)[j * ld_t + i] =
                        __float2bfloat16_rn(x - __bfloat162float(hi));
            }
        }
    }
}

template <bool F64>
__global__ void ingest_split_kernel(const float *__restrict__ A, int64_t m, int64_t n, int64_t lda,
                                    float tau, void *xs_hi, void *xs_lo, int64_t ld_s, void *xt_hi,
                                    void *xt_lo, int64_t ld_t, double *scal)
{
    split_block<F64>(A, m, n, lda, tau, xs_hi, xs_lo, ld_s, xt_hi, xt_lo, ld_t, scal, blockIdx.x,
                     blockIdx.y, threadIdx.x, threadIdx.y);
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

__global__ void grouped_reduce_kernel(const AuxRec *recs, const CallRec *calls, int count)
{
    const int i = find_rec(recs, count, blockIdx.x, false);
    const AuxRec &r = recs[i];
    const CallRec &c = calls[i];
    const int lb = blockIdx.x - r.blk_reduce;
    if (!r.wide) {
        const int gx = (int)((r.n + 31) / 32);
        colnorm_block(c.A, r.m, r.n, c.lda, r.colnorm, r.scal, r.status, lb % gx, lb / gx,
                      threadIdx.x & 31, threadIdx.x >> 5);
    } else {
        rownorm_block(c.A, r.m, r.n, c.lda, r.colnorm, r.scal, r.status, lb, threadIdx.x);
    }
}

__global__ void grouped_split_kernel(const AuxRec *recs, const CallRec *calls, int count)
{
    const int i = find_rec(recs, count, blockIdx.x, true);
    const AuxRec &r = recs[i];
    const CallRec &c = calls[i];
    const int lb = blockIdx.x - r.blk_split;
    const int gx = (int)((r.n + 31) / 32);
    if (r.f64)
        split_block<true>(c.A, r.m, r.n, c.lda, c.tau, r.xs_hi, nullptr, r.ld_s, r.xt_hi, nullptr,
                          r.ld_t, r.scal, lb % gx, lb / gx, threadIdx.x & 31, threadIdx.x >> 5);
    else
        split_block<false>(c.A, r.m, r.n, c.lda, c.tau, r.xs_hi, r.xs_lo, r.ld_s, r.xt_hi, r.xt_lo,
                           r.ld_t, r.scal, lb % gx, lb / gx, threadIdx.x & 31, threadIdx.x >> 5);
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
                                 double *colnorm2, double *scal, int *status, cudaStream_t s)
{
    if (!wide) {
        dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + kRowsPerBlock - 1) / kRowsPerBlock));
        ingest_colnorm_kernel<<<grid, dim3(32, 8), 0, s>>>(A, m, n, lda, colnorm2, scal, status);
    } else {
        unsigned blocks = (unsigned)((m + 7) / 8);
        ingest_rownorm_kernel<<<blocks, 256, 0, s>>>(A, m, n, lda, colnorm2, scal, status);
    }
    return cudaGetLastError();
}

cudaError_t ingest_split_launch(const float *A, int64_t m, int64_t n, int64_t lda, float tau,
                                int f64, void *xs_hi, void *xs_lo, int64_t ld_s, void *xt_hi,
                                void *xt_lo, int64_t ld_t, double *scal, int *status,
                                cudaStream_t s)
{
    (void)status;
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32));
    if (f64)
        ingest_split_kernel<true><<<grid, dim3(32, 8), 0, s>>>(A, m, n, lda, tau, xs_hi, nullptr,
                                                                ld_s, xt_hi, nullptr, ld_t, scal);
    else
        ingest_split_kernel<false><<<grid, dim3(32, 8), 0, s>>>(A, m, n, lda, tau, xs_hi, xs_lo,
                                                                 ld_s, xt_hi, xt_lo, ld_t, scal);
    return cudaGetLastError();
}

int grouped_reduce_blocks(int64_t m, int64_t n, int wide)
{
    if (!wide)
        return (int)(((n + 31) / 32) * ((m + kRowsPerBlock - 1) / kRowsPerBlock));
    return (int)((m + 7) / 8);
}

int grouped_split_blocks(int64_t m, int64_t n) { return (int)(((n + 31) / 32) * ((m + 31) / 32)); }

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
