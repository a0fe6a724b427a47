// Tensor-core product kernel for sm_103a: D = sum_s L_s R_s^T with BF16
// operands staged by TMA into 128-byte-swizzled shared memory, tcgen05.mma
// (kind::f16, BF16 x BF16 -> FP32) accumulating in tensor memory, and a fused
// epilogue that reads the accumulator back with tcgen05.ld. Problems flagged fp8
// (the FP8 experiment) take e4m3 operands through kind::f8f6f4 instead; the operand
// kind, like the epilogue's chunk loop (one copy per product kind), is chosen once
// per tile.
//
// This one kernel carries every dense product of the method (Section 2): the
// shifted Gram A^T A - tau^2 I, the polynomial steps X (a I + b X^T X +
// c (X^T X)^2) of both polar chains, the polish step and the final combine
// 1/2 (A - tau P)(I + S) of Proposition 1.
//
// Structure (persistent, one CTA per SM, 320 threads):
//   warp 0    : TMA producer (one thread), STAGES-deep shared-memory ring.
//   warp 1    : tensor-memory allocator and MMA issuer (one thread).
//   warps 2-9 : epilogue; warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31, and
//               the two warps of a lane quadrant take alternate 32-column chunks.
// Two accumulator buffers of BN FP32 columns each let the epilogue of one tile
// overlap the MMAs of the next.
//
// CTA-pair mode (PAIR): a cluster of two CTAs computes one 256 x 256 tile with
// tcgen05.mma.cta_group::2. Each CTA stages its own 128 rows of L and one half
// (128 rows) of the tile's R, so a pipeline stage is 32 KiB instead of 48 KiB
// and every operand byte crosses L2 -> SM once per pair instead of once per CTA.
// The even CTA (leader) issues the MMAs for both, its barriers collect both
// CTAs' TMA bytes and both CTAs' epilogue releases; MMA completion is multicast
// to both CTAs, whose epilogues each drain their own 128 x 256 accumulator.
//
// Every wait on an mbarrier is bounded (kWaitTimeoutNs of global time); on
// expiry the kernel records SVT_ERR_TIMEOUT in the problem's status word, the
// other roles stop at their next wait, in-flight copies and MMAs are drained
// (again with a bound) and tensor memory is released before the kernel returns.
#include <algorithm>
#include <cstddef>

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "svt_internal.h"

namespace svt {

namespace {

constexpr uint64_t kWaitTimeoutNs = 2000000000ull;  // 2 s
constexpr int kThreads = 320;  // 2 producer/MMA warps + 8 epilogue warps
constexpr int kEpiWarps = 8;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase with the given parity to complete. Returns false
// when the kernel is aborting (another role timed out) or this wait timed out.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                          int *status, uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag)
                return false;
            uint64_t now = global_timer_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > limit_ns) {
                *abort_flag = 1;
                if (status)
                    atomicCAS(status, 0, (int)SVT_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

// Waits on barriers that another CTA of the cluster signals use acquire at
// cluster scope.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                  int *status, uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait_cluster(bar, parity))
            return true;
        if ((it & 255u) == 255u) {
            if (*abort_flag)
                return false;
            uint64_t now = global_timer_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > limit_ns) {
                *abort_flag = 1;
                if (status)
                    atomicCAS(status, 0, (int)SVT_ERR_TIMEOUT);
                return false;
            }
        }
    }
}

template <bool CLUSTER>
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                         int *status, uint64_t limit_ns)
{
    return CLUSTER ? mbar_wait_cluster(bar, parity, abort_flag, status, limit_ns)
                   : mbar_wait(bar, parity, abort_flag, status, limit_ns);
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t peer_addr(const void *p, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
                 : "memory");
}

__device__ __forceinline__ void st_remote_u32(uint32_t cluster_addr, int v)
{
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA load into this CTA's shared memory whose completion is counted on a
// barrier of either CTA of the pair (a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void *smem_dst, const CUtensorMap *map, int x,
                                                 int y, uint32_t bar_cluster_addr)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster_addr)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(smem_dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *smem_src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(smem_src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// At most N of this thread's most recent bulk groups may still be reading shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait until *counter >= target (another CTA's completion count).
__device__ bool wait_counter(const int *counter, int target, volatile int *abort_flag, int *status,
                             uint64_t limit_ns)
{
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        if (ld_acquire_gpu(counter) >= target)
            return true;
        if ((it & 63u) == 63u) {
            if (*abort_flag)
                return false;
            uint64_t now = global_timer_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > limit_ns) {
                *abort_flag = 1;
                if (status)
                    atomicCAS(status, 0, (int)SVT_ERR_TIMEOUT);
                return false;
            }
            __nanosleep(64);
        }
    }
}

// Limit of the waits on other tiles' results (the launch's debug setting, else 2 s).
__device__ __forceinline__ uint64_t dep_limit(const TcLaunch &L)
{
    return L.dep_wait_ns ? (uint64_t)L.dep_wait_ns : kWaitTimeoutNs;
}

// Wait for strip `idx` of dependency k of problem P (see TcProblem::sdep_*), unless the
// producing problem is already known (src_done) or found to be complete as a whole,
// which covers every strip; a role then stops checking that source.
__device__ __forceinline__ bool wait_strip(const TcLaunch &L, const TcProblem &P, int k, int idx,
                                           bool &src_done, volatile int *abort_flag, int *status)
{
    if (src_done)
        return true;
    if (ld_acquire_gpu(&L.done[P.sdep_src[k]]) >= P.sdep_whole[k]) {
        src_done = true;
        return true;
    }
    return wait_counter(&L.strips[P.sdep_base[k] + idx], P.sdep_target[k], abort_flag, status,
                        dep_limit(L));
}

// Shared-memory matrix descriptor for a K-major operand tile laid out by TMA
// with 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)(16u >> 4) << 16;          // leading byte offset (unused here)
    d |= (uint64_t)(1024u >> 4) << 32;        // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4)                       // D format FP32
           | (1u << 7)                     // A format BF16
           | (1u << 10)                    // B format BF16
           | ((uint32_t)(n >> 3) << 17)    // N / 8
           | ((uint32_t)(m >> 4) << 24);   // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Instruction descriptor of kind::f8f6f4: e4m3 x e4m3 -> FP32 (A and B format code 0),
// both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_e4m3(int m, int n)
{
    return (1u << 4)                       // D format FP32
           | ((uint32_t)(n >> 3) << 17)    // N / 8
           | ((uint32_t)(m >> 4) << 24);   // M / 16
}

// A compile-time bool passed as a value (selects a loop body's instruction kind).
template <bool B>
struct BoolTag {
    static constexpr bool value = B;
};

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_e4m3_pair(uint32_t d_tmem, uint64_t a, uint64_t b,
                                              uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a, uint64_t b,
                                              uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Completion of this thread's pair MMAs arrives on the barrier at the same
// offset in both CTAs of the pair.
__device__ __forceinline__ void mma_commit_both(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

__device__ __forceinline__ void mma_commit_pair_local(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

template <bool PAIR>
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t cols)
{
    if (PAIR)
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(slot)),
                     "r"(cols));
    else
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(slot)),
                     "r"(cols));
}

template <bool PAIR>
__device__ __forceinline__ void tmem_relinquish()
{
    if (PAIR)
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
    else
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

template <bool PAIR>
__device__ __forceinline__ void tmem_dealloc(uint32_t base, uint32_t cols)
{
    if (PAIR)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols));
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(cols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 32 consecutive FP32 columns of tensor memory into registers.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i)
        v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- tiles

struct TileCoord {
    int prob, tm, tn;
    bool valid;
};

__device__ __forceinline__ const TcProblem &prob_at(const TcLaunch &L, int p)
{
    return L.gtab ? L.gtab[p] : L.p[p];
}

// Linear tile index -> (problem, tile row, tile column) for tiles of TM x BN.
// Dense problems: column-major over the tile grid. Symmetric problems: only
// tiles holding some element with row <= col; column tn holds r (tn + 1) row
// tiles (r = BN / TM), so the first tile of column tn is r tn (tn + 1) / 2
// (ROWMAJOR_SYM with square tiles: row-major instead, see below).
// A role's tile indices only increase, so the problem search gallops forward from
// the previous answer (`hint`) instead of bisecting the whole table: a few
// dependent loads of the tile prefix sums instead of log2(problems).
template <int BN, int TM, bool ROWMAJOR_SYM>
__device__ TileCoord decode_tile(const TcLaunch &L, int t, int &hint)
{
    TileCoord tc{0, 0, 0, false};
    int p = 0, start = 0;
    if (L.gtab) {
        p = hint;
        if (p < 0 || p >= L.gcount || L.gstart[p] > t)
            p = 0;
        int step = 1, q = p + 1;  // first q > p with gstart[q] > t lies in (p, q]
        while (q < L.gcount && L.gstart[q] <= t) {
            p = q;
            step <<= 1;
            q = p + step;
        }
        int hi = (q < L.gcount ? q : L.gcount) - 1;  // last p with gstart[p] <= t
        while (p < hi) {
            const int mid = (p + hi + 1) >> 1;
            if (L.gstart[mid] <= t)
                p = mid;
            else
                hi = mid - 1;
        }
        hint = p;
        start = L.gstart[p];
    } else {
        while (p + 1 < L.nprob && t >= L.tile_start[p + 1])
            ++p;
        start = L.tile_start[p];
    }
    const TcProblem &P = prob_at(L, p);
    int local = t - start;
    tc.prob = p;
    if (!P.sym) {
        tc.tm = local % P.tiles_m;
        tc.tn = local / P.tiles_m;
        tc.valid = true;
        return tc;
    }
    constexpr int r = BN / TM;
    if (ROWMAJOR_SYM && r == 1) {
        // Square tiles: row-major over the upper triangle (row tm holds columns
        // tm .. T - 1, first index tm T - tm (tm - 1) / 2), so that the strips of a
        // symmetric product complete in order.
        const int T = P.tiles_n;
        auto first = [T](int i) { return i * T - i * (i - 1) / 2; };
        const float b = 2.0f * (float)T + 1.0f;
        int tm = (int)((b - sqrtf(fmaxf(b * b - 8.0f * (float)local, 0.0f))) * 0.5f);
        tm = tm < 0 ? 0 : (tm > T - 1 ? T - 1 : tm);
        while (tm > 0 && first(tm) > local)
            --tm;
        while (tm + 1 < T && first(tm + 1) <= local)
            ++tm;
        tc.tm = tm;
        tc.tn = tm + (local - first(tm));
        tc.valid = (tm < P.tiles_m) && (tc.tn < P.tiles_n);
        return tc;
    }
    int tn = (int)((sqrtf(8.0f * (float)local / (float)r + 1.0f) - 1.0f) * 0.5f);
    while (tn > 0 && r * tn * (tn + 1) / 2 > local)
        --tn;
    while (r * (tn + 1) * (tn + 2) / 2 <= local)
        ++tn;
    int tm = local - r * tn * (tn + 1) / 2;
    tc.tm = tm;
    tc.tn = tn;
    tc.valid = (tm < P.tiles_m) && (tn < P.tiles_n);
    return tc;
}

// ------------------------------------------------------------- epilogue

struct EpiScales {
    float alpha, beta, gamma;
};

__device__ __forceinline__ EpiScales epi_scales(const Epi &e, double alpha)
{
    EpiScales s{(float)alpha, (float)e.beta, (float)e.gamma};
    if (e.theta_src) {
        double theta = pow(*e.theta_src, e.theta_pow);
        if (theta > 0.0 && isfinite(theta)) {
            s.alpha = (float)(alpha * pow(theta, -e.ea));
            s.beta = (float)(e.beta * pow(theta, -e.eb));
            s.gamma = (float)(e.gamma * pow(theta, -e.eg));
        } else if (!isfinite(theta) && e.status) {
            atomicCAS(e.status, 0, (int)SVT_ERR_DIVERGED);
        }  // theta == 0: the chain's matrix is zero; nothing to scale
    }
    return s;
}

__device__ __forceinline__ bool aligned16(const void *p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15u) == 0;
}

// The fields of the current problem that the epilogue reads for every 32 x 32
// block, loaded once per change of problem into registers: the problem table
// lives in global memory, and every memory-clobbering TMA or fence instruction
// of the epilogue would otherwise force these loads to be repeated.
struct EpiHot {
    const void *c0, *c1;
    void *o0, *o1, *t0, *t1;
    const CUtensorMap *maps;  // mapO[0..1] then mapT[0..1] of the problem
    double *norm_acc;
    const double *diag, *dss;
    int64_t ldc, ldo, ldt;
    float alpha, beta, gamma;
    int M, N, sym, otma, ttma, c_kind, c_trans, o_kind, o_trans, t_kind;
    void *f0;          // e4m3 copy (FP8 experiment), null: none
    int64_t ldf;
    float fscale;
    int strip_base, tiles_m;  // fused solves: the problem's strip counters
};

// Raw C values of one lane's 32-column row segment: BF16 hi in q[0..3] (lo of a
// pair in q[4..7]) or FP32 in q[0..7].
struct CRaw {
    uint4 q[8];
};

// Issue the loads of C(r, c0 .. c0 + 31) into registers. Returns false where the
// vector form does not apply (no C, row outside, transposed C, a ragged right edge,
// or a row address that is not 16-byte aligned); c_apply then reads C directly.
__device__ __forceinline__ bool c_load(const EpiHot &h, int64_t r, int64_t c0, bool full_row,
                                       CRaw &cr)
{
    if (h.c_kind == C_NONE || h.c_trans || !full_row)
        return false;
    const int64_t off = r * h.ldc + c0;
    if (h.c_kind == C_F32) {
        const float *p = static_cast<const float *>(h.c0) + off;
        if (!aligned16(p))
            return false;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            cr.q[q] = __ldg(reinterpret_cast<const uint4 *>(p) + q);
        return true;
    }
    const __nv_bfloat16 *ph = static_cast<const __nv_bfloat16 *>(h.c0) + off;
    const __nv_bfloat16 *pl = static_cast<const __nv_bfloat16 *>(h.c1) + off;
    if (!aligned16(ph) || (h.c_kind == C_PAIR && !aligned16(pl)))
        return false;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        cr.q[q] = __ldg(reinterpret_cast<const uint4 *>(ph) + q);
    if (h.c_kind == C_PAIR) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            cr.q[4 + q] = __ldg(reinterpret_cast<const uint4 *>(pl) + q);
    }
    return true;
}

// v[i] += beta * C(r, c0 + i) for i < ncol, from registers loaded by c_load (vec)
// or read directly (any layout, alignment or edge).
__device__ __forceinline__ void c_apply(const EpiHot &h, const CRaw &cr, bool vec, int64_t r,
                                        int64_t c0, int ncol, bool row_ok, float *v)
{
    if (h.c_kind == C_NONE || !row_ok)
        return;
    const float beta = h.beta;
    if (vec) {
        if (h.c_kind == C_F32) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                v[4 * q] += beta * __uint_as_float(cr.q[q].x);
                v[4 * q + 1] += beta * __uint_as_float(cr.q[q].y);
                v[4 * q + 2] += beta * __uint_as_float(cr.q[q].z);
                v[4 * q + 3] += beta * __uint_as_float(cr.q[q].w);
            }
            return;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const __nv_bfloat162 *b = reinterpret_cast<const __nv_bfloat162 *>(&cr.q[q]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float2 f = __bfloat1622float2(b[j]);
                v[q * 8 + 2 * j] += beta * f.x;
                v[q * 8 + 2 * j + 1] += beta * f.y;
            }
        }
        if (h.c_kind == C_PAIR) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const __nv_bfloat162 *b = reinterpret_cast<const __nv_bfloat162 *>(&cr.q[4 + q]);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 f = __bfloat1622float2(b[j]);
                    v[q * 8 + 2 * j] += beta * f.x;
                    v[q * 8 + 2 * j + 1] += beta * f.y;
                }
            }
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        if (i >= ncol)
            continue;
        const int64_t c = c0 + i;
        const int64_t off = h.c_trans ? c * h.ldc + r : r * h.ldc + c;
        float x;
        if (h.c_kind == C_F32)
            x = static_cast<const float *>(h.c0)[off];
        else {
            x = __bfloat162float(static_cast<const __nv_bfloat16 *>(h.c0)[off]);
            if (h.c_kind == C_PAIR)
                x += __bfloat162float(static_cast<const __nv_bfloat16 *>(h.c1)[off]);
        }
        v[i] += beta * x;
    }
}

// Fallback staging: 32 x 32 floats, element (a, b) at a * 32 + (b ^ a); rows and
// columns are both free of bank conflicts.
__device__ __forceinline__ int xs_idx(int a, int b) { return a * 32 + (b ^ a); }

// e4m3 bytes of scale * v, saturated (the FP8 experiment's operand copies), in the
// layout store_block uses: 16 rows x 32 bytes per instruction. Kept out of line so
// that the BF16 epilogue's code is what it is without it.
__device__ __noinline__ void store_block_e4m3(const float *st, void *p0, int64_t ld, int64_t r0,
                                              int64_t c0, int64_t M, int64_t N, bool trans,
                                              bool symdiag, int lane, float scale)
{
    const int64_t orow0 = trans ? c0 : r0, ocol0 = trans ? r0 : c0;
    const int64_t orows = trans ? N : M, ocols = trans ? M : N;
    // e4m3 bytes of scale * v, saturated: 16 rows x 32 bytes per instruction
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int a = k * 16 + (lane >> 1);
        const int q = lane & 1;  // columns 16 q .. 16 q + 15
        const int64_t R = orow0 + a;
        float x[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int b = q * 16 + j;
            int sa, sb;
            if (trans) { sa = b; sb = a; }
            else if (symdiag && a > b) { sa = b; sb = a; }
            else { sa = a; sb = b; }
            x[j] = scale * st[xs_idx(sa, sb)];
        }
        if (R >= orows)
            continue;
        const int64_t C = ocol0 + q * 16;
        uint8_t *p = static_cast<uint8_t *>(p0) + R * ld + C;
        if (C + 16 <= ocols && aligned16(p)) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(x[4 * j], x[4 * j + 1]),
                                                             __NV_SATFINITE, __NV_E4M3);
                const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(x[4 * j + 2], x[4 * j + 3]),
                                                             __NV_SATFINITE, __NV_E4M3);
                w[j] = lo | (hi << 16);
            }
            *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (C + j < ocols)
                    p[j] = __nv_cvt_float_to_fp8(x[j], __NV_SATFINITE, __NV_E4M3);
        }
    }
}

// Store a 32 x 32 block held in shared memory `st` (st[a][b] = value of tile
// element (r0 + a, c0 + b)) to global memory, coalesced: warp lanes cover whole
// row segments (8 rows x 64 B for BF16, 4 rows x 128 B for FP32 per instruction).
//   trans = 0: element (r0 + a, c0 + b) -> p[(r0 + a) * ld + c0 + b];
//              symdiag: the block sits on the diagonal and (a > b) takes st[b][a].
//   trans = 1: element (r0 + b, c0 + a) -> p[(c0 + a) * ld + r0 + b].
// Only elements with row < M and col < N (tile coordinates) are written.
__device__ __forceinline__ void store_block(const float *st, int kind, void *p0, void *p1,
                                            int64_t ld, int64_t r0, int64_t c0, int64_t M,
                                            int64_t N, bool trans, bool symdiag, int lane)
{
    // output rows: tile rows (trans = 0) or tile columns (trans = 1)
    const int64_t orow0 = trans ? c0 : r0, ocol0 = trans ? r0 : c0;
    const int64_t orows = trans ? N : M, ocols = trans ? M : N;
    if (kind == O_BF16 || kind == O_PAIR) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int a = k * 8 + (lane >> 2);  // output row within the block
            const int q = lane & 3;             // 16-byte chunk: columns 8q .. 8q + 7
            const int64_t R = orow0 + a;
            float x[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int b = q * 8 + j;
                int sa, sb;  // staging coordinates
                if (trans) { sa = b; sb = a; }
                else if (symdiag && a > b) { sa = b; sb = a; }
                else { sa = a; sb = b; }
                x[j] = st[xs_idx(sa, sb)];
            }
            if (R >= orows)
                continue;
            const int64_t C = ocol0 + q * 8;
            const int64_t off = R * ld + C;
            if (C + 8 <= ocols && aligned16(static_cast<__nv_bfloat16 *>(p0) + off) &&
                (kind != O_PAIR || aligned16(static_cast<__nv_bfloat16 *>(p1) + off))) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    __nv_bfloat162 h2 = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
                    hw[j] = *reinterpret_cast<uint32_t *>(&h2);
                    __nv_bfloat162 l2 = __floats2bfloat162_rn(x[2 * j] - __low2float(h2),
                                                              x[2 * j + 1] - __high2float(h2));
                    lw[j] = *reinterpret_cast<uint32_t *>(&l2);
                }
                *reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(p0) + off) =
                    make_uint4(hw[0], hw[1], hw[2], hw[3]);
                if (kind == O_PAIR)
                    *reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(p1) + off) =
                        make_uint4(lw[0], lw[1], lw[2], lw[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (C + j < ocols) {
                        __nv_bfloat16 h = __float2bfloat16_rn(x[j]);
                        static_cast<__nv_bfloat16 *>(p0)[off + j] = h;
                        if (kind == O_PAIR)
                            static_cast<__nv_bfloat16 *>(p1)[off + j] =
                                __float2bfloat16_rn(x[j] - __bfloat162float(h));
                    }
                }
            }
        }
    } else if (kind == O_F32) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int a = k * 4 + (lane >> 3);
            const int q = lane & 7;  // columns 4q .. 4q + 3
            const int64_t R = orow0 + a;
            float x[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int b = q * 4 + j;
                int sa, sb;
                if (trans) { sa = b; sb = a; }
                else if (symdiag && a > b) { sa = b; sb = a; }
                else { sa = a; sb = b; }
                x[j] = st[xs_idx(sa, sb)];
            }
            if (R >= orows)
                continue;
            const int64_t C = ocol0 + q * 4;
            const int64_t off = R * ld + C;
            if (C + 4 <= ocols && aligned16(static_cast<float *>(p0) + off)) {
                *reinterpret_cast<float4 *>(static_cast<float *>(p0) + off) =
                    make_float4(x[0], x[1], x[2], x[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (C + j < ocols)
                        static_cast<float *>(p0)[off + j] = x[j];
            }
        }
    }
}

// Byte offset of element (row, col) of a 32 x 32 staging block laid out the way
// the TMA unit reads it: FP32 rows of 128 B with the 128-byte swizzle (16-byte
// chunk index XOR row % 8), BF16 rows of 64 B with the 64-byte swizzle (chunk
// index XOR (row / 2) % 4). Both orders of writing -- a lane per row with 16-byte
// vectors, or a lane per column with scalars -- are free of bank conflicts.
__device__ __forceinline__ uint32_t stg_off_f32(int row, int col)
{
    return (uint32_t)(row * 128 + ((((col >> 2) ^ (row & 7))) << 4) + (col & 3) * 4);
}
__device__ __forceinline__ uint32_t stg_off_b16(int row, int col)
{
    return (uint32_t)(row * 64 + ((((col >> 3) ^ ((row >> 1) & 3))) << 4) + (col & 7) * 2);
}

// Stage the warp's 32 x 32 block (lane = block row, x[] = its 32 columns) and
// store it with one or two TMA stores (one bulk group): at tile coordinates
// (x = c0, y = r0), or transposed at (x = r0, y = c0). `kind` is O_F32, O_BF16 or
// O_PAIR (hi through m0, lo through m1). The warp owns NSTG 4 KiB staging slots
// (1024-byte aligned) used in turn, so a store's shared-memory read overlaps the
// staging of the next NSTG - 1 blocks; an FP32 block fills a slot, BF16 hi and lo
// take its two halves.
template <int NSTG>
__device__ __forceinline__ void tma_store_block(const float *x, int kind, bool trans,
                                                const CUtensorMap *m0, const CUtensorMap *m1,
                                                int r0, int c0, uint8_t *stg_base, int &slot,
                                                int lane)
{
    uint8_t *stg0 = stg_base + slot * 4096, *stg1 = stg0 + 2048;
    if (++slot == NSTG)
        slot = 0;
    if (lane == 0)
        bulk_wait_read<NSTG - 1>();  // the store that last used this slot has read it
    __syncwarp();
    if (kind == O_F32) {
        if (!trans) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                *reinterpret_cast<float4 *>(stg0 + stg_off_f32(lane, 4 * q)) =
                    make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
        } else {
#pragma unroll
            for (int c = 0; c < 32; ++c)
                *reinterpret_cast<float *>(stg0 + stg_off_f32(c, lane)) = x[c];
        }
    } else {
        const bool pair = (kind == O_PAIR);
        if (!trans) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    __nv_bfloat162 h2 = __floats2bfloat162_rn(x[8 * q + 2 * j], x[8 * q + 2 * j + 1]);
                    hw[j] = *reinterpret_cast<uint32_t *>(&h2);
                    __nv_bfloat162 l2 = __floats2bfloat162_rn(x[8 * q + 2 * j] - __low2float(h2),
                                                              x[8 * q + 2 * j + 1] - __high2float(h2));
                    lw[j] = *reinterpret_cast<uint32_t *>(&l2);
                }
                *reinterpret_cast<uint4 *>(stg0 + stg_off_b16(lane, 8 * q)) =
                    make_uint4(hw[0], hw[1], hw[2], hw[3]);
                if (pair)
                    *reinterpret_cast<uint4 *>(stg1 + stg_off_b16(lane, 8 * q)) =
                        make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                __nv_bfloat16 h = __float2bfloat16_rn(x[c]);
                *reinterpret_cast<__nv_bfloat16 *>(stg0 + stg_off_b16(c, lane)) = h;
                if (pair)
                    *reinterpret_cast<__nv_bfloat16 *>(stg1 + stg_off_b16(c, lane)) =
                        __float2bfloat16_rn(x[c] - __bfloat162float(h));
            }
        }
    }
    fence_async_smem();
    __syncwarp();
    if (lane == 0) {
        const int sx = trans ? r0 : c0, sy = trans ? c0 : r0;
        tma_store_2d(m0, sx, sy, stg0);
        if (kind == O_PAIR)
            tma_store_2d(m1, sx, sy, stg1);
        bulk_commit();
    }
}

// Rest of the epilogue of one 32 x 32 block after alpha D + beta C: the identity
// term (or the FP64 shifted-Gram diagonal) on the diagonal, the squared-norm
// contribution, then the stores. lane = tile row r0 + lane, columns c0 .. c0 + 31.
// Values are staged in shared memory and stored coalesced to every requested
// destination: the output (row-major or transposed), the extra transposed copy
// and, for symmetric products, the mirror.
template <int NSTG>
__device__ __forceinline__ void epilogue_finish(const EpiHot &h, int64_t r0, int64_t c0, float *v,
                                                double &nrm, uint8_t *stg, int &slot, int lane)
{
    const int64_t r = r0 + lane;
    const bool row_ok = r < h.M;
    const int64_t rem = (int64_t)h.N - c0;
    const int ncol = rem < 32 ? (int)rem : 32;
    const bool diag_block = (r0 == c0);
    if (diag_block) {  // this lane's diagonal element is column i == lane
        const bool dg = h.diag != nullptr;
        const float dval = (dg && row_ok) ? (float)(h.diag[r] * h.dss[0] - h.dss[1]) : 0.f;
        const float g = h.gamma;
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (i == lane)
                v[i] = dg ? dval : v[i] + g;
    }
    if (h.norm_acc && row_ok) {
        // FP32 within the row's 32 values (relative error <= 32 * 2^-24), FP64 across.
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            float w = (i < ncol) ? 1.f : 0.f;
            if (h.sym) {
                const int64_t c = c0 + i;
                w = (r < c) ? 2.f * w : (r == c ? w : 0.f);
            }
            acc = fmaf(w * v[i], v[i], acc);
        }
        nrm += (double)acc;
    }
    const bool symdiag = h.sym && diag_block;
    // Outputs through TMA stores (all but diagonal blocks of symmetric products).
    const bool o_tma = h.otma && h.o_kind != O_NONE && !symdiag;
    if (o_tma)
        tma_store_block<NSTG>(v, h.o_kind, h.o_trans != 0, &h.maps[0], &h.maps[1], (int)r0,
                              (int)c0, stg, slot, lane);
    if (h.sym && !diag_block && h.otma)  // mirror of a block strictly above the diagonal
        tma_store_block<NSTG>(v, h.o_kind, true, &h.maps[0], &h.maps[1], (int)r0, (int)c0, stg,
                              slot, lane);
    if (h.ttma && h.t_kind != O_NONE)
        tma_store_block<NSTG>(v, h.t_kind, true, &h.maps[2], &h.maps[3], (int)r0, (int)c0, stg,
                              slot, lane);
    const bool need_plain = (h.o_kind != O_NONE && !o_tma) || (h.sym && !diag_block && !h.otma) ||
                            (h.t_kind != O_NONE && !h.ttma) || h.f0 != nullptr;
    if (!need_plain)
        return;
    // Coalesced plain-store path: stage with a swizzled pitch, then whole row segments.
    if (lane == 0)
        bulk_wait_read0();
    __syncwarp();
    float *st = reinterpret_cast<float *>(stg);
#pragma unroll
    for (int i = 0; i < 32; ++i)
        st[xs_idx(lane, i)] = v[i];
    __syncwarp();
    if (h.o_kind != O_NONE && !o_tma)
        store_block(st, h.o_kind, h.o0, h.o1, h.ldo, r0, c0, h.M, h.N, h.o_trans != 0, symdiag, lane);
    if (h.sym && !diag_block && !h.otma)
        store_block(st, h.o_kind, h.o0, h.o1, h.ldo, r0, c0, h.M, h.N, true, false, lane);
    if (h.t_kind != O_NONE && !h.ttma)
        store_block(st, h.t_kind, h.t0, h.t1, h.ldt, r0, c0, h.M, h.N, true, false, lane);
    if (h.f0) {  // the e4m3 copy, mirrored like the output for symmetric products
        store_block_e4m3(st, h.f0, h.ldf, r0, c0, h.M, h.N, false, symdiag, lane, h.fscale);
        if (h.sym && !diag_block)
            store_block_e4m3(st, h.f0, h.ldf, r0, c0, h.M, h.N, true, false, lane, h.fscale);
    }
    __syncwarp();
}

// Product kinds whose epilogue runs a specialised chunk loop (chosen once per tile):
// BF16 or hi/lo-pair output through TMA stores, no norm, no FP64 diagonal, no e4m3
// copy, untransposed output, and one of
//   symmetric, no C                 (Y = X^T X, Y = S^2, S Z)
//   symmetric, C of the output kind (Z = a I + b Y + c Y^2)
//   general, no C, transposed copy of the output kind (X Z and its X^T)
// Everything else runs the generic loop (code -1). Code = 3 * (output is a pair) +
// (0 symmetric, 1 symmetric with C, 2 general with copy).
template <int S>
struct EpiSpec {
    static constexpr bool generic = S < 0;
    static constexpr int okind = S >= 3 ? O_PAIR : O_BF16;
    static constexpr bool sym = S >= 0 && S % 3 != 2;
    static constexpr int ckind = (S >= 0 && S % 3 == 1) ? (S >= 3 ? C_PAIR : C_BF16) : C_NONE;
    static constexpr bool has_t = S >= 0 && S % 3 == 2;
};

__device__ __forceinline__ int epi_spec(const EpiHot &h)
{
    if ((h.o_kind != O_BF16 && h.o_kind != O_PAIR) || !h.otma || h.o_trans || h.norm_acc || h.f0 ||
        h.diag)
        return -1;
    const bool pair = h.o_kind == O_PAIR;
    const int base = pair ? 3 : 0;
    if (h.sym && h.t_kind == O_NONE) {
        if (h.c_kind == C_NONE)
            return base;
        if (h.c_kind == (pair ? C_PAIR : C_BF16) && !h.c_trans)
            return base + 1;
        return -1;
    }
    if (!h.sym && h.t_kind == h.o_kind && h.ttma && h.c_kind == C_NONE && h.gamma == 0.f)
        return base + 2;
    return -1;
}

// c_load / c_apply for an untransposed C in BF16 (CK = C_BF16) or as a hi/lo pair.
template <int CK>
__device__ __forceinline__ bool c_load_spec(const EpiHot &h, int64_t r, int64_t c0, bool full_row,
                                            CRaw &cr)
{
    if (!full_row)
        return false;
    const int64_t off = r * h.ldc + c0;
    const __nv_bfloat16 *ph = static_cast<const __nv_bfloat16 *>(h.c0) + off;
    const __nv_bfloat16 *pl = static_cast<const __nv_bfloat16 *>(h.c1) + off;
    if (!aligned16(ph) || (CK == C_PAIR && !aligned16(pl)))
        return false;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        cr.q[q] = __ldg(reinterpret_cast<const uint4 *>(ph) + q);
    if (CK == C_PAIR) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            cr.q[4 + q] = __ldg(reinterpret_cast<const uint4 *>(pl) + q);
    }
    return true;
}

template <int CK>
__device__ __forceinline__ void c_apply_spec(const EpiHot &h, const CRaw &cr, bool vec, int64_t r,
                                             int64_t c0, int ncol, bool row_ok, float *v)
{
    if (!row_ok)
        return;
    const float beta = h.beta;
    if (vec) {
#pragma unroll
        for (int half = 0; half < (CK == C_PAIR ? 2 : 1); ++half) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const __nv_bfloat162 *b = reinterpret_cast<const __nv_bfloat162 *>(&cr.q[4 * half + q]);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 f = __bfloat1622float2(b[j]);
                    v[q * 8 + 2 * j] += beta * f.x;
                    v[q * 8 + 2 * j + 1] += beta * f.y;
                }
            }
        }
        return;
    }
    const int64_t off = r * h.ldc + c0;
    const __nv_bfloat16 *ph = static_cast<const __nv_bfloat16 *>(h.c0) + off;
    const __nv_bfloat16 *pl = static_cast<const __nv_bfloat16 *>(h.c1) + off;
#pragma unroll
    for (int i = 0; i < 32; ++i)
        if (i < ncol) {
            float x = __bfloat162float(ph[i]);
            if (CK == C_PAIR)
                x += __bfloat162float(pl[i]);
            v[i] += beta * x;
        }
}

// epilogue_finish for the specialised kinds (output kind OK): the identity term on the
// diagonal of a symmetric product, then TMA stores of the block, its mirror (symmetric,
// off the diagonal) or its transposed copy; diagonal blocks of symmetric products are
// stored whole from shared memory with their upper triangle mirrored, as in the generic
// path.
template <int NSTG, int OK, bool SYM, bool HAST>
__device__ __forceinline__ void epilogue_finish_spec(const EpiHot &h, int64_t r0, int64_t c0,
                                                     float *v, uint8_t *stg, int &slot, int lane)
{
    if (SYM) {
        if (r0 == c0) {
            const float g = h.gamma;
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (i == lane)
                    v[i] += g;
            if (lane == 0)
                bulk_wait_read0();
            __syncwarp();
            float *st = reinterpret_cast<float *>(stg);
#pragma unroll
            for (int i = 0; i < 32; ++i)
                st[xs_idx(lane, i)] = v[i];
            __syncwarp();
            store_block(st, OK, h.o0, h.o1, h.ldo, r0, c0, h.M, h.N, false, true, lane);
            __syncwarp();
            return;
        }
        tma_store_block<NSTG>(v, OK, false, &h.maps[0], &h.maps[1], (int)r0, (int)c0, stg, slot, lane);
        tma_store_block<NSTG>(v, OK, true, &h.maps[0], &h.maps[1], (int)r0, (int)c0, stg, slot, lane);
        return;
    }
    tma_store_block<NSTG>(v, OK, false, &h.maps[0], &h.maps[1], (int)r0, (int)c0, stg, slot, lane);
    if (HAST)
        tma_store_block<NSTG>(v, OK, true, &h.maps[2], &h.maps[3], (int)r0, (int)c0, stg, slot, lane);
}

// Load the epilogue fields of problem P (with the per-call fields of a grouped or
// fused launch) into registers.
__device__ __forceinline__ void load_hot(EpiHot &h, const TcProblem &P, const CallRec *calls)
{
    const Epi &e = P.ep;
    h.c0 = e.c0;
    h.c1 = e.c1;
    h.ldc = e.ldc;
    h.o0 = e.o0;
    h.o1 = e.o1;
    h.ldo = e.ldo;
    h.t0 = e.t0;
    h.t1 = e.t1;
    h.ldt = e.ldt;
    h.maps = &P.mapO[0];
    h.norm_acc = e.norm_acc;
    h.diag = e.diag;
    h.dss = e.dss;
    h.M = P.M;
    h.N = P.N;
    h.sym = P.sym;
    h.otma = P.o_tma;
    h.ttma = P.t_tma;
    h.c_kind = e.c_kind;
    h.c_trans = e.c_trans;
    h.strip_base = P.strip_base;  // read only by strip launches
    h.tiles_m = P.tiles_m;
    h.o_kind = e.o_kind;
    h.o_trans = e.o_trans;
    h.t_kind = e.t_kind;
    h.f0 = e.f0;
    h.ldf = e.ldf;
    h.fscale = e.fscale;
    double alpha = e.alpha;
    if (P.patch) {  // grouped / fused launch: per-call fields
        const CallRec &cr = calls[P.call_idx];
        if (P.patch & PT_C_IS_A) {
            h.c0 = cr.A;
            h.ldc = cr.lda;
        }
        if (P.patch & PT_O_IS_Y) {
            h.o0 = cr.Y;
            h.ldo = cr.ldy;
            h.otma = 0;
        }
        if (P.patch & PT_ALPHA_NEG_TAU)
            alpha = -(double)cr.tau;
    }
    const EpiScales sc = epi_scales(e, alpha);
    h.alpha = sc.alpha;
    h.beta = sc.beta;
    h.gamma = sc.gamma;
}

// --------------------------------------------------------------- kernel

constexpr int kRingTiles = 4;  // fused launches: tile ids in flight between the roles

template <int BN, int STAGES, bool CHAIN, bool PAIR, int NSTG, bool STRIPS>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(const __grid_constant__ TcLaunch L)
{
    static_assert(!STRIPS || CHAIN, "strip dependencies exist in fused launches only");
    static_assert(!PAIR || BN == 256, "CTA pairs compute 256 x 256 tiles");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                ~static_cast<uintptr_t>(1023));
    constexpr int A_BYTES = kBM * kBK * 2;
    constexpr int B_ROWS = PAIR ? BN / 2 : BN;  // rows of R this CTA stages per k-block
    constexpr int B_BYTES = B_ROWS * kBK * 2;
    constexpr int TILE_ROWS = PAIR ? 2 * kBM : kBM;
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint8_t *stage_all = sB + STAGES * B_BYTES;  // kEpiWarps x NSTG x 4 KiB, 1024-aligned
    uint64_t *full = reinterpret_cast<uint64_t *>(stage_all + kEpiWarps * NSTG * 4096);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *skip_flag = reinterpret_cast<int *>(tmem_slot + 2);
    // Fused launches: a ring of tile ids from the producer to the MMA and epilogue roles.
    uint64_t *rfull = reinterpret_cast<uint64_t *>(
        (reinterpret_cast<uintptr_t>(tmem_slot + 3) + 7) & ~static_cast<uintptr_t>(7));
    uint64_t *rempty = rfull + kRingTiles;
    // Ring entry i: tring[4 i .. 4 i + 3] = tile index (-1: no more tiles), problem
    // (-1: nothing to compute), tile row, tile column -- decoded once by the producer.
    volatile int *tring = reinterpret_cast<volatile int *>(rempty + kRingTiles);
    const CallRec *calls = L.calls ? L.calls : &L.call_inline;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    int *status0 = prob_at(L, 0).ep.status;
    // CTA pairs: rank 0 (leader) issues the MMAs and hands out tile ids.
    const uint32_t rank = PAIR ? cluster_rank() : 0u;
    const bool leader = rank == 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            // Pairs: one release per epilogue warp of both CTAs, on the leader's barrier.
            mbar_init(&tempty[b], PAIR ? 2 * kEpiWarps : 32 * kEpiWarps);
        }
        mbar_init(drain, 1);
        for (int i = 0; i < kRingTiles; ++i) {
            mbar_init(&rfull[i], 1);
            // Consumers of a ring entry: the MMA issuer and the epilogue warps; for
            // pairs also the peer's producer and epilogue warps.
            mbar_init(&rempty[i], PAIR ? 2 * (1 + kEpiWarps) : 1 + kEpiWarps);
        }
        *abort_flag = 0;
        // A solve whose earlier launch already timed out does no further work.
        *skip_flag = (status0 && *reinterpret_cast<volatile int *>(status0) == (int)SVT_ERR_TIMEOUT);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (PAIR) {
        // The peer's barriers exist before either CTA signals them.
        __syncthreads();
        cluster_sync_all();
    }
    if (warp == 1) {
        tmem_alloc<PAIR>(tmem_slot, 2 * BN);
        tmem_relinquish<PAIR>();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int total = *skip_flag ? 0
                                 : (L.gtab ? (L.tile_hi > 0 ? L.tile_hi : L.gstart[L.gcount])
                                           : L.tile_start[L.nprob]);
    // Static schedule (non-fused launches): CTA (pair) i takes tiles i, i + grid, ...
    const int t_first = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int t_step = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------ TMA producer
        int stage = 0;
        uint32_t phase = 0;
        uint32_t issued = 0, issued_parity = 0;  // bit s: stage s loaded / parity of its last load
        bool ok = true;
        int ri = 0;
        uint32_t rphase = 0;
        int hint = 0;
        int dep_prob = -1;       // problem whose whole dependencies have been waited for
        bool src_done[2] = {false, false};
        int smode[2] = {0, 0};   // that problem's strip dependencies of L and R
        for (int t = t_first; ok; t += t_step) {
            TileCoord tc;
            if (CHAIN) {
                if (!PAIR || leader) {
                    // Take the next tile in table order, decode it and hand it to the
                    // other roles (and to the peer CTA of a pair).
                    if (!wait_bar<PAIR>(&rempty[ri], rphase ^ 1u, abort_flag, status0, kWaitTimeoutNs))
                        break;
                    t = L.tile_lo + atomicAdd(L.tile_counter, 1);
                    t = (t < total) ? t : -1;
                    tc = TileCoord{-1, 0, 0, false};
                    if (t >= 0)
                        tc = decode_tile<BN, TILE_ROWS, STRIPS>(L, t, hint);
                    const int ent[4] = {t, tc.valid ? tc.prob : -1, tc.tm, tc.tn};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tring[4 * ri + k] = ent[k];
                    if (PAIR) {
#pragma unroll
                        for (int k = 0; k < 4; ++k)
                            st_remote_u32(peer_addr((const void *)&tring[4 * ri + k], 1), ent[k]);
                        mbar_arrive_remote(peer_addr(&rfull[ri], 1));
                    }
                    mbar_arrive(&rfull[ri]);
                } else {
                    // Peer CTA: the leader's tile.
                    if (!mbar_wait_cluster(&rfull[ri], rphase, abort_flag, status0, kWaitTimeoutNs))
                        break;
                    t = tring[4 * ri];
                    tc.prob = tring[4 * ri + 1];
                    tc.tm = tring[4 * ri + 2];
                    tc.tn = tring[4 * ri + 3];
                    tc.valid = tc.prob >= 0;
                    mbar_arrive_remote(peer_addr(&rempty[ri], 0));
                }
                if (++ri == kRingTiles) {
                    ri = 0;
                    rphase ^= 1u;
                }
                if (t < 0)
                    break;
            } else {
                if (t >= total)
                    break;
                tc = decode_tile<BN, TILE_ROWS, STRIPS>(L, t, hint);
            }
            if (!tc.valid)
                continue;
            const TcProblem &P = prob_at(L, tc.prob);
            {
                // The epilogue reads this problem's fields after o_tma (and the Epi) when
                // it reaches the tile, a few tiles later: bring their lines into L1 now.
                const char *pb = reinterpret_cast<const char *>(&P.o_tma);
                const int nlines =
                    (int)((sizeof(TcProblem) - offsetof(TcProblem, o_tma) + 127) / 128) + 1;
                for (int k = 0; k < nlines; ++k)
                    asm volatile("prefetch.L1 [%0];" ::"l"(pb + 128 * k));
            }
            // A k-block is one 128-byte swizzle row: 64 BF16 or 128 e4m3 elements.
            const int kshift = P.fp8 ? 7 : 6;
            const int kblocks = (P.K + (1 << kshift) - 1) >> kshift;
            const int row0 = (PAIR ? 2 * tc.tm + (int)rank : tc.tm) * kBM;
            const int col0 = tc.tn * BN + (int)rank * B_ROWS;
            if (CHAIN) {
                // Operands are results of earlier problems: wait until they are complete
                // (whole problems), or until the strips this tile reads are (L: the
                // strip of this tile's row, R: of its column).
                if (STRIPS) {
                    if (tc.prob != dep_prob) {  // once per problem: counts only grow
                        for (int d = 0; d < 2 && ok; ++d)
                            if (P.dep[d] >= 0)
                                ok = wait_counter(&L.done[P.dep[d]], P.dep_target[d], abort_flag,
                                                  status0, dep_limit(L));
                        dep_prob = tc.prob;
                        smode[0] = P.sdep_mode[0];
                        smode[1] = P.sdep_mode[1];
                        src_done[0] = !smode[0];
                        src_done[1] = !smode[1];
                    }
                    for (int q = 0; q < 2 && ok; ++q)
                        if (!src_done[q])
                            ok = wait_strip(L, P, q, q ? tc.tn : tc.tm, src_done[q], abort_flag,
                                            status0);
                } else {
                    for (int d = 0; d < 2 && ok; ++d)
                        if (P.dep[d] >= 0)
                            ok = wait_counter(&L.done[P.dep[d]], P.dep_target[d], abort_flag,
                                              status0, dep_limit(L));
                }
                fence_async_global();  // the TMA reads below come after the acquire
                if (!ok)
                    break;
            }
            for (int sg = 0; sg < P.nseg && ok; ++sg) {
                const CUtensorMap *mL = &P.mapL[P.segL[sg]];
                const CUtensorMap *mR = &P.mapR[P.segR[sg]];
                for (int kb = 0; kb < kblocks; ++kb) {
                    if (!wait_bar<PAIR>(&empty[stage], phase ^ 1u, abort_flag, status0, kWaitTimeoutNs)) {
                        ok = false;
                        break;
                    }
                    if (PAIR) {
                        // Both CTAs' bytes complete on the leader's barrier.
                        const uint32_t fb = peer_addr(&full[stage], 0);
                        if (leader)
                            mbar_expect_tx(&full[stage], 2u * (uint32_t)(A_BYTES + B_BYTES));
                        tma_load_2d_pair(sA + stage * A_BYTES, mL, kb << kshift, row0, fb);
                        tma_load_2d_pair(sB + stage * B_BYTES, mR, kb << kshift, col0, fb);
                    } else {
                        mbar_expect_tx(&full[stage], (uint32_t)(A_BYTES + B_BYTES));
                        tma_load_2d(sA + stage * A_BYTES, mL, kb << kshift, row0, &full[stage]);
                        tma_load_2d(sB + stage * B_BYTES, mR, kb << kshift, col0, &full[stage]);
                    }
                    issued |= 1u << stage;
                    issued_parity = (issued_parity & ~(1u << stage)) | (phase << stage);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
        // Drain: the last copy into every stage must have landed before exit. The
        // peer of a pair sees its copies land through the leader's MMA consuming them.
        for (int s = 0; s < STAGES; ++s)
            if ((issued >> s) & 1u) {
                volatile int no_abort = 0;
                if (!PAIR || leader)
                    mbar_wait(&full[s], (issued_parity >> s) & 1u, &no_abort, nullptr, kWaitTimeoutNs / 4);
                else
                    mbar_wait_cluster(&empty[s], (issued_parity >> s) & 1u, &no_abort, nullptr,
                                      kWaitTimeoutNs / 4);
            }
    } else if (warp == 1 && lane == 0 && (!PAIR || leader)) {
        // ------------------------------------------------ MMA issuer
        int stage = 0;
        uint32_t phase = 0;
        int buf = 0;
        uint32_t tphase = 0;
        bool ok = true;
        int ri = 0;
        uint32_t rphase = 0;
        int hint = 0;
        for (int t = t_first; ok; t += t_step) {
            TileCoord tc;
            if (CHAIN) {
                if (!mbar_wait(&rfull[ri], rphase, abort_flag, status0, kWaitTimeoutNs))
                    break;
                t = tring[4 * ri];
                tc.prob = tring[4 * ri + 1];
                tc.tm = tring[4 * ri + 2];
                tc.tn = tring[4 * ri + 3];
                tc.valid = tc.prob >= 0;
                mbar_arrive(&rempty[ri]);
                if (++ri == kRingTiles) {
                    ri = 0;
                    rphase ^= 1u;
                }
                if (t < 0)
                    break;
            } else {
                if (t >= total)
                    break;
                tc = decode_tile<BN, TILE_ROWS, STRIPS>(L, t, hint);
            }
            if (!tc.valid)
                continue;
            const TcProblem &P = prob_at(L, tc.prob);
            if (!wait_bar<PAIR>(&tempty[buf], tphase ^ 1u, abort_flag, status0, kWaitTimeoutNs))
                break;
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(buf * BN);
            // The tile's k-loop, one copy per operand kind chosen once per tile, so that
            // the BF16 loop carries no test of the kind: for each segment and k-block,
            // wait for the stage's copies, issue four MMAs over its 128 bytes of each row
            // (K = 16 BF16 or 32 e4m3 elements each) and release the stage.
            auto k_loop = [&](auto f8_tag) -> bool {
                constexpr bool F8 = decltype(f8_tag)::value;
                constexpr uint32_t id = F8 ? idesc_e4m3(TILE_ROWS, BN) : idesc_bf16(TILE_ROWS, BN);
                const int kblocks = F8 ? (P.K + 2 * kBK - 1) / (2 * kBK) : (P.K + kBK - 1) / kBK;
                uint32_t acc = 0;
                for (int sg = 0; sg < P.nseg; ++sg) {
                    for (int kb = 0; kb < kblocks; ++kb) {
                        if (!mbar_wait(&full[stage], phase, abort_flag, status0, kWaitTimeoutNs))
                            return false;
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(sA + stage * A_BYTES);
                        const uint32_t b0 = smem_u32(sB + stage * B_BYTES);
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
                            const uint64_t ad = sw128_desc(a0 + kk * 32), bd = sw128_desc(b0 + kk * 32);
                            if (F8) {
                                if (PAIR)
                                    mma_e4m3_pair(d_tmem, ad, bd, id, acc);
                                else
                                    mma_e4m3(d_tmem, ad, bd, id, acc);
                            } else {
                                if (PAIR)
                                    mma_bf16_pair(d_tmem, ad, bd, id, acc);
                                else
                                    mma_bf16(d_tmem, ad, bd, id, acc);
                            }
                            acc = 1;
                        }
                        if (PAIR)
                            mma_commit_both(&empty[stage]);
                        else
                            mma_commit(&empty[stage]);
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                }
                return true;
            };
            ok = P.fp8 ? k_loop(BoolTag<true>{}) : k_loop(BoolTag<false>{});
            if (!ok)
                break;
            if (PAIR)
                mma_commit_both(&tfull[buf]);
            else
                mma_commit(&tfull[buf]);
            if (++buf == 2) {
                buf = 0;
                tphase ^= 1u;
            }
        }
        // Drain: every MMA issued so far completes before tensor memory is freed.
        if (PAIR)
            mma_commit_pair_local(drain);
        else
            mma_commit(drain);
        volatile int no_abort = 0;
        mbar_wait(drain, 0, &no_abort, nullptr, kWaitTimeoutNs / 4);
    } else if (warp >= 2) {
        // ------------------------------------------------ epilogue
        const int quad = warp & 3;  // TMEM lane quadrant this warp may access
        const int half = (warp - 2) >> 2;  // two warps per quadrant split the column chunks
        uint8_t *stage_buf = stage_all + (warp - 2) * NSTG * 4096;
        int slot = 0;  // next staging slot of this warp
        int buf = 0;
        uint32_t tphase = 0;
        int last_prob = -1;
        bool c_done = true;
        int ri = 0;
        uint32_t rphase = 0;
        int hint = 0;
        for (int t = t_first;; t += t_step) {
            TileCoord tc;
            if (CHAIN) {
                if (!wait_bar<PAIR>(&rfull[ri], rphase, abort_flag, status0, kWaitTimeoutNs))
                    break;
                t = tring[4 * ri];
                tc.prob = tring[4 * ri + 1];
                tc.tm = tring[4 * ri + 2];
                tc.tn = tring[4 * ri + 3];
                tc.valid = tc.prob >= 0;
                __syncwarp();
                if (lane == 0) {
                    if (PAIR && !leader)
                        mbar_arrive_remote(peer_addr(&rempty[ri], 0));
                    else
                        mbar_arrive(&rempty[ri]);
                }
                if (++ri == kRingTiles) {
                    ri = 0;
                    rphase ^= 1u;
                }
                if (t < 0)
                    break;
            } else {
                if (t >= total)
                    break;
                tc = decode_tile<BN, TILE_ROWS, STRIPS>(L, t, hint);
            }
            if (!tc.valid)
                continue;
            const TcProblem &P = prob_at(L, tc.prob);
            if (CHAIN && !STRIPS && (P.ep.c_kind != C_NONE || P.ep.theta_src)) {
                // C or the norm bound is an earlier result: make it visible to these loads.
                for (int d = 0; d < 2; ++d)
                    if (P.dep[d] >= 0 && lane == 0)
                        wait_counter(&L.done[P.dep[d]], P.dep_target[d], abort_flag, status0,
                                     dep_limit(L));
                __syncwarp();
            }
            if (STRIPS) {
                // C or the norm bound is an earlier result: make it visible to these loads;
                // earlier readers of the buffers this tile overwrites must be done.
                if (lane == 0) {
                    if (tc.prob != last_prob) {  // once per problem: counts only grow
                        if (P.ep.c_kind != C_NONE || P.ep.theta_src)
                            for (int d = 0; d < 2; ++d)
                                if (P.dep[d] >= 0)
                                    wait_counter(&L.done[P.dep[d]], P.dep_target[d], abort_flag,
                                                 status0, dep_limit(L));
                        for (int d = 0; d < P.nwdep; ++d)
                            wait_counter(&L.done[P.wdep[d]], P.wdep_target[d], abort_flag,
                                         status0, dep_limit(L));
                        c_done = !P.sdep_mode[2];
                    }
                    if (!c_done)
                        wait_strip(L, P, 2, tc.tm, c_done, abort_flag, status0);
                }
                __syncwarp();
            }
            if (PAIR)
                tc.tm = 2 * tc.tm + (int)rank;  // this CTA's 128-row half of the tile
            EpiHot h;  // per tile: its registers are free outside the tile's loops
            load_hot(h, P, calls);
            const int spec = epi_spec(h);
            last_prob = tc.prob;
            const int64_t warp_row0 = (int64_t)tc.tm * kBM + quad * 32;
            const int64_t row = warp_row0 + lane;
            const bool row_ok = row < h.M;
            // This warp's 32-column chunks: every other one, skipping chunks right of
            // N or wholly below the diagonal (warp-uniform).
            auto next_chunk = [&](int ch) {
                for (; ch < BN / 32; ch += 2) {
                    const int64_t c0 = (int64_t)tc.tn * BN + ch * 32;
                    if (c0 < h.N && warp_row0 < h.M && !(h.sym && warp_row0 > c0 + 31))
                        break;
                }
                return ch;
            };
            auto full_row = [&](int ch) {
                return row_ok && (int64_t)h.N - ((int64_t)tc.tn * BN + ch * 32) >= 32;
            };
            int ch = next_chunk(half);
            // The first chunk's C is loaded while the accumulator is still being computed.
            CRaw cr;
            bool cvec = false;
            if (ch < BN / 32)
                cvec = c_load(h, row, (int64_t)tc.tn * BN + ch * 32, full_row(ch), cr);
            if (!wait_bar<PAIR>(&tfull[buf], tphase, abort_flag, status0, kWaitTimeoutNs))
                break;
            tc_fence_after();
            double nrm = 0.0;
            // The chunk loop, one copy per product kind (epi_spec, chosen once per tile):
            // the specialised copies carry no tests of output, C, norm and copy kinds.
            auto chunk_loop = [&](auto spec_tag) {
                using Spec = decltype(spec_tag);
#pragma unroll 1
                while (ch < BN / 32) {
                    const int nx = next_chunk(ch + 2);
                    const int64_t c0 = (int64_t)tc.tn * BN + ch * 32;
                    const int64_t rem = (int64_t)h.N - c0;
                    float v[32];
                    tmem_ld32(tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BN + ch * 32),
                              v);
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        v[i] *= h.alpha;
                    if constexpr (Spec::generic) {
                        c_apply(h, cr, cvec, row, c0, rem < 32 ? (int)rem : 32, row_ok, v);
                        // The next chunk's C is in flight while this chunk is stored.
                        if (nx < BN / 32)
                            cvec = c_load(h, row, (int64_t)tc.tn * BN + nx * 32, full_row(nx), cr);
                        epilogue_finish<NSTG>(h, warp_row0, c0, v, nrm, stage_buf, slot, lane);
                    } else {
                        if constexpr (Spec::ckind != C_NONE) {
                            c_apply_spec<Spec::ckind>(h, cr, cvec, row, c0, rem < 32 ? (int)rem : 32,
                                                      row_ok, v);
                            if (nx < BN / 32)
                                cvec = c_load_spec<Spec::ckind>(h, row, (int64_t)tc.tn * BN + nx * 32,
                                                                full_row(nx), cr);
                        }
                        epilogue_finish_spec<NSTG, Spec::okind, Spec::sym, Spec::has_t>(
                            h, warp_row0, c0, v, stage_buf, slot, lane);
                    }
                    ch = nx;
                }
            };
            switch (spec) {
            case 0: chunk_loop(EpiSpec<0>{}); break;
            case 1: chunk_loop(EpiSpec<1>{}); break;
            case 2: chunk_loop(EpiSpec<2>{}); break;
            case 3: chunk_loop(EpiSpec<3>{}); break;
            case 4: chunk_loop(EpiSpec<4>{}); break;
            case 5: chunk_loop(EpiSpec<5>{}); break;
            default: chunk_loop(EpiSpec<-1>{}); break;
            }
            if (h.norm_acc) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
                if (lane == 0 && nrm != 0.0)
                    atomicAdd(h.norm_acc, nrm);
            }
            tc_fence_before();
            if (PAIR) {
                // One release per warp, on the leader's barrier (it issues the next MMAs).
                __syncwarp();
                if (lane == 0)
                    mbar_arrive_remote(peer_addr(&tempty[buf], 0));
            } else {
                mbar_arrive(&tempty[buf]);
            }
            if (++buf == 2) {
                buf = 0;
                tphase ^= 1u;
            }
            if (CHAIN) {
                // Publish: this warp's part of the tile is in global memory. The lanes'
                // plain stores (diagonal blocks of symmetric products, ragged edges) are
                // ordered before lane 0's accesses by __syncwarp; lane 0's GPU-scope fence
                // is cumulative over them and over its TMA stores (waited for and fenced
                // into the generic proxy), and its counter increment releases them all to
                // the tiles that acquire the counter.
                __syncwarp();
                if (lane == 0) {
                    bulk_wait_all0();
                    fence_async_global();
                    __threadfence();
                    atomicAdd(&L.done[P.pid], 1);
                    if (STRIPS && h.strip_base >= 0) {  // the strips this tile completes a part of
                        int *sp = L.strips + h.strip_base;
                        const int sr = PAIR ? (tc.tm >> 1) : tc.tm;  // tile (pair) row
                        atomicAdd(sp + sr, 1);
                        if (!h.sym)
                            atomicAdd(sp + h.tiles_m + tc.tn, 1);
                        else if (tc.tn != sr)
                            atomicAdd(sp + tc.tn, 1);
                    }
                }
                __syncwarp();
            }
        }
        // All TMA stores of this warp complete before the CTA may exit.
        if (lane == 0)
            bulk_wait_all0();
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    if (PAIR)
        cluster_sync_all();  // neither CTA leaves while its peer may still signal it
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc<PAIR>(tmem_base, 2 * BN);
    }
}

static_assert(offsetof(TcProblem, mapT) == offsetof(TcProblem, mapO) + 2 * sizeof(CUtensorMap),
              "the epilogue addresses mapO[0..1] and mapT[0..1] as one array");

template <int BN, int STAGES, bool PAIR, int NSTG>
constexpr int smem_bytes()
{
    return STAGES * (kBM + (PAIR ? BN / 2 : BN)) * kBK * 2 +
           kEpiWarps * NSTG * 4096 /* epilogue staging */ + 1024 /* alignment slack */ +
           512 /* barriers, tile ring */;
}

// One launch of the product kernel over total_tiles tiles (tile-width code's
// tiles: CTA pairs for kBnPair). Persistent: at most one CTA (pair) per SM (pair).
template <int BN, int STAGES, bool CHAIN, bool PAIR, int NSTG, bool STRIPS = false>
cudaError_t launch_kernel(const TcLaunch &l, int total_tiles, int num_sms, cudaStream_t s)
{
    constexpr int smem = smem_bytes<BN, STAGES, PAIR, NSTG>();
    static_assert(smem <= 232448, "shared memory per CTA");
    auto kern = tc_gemm_kernel<BN, STAGES, CHAIN, PAIR, NSTG, STRIPS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    if (total_tiles <= 0)
        return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    int grid = total_tiles < num_sms ? total_tiles : num_sms;
    if (PAIR) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        // Pairs that can be resident at once (SMs pair up within a GPC).
        static int max_pairs = -1;
        if (max_pairs < 0) {
            cfg.gridDim = dim3((unsigned)(num_sms & ~1), 1, 1);
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess || nc <= 0) {
                cudaGetLastError();
                nc = num_sms / 2;
            }
            max_pairs = nc;
        }
        const int cap = std::min(max_pairs, num_sms / 2);  // a caller's SM budget caps it too
        const int pairs = std::max(1, std::min(total_tiles, cap));
        grid = 2 * pairs;
    }
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    return cudaLaunchKernelEx(&cfg, kern, l);
}

template <bool CHAIN>
cudaError_t launch_width(const TcLaunch &l, int bn, int total_tiles, int num_sms, cudaStream_t s)
{
    // 128 x 128 tiles serve small problems (short K): 5 stages and two staging slots
    // per epilogue warp, so that stores overlap; the wide tiles keep every byte for
    // pipeline stages.
    if (bn == 256)
        return launch_kernel<256, 4, CHAIN, false, 1>(l, total_tiles, num_sms, s);
    if (bn == 128)
        return launch_kernel<128, 5, CHAIN, false, 2>(l, total_tiles, num_sms, s);
    if (bn == kBnPair)
        return launch_kernel<256, 6, CHAIN, true, 1>(l, total_tiles, num_sms, s);
    return cudaErrorInvalidValue;
}

} // namespace

cudaError_t tc_gemm_launch_grouped(const TcLaunch &l, int bn, int total_tiles, int num_sms,
                                   cudaStream_t s)
{
    TcLaunch g = l;
    g.nprob = 0;
    return launch_width<false>(g, bn, total_tiles, num_sms, s);
}

cudaError_t tc_gemm_launch_fused(const TcLaunch &l, int bn, int total_tiles, int num_sms,
                                 cudaStream_t s, bool strips)
{
    TcLaunch g = l;
    g.nprob = 0;
    if (strips) {  // square tiles only: per-strip dependencies
        if (bn == 128)
            return launch_kernel<128, 5, true, false, 2, true>(g, total_tiles, num_sms, s);
        if (bn == kBnPair)
            return launch_kernel<256, 6, true, true, 1, true>(g, total_tiles, num_sms, s);
        return cudaErrorInvalidValue;
    }
    return launch_width<true>(g, bn, total_tiles, num_sms, s);
}

int tc_num_tiles(const TcProblem &p, int bn)
{
    if (!p.sym)
        return p.tiles_m * p.tiles_n;
    const int r = tile_cols(bn) / tile_rows(bn);
    return r * p.tiles_n * (p.tiles_n + 1) / 2;
}

int tc_valid_ctas(const TcProblem &p, int bn)
{
    int n = 0;
    if (!p.sym) {
        n = p.tiles_m * p.tiles_n;
    } else {
        const int r = tile_cols(bn) / tile_rows(bn);
        for (int tn = 0; tn < p.tiles_n; ++tn)
            n += std::min(r * (tn + 1), p.tiles_m);
    }
    return n * ctas_per_tile(bn);
}

cudaError_t tc_gemm_launch(const TcLaunch &l, int bn, int num_sms, cudaStream_t s)
{
    if (l.gtab)
        return cudaErrorInvalidValue;
    return launch_width<false>(l, bn, l.tile_start[l.nprob], num_sms, s);
}

} // namespace svt
