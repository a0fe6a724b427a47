// libsvt host side: context, workspace layout, launch plans and the solve
// sequence of Proposition 1 in the factored form A_tau = 1/2 (A - tau P)(I + S).
//
// One solve of an m x n matrix works on the tall orientation (M, N) =
// (max(m, n), min(m, n)); the wide case (n > m) is the footnote's A A^T branch,
// i.e. the tall problem of A^T, with the result written transposed.
//
//   ingest   : FP64 ||A||_F^2 and Gram diagonal; X0 = A / alpha (alpha a power
//              of two) as BF16 (or FP64) in both orientations.
//   Gram     : S0 = (A^T A - tau^2 I) / alpha^2, FP32-class product (three
//              BF16 products of hi/lo parts), diagonal recomputed in FP64 with
//              the tau^2 shift (Section 4 shifts by tau**2), ||S0||_F^2 in FP64.
//   chains   : per step t, for P (X: M x N) and S (symmetric N x N) together:
//                Y = X^T X;  Z = c_t Y^2 + b_t Y + a_t I;  X <- X Z,
//              the first step scaled by the chain's norm bound theta.
//   polish   : one cubic Newton-Schulz step per chain in the FP32-class tier;
//              the P polish writes B = A - tau P directly.
//   combine  : Y = 1/2 (B S + B) in the FP32-class tier, stored as FP32.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "fused_deps.h"
#include "plan.h"
#include "segments.h"
#include "tuning_json.h"

namespace svt {

// ------------------------------------------------------------ tensor maps

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;
std::once_flag g_encode_once;

void resolve_encode()
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        g_encode = reinterpret_cast<EncodeTiledFn>(fn);
}
} // namespace

bool encode_bf16_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld,
                     int box_rows)
{
    std::call_once(g_encode_once, resolve_encode);
    if (!g_encode || !ptr || rows <= 0 || cols <= 0 || (ld % 8) != 0 ||
        (reinterpret_cast<uintptr_t>(ptr) & 15) != 0)
        return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_e4m3_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld,
                     int box_rows)
{
    std::call_once(g_encode_once, resolve_encode);
    if (!g_encode || !ptr || rows <= 0 || cols <= 0 || (ld % 16) != 0 ||
        (reinterpret_cast<uintptr_t>(ptr) & 15) != 0)
        return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld};
    cuuint32_t box[2] = {(cuuint32_t)(2 * kBK), (cuuint32_t)box_rows};  // one 128-byte row
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(ptr), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool encode_store_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld,
                      bool f32)
{
    std::call_once(g_encode_once, resolve_encode);
    const int64_t esz = f32 ? 4 : 2;
    if (!g_encode || !ptr || rows <= 0 || cols <= 0 || ((ld * esz) % 16) != 0 ||
        (reinterpret_cast<uintptr_t>(ptr) & 15) != 0)
        return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                          2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          f32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

void attach_store_maps(TcProblem &p)
{
    const Epi &e = p.ep;
    p.o_tma = 0;
    p.t_tma = 0;
    // Output: tile-oriented M x N, or transposed N x M when o_trans.
    if (e.o_kind == O_BF16 || e.o_kind == O_PAIR || e.o_kind == O_F32) {
        const bool f32 = e.o_kind == O_F32;
        const int64_t rows = e.o_trans ? p.N : p.M, cols = e.o_trans ? p.M : p.N;
        bool ok = encode_store_map(&p.mapO[0], e.o0, rows, cols, e.ldo, f32);
        if (ok && e.o_kind == O_PAIR)
            ok = encode_store_map(&p.mapO[1], e.o1, rows, cols, e.ldo, false);
        p.o_tma = ok ? 1 : 0;
    }
    // Transposed copy: N x M.
    if (e.t_kind == O_BF16 || e.t_kind == O_PAIR) {
        bool ok = encode_store_map(&p.mapT[0], e.t0, p.N, p.M, e.ldt, false);
        if (ok && e.t_kind == O_PAIR)
            ok = encode_store_map(&p.mapT[1], e.t1, p.N, p.M, e.ldt, false);
        p.t_tma = ok ? 1 : 0;
    }
}


svt_status resolve_status(const svt_options *in, Resolved *r)
{
    if (in && in->prec == SVT_FP8_EXPERIMENTAL)
        return SVT_ERR_UNSUPPORTED;
    return resolve(in, r) ? SVT_OK : SVT_ERR_INVALID;
}

bool resolve(const svt_options *in, Resolved *r)
{
    svt_options o;
    if (in)
        o = *in;
    else
        svt_options_default(&o);
    if (o.iters < 0 || o.iters > 1000 || !std::isfinite(o.ell0) || !std::isfinite(o.delta))
        return false;
    if (o.prec != SVT_FP64 && o.prec != SVT_FP32 && o.prec != SVT_BF16)
        return false;
    r->iters = o.iters;
    r->prec = o.prec;
    r->schedule = (o.schedule == SVT_SCHED_NS3) ? SVT_SCHED_NS3 : SVT_SCHED_PE5;
    if (o.schedule != SVT_SCHED_AUTO && o.schedule != SVT_SCHED_PE5 && o.schedule != SVT_SCHED_NS3)
        return false;
    if (o.norm == SVT_NORM_AUTO)
        r->norm = (r->schedule == SVT_SCHED_PE5) ? SVT_NORM_GRAM : SVT_NORM_FRO;
    else if (o.norm == SVT_NORM_FRO || o.norm == SVT_NORM_GRAM)
        r->norm = o.norm;
    else
        return false;
    r->ell0 = (o.ell0 > 0.0) ? o.ell0 : 1e-3;
    if (!(r->ell0 < 1.0))
        return false;
    if (o.delta < 0.0)
        r->delta = (o.prec == SVT_BF16) ? 0.01 : (o.prec == SVT_FP32 ? 1e-4 : 0.0);
    else
        r->delta = o.delta;
    r->polish = o.polish ? 1 : 0;
    if (o.mode != SVT_MODE_SVT && o.mode != SVT_MODE_RANK_R)
        return false;
    r->mode = o.mode;
    if (o.hp_steps < -1)
        return false;
    r->hp_steps = (o.prec == SVT_BF16) ? o.hp_steps : 0;
    r->fuse = (o.fuse && o.prec != SVT_FP64) ? 1 : 0;
    if (o.tile != 0 && o.tile != 128 && o.tile != 256 && o.tile != kBnPair)
        return false;
    r->tile = (o.prec == SVT_FP64) ? 0 : o.tile;
    r->out64 = 0;
    r->fp8_p = r->fp8_s = 0;
    r->fp8_s_y2 = 0;
    return true;
}

namespace {
struct Alloc {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t o = off;
        off = align_up(off + bytes, kAlign);
        return o;
    }
};

} // namespace

static Buf make_buf(Alloc &a, int64_t rows, int64_t cols, size_t esz, bool pair)
{
    Buf b;
    b.rows = rows;
    b.cols = cols;
    b.ld = ld_of(cols);
    size_t bytes = (size_t)rows * (size_t)b.ld * esz;
    b.hi = a.take(bytes);
    b.has_lo = pair;
    if (pair)
        b.lo = a.take(bytes);
    return b;
}

Layout make_layout(int64_t m, int64_t n, const Resolved &r)
{
    Layout L;
    L.M = std::max(m, n);
    L.N = std::min(m, n);
    L.ldM = ld_of(L.M);
    L.ldN = ld_of(L.N);
    const bool f64 = r.prec == SVT_FP64;
    const bool fp32 = r.prec == SVT_FP32;
    L.esz = f64 ? 8 : 2;
    const bool skipP = r.mode == SVT_MODE_RANK_R;
    Alloc a;
    L.scal = a.take(SC_COUNT * sizeof(double));
    L.status = a.take(sizeof(int) * 4);
    // Product launches of a solve: Gram, 3 per step, 2 polish, combine; <= 2 problems each.
    L.max_problems = 2 * (1 + 3 * std::max(0, r.iters) + 2 + 1);
    // done[] and one tile counter per launch of a fused solve
    L.counters = a.take(sizeof(int) * (size_t)(L.max_problems + kMaxFusedSegments));
    L.colnorm = a.take((size_t)L.N * sizeof(double));
    const bool pairs = fp32;  // iterates carried as hi/lo pairs
    for (int i = 0; i < 2; ++i) {
        if (!skipP || i == 0)
            L.X[i] = make_buf(a, L.M, L.N, L.esz, pairs && !f64);
        if (!skipP || i == 0)
            L.Xt[i] = make_buf(a, L.N, L.M, L.esz, pairs && !f64);
    }
    if (!f64 && !pairs)
        L.XtLo0 = make_buf(a, L.N, L.M, L.esz, false);
    // S-chain buffers hold hi/lo pairs when any S step runs in the FP32-class tier.
    const bool pairsS = pairs || (r.prec == SVT_BF16 && r.hp_steps != 0);
    for (int i = 0; i < 2; ++i)
        L.S[i] = make_buf(a, L.N, L.N, L.esz, pairsS);
    if (!skipP) {
        L.Yp = make_buf(a, L.N, L.N, L.esz, pairs);
        L.Zp = make_buf(a, L.N, L.N, L.esz, pairs);
        L.ZPp = make_buf(a, L.N, L.N, L.esz, !f64);
    }
    L.Ys = make_buf(a, L.N, L.N, L.esz, pairsS);
    L.Zs = make_buf(a, L.N, L.N, L.esz, pairsS);
    L.ZSp = make_buf(a, L.N, L.N, L.esz, !f64);
    L.B = make_buf(a, L.M, L.N, L.esz, !f64);
    L.Sp = make_buf(a, L.N, L.N, L.esz, !f64);
    if (r.fp8_p && !skipP)
        L.Yp8 = make_buf(a, L.N, L.N, 1, false);
    if (r.fp8_s) {
        for (int i = 0; i < 2; ++i)
            L.S8[i] = make_buf(a, L.N, L.N, 1, false);
        L.Ys8 = make_buf(a, L.N, L.N, 1, false);
        L.Zs8 = make_buf(a, L.N, L.N, 1, false);
    }
    if (!f64 && r.fuse) {
        L.fused_tab_bytes = align_up(sizeof(TcProblem) * (size_t)L.max_problems, kAlign) +
                            align_up(sizeof(int) * (size_t)(L.max_problems + 1), kAlign);
        L.fused_tab = a.take(L.fused_tab_bytes);
        // Strip counters of a fused solve, at the end so that they move no buffer: per
        // problem at most one per 128-row tile row and 128-column tile column.
        L.max_strips = (int)((L.M + kBM - 1) / kBM + (L.N + kBM - 1) / kBM);
        L.strips_bytes = sizeof(int) * (size_t)L.max_problems * (size_t)L.max_strips;
        L.strips = a.take(L.strips_bytes);
    }
    L.total = a.off;
    return L;
}

} // namespace svt

namespace svt {
namespace {

// ---------------------------------------------------------- plan builder

struct Builder {
    svt_ctx *ctx;
    Plan *plan;
    uint8_t *base;       // workspace base for this plan
    int bn_default;

    void *ptr(size_t off) { return base + off; }
    double *scal(int slot) { return reinterpret_cast<double *>(base + plan->lay.scal) + slot; }
    int *status() { return reinterpret_cast<int *>(base + plan->lay.status); }

    Epi epi0()
    {
        Epi e;
        std::memset(&e, 0, sizeof(e));
        e.alpha = 1.0;
        e.status = status();
        return e;
    }

    // Output description for a Buf: BF16, pair or FP64.
    void set_out(Epi &e, const Buf &b, bool pair)
    {
        const bool f64 = plan->opt.prec == SVT_FP64;
        e.o_kind = f64 ? O_F64 : (pair ? O_PAIR : O_BF16);
        e.o0 = ptr(b.hi);
        e.o1 = pair ? ptr(b.lo) : nullptr;
        e.ldo = b.ld;
    }
    void set_t(Epi &e, const Buf &b, bool pair)
    {
        const bool f64 = plan->opt.prec == SVT_FP64;
        e.t_kind = f64 ? O_F64 : (pair ? O_PAIR : O_BF16);
        e.t0 = ptr(b.hi);
        e.t1 = pair ? ptr(b.lo) : nullptr;
        e.ldt = b.ld;
    }
    // The e4m3 copy of a product's result (FP8 experiment), scaled by `scale`.
    void set_f(Epi &e, const Buf &b, float scale)
    {
        e.f0 = ptr(b.hi);
        e.ldf = b.ld;
        e.fscale = scale;
    }
    void set_c(Epi &e, const Buf &b, double beta)
    {
        const bool f64 = plan->opt.prec == SVT_FP64;
        e.c_kind = f64 ? C_F64 : (b.has_lo ? C_PAIR : C_BF16);
        e.c0 = ptr(b.hi);
        e.c1 = b.has_lo ? ptr(b.lo) : nullptr;
        e.ldc = b.ld;
        e.beta = beta;
    }

    // One product D = L R^T over the segment pattern implied by the operands'
    // hi/lo parts (1, 2 or 3 BF16 products).
    bool tc_problem(TcProblem &p, const Buf &L, const Buf &R, int M, int N, int K, bool sym,
                    const Epi &e, int bn, bool fp8 = false)
    {
        std::memset(&p, 0, sizeof(p));
        if (fp8) {  // e4m3 operands (FP8 experiment): one segment, hi buffers only
            if (!encode_e4m3_map(&p.mapL[0], ptr(L.hi), L.rows, L.cols, L.ld, kBM) ||
                !encode_e4m3_map(&p.mapR[0], ptr(R.hi), R.rows, R.cols, R.ld, r_box_rows(bn)))
                return false;
            p.fp8 = 1;
            p.nseg = 1;
            p.M = M;
            p.N = N;
            p.K = K;
            p.sym = sym ? 1 : 0;
            p.strip_base = -1;
            p.tiles_m = (M + tile_rows(bn) - 1) / tile_rows(bn);
            p.tiles_n = (N + tile_cols(bn) - 1) / tile_cols(bn);
            p.ep = e;
            attach_store_maps(p);
            return true;
        }
        if (!encode_bf16_map(&p.mapL[0], ptr(L.hi), L.rows, L.cols, L.ld, kBM))
            return false;
        if (!encode_bf16_map(&p.mapR[0], ptr(R.hi), R.rows, R.cols, R.ld, r_box_rows(bn)))
            return false;
        if (L.has_lo && !encode_bf16_map(&p.mapL[1], ptr(L.lo), L.rows, L.cols, L.ld, kBM))
            return false;
        if (R.has_lo && !encode_bf16_map(&p.mapR[1], ptr(R.lo), R.rows, R.cols, R.ld, r_box_rows(bn)))
            return false;
        int ns = 0;
        p.segL[ns] = 0; p.segR[ns] = 0; ++ns;
        if (R.has_lo) { p.segL[ns] = 0; p.segR[ns] = 1; ++ns; }
        if (L.has_lo) { p.segL[ns] = 1; p.segR[ns] = 0; ++ns; }
        p.nseg = ns;
        p.M = M;
        p.N = N;
        p.K = K;
        p.sym = sym ? 1 : 0;
        p.strip_base = -1;
        p.tiles_m = (M + tile_rows(bn) - 1) / tile_rows(bn);
        p.tiles_n = (N + tile_cols(bn) - 1) / tile_cols(bn);
        p.ep = e;
        attach_store_maps(p);
        return true;
    }

    void f64_problem(F64Problem &p, const Buf &L, const Buf &R, int M, int N, int K, bool sym,
                     const Epi &e)
    {
        std::memset(&p, 0, sizeof(p));
        p.L = static_cast<const double *>(ptr(L.hi));
        p.R = static_cast<const double *>(ptr(R.hi));
        p.ldl = L.ld;
        p.ldr = R.ld;
        p.M = M;
        p.N = N;
        p.K = K;
        p.sym = sym ? 1 : 0;
        p.ep = e;
    }

    // Grouped launch of up to two products (P chain and S chain of one step).
    struct Prod {
        const Buf *L, *R;
        int M, N, K;
        bool sym;
        Epi e;
        int patch;
        int chain = 0;  // 0 P chain, 1 S chain, 2 both (combine)
        bool fp8 = false;  // e4m3 operands (FP8 experiment)
    };

    bool emit(const std::vector<Prod> &prods)
    {
        if (prods.empty())
            return true;
        if (plan->opt.prec == SVT_FP64) {
            F64Launch l;
            std::memset(&l, 0, sizeof(l));
            l.nprob = (int)prods.size();
            for (size_t i = 0; i < prods.size(); ++i) {
                const Prod &q = prods[i];
                f64_problem(l.p[i], *q.L, *q.R, q.M, q.N, q.K, q.sym, q.e);
                if (q.patch)
                    plan->patches.push_back({OP_F64, (int)plan->f64.size(), (int)i, q.patch});
            }
            plan->ops.push_back({OP_F64, (int)plan->f64.size(), 0});
            plan->f64.push_back(l);
            plan->kernel_launches += 1;
            return true;
        }
        int bn = 128;
        for (const Prod &q : prods)
            if (q.N > 128)
                bn = 256;
        if (plan->force_bn > 0)
            bn = plan->force_bn;
        else if (plan->force_bn < 0 && plan->tc.size() < plan->bn_choice.size())
            bn = plan->bn_choice[plan->tc.size()];
        TcLaunch l;
        std::memset(&l, 0, sizeof(l));
        l.nprob = (int)prods.size();
        int start = 0;
        for (size_t i = 0; i < prods.size(); ++i) {
            const Prod &q = prods[i];
            if (!tc_problem(l.p[i], *q.L, *q.R, q.M, q.N, q.K, q.sym, q.e, bn, q.fp8))
                return false;
            plan->tc_chain.push_back(q.chain);
            plan->tc_io.push_back({ptr(q.L->hi), ptr(q.R->hi),
                                   (q.patch & PT_C_IS_A) ? nullptr : q.e.c0,
                                   (q.patch & PT_O_IS_Y) ? nullptr : q.e.o0, q.e.t0,
                                   q.e.o_trans, q.e.theta_src, q.e.norm_acc, q.e.f0});
            l.tile_start[i] = start;
            start += tc_num_tiles(l.p[i], bn);
            if (q.patch)
                plan->patches.push_back({OP_TC, (int)plan->tc.size(), (int)i, q.patch});
        }
        l.tile_start[prods.size()] = start;
        // Algorithmic flops: 2 M N K per product, symmetric products counted at half;
        // the hi/lo segments of FP32-class products are not counted again.
        double fl = 0.0, tfl = 0.0;
        for (const Prod &q : prods)
            fl += (q.sym ? 1.0 : 2.0) * (double)q.M * (double)q.N * (double)q.K;
        for (int i = 0; i < l.nprob; ++i) {
            const TcProblem &tp = l.p[i];
            const int kb = tp.fp8 ? 2 * kBK : kBK;
            const double kpad = (double)((tp.K + kb - 1) / kb * kb);
            // each CTA tile: 128 rows x tile_cols(bn) columns over the padded K
            tfl += (double)tp.nseg * (double)tc_valid_ctas(tp, bn) * 2.0 * kBM *
                   (double)tile_cols(bn) * kpad;
        }
        plan->tc_flops.push_back(fl);
        plan->tc_tensor_flops.push_back(tfl);
        plan->ops.push_back({OP_TC, (int)plan->tc.size(), bn});
        plan->tc.push_back(l);
        plan->kernel_launches += 1;
        plan->tc_launches_per_solve += 1;
        return true;
    }

    // The same buffer used with or without its lo part.
    static Buf view(const Buf &b, bool pair)
    {
        Buf v = b;
        v.has_lo = pair && b.has_lo;
        return v;
    }

    bool build()
    {
        Plan &P = *plan;
        const Layout &L = P.lay;
        const Resolved &o = P.opt;
        const bool f64 = o.prec == SVT_FP64;
        const bool pairs = o.prec == SVT_FP32;
        const bool skipP = o.mode == SVT_MODE_RANK_R;
        const int M = (int)L.M, N = (int)L.N;
        // Leading S-chain steps run in the FP32-class tier: all of them in the FP32
        // tier; in the BF16 tier the first hp_steps (auto: the steps whose design
        // interval starts below 0.1, while the shifted Gram's small eigenvalues are
        // still below BF16 resolution relative to the largest).
        int hpS = 0;
        if (pairs) {
            hpS = o.iters;
        } else if (o.prec == SVT_BF16) {
            if (o.hp_steps >= 0) {
                hpS = std::min(o.hp_steps, o.iters);
            } else {
                for (int t = 0; t < o.iters; ++t)
                    if (P.lo[t] < 0.1)
                        hpS = t + 1;
            }
        }
        // S after t steps is a pair iff step t (its consumer) runs FP32-class.
        auto s_pair = [&](int t) { return pairs || t < hpS; };
        P.hp_steps_s = hpS;
        P.final_s_pair = s_pair(o.iters);

        P.ops.push_back({OP_MEMSET, 0, 0});
        P.ops.push_back({OP_REDUCE, 0, 0});
        P.ops.push_back({OP_SPLIT, 0, 0});
        P.kernel_launches += 2;

        // Gram: S0 = Xt0 Xt0^T with FP64 diagonal colnorm2 / alpha^2 - tau^2 / alpha^2.
        {
            Buf Lg = L.Xt[0];
            if (!f64 && !pairs) {  // BF16 tier keeps the lo part of X0^T separately
                Lg.has_lo = true;
                Lg.lo = L.XtLo0.hi;
            }
            Epi e = epi0();
            set_out(e, L.S[0], s_pair(0));
            e.diag = reinterpret_cast<const double *>(base + L.colnorm);
            e.dss = scal(SC_INV_ALPHA2);  // [INV_ALPHA2, TAU2_SCALED]
            e.norm_acc = scal(SC_NRM_S0);
            if (!emit({{&Lg, &Lg, N, N, M, true, e, 0, 1}}))
                return false;
        }

        // FP8 experiment: S-chain step t runs all three products on e4m3 copies (a BF16
        // quintic step after the first); the copies it reads are written by the products
        // that produce S, Y and Z. Scales are powers of two from the iterates' bounds:
        // the normalised iterates and their squares stay below ~1.03 (x 256 < 448, the
        // largest e4m3), the P chain's first Y = X0^T X0 below ||X0||_F^2 < 2 (x 128), and
        // Z = a + b y + c y^2 below its maximum over y in [0, 1.1].
        auto f8s_all_at = [&](int t) {
            return t >= 1 && t < o.iters && o.schedule == SVT_SCHED_PE5 && !s_pair(t) &&
                   ((o.fp8_s >> t) & 1ull) && !o.fp8_s_y2;
        };
        auto e4m3_scale = [](double bound) {
            double sc = 1.0;
            while (sc * 2.0 * bound <= 448.0 && sc < 32768.0)
                sc *= 2.0;
            return (float)sc;
        };
        const float s_it = 256.f;
        // Chains.
        int cur = 0;
        for (int t = 0; t < o.iters; ++t) {
            const double a = P.coef[3 * t], b = P.coef[3 * t + 1], c = P.coef[3 * t + 2];
            const bool first = (t == 0);
            const bool quintic = (o.schedule == SVT_SCHED_PE5) || (first && o.norm == SVT_NORM_GRAM);
            const int nxt = 1 - cur;
            const bool hp = s_pair(t);  // this S step in the FP32-class tier
            const Buf Sc = view(L.S[cur], hp), Ysv = view(L.Ys, hp), Zsv = view(L.Zs, hp);
            const bool f8p = quintic && !skipP && ((o.fp8_p >> t) & 1ull);
            const bool f8s = quintic && !hp && t >= 1 && ((o.fp8_s >> t) & 1ull);
            const bool f8s_all = f8s_all_at(t), f8s_next = f8s_all_at(t + 1);
            const float s_yp = first ? 128.f : 256.f;
            double zmax = std::max(std::fabs(a), std::fabs(a + 1.1 * b + 1.21 * c));
            if (c != 0.0) {
                const double yv = -b / (2.0 * c);
                if (yv > 0.0 && yv < 1.1)
                    zmax = std::max(zmax, std::fabs(a + b * yv + c * yv * yv));
            }
            const float s_z = e4m3_scale(zmax);
            // theta sources for the first step
            const double *thP = nullptr, *thS = nullptr;
            double powP = 0.5, powS = 0.5;
            if (first) {
                if (o.norm == SVT_NORM_FRO) {
                    thP = scal(SC_NRM_X0);
                    thS = scal(SC_NRM_S0);
                } else {
                    thP = scal(SC_NRM_YP);
                    thS = scal(SC_NRM_YS);
                    powP = powS = 0.25;
                }
            }
            auto theta = [&](Epi &e, const double *src, double pw, double ea, double eb, double eg) {
                if (!src)
                    return;
                e.theta_src = src;
                e.theta_pow = pw;
                e.ea = ea;
                e.eb = eb;
                e.eg = eg;
            };
            if (quintic) {
                // Y = X^T X (P: Xt Xt^T; S: S S)
                std::vector<Prod> s1;
                if (!skipP) {
                    Epi e = epi0();
                    set_out(e, L.Yp, pairs);
                    if (first && o.norm == SVT_NORM_GRAM)
                        e.norm_acc = scal(SC_NRM_YP);
                    if (f8p)
                        set_f(e, L.Yp8, s_yp);
                    s1.push_back({&L.Xt[cur], &L.Xt[cur], N, N, M, true, e, 0});
                }
                {
                    Epi e = epi0();
                    set_out(e, L.Ys, hp);
                    if (first && o.norm == SVT_NORM_GRAM)
                        e.norm_acc = scal(SC_NRM_YS);
                    if (f8s)
                        set_f(e, L.Ys8, s_it);
                    if (f8s_all) {
                        e.alpha = 1.0 / ((double)s_it * s_it);
                        s1.push_back({&L.S8[cur], &L.S8[cur], N, N, N, true, e, 0, 1, true});
                    } else {
                        s1.push_back({&Sc, &Sc, N, N, N, true, e, 0, 1});
                    }
                }
                if (!emit(s1))
                    return false;
                // Z = c Y^2 + b Y + a I
                std::vector<Prod> s2;
                if (!skipP) {
                    Epi e = epi0();
                    e.alpha = c;
                    e.gamma = a;
                    set_c(e, L.Yp, b);
                    set_out(e, L.Zp, pairs);
                    theta(e, thP, powP, 5, 3, 1);
                    if (f8p) {  // Y^2 from the e4m3 copy of Y: undo its scale squared
                        e.alpha = c / ((double)s_yp * s_yp);
                        s2.push_back({&L.Yp8, &L.Yp8, N, N, N, true, e, 0, 0, true});
                    } else {
                        s2.push_back({&L.Yp, &L.Yp, N, N, N, true, e, 0});
                    }
                }
                {
                    Epi e = epi0();
                    e.alpha = c;
                    e.gamma = a;
                    set_c(e, Ysv, b);
                    set_out(e, L.Zs, hp);
                    theta(e, thS, powS, 5, 3, 1);
                    if (f8s_all)
                        set_f(e, L.Zs8, s_z);
                    if (f8s) {
                        e.alpha = c / ((double)s_it * s_it);
                        s2.push_back({&L.Ys8, &L.Ys8, N, N, N, true, e, 0, 1, true});
                    } else {
                        s2.push_back({&Ysv, &Ysv, N, N, N, true, e, 0, 1});
                    }
                }
                if (!emit(s2))
                    return false;
            } else {
                // cubic: Z = b Y + a I straight from the Y product
                std::vector<Prod> s1;
                if (!skipP) {
                    Epi e = epi0();
                    e.alpha = b;
                    e.gamma = a;
                    set_out(e, L.Zp, pairs);
                    theta(e, thP, powP, 3, 0, 1);
                    s1.push_back({&L.Xt[cur], &L.Xt[cur], N, N, M, true, e, 0});
                }
                {
                    Epi e = epi0();
                    e.alpha = b;
                    e.gamma = a;
                    set_out(e, L.Zs, hp);
                    theta(e, thS, powS, 3, 0, 1);
                    s1.push_back({&Sc, &Sc, N, N, N, true, e, 0, 1});
                }
                if (!emit(s1))
                    return false;
            }
            // X <- X Z (P: also write X^T), S <- S Z (symmetric)
            std::vector<Prod> s3;
            if (!skipP) {
                Epi e = epi0();
                set_out(e, L.X[nxt], pairs);
                set_t(e, L.Xt[nxt], pairs);
                s3.push_back({&L.X[cur], &L.Zp, M, N, N, false, e, 0});
            }
            {
                Epi e = epi0();
                set_out(e, L.S[nxt], s_pair(t + 1));
                if (f8s_next)
                    set_f(e, L.S8[nxt], s_it);
                if (f8s_all) {
                    e.alpha = 1.0 / ((double)s_it * s_z);
                    s3.push_back({&L.S8[cur], &L.Zs8, N, N, N, true, e, 0, 1, true});
                } else {
                    s3.push_back({&Sc, &Zsv, N, N, N, true, e, 0, 1});
                }
            }
            if (!emit(s3))
                return false;
            cur = nxt;
        }

        // Polish (FP32-class): Z = 3/2 I - 1/2 X^T X; P' = X Z -> B = A - tau P'; S' = S Z.
        const Buf Sfin = view(L.S[cur], s_pair(o.iters));
        if (o.polish || f64) {
            std::vector<Prod> s1;
            if (!skipP) {
                Epi e = epi0();
                e.alpha = -0.5;
                e.gamma = 1.5;
                set_out(e, L.ZPp, !f64);
                s1.push_back({&L.Xt[cur], &L.Xt[cur], N, N, M, true, e, 0});
            }
            {
                Epi e = epi0();
                e.alpha = -0.5;
                e.gamma = 1.5;
                set_out(e, L.ZSp, !f64);
                s1.push_back({&Sfin, &Sfin, N, N, N, true, e, 0, 1});
            }
            if (!emit(s1))
                return false;
            std::vector<Prod> s2;
            if (!skipP) {
                Epi e = epi0();
                e.alpha = -1.0;  // patched to -tau per call
                e.beta = 1.0;    // C = A (patched)
                e.c_kind = f64 ? C_F32 : C_F32;
                e.c_trans = P.wide ? 1 : 0;
                set_out(e, L.B, !f64);
                s2.push_back({&L.X[cur], &L.ZPp, M, N, N, false, e, PT_C_IS_A | PT_ALPHA_NEG_TAU});
            }
            {
                Epi e = epi0();
                set_out(e, L.Sp, !f64);
                s2.push_back({&Sfin, &L.ZSp, N, N, N, true, e, 0, 1});
            }
            if (!emit(s2))
                return false;
            if (skipP) {
                P.ops.push_back({OP_PREP, 1, 0});  // B = A (no P term)
                P.kernel_launches += 1;
            }
        } else {
            P.ops.push_back({OP_PREP, skipP ? 1 : 0, 0});  // B = A - tau X, S' = S
            P.kernel_launches += 1;
        }

        // Combine: Y = 1/2 B S' + 1/2 B (FP32 out, or FP64 for svt_polar_f64; transposed
        // back for wide input).
        {
            Epi e = epi0();
            e.alpha = 0.5;
            set_c(e, L.B, 0.5);
            e.o_kind = (f64 && o.out64) ? O_F64 : O_F32;
            e.o_trans = P.wide ? 1 : 0;
            e.norm_acc = scal(SC_NRM_OUT);
            if (!emit({{&L.B, &L.Sp, M, N, N, false, e, PT_O_IS_Y, 2}}))
                return false;
        }
        P.ops.push_back({OP_FINAL, 0, 0});
        P.kernel_launches += 1;
        return true;
    }
};

// B = A_tall - tau * X (or A_tall alone), S' = S, when the polish is off or
// the P chain is skipped.
__global__ void prep_kernel(const float *__restrict__ A, int64_t lda, int wide, int64_t M,
                            int64_t N, float tau, int xkind, const void *x0, const void *x1,
                            int64_t ldx, int bkind, void *b0, void *b1, int64_t ldb,
                            const void *s0, const void *s1, int skind, void *sp0, void *sp1,
                            int64_t lds)
{
    const int64_t total = M * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / N, c = i % N;
        double a = wide ? (double)A[c * lda + r] : (double)A[r * lda + c];
        double x = 0.0;
        if (xkind == C_BF16)
            x = __bfloat162float(static_cast<const __nv_bfloat16 *>(x0)[r * ldx + c]);
        else if (xkind == C_PAIR)
            x = (double)__bfloat162float(static_cast<const __nv_bfloat16 *>(x0)[r * ldx + c]) +
                (double)__bfloat162float(static_cast<const __nv_bfloat16 *>(x1)[r * ldx + c]);
        else if (xkind == C_F64)
            x = static_cast<const double *>(x0)[r * ldx + c];
        double v = a - (double)tau * x;
        if (bkind == O_F64) {
            static_cast<double *>(b0)[r * ldb + c] = v;
        } else {
            __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
            static_cast<__nv_bfloat16 *>(b0)[r * ldb + c] = hi;
            static_cast<__nv_bfloat16 *>(b1)[r * ldb + c] =
                __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
        }
        if (s0 && r < N) {
            if (skind == C_F64) {
                static_cast<double *>(sp0)[r * lds + c] = static_cast<const double *>(s0)[r * lds + c];
            } else {
                __nv_bfloat16 h = static_cast<const __nv_bfloat16 *>(s0)[r * lds + c];
                __nv_bfloat16 l = (skind == C_PAIR) ? static_cast<const __nv_bfloat16 *>(s1)[r * lds + c]
                                                    : __float2bfloat16_rn(0.0f);
                static_cast<__nv_bfloat16 *>(sp0)[r * lds + c] = h;
                static_cast<__nv_bfloat16 *>(sp1)[r * lds + c] = l;
            }
        }
    }
}


} // namespace

svt_status run_ops(svt_ctx *ctx, Plan &P, const CallArgs &a, cudaStream_t s, size_t first,
                   size_t last, int sms)
{
    const int grid_sms = (sms > 0 && sms < ctx->num_sms) ? sms : ctx->num_sms;
    uint8_t *base = ctx->ws + P.ws_base;
    const Layout &L = P.lay;
    double *scal = reinterpret_cast<double *>(base + L.scal);
    int *status = reinterpret_cast<int *>(base + L.status);
    double *colnorm = reinterpret_cast<double *>(base + L.colnorm);
    const bool f64 = P.opt.prec == SVT_FP64;
    const bool pairs = P.opt.prec == SVT_FP32;
    const bool skipP = P.opt.mode == SVT_MODE_RANK_R;
    cudaError_t err = cudaSuccess;
    int cur_final = P.opt.iters % 2;
    int launched = 0;
    const bool fused = P.fused && first == 0 && last >= P.ops.size();
    const bool prof = ctx->profile && !a.in_graph;
    bool fused_done = false;
    ctx->table_owner = nullptr;  // this solve overwrites part of the workspace
    for (size_t oi = first; oi < last && oi < P.ops.size(); ++oi) {
        const Op &op = P.ops[oi];
        if (fused && op.kind == OP_TC) {
            if (fused_done)
                continue;
            fused_done = true;
            // The table region is shared with other plans: refresh it from the host image.
            if (!a.in_graph && upload_fused_table(ctx, P, s) != SVT_OK)
                return SVT_ERR_CUDA;
            TcLaunch l = P.fused_launch;
            l.dep_wait_ns = ctx->dbg_wait_ns;
            l.call_inline.A = a.A;
            l.call_inline.Y = a.Y;
            l.call_inline.lda = a.lda;
            l.call_inline.ldy = a.ldy;
            l.call_inline.tau = a.tau;
            l.call_inline.d_status = a.d_status;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (prof) {
                if (ctx->prof_next + 2 > ctx->prof_pool.size()) {
                    for (int k = 0; k < 64; ++k) {
                        cudaEvent_t ev;
                        if (cudaEventCreate(&ev) != cudaSuccess)
                            return SVT_ERR_CUDA;
                        ctx->prof_pool.push_back(ev);
                    }
                }
                e0 = ctx->prof_pool[ctx->prof_next++];
                e1 = ctx->prof_pool[ctx->prof_next++];
                cudaEventRecord(e0, s);
            }
            err = tc_gemm_launch_fused(l, P.fused_bn, P.fused_tiles, grid_sms, s, P.uses_strips);
            if (prof) {
                cudaEventRecord(e1, s);
                ctx->prof_pending.push_back({e0, e1, P.fused_flops, P.fused_tensor_flops});
            }
            ++launched;
            if (err != cudaSuccess)
                return SVT_ERR_CUDA;
            continue;
        }
        if (op.kind != OP_MEMSET)
            ++launched;
        switch (op.kind) {
        case OP_MEMSET:
            // scalars, status, counters and Gram diagonal are contiguous from L.scal
            err = cudaMemsetAsync(base + L.scal, 0, L.colnorm + (size_t)L.N * sizeof(double) - L.scal, s);
            if (err == cudaSuccess && P.fused && P.uses_strips)
                err = cudaMemsetAsync(base + L.strips, 0, L.strips_bytes, s);
            break;
        case OP_REDUCE:
            err = ingest_reduce_launch(a.A, P.m, P.n, a.lda, P.wide ? 1 : 0, f64 ? 1 : 0, colnorm,
                                       scal, status, s);
            break;
        case OP_SPLIT: {
            // same orientation as A: X (tall) when !wide, X^T when wide.
            const Buf &same = P.wide ? L.Xt[0] : L.X[0];
            const Buf &tran = P.wide ? L.X[0] : L.Xt[0];
            void *same_lo = same.has_lo ? base + same.lo : nullptr;
            void *tran_lo = tran.has_lo ? base + tran.lo : nullptr;
            if (!f64 && !pairs) {  // BF16 tier: lo part of X0^T only, for the Gram
                if (P.wide)
                    same_lo = base + L.XtLo0.hi;
                else
                    tran_lo = base + L.XtLo0.hi;
            }
            err = ingest_split_launch(a.A, P.m, P.n, a.lda, a.tau, f64 ? 1 : 0, base + same.hi,
                                      same_lo, same.ld, base + tran.hi, tran_lo, tran.ld, scal,
                                      status, s);
            break;
        }
        case OP_TC: {
            TcLaunch l = P.tc[op.idx];
            l.dep_wait_ns = ctx->dbg_wait_ns;
            for (const PatchRec &pr : P.patches)
                if (pr.kind == OP_TC && pr.launch == op.idx) {
                    Epi &e = l.p[pr.prob].ep;
                    if (pr.flags & PT_C_IS_A) {
                        e.c0 = a.A;
                        e.ldc = a.lda;
                    }
                    if (pr.flags & PT_O_IS_Y) {
                        e.o0 = a.Y;
                        e.ldo = a.ldy;
                    }
                    if (pr.flags & PT_ALPHA_NEG_TAU)
                        e.alpha = -(double)a.tau;
                }
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (prof) {
                if (ctx->prof_next + 2 > ctx->prof_pool.size()) {
                    for (int k = 0; k < 64; ++k) {
                        cudaEvent_t ev;
                        if (cudaEventCreate(&ev) != cudaSuccess)
                            return SVT_ERR_CUDA;
                        ctx->prof_pool.push_back(ev);
                    }
                }
                e0 = ctx->prof_pool[ctx->prof_next++];
                e1 = ctx->prof_pool[ctx->prof_next++];
                cudaEventRecord(e0, s);
            }
            err = tc_gemm_launch(l, op.bn, grid_sms, s);
            if (prof) {
                cudaEventRecord(e1, s);
                ctx->prof_pending.push_back({e0, e1, P.tc_flops[op.idx], P.tc_tensor_flops[op.idx]});
            }
            break;
        }
        case OP_F64: {
            F64Launch l = P.f64[op.idx];
            for (const PatchRec &pr : P.patches)
                if (pr.kind == OP_F64 && pr.launch == op.idx) {
                    Epi &e = l.p[pr.prob].ep;
                    if (pr.flags & PT_C_IS_A) {
                        e.c0 = a.A;
                        e.ldc = a.lda;
                    }
                    if (pr.flags & PT_O_IS_Y) {
                        e.o0 = a.Y;
                        e.ldo = a.ldy;
                    }
                    if (pr.flags & PT_ALPHA_NEG_TAU)
                        e.alpha = -(double)a.tau;
                }
            err = f64_gemm_launch(l, s);
            break;
        }
        case OP_PREP: {
            const Buf &X = L.X[cur_final];
            const Buf &S = L.S[cur_final];
            int xkind = (op.idx == 1 || skipP) ? C_NONE : (f64 ? C_F64 : (X.has_lo ? C_PAIR : C_BF16));
            int skind = f64 ? C_F64 : (P.final_s_pair ? C_PAIR : C_BF16);
            bool copyS = !(P.opt.polish || f64);
            int64_t total = L.M * L.N;
            int blocks = (int)std::min<int64_t>((total + 255) / 256, 4 * ctx->num_sms * 8);
            prep_kernel<<<blocks, 256, 0, s>>>(
                a.A, a.lda, P.wide ? 1 : 0, L.M, L.N, skipP ? 0.0f : a.tau, xkind,
                xkind ? base + X.hi : nullptr, X.has_lo ? base + X.lo : nullptr, X.ld,
                f64 ? O_F64 : O_PAIR, base + L.B.hi, f64 ? nullptr : base + L.B.lo, L.B.ld,
                copyS ? base + S.hi : nullptr, (copyS && P.final_s_pair) ? base + S.lo : nullptr, skind,
                base + L.Sp.hi, f64 ? nullptr : base + L.Sp.lo, L.Sp.ld);
            err = cudaGetLastError();
            break;
        }
        case OP_FINAL:
            err = finalize_launch(scal, status, a.d_status, s);
            break;
        }
        if (err != cudaSuccess)
            return SVT_ERR_CUDA;
    }
    if (!a.in_graph)
        ctx->launches += (uint64_t)launched;
    return SVT_OK;
}

svt_status upload_fused_table(svt_ctx *ctx, Plan &P, cudaStream_t s)
{
    if (!P.fused)
        return SVT_OK;
    ctx->table_owner = nullptr;
    return cudaMemcpyAsync(const_cast<TcProblem *>(P.fused_launch.gtab), P.h_fused, P.fused_bytes,
                           cudaMemcpyHostToDevice, s) == cudaSuccess
               ? SVT_OK
               : SVT_ERR_CUDA;
}

svt_status run_plan(svt_ctx *ctx, Plan &P, const CallArgs &a, cudaStream_t s, int sms)
{
    return run_ops(ctx, P, a, s, 0, P.ops.size(), sms);
}

Segments plan_segments(const Plan &P, double target)
{
    Segments seg;
    seg.fused = P.fused;
    // Work of each unit: a problem of the fused table, or an op of the plan.
    std::vector<double> unit;
    if (P.fused) {
        unit = P.fused_work;
    } else {
        for (const Op &op : P.ops)
            unit.push_back(op.kind == OP_TC ? P.tc_tensor_flops[op.idx] : 0.0);
    }
    seg.bounds = split_units(unit, target, kMaxFusedSegments);
    for (int k = 0; k + 1 < (int)seg.bounds.size(); ++k) {
        double w = 0.0;
        for (int i = seg.bounds[k]; i < seg.bounds[k + 1]; ++i)
            w += unit[i];
        seg.work.push_back(w);
    }
    return seg;
}

svt_status run_plan_segment(svt_ctx *ctx, Plan &P, const CallArgs &a, cudaStream_t s,
                            const Segments &seg, int k, int sms)
{
    const int nseg = seg.count();
    if (k < 0 || k >= nseg || nseg > kMaxFusedSegments || a.in_graph || seg.fused != P.fused)
        return SVT_ERR_INVALID;
    if (!seg.fused)
        return run_ops(ctx, P, a, s, (size_t)seg.bounds[k], (size_t)seg.bounds[k + 1], sms);
    svt_status st;
    if (k == 0) {
        if ((st = run_ops(ctx, P, a, s, 0, P.fused_first_op, sms)) != SVT_OK)
            return st;
        if ((st = upload_fused_table(ctx, P, s)) != SVT_OK)
            return st;
    }
    TcLaunch l = P.fused_launch;
    l.dep_wait_ns = ctx->dbg_wait_ns;
    l.call_inline.A = a.A;
    l.call_inline.Y = a.Y;
    l.call_inline.lda = a.lda;
    l.call_inline.ldy = a.ldy;
    l.call_inline.tau = a.tau;
    l.call_inline.d_status = a.d_status;
    l.tile_lo = P.fused_starts[seg.bounds[k]];
    l.tile_hi = P.fused_starts[seg.bounds[k + 1]];
    l.tile_counter = P.fused_launch.tile_counter + k;  // zeroed with the solve's scratch
    const int grid_sms = (sms > 0 && sms < ctx->num_sms) ? sms : ctx->num_sms;
    if (l.tile_hi > l.tile_lo) {
        cudaError_t err = tc_gemm_launch_fused(l, P.fused_bn, l.tile_hi - l.tile_lo, grid_sms, s,
                                               P.uses_strips);
        ctx->launches += 1;
        if (err != cudaSuccess)
            return SVT_ERR_CUDA;
    }
    if (k == nseg - 1)
        return run_ops(ctx, P, a, s, P.fused_last_op + 1, P.ops.size(), sms);
    return SVT_OK;
}

namespace {

// One persistent launch for all products of the plan: problems in program order,
// each depending on the previous problem of its chain (the combine on both chains).
// Eligible when the products are contiguous in the op list and share one tile width.
svt_status build_fused(svt_ctx *ctx, Plan &P)
{
    P.fused = false;
    if (!P.lay.fused_tab_bytes)
        return SVT_OK;
    size_t first = P.ops.size(), last = 0;
    int bn = 0;
    for (size_t i = 0; i < P.ops.size(); ++i) {
        if (P.ops[i].kind != OP_TC)
            continue;
        first = std::min(first, i);
        last = i;
        if (bn && P.ops[i].bn != bn)
            return SVT_OK;
        bn = P.ops[i].bn;
    }
    if (first > last)
        return SVT_OK;
    for (size_t i = first; i <= last; ++i)
        if (P.ops[i].kind != OP_TC)
            return SVT_OK;
    // Dependencies (fused_deps.h): whole previous problem of the chain, or per strip.
    // Strips pay on CTA-pair tiles where products are 10 to 15 tiles wide (the smaller
    // side from 2560 to under 4096: 8 % at 3072^2). On narrower products a tile's MMAs
    // take about as long as the extra acquire loads in front of its operand copies; on
    // wider ones the chains rarely wait for each other.
    const int64_t tiles_wide = std::min(P.lay.M, P.lay.N) / tile_cols(bn);
    const bool strips_ok = bn == kBnPair && tiles_wide >= 10 && tiles_wide < 16;
    std::vector<TcProblem> probs;
    std::vector<DepProduct> dps;
    std::vector<int> starts;
    std::vector<double> work;
    size_t ci = 0;
    int total = 0;
    for (size_t i = first; i <= last; ++i) {
        const int li = P.ops[i].idx;
        const TcLaunch &l = P.tc[li];
        for (int q = 0; q < l.nprob; ++q) {
            TcProblem tp = l.p[q];
            const Plan::ProbIO io = P.tc_io[ci];
            const int chain = P.tc_chain[ci++];
            tp.pid = (int)probs.size();
            tp.patch = 0;
            tp.call_idx = 0;
            for (const PatchRec &pr : P.patches)
                if (pr.kind == OP_TC && pr.launch == li && pr.prob == q)
                    tp.patch |= pr.flags;
            if (tp.patch & PT_O_IS_Y)
                tp.o_tma = 0;  // the caller's output: plain coalesced stores
            dps.push_back({io.l, io.r, io.c, io.o, io.t, io.o_trans, tp.sym, chain, tp.tiles_m,
                           tp.tiles_n, tc_valid_ctas(tp, bn), io.theta_src, io.norm_acc, io.f});
            starts.push_back(total);
            total += tc_num_tiles(tp, bn);
            const int kb = tp.fp8 ? 2 * kBK : kBK;
            work.push_back((double)tp.nseg * (double)tc_valid_ctas(tp, bn) * 2.0 * kBM *
                           (double)tile_cols(bn) * (double)((tp.K + kb - 1) / kb * kb));
            probs.push_back(tp);
        }
    }
    std::vector<DepResult> deps;
    if (!derive_fused_deps(dps, strips_ok, kEpiWarpsPublic, kEpiWarpsPublic * ctas_per_tile(bn),
                           P.lay.max_problems * P.lay.max_strips, deps))
        return SVT_OK;  // not representable: the plan runs launch by launch
    for (size_t k = 0; k < probs.size(); ++k) {
        TcProblem &tp = probs[k];
        const DepResult &d = deps[k];
        for (int j = 0; j < 2; ++j) {
            tp.dep[j] = d.dep[j];
            tp.dep_target[j] = d.dep_target[j];
        }
        tp.nwdep = d.nwdep;
        for (int j = 0; j < 4; ++j) {
            tp.wdep[j] = d.wdep[j];
            tp.wdep_target[j] = d.wdep_target[j];
        }
        for (int j = 0; j < 3; ++j) {
            tp.sdep_mode[j] = d.sdep_mode[j];
            tp.sdep_base[j] = d.sdep_base[j];
            tp.sdep_target[j] = d.sdep_target[j];
            tp.sdep_src[j] = d.sdep_src[j];
            tp.sdep_whole[j] = d.sdep_whole[j];
        }
        tp.strip_base = d.strip_base;
    }
    P.uses_strips = strips_ok;
    starts.push_back(total);
    if ((int)probs.size() > P.lay.max_problems)
        return SVT_OK;
    uint8_t *base = ctx->ws + P.ws_base;
    const size_t tab_bytes = align_up(sizeof(TcProblem) * (size_t)P.lay.max_problems, kAlign);
    TcProblem *dp = reinterpret_cast<TcProblem *>(base + P.lay.fused_tab);
    int *ds = reinterpret_cast<int *>(base + P.lay.fused_tab + tab_bytes);
    // Pinned host image of [problems | starts], copied to the device at every call.
    P.fused_bytes = tab_bytes + sizeof(int) * starts.size();
    if (cudaMallocHost(reinterpret_cast<void **>(&P.h_fused), P.fused_bytes) != cudaSuccess)
        return SVT_ERR_CUDA;
    std::memset(P.h_fused, 0, P.fused_bytes);
    std::memcpy(P.h_fused, probs.data(), sizeof(TcProblem) * probs.size());
    std::memcpy(P.h_fused + tab_bytes, starts.data(), sizeof(int) * starts.size());
    std::memset(&P.fused_launch, 0, sizeof(P.fused_launch));
    P.fused_launch.gtab = dp;
    P.fused_launch.gstart = ds;
    P.fused_launch.gcount = (int)probs.size();
    int *counters = reinterpret_cast<int *>(base + P.lay.counters);
    P.fused_launch.done = counters;
    P.fused_launch.tile_counter = counters + P.lay.max_problems;
    P.fused_launch.strips = reinterpret_cast<int *>(base + P.lay.strips);
    P.fused_tiles = total;
    P.fused_bn = bn;
    P.fused_starts = starts;
    P.fused_work = work;
    P.fused_first_op = first;
    P.fused_last_op = last;
    P.fused_flops = 0.0;
    for (double f : P.tc_flops)
        P.fused_flops += f;
    P.fused_tensor_flops = 0.0;
    for (double f : P.tc_tensor_flops)
        P.fused_tensor_flops += f;
    P.fused = true;
    return SVT_OK;
}

} // namespace

void evict_plans(svt_ctx *ctx, size_t max_entries)
{
    if (ctx->plans.size() <= max_entries)
        return;
    for (auto it = ctx->plans.begin(); it != ctx->plans.end();) {
        if (it->second.use_count() == 1)
            it = ctx->plans.erase(it);
        else
            ++it;
    }
}

// Tile mode of a fused solve when none is requested or tuned, from whole-solve timings on
// GB300 (BF16 tier, 20 steps): 128 x 128 tiles while the small side is at most 1536 (more
// tiles per product keep all SMs busy: 1.31x over 128 x 256 at 1024^2), CTA pairs above
// (1.01x at 2048^2, 1.035x at 3072^2 and 4096^2, 1.04x at 8192 x 2048, 1.08x at 6144^2,
// 8192^2 and 16384 x 4096).
int fused_auto_width(int64_t m, int64_t n)
{
    return std::min(m, n) <= 1536 ? 128 : kBnPair;
}

svt_status get_plan(svt_ctx *ctx, int64_t m, int64_t n, const Resolved &r, size_t ws_base,
                    size_t ws_avail, Plan **out, int force_bn, std::shared_ptr<Plan> *keep)
{
    if (force_bn == 0 && r.fuse && r.prec != SVT_FP64)
        force_bn = fused_auto_width(m, n);
    Key k{m, n, r.iters, r.prec, r.schedule, r.norm, r.polish, r.mode, r.hp_steps, r.ell0, r.delta,
          ws_base, force_bn, r.fuse, r.out64, r.fp8_p, r.fp8_s, r.fp8_s_y2};
    auto it = ctx->plans.find(k);
    if (it != ctx->plans.end()) {
        *out = it->second.get();
        if (keep)
            *keep = it->second;
        return SVT_OK;
    }
    // Host-side fault injection (svt_ctx_debug): the Nth plan build fails.
    if (ctx->dbg_fail_plan > 0 && --ctx->dbg_fail_plan == 0)
        return SVT_ERR_OOM;
    NvtxRange nvtx_build("svt plan build");
    auto plan = std::make_shared<Plan>();
    plan->m = m;
    plan->n = n;
    plan->wide = n > m;
    plan->opt = r;
    plan->lay = make_layout(m, n, r);
    plan->ws_base = ws_base;
    plan->force_bn = force_bn;
    if (force_bn < 0) {
        auto t = ctx->tuning.find(tune_key(m, n, r));
        if (t == ctx->tuning.end())
            return SVT_ERR_INVALID;
        plan->bn_choice = t->second;
    }
    if (plan->lay.total > ws_avail)
        return SVT_ERR_OOM;
    plan->coef.assign((size_t)std::max(1, 3 * r.iters), 0.0);
    plan->lo.assign((size_t)std::max(1, r.iters), 0.0);
    if (schedule_coeffs(r.schedule, r.iters, r.ell0, r.delta, plan->coef.data(),
                        plan->lo.data()) != 0)
        return SVT_ERR_INVALID;
    Builder b{ctx, plan.get(), ctx->ws + ws_base, 256};
    if (!b.build())
        return SVT_ERR_CUDA;
    if (r.fuse && build_fused(ctx, *plan) != SVT_OK)
        return SVT_ERR_CUDA;
    *out = plan.get();
    if (keep)
        *keep = plan;
    ctx->plans[k] = std::move(plan);
    return SVT_OK;
}

svt_status plan_for_solve(svt_ctx *ctx, int64_t m, int64_t n, const Resolved &r, Plan **out,
                          std::shared_ptr<Plan> *keep)
{
    const int fbn = r.tile ? r.tile : (ctx->tuning.count(tune_key(m, n, r)) ? -1 : 0);
    return get_plan(ctx, m, n, r, 0, ctx->ws_bytes, out, fbn, keep);
}

svt_status plan_status_copy(svt_ctx *ctx, const Plan &P, int *host_dst, cudaStream_t s)
{
    const int *src = reinterpret_cast<const int *>(ctx->ws + P.ws_base + P.lay.status);
    return cudaMemcpyAsync(host_dst, src, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess
               ? SVT_OK
               : SVT_ERR_CUDA;
}

static bool finite_tau(float tau) { return std::isfinite(tau) && tau >= 0.0f; }

svt_status validate_out(const float *A, int64_t m, int64_t n, int64_t lda, float tau,
                        const void *Y, int64_t ldy, size_t ysz)
{
    if (!A || !Y || m <= 0 || n <= 0 || lda < n || ldy < n || !finite_tau(tau))
        return SVT_ERR_INVALID;
    if (m > (int64_t)1 << 20 || n > (int64_t)1 << 20)
        return SVT_ERR_UNSUPPORTED;
    // A and Y must not overlap
    const size_t abytes = ((size_t)(m - 1) * (size_t)lda + (size_t)n) * sizeof(float);
    const size_t ybytes = ((size_t)(m - 1) * (size_t)ldy + (size_t)n) * ysz;
    if (overlaps(A, abytes, Y, ybytes))
        return SVT_ERR_INVALID;
    return SVT_OK;
}

svt_status validate(const float *A, int64_t m, int64_t n, int64_t lda, float tau, const float *Y,
                    int64_t ldy)
{
    return validate_out(A, m, n, lda, tau, Y, ldy, sizeof(float));
}

} // namespace svt

using namespace svt;

extern "C" {

const char *svt_status_str(svt_status s)
{
    switch (s) {
    case SVT_OK: return "SVT_OK";
    case SVT_ERR_INVALID: return "SVT_ERR_INVALID";
    case SVT_ERR_OOM: return "SVT_ERR_OOM";
    case SVT_ERR_CUDA: return "SVT_ERR_CUDA";
    case SVT_ERR_NONFINITE: return "SVT_ERR_NONFINITE";
    case SVT_ERR_DIVERGED: return "SVT_ERR_DIVERGED";
    case SVT_ERR_TIMEOUT: return "SVT_ERR_TIMEOUT";
    case SVT_ERR_NOT_READY: return "SVT_ERR_NOT_READY";
    case SVT_ERR_BUSY: return "SVT_ERR_BUSY";
    case SVT_ERR_UNSUPPORTED: return "SVT_ERR_UNSUPPORTED";
    case SVT_ERR_CANCELLED: return "SVT_ERR_CANCELLED";
    }
    return "SVT_ERR_UNKNOWN";
}

void svt_options_default(svt_options *o)
{
    if (!o)
        return;
    o->iters = 20;
    o->prec = SVT_BF16;
    o->schedule = SVT_SCHED_AUTO;
    o->norm = SVT_NORM_AUTO;
    o->ell0 = 1e-3;
    o->delta = -1.0;
    o->polish = 1;
    o->mode = SVT_MODE_SVT;
    o->hp_steps = -1;
    o->fuse = 1;
    o->tile = 0;
}

svt_status svt_workspace_bytes_ex(int64_t m, int64_t n, const svt_options *opt, size_t *out)
{
    Resolved r;
    if (!out || m <= 0 || n <= 0)
        return SVT_ERR_INVALID;
    if (svt_status rs = resolve_status(opt, &r))
        return rs;
    *out = make_layout(m, n, r).total;
    return SVT_OK;
}

svt_status svt_workspace_bytes(int64_t m, int64_t n, svt_precision prec, size_t *out)
{
    svt_options o;
    svt_options_default(&o);
    o.prec = prec;
    return svt_workspace_bytes_ex(m, n, &o, out);
}

svt_status svt_schedule_coeffs(svt_schedule_kind kind, int iters, double ell0, double delta,
                               double *coef)
{
    int k = (kind == SVT_SCHED_NS3) ? SVT_SCHED_NS3 : SVT_SCHED_PE5;
    if (kind != SVT_SCHED_AUTO && kind != SVT_SCHED_PE5 && kind != SVT_SCHED_NS3)
        return SVT_ERR_INVALID;
    return schedule_coeffs(k, iters, ell0, delta, coef) == 0 ? SVT_OK : SVT_ERR_INVALID;
}

svt_status svt_ctx_create(int device, void *workspace, size_t ws_bytes, svt_ctx_t *out)
{
    if (!out || (ws_bytes > 0 && !workspace) ||
        (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0)
        return SVT_ERR_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return SVT_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess)
        return SVT_ERR_CUDA;
    auto *c = new svt_ctx();
    c->device = device;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return SVT_ERR_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return SVT_ERR_CUDA;
    }
    std::snprintf(c->gpu_name, sizeof(c->gpu_name), "%s", prop.name);
    c->ws = static_cast<uint8_t *>(workspace);
    c->ws_bytes = ws_bytes;
    *out = c;
    return SVT_OK;
}

svt_status svt_ctx_debug(svt_ctx_t ctx, svt_debug_flag flag, int64_t value)
{
    if (!ctx || value < 0)
        return SVT_ERR_INVALID;
    std::lock_guard<std::mutex> g(ctx->mu);
    switch (flag) {
    case SVT_DEBUG_FAIL_PLAN: ctx->dbg_fail_plan = value; return SVT_OK;
    case SVT_DEBUG_ADMIT_DELAY_US: ctx->dbg_admit_delay_us = value; return SVT_OK;
    case SVT_DEBUG_WAIT_LIMIT_NS: ctx->dbg_wait_ns = (uint64_t)value; return SVT_OK;
    }
    return SVT_ERR_INVALID;
}

svt_status svt_tuning_export(svt_ctx_t ctx, char *buf, size_t cap, size_t *len)
{
    if (!ctx || !len || (cap > 0 && !buf))
        return SVT_ERR_INVALID;
    std::string text;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        text = tuning_to_json(ctx->gpu_name, ctx->num_sms, ctx->tuning);
    }
    *len = text.size();
    if (cap < text.size() + 1)
        return SVT_ERR_OOM;
    std::memcpy(buf, text.c_str(), text.size() + 1);
    return SVT_OK;
}

svt_status svt_tuning_import(svt_ctx_t ctx, const char *json)
{
    if (!ctx || !json)
        return SVT_ERR_INVALID;
    std::map<TuneKey, std::vector<int>> entries;
    if (!tuning_from_json(json, ctx->gpu_name, ctx->num_sms, &entries))
        return SVT_ERR_INVALID;
    std::lock_guard<std::mutex> g(ctx->mu);
    for (auto &kv : entries) {
        // cached plans built from an earlier tuning of this shape are stale
        for (auto it = ctx->plans.begin(); it != ctx->plans.end();) {
            const Key &k = it->first;
            if (k.force_bn < 0 && k.m == kv.first.m && k.n == kv.first.n && k.fuse == kv.first.fuse)
                it = ctx->plans.erase(it);
            else
                ++it;
        }
        ctx->tuning[kv.first] = kv.second;
    }
    return SVT_OK;
}

svt_status svt_ctx_destroy(svt_ctx_t ctx)
{
    if (!ctx)
        return SVT_ERR_INVALID;
    serve_shutdown(ctx);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    completion_release(ctx);
    for (cudaEvent_t e : ctx->prof_pool)
        cudaEventDestroy(e);
    delete ctx;
    return SVT_OK;
}

svt_status svt_polar_ex(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda,
                        float tau, const svt_options *opt, float *Y, int64_t ldy,
                        svt_status *d_status, void *stream)
{
    if (!ctx)
        return SVT_ERR_INVALID;
    svt_status st = validate(A, m, n, lda, tau, Y, ldy);
    if (st != SVT_OK)
        return st;
    Resolved r;
    if ((st = resolve_status(opt, &r)) != SVT_OK)
        return st;
    if (r.prec == SVT_FP64 && (m > kF64MaxDim || n > kF64MaxDim))
        return SVT_ERR_UNSUPPORTED;
    if (serve_busy(ctx))
        return SVT_ERR_BUSY;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    NvtxRange nvtx_solve("svt_polar");
    Plan *plan = nullptr;
    st = plan_for_solve(ctx, m, n, r, &plan);
    if (st != SVT_OK)
        return st;
    CallArgs a{A, lda, tau, Y, ldy, d_status};
    return run_plan(ctx, *plan, a, static_cast<cudaStream_t>(stream));
}

svt_status svt_polar_f64(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda,
                         float tau, const svt_options *opt, double *Y, int64_t ldy,
                         svt_status *d_status, void *stream)
{
    if (!ctx)
        return SVT_ERR_INVALID;
    svt_status st = validate_out(A, m, n, lda, tau, Y, ldy, sizeof(double));
    if (st != SVT_OK)
        return st;
    Resolved r;
    if ((st = resolve_status(opt, &r)) != SVT_OK)
        return st;
    if (r.prec != SVT_FP64)
        return SVT_ERR_INVALID;  // only the FP64 tier has an FP64 result
    if (m > kF64MaxDim || n > kF64MaxDim)
        return SVT_ERR_UNSUPPORTED;
    r.out64 = 1;
    if (serve_busy(ctx))
        return SVT_ERR_BUSY;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    Plan *plan = nullptr;
    st = get_plan(ctx, m, n, r, 0, ctx->ws_bytes, &plan);
    if (st != SVT_OK)
        return st;
    // The plan's combine stores FP64; the output pointer travels as the call's Y.
    CallArgs a{A, lda, tau, reinterpret_cast<float *>(Y), ldy, d_status};
    return run_plan(ctx, *plan, a, static_cast<cudaStream_t>(stream));
}

svt_status svt_autotune(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda,
                        float tau, const svt_options *opt, float *Y, int64_t ldy, int reps,
                        void *stream)
{
    if (!ctx)
        return SVT_ERR_INVALID;
    svt_status st = validate(A, m, n, lda, tau, Y, ldy);
    if (st != SVT_OK)
        return st;
    Resolved r;
    if (reps < 1)
        return SVT_ERR_INVALID;
    if ((st = resolve_status(opt, &r)) != SVT_OK)
        return st;
    if (r.prec == SVT_FP64)
        return SVT_OK;  // the FP64 tier has no tile choice
    if (serve_busy(ctx))
        return SVT_ERR_BUSY;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CallArgs a{A, lda, tau, Y, ldy, nullptr};
    const int widths[3] = {128, 256, kBnPair};
    std::vector<int> choice;
    if (r.fuse) {
        // Fused solves: one width for all products; time whole solves with each.
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess)
            return SVT_ERR_CUDA;
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return SVT_ERR_CUDA;
        }
        double best = -1.0;
        int best_w = 0;
        size_t n_tc = 0;
        for (int w = 0; w < 3 && st == SVT_OK; ++w) {
            Plan *plan = nullptr;
            st = get_plan(ctx, m, n, r, 0, ctx->ws_bytes, &plan, widths[w]);
            if (st != SVT_OK)
                break;
            if (!plan->fused)
                continue;  // this width cannot run as one launch here
            st = run_plan(ctx, *plan, a, s);  // warm-up
            if (st != SVT_OK)
                break;
            cudaEventRecord(e0, s);
            for (int k = 0; k < reps && st == SVT_OK; ++k)
                st = run_plan(ctx, *plan, a, s);
            cudaEventRecord(e1, s);
            if (st != SVT_OK)
                break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = SVT_ERR_CUDA;
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (best < 0.0 || t < best) {
                best = t;
                best_w = widths[w];
                n_tc = plan->tc.size();
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st != SVT_OK)
            return st;
        if (best_w == 0)
            return SVT_OK;  // no width runs fused: keep the automatic choice
        choice.assign(n_tc, best_w);
    } else {
        std::vector<double> ms[3];
        const bool prev_profile = ctx->profile;
        for (int w = 0; w < 3; ++w) {
            Plan *plan = nullptr;
            st = get_plan(ctx, m, n, r, 0, ctx->ws_bytes, &plan, widths[w]);
            if (st != SVT_OK)
                return st;
            st = run_plan(ctx, *plan, a, s);  // warm-up
            if (st != SVT_OK)
                return st;
            ctx->profile = true;
            ctx->prof_pending.clear();
            ctx->prof_next = 0;
            for (int k = 0; k < reps; ++k) {
                st = run_plan(ctx, *plan, a, s);
                if (st != SVT_OK) {
                    ctx->profile = prev_profile;
                    return st;
                }
            }
            const size_t per = plan->tc.size();
            ms[w].assign(per, 0.0);
            for (size_t i = 0; i < ctx->prof_pending.size(); ++i) {
                auto &pr = ctx->prof_pending[i];
                if (cudaEventSynchronize(pr.b) != cudaSuccess) {
                    ctx->profile = prev_profile;
                    return SVT_ERR_CUDA;
                }
                float t = 0.f;
                cudaEventElapsedTime(&t, pr.a, pr.b);
                ms[w][i % per] += t;
            }
            ctx->prof_pending.clear();
            ctx->prof_next = 0;
            ctx->profile = prev_profile;
        }
        choice.assign(ms[0].size(), 128);
        for (size_t i = 0; i < choice.size(); ++i) {
            int bw = 0;
            for (int w = 1; w < 3; ++w)
                if (ms[w][i] < ms[bw][i])
                    bw = w;
            choice[i] = widths[bw];
        }
    }
    // Plans built from an earlier tuning of this shape are stale.
    for (auto it = ctx->plans.begin(); it != ctx->plans.end();) {
        const Key &k = it->first;
        if (k.force_bn < 0 && k.m == m && k.n == n && k.fuse == r.fuse)
            it = ctx->plans.erase(it);
        else
            ++it;
    }
    ctx->tuning[tune_key(m, n, r)] = choice;
    return SVT_OK;
}

svt_status svt_polar(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda, float tau,
                     int iters, svt_precision prec, float *Y, int64_t ldy, svt_status *d_status,
                     void *stream)
{
    svt_options o;
    svt_options_default(&o);
    o.iters = iters;
    o.prec = prec;
    return svt_polar_ex(ctx, A, m, n, lda, tau, &o, Y, ldy, d_status, stream);
}

svt_status svt_ctx_sync(svt_ctx_t ctx, void *stream)
{
    if (!ctx)
        return SVT_ERR_INVALID;
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return SVT_ERR_CUDA;
    return SVT_OK;
}

uint64_t svt_ctx_launch_count(svt_ctx_t ctx) { return ctx ? ctx->launches : 0; }

svt_status svt_ctx_profile(svt_ctx_t ctx, int enable)
{
    if (!ctx)
        return SVT_ERR_INVALID;
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->profile = enable != 0;
    ctx->prof_pending.clear();
    ctx->prof_next = 0;
    return SVT_OK;
}

svt_status svt_ctx_profile_read_ex(svt_ctx_t ctx, double *tc_ms, double *tc_flops,
                                   double *tc_tensor_flops, uint64_t *tc_launches)
{
    if (!ctx || !tc_ms || !tc_flops || !tc_launches)
        return SVT_ERR_INVALID;
    std::lock_guard<std::mutex> g(ctx->mu);
    double ms = 0.0, fl = 0.0, tfl = 0.0;
    for (auto &r : ctx->prof_pending) {
        if (cudaEventSynchronize(r.b) != cudaSuccess)
            return SVT_ERR_CUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess)
            return SVT_ERR_CUDA;
        ms += t;
        fl += r.flops;
        tfl += r.tensor_flops;
    }
    *tc_ms = ms;
    *tc_flops = fl;
    if (tc_tensor_flops)
        *tc_tensor_flops = tfl;
    *tc_launches = ctx->prof_pending.size();
    ctx->prof_pending.clear();
    ctx->prof_next = 0;
    return SVT_OK;
}

svt_status svt_ctx_profile_read(svt_ctx_t ctx, double *tc_ms, double *tc_flops,
                                uint64_t *tc_launches)
{
    return svt_ctx_profile_read_ex(ctx, tc_ms, tc_flops, nullptr, tc_launches);
}

svt_status svt_debug_gemm_bf16_ex(svt_ctx_t ctx, int nseg, const void *L_hi, const void *L_lo,
                                  const void *R_hi, const void *R_lo, int64_t M, int64_t N,
                                  int64_t K, int64_t ldl, int64_t ldr, float *D, int64_t ldd,
                                  int sym, int tile, void *stream)
{
    if (!ctx || nseg < 1 || nseg > 3 || !L_hi || !R_hi || !D || M <= 0 || N <= 0 || K <= 0 ||
        ldl < K || ldr < K || ldd < N || (ldl % 8) || (ldr % 8) || (sym && M != N))
        return SVT_ERR_INVALID;
    if ((nseg >= 2 && !R_lo) || (nseg == 3 && !L_lo))
        return SVT_ERR_INVALID;
    if (tile != 0 && tile != 128 && tile != 256 && tile != kBnPair)
        return SVT_ERR_INVALID;
    if (M > INT32_MAX / 2 || N > INT32_MAX / 2 || K > INT32_MAX / 2)
        return SVT_ERR_UNSUPPORTED;
    const int bn = tile ? tile : (N > 128 ? 256 : 128);
    TcLaunch l;
    std::memset(&l, 0, sizeof(l));
    l.nprob = 1;
    TcProblem &p = l.p[0];
    if (!encode_bf16_map(&p.mapL[0], L_hi, M, K, ldl, kBM) ||
        !encode_bf16_map(&p.mapR[0], R_hi, N, K, ldr, r_box_rows(bn)))
        return SVT_ERR_INVALID;
    if (nseg >= 2 && !encode_bf16_map(&p.mapR[1], R_lo, N, K, ldr, r_box_rows(bn)))
        return SVT_ERR_INVALID;
    if (nseg == 3 && !encode_bf16_map(&p.mapL[1], L_lo, M, K, ldl, kBM))
        return SVT_ERR_INVALID;
    const int sl[3] = {0, 0, 1}, sr[3] = {0, 1, 0};
    p.nseg = nseg;
    for (int i = 0; i < nseg; ++i) {
        p.segL[i] = sl[i];
        p.segR[i] = sr[i];
    }
    p.M = (int)M;
    p.N = (int)N;
    p.K = (int)K;
    p.sym = sym ? 1 : 0;
    p.strip_base = -1;
    p.tiles_m = (int)((M + tile_rows(bn) - 1) / tile_rows(bn));
    p.tiles_n = (int)((N + tile_cols(bn) - 1) / tile_cols(bn));
    std::memset(&p.ep, 0, sizeof(p.ep));
    p.ep.alpha = 1.0;
    p.ep.o_kind = O_F32;
    p.ep.o0 = D;
    p.ep.ldo = ldd;
    attach_store_maps(p);
    l.tile_start[0] = 0;
    l.tile_start[1] = tc_num_tiles(p, bn);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    cudaError_t e = tc_gemm_launch(l, bn, ctx->num_sms, static_cast<cudaStream_t>(stream));
    ctx->launches += 1;
    return e == cudaSuccess ? SVT_OK : SVT_ERR_CUDA;
}

svt_status svt_debug_gemm_e4m3(svt_ctx_t ctx, const void *L, const void *R, int64_t M, int64_t N,
                               int64_t K, int64_t ldl, int64_t ldr, float *D, int64_t ldd, int tile,
                               void *stream)
{
    if (!ctx || !L || !R || !D || M <= 0 || N <= 0 || K <= 0 || ldl < K || ldr < K || ldd < N ||
        (ldl % 16) || (ldr % 16))
        return SVT_ERR_INVALID;
    if (tile != 0 && tile != 128 && tile != 256 && tile != kBnPair)
        return SVT_ERR_INVALID;
    if (M > INT32_MAX / 2 || N > INT32_MAX / 2 || K > INT32_MAX / 2)
        return SVT_ERR_UNSUPPORTED;
    const int bn = tile ? tile : (N > 128 ? 256 : 128);
    TcLaunch l;
    std::memset(&l, 0, sizeof(l));
    l.nprob = 1;
    TcProblem &p = l.p[0];
    if (!encode_e4m3_map(&p.mapL[0], L, M, K, ldl, kBM) ||
        !encode_e4m3_map(&p.mapR[0], R, N, K, ldr, r_box_rows(bn)))
        return SVT_ERR_INVALID;
    p.fp8 = 1;
    p.nseg = 1;
    p.M = (int)M;
    p.N = (int)N;
    p.K = (int)K;
    p.strip_base = -1;
    p.tiles_m = (int)((M + tile_rows(bn) - 1) / tile_rows(bn));
    p.tiles_n = (int)((N + tile_cols(bn) - 1) / tile_cols(bn));
    p.ep.alpha = 1.0;
    p.ep.o_kind = O_F32;
    p.ep.o0 = D;
    p.ep.ldo = ldd;
    attach_store_maps(p);
    l.tile_start[0] = 0;
    l.tile_start[1] = tc_num_tiles(p, bn);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    cudaError_t e = tc_gemm_launch(l, bn, ctx->num_sms, static_cast<cudaStream_t>(stream));
    ctx->launches += 1;
    return e == cudaSuccess ? SVT_OK : SVT_ERR_CUDA;
}

// The BF16 tier's resolved options with an FP8 policy's steps on e4m3 operands.
static svt_status resolve_fp8(const svt_options *opt, const svt_fp8_policy *policy, Resolved *r)
{
    if (!policy || policy->reserved != 0)
        return SVT_ERR_INVALID;
    svt_options o;
    if (opt)
        o = *opt;
    else
        svt_options_default(&o);
    if (o.prec == SVT_FP8_EXPERIMENTAL)
        o.prec = SVT_BF16;
    if (o.prec != SVT_BF16)
        return SVT_ERR_INVALID;
    if (svt_status st = resolve_status(&o, r))
        return st;
    r->fp8_p = policy->p_steps;
    r->fp8_s = policy->s_steps;
    r->fp8_s_y2 = policy->s_y2_only ? 1 : 0;
    return SVT_OK;
}

svt_status svt_workspace_bytes_fp8(int64_t m, int64_t n, const svt_options *opt,
                                   const svt_fp8_policy *policy, size_t *out)
{
    Resolved r;
    if (!out || m <= 0 || n <= 0)
        return SVT_ERR_INVALID;
    if (svt_status st = resolve_fp8(opt, policy, &r))
        return st;
    *out = make_layout(m, n, r).total;
    return SVT_OK;
}

svt_status svt_polar_fp8(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda,
                         float tau, const svt_options *opt, const svt_fp8_policy *policy, float *Y,
                         int64_t ldy, svt_status *d_status, void *stream)
{
    if (!ctx)
        return SVT_ERR_INVALID;
    svt_status st = validate(A, m, n, lda, tau, Y, ldy);
    if (st != SVT_OK)
        return st;
    Resolved r;
    if ((st = resolve_fp8(opt, policy, &r)) != SVT_OK)
        return st;
    if (serve_busy(ctx))
        return SVT_ERR_BUSY;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    Plan *plan = nullptr;
    st = plan_for_solve(ctx, m, n, r, &plan);
    if (st != SVT_OK)
        return st;
    CallArgs a{A, lda, tau, Y, ldy, d_status};
    return run_plan(ctx, *plan, a, static_cast<cudaStream_t>(stream));
}

svt_status svt_debug_wait_timeout(svt_ctx_t ctx, svt_status *d_status, void *stream)
{
    if (!ctx || !d_status)
        return SVT_ERR_INVALID;
    // [one problem | tile starts 0, 1 | done[0], tile counter] at the workspace start
    const size_t tab = align_up(sizeof(TcProblem), kAlign);
    const size_t bytes = tab + 4 * sizeof(int);
    if (ctx->ws_bytes < bytes)
        return SVT_ERR_OOM;
    if (serve_busy(ctx))
        return SVT_ERR_BUSY;
    std::lock_guard<std::mutex> g(ctx->mu);
    if (cudaSetDevice(ctx->device) != cudaSuccess)
        return SVT_ERR_CUDA;
    std::vector<uint8_t> img(bytes, 0);
    TcProblem &p = *reinterpret_cast<TcProblem *>(img.data());
    p.M = p.N = p.K = kBM;
    p.tiles_m = p.tiles_n = 1;
    p.nseg = 1;
    p.pid = 0;
    p.dep[0] = 0;  // the tile waits for its own problem to complete: it never does
    p.dep_target[0] = 1;
    p.dep[1] = -1;
    p.strip_base = -1;
    p.ep.alpha = 1.0;
    p.ep.status = reinterpret_cast<int *>(d_status);
    int *ints = reinterpret_cast<int *>(img.data() + tab);
    ints[0] = 0;
    ints[1] = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    ctx->table_owner = nullptr;  // the workspace start is overwritten
    if (cudaMemcpyAsync(ctx->ws, img.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SVT_ERR_CUDA;
    TcLaunch l;
    std::memset(&l, 0, sizeof(l));
    l.gtab = reinterpret_cast<const TcProblem *>(ctx->ws);
    l.gstart = reinterpret_cast<const int *>(ctx->ws + tab);
    l.gcount = 1;
    l.done = reinterpret_cast<int *>(ctx->ws + tab) + 2;
    l.tile_counter = l.done + 1;
    const cudaError_t e = tc_gemm_launch_fused(l, 128, 1, ctx->num_sms, s, false);
    ctx->launches += 1;
    return e == cudaSuccess ? SVT_OK : SVT_ERR_CUDA;
}

svt_status svt_debug_gemm_bf16(svt_ctx_t ctx, int nseg, const void *L_hi, const void *L_lo,
                               const void *R_hi, const void *R_lo, int64_t M, int64_t N,
                               int64_t K, int64_t ldl, int64_t ldr, float *D, int64_t ldd,
                               int sym, void *stream)
{
    return svt_debug_gemm_bf16_ex(ctx, nseg, L_hi, L_lo, R_hi, R_lo, M, N, K, ldl, ldr, D, ldd,
                                  sym, 0, stream);
}

} // extern "C"
