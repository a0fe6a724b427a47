// Internal declarations shared by the libsvt translation units.
//
// The library computes singular value soft-thresholding (Eq. 1) through
// Proposition 1 in its factored form A_tau = 1/2 (A - tau P)(I + S), with the
// tall orientation M >= N: a wide input (n > m, the footnote's A A^T branch) is
// solved as the tall problem of A^T and its result is stored transposed.
//
// Every dense product is D = sum_s L_s R_s^T with both operands K-major
// (row-major, contraction along rows), and a fused epilogue
//   v = alpha * D + beta * C + gamma * [r == c]
// (alpha, beta, gamma optionally scaled by powers of a device-side norm), with
// an FP64 diagonal override for the tau^2 shift and an FP64 sum of squares.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/svt.h"

namespace svt {

constexpr int kMaxProblems = 2;   // problems per by-value grouped launch (P and S chains)
constexpr int kMaxFusedSegments = 64;  // launches a fused solve may be split into
constexpr int kBM = 128;          // tile rows (tcgen05 M)
constexpr int kBK = 64;           // K per pipeline stage: one 128-byte swizzle row of BF16

// Tile-width codes of the product kernel. 128 and 256: one CTA per 128 x bn
// output tile. kBnPair: a cluster of two CTAs per 256 x 256 tile
// (tcgen05 cta_group::2), each CTA holding 128 x 256 of it and staging half of
// the tile's R rows.
constexpr int kBnPair = 512;
inline int tile_rows(int bn) { return bn == kBnPair ? 2 * kBM : kBM; }
inline int tile_cols(int bn) { return bn == kBnPair ? 256 : bn; }
inline int r_box_rows(int bn) { return bn == kBnPair ? 128 : bn; }  // R rows one CTA loads
inline int ctas_per_tile(int bn) { return bn == kBnPair ? 2 : 1; }

enum CKind : int { C_NONE = 0, C_BF16 = 1, C_PAIR = 2, C_F32 = 3, C_F64 = 4 };
enum OKind : int { O_NONE = 0, O_BF16 = 1, O_PAIR = 2, O_F32 = 3, O_F64 = 4, O_E4M3 = 5 };

// Device-side scalar slots of one solve (FP64, in the workspace).
enum Scal : int {
    SC_NRM_A2 = 0,      // ||A||_F^2
    SC_ALPHA = 1,       // power of two near ||A||_F; X0 = A / alpha exactly
    SC_INV_ALPHA2 = 2,  // 1 / alpha^2
    SC_TAU2_SCALED = 3, // tau^2 / alpha^2
    SC_NRM_X0 = 4,      // ||X0||_F^2 = ||A||_F^2 / alpha^2
    SC_NRM_S0 = 5,      // ||S0||_F^2 (S0 = (A^T A - tau^2 I) / alpha^2)
    SC_NRM_YP = 6,      // ||X0^T X0||_F^2 of the P chain's first step
    SC_NRM_YS = 7,      // ||S0^2||_F^2 of the S chain's first step
    SC_NRM_OUT = 8,     // ||Y||_F^2 of the output
    SC_COUNT = 16
};

struct Epi {
    double alpha, beta, gamma;       // v = alpha D + beta C + gamma [r == c]
    double ea, eb, eg;               // exponents: alpha *= theta^-ea, ...
    const double *theta_src;         // theta = (*theta_src)^theta_pow; null: theta = 1
    double theta_pow;
    int c_kind, c_trans;             // C source; c_trans: C(r, c) = c0[c * ldc + r]
    const void *c0, *c1;
    int64_t ldc;
    int o_kind, o_trans;             // output; o_trans: stored at [c * ldo + r]
    void *o0, *o1;
    int64_t ldo;
    int t_kind;                      // extra transposed copy (O_NONE, O_BF16, O_PAIR, O_F64)
    void *t0, *t1;
    int64_t ldt;
    double *norm_acc;                // += sum of v^2 over the full matrix
    const double *diag;              // v(r, r) = diag[r] * dss[0] - dss[1] (FP64)
    const double *dss;
    int *status;                     // device status word of the solve
    // Extra e4m3 copy of the output (FP8 experiment): fscale * v, saturated, same
    // orientation as the output (mirrored for symmetric products); f0 == null: none.
    void *f0;
    int64_t ldf;
    float fscale;
    int pad_f;
};

// Per-call arguments of one matrix, read by the kernels of a grouped launch
// (device table, uploaded per call).
struct CallRec {
    const float *A;
    float *Y;
    int64_t lda, ldy;
    float tau;
    int pad;
    svt_status *d_status;
};

// Problem fields that come from the call table in grouped launches.
enum Patch { PT_C_IS_A = 1, PT_O_IS_Y = 2, PT_ALPHA_NEG_TAU = 4 };

// One product of a grouped tensor-core launch.
struct TcProblem {
    CUtensorMap mapL[2];             // L operands, box 64 x 128
    CUtensorMap mapR[2];             // R operands, box 64 x BN
    CUtensorMap mapO[2];             // output hi/lo (or FP32), box 32 x 32, for TMA stores
    CUtensorMap mapT[2];             // transposed copy hi/lo, box 32 x 32
    int o_tma, t_tma;                // 1: store through mapO / mapT
    int patch, call_idx;             // grouped launches: fields taken from calls[call_idx]
    // Fused (chained) launches: completion counter index of this problem, and the
    // problems whose results it reads with the counts that mean "complete".
    int pid;
    int dep[2];
    int dep_target[2];
    // Finer dependencies of a fused solve (tiles with TM == BN, one strip per tile
    // row or column): sdep[0] / [1] / [2] for the L, R and C operands, the producing
    // problem's strip counters at sdep_base, strip index = this tile's row (L, C) or
    // column (R), complete at sdep_target. sdep_mode: 0 none, 1 row strip of a
    // row-major output, 2 column strip (the producer's transposed output), 3 strip of
    // a symmetric product (its rows and columns). wdep: whole problems the epilogue
    // waits for before its stores (earlier readers of the buffers it overwrites, the
    // problems that accumulate the norms it scales by).
    int sdep_mode[3], sdep_base[3], sdep_target[3];
    int sdep_src[3], sdep_whole[3];  // producing problem and its whole-completion count
    int strip_base;  // this problem's strip counters (-1: none): rows then columns
    int nwdep;
    int wdep[4], wdep_target[4];
    int nseg;
    int segL[3], segR[3];
    int M, N, K;
    int fp8;                         // operands are e4m3 (kind::f8f6f4): 128 of K per k-block
    int sym;                         // upper tiles only, mirrored store (M == N)
    int tiles_m, tiles_n;
    Epi ep;
};

struct TcLaunch {
    int nprob;
    int tile_start[kMaxProblems + 1];
    TcProblem p[kMaxProblems];
    // Grouped launches: problems and tile prefix sums in device memory instead.
    const TcProblem *gtab;
    const int *gstart;               // gcount + 1 entries
    int gcount;
    const CallRec *calls;
    // Fused launch (all products of a solve, device-side dependencies): tiles are
    // taken in table order from *tile_counter; done[pid] counts finished
    // (tile, epilogue warp) pairs. Both live in the solve's zeroed scratch.
    int *tile_counter;
    int *done;
    // Fused launches over part of the table (a segment of a solve issued as several
    // launches): tiles [tile_lo, tile_hi) in table order; tile_hi == 0: the whole table.
    int tile_lo, tile_hi;
    int *strips;  // fused solves: per-problem strip completion counters
    CallRec call_inline;             // per-call fields when calls == nullptr
    // Limit of the waits on other tiles' results (dependency counters), ns; 0: the
    // kernel's default. Set from the context's SVT_DEBUG_WAIT_LIMIT_NS.
    unsigned long long dep_wait_ns;
};

// One product of the FP64 SIMT path: D = L R^T, L M x K (ldl), R N x K (ldr).
struct F64Problem {
    const double *L, *R;
    int64_t ldl, ldr;
    int M, N, K;
    int sym;
    Epi ep;
};

struct F64Launch {
    int nprob;
    F64Problem p[2];
};

// ---- launchers (defined in the .cu files) ----
int tc_num_tiles(const TcProblem &p, int bn);
// CTA tiles (128 rows each) of a problem that publish completion in a fused
// launch: tiles with work, times the CTAs per tile.
int tc_valid_ctas(const TcProblem &p, int bn);
cudaError_t tc_gemm_launch(const TcLaunch &l, int bn, int num_sms, cudaStream_t s);
// Grouped launch: l.gtab / l.gstart / l.gcount / l.calls point to device memory;
// total_tiles (host copy of gstart[gcount]) sizes the grid.
cudaError_t tc_gemm_launch_grouped(const TcLaunch &l, int bn, int total_tiles, int num_sms,
                                   cudaStream_t s);
// Fused launch: l.gtab / l.gstart / l.gcount hold every product of a solve in
// dependency order; l.tile_counter and l.done point to zeroed device counters.
// strips: the table carries per-strip dependencies (square tiles: bn 128 or kBnPair).
cudaError_t tc_gemm_launch_fused(const TcLaunch &l, int bn, int total_tiles, int num_sms,
                                 cudaStream_t s, bool strips = false);
constexpr int kEpiWarpsPublic = 8;  // completion count per tile of a fused launch
cudaError_t f64_gemm_launch(const F64Launch &l, cudaStream_t s);

// Ingest: column norms of the tall matrix and ||A||_F^2, summed in FP64 (squares in
// FP32 over four values first unless f64, the FP64 tier).
// wide = 0: tall matrix is A (M = m, N = n), colnorm2[j] = sum_i A[i][j]^2.
// wide = 1: tall matrix is A^T (M = n, N = m), colnorm2[i] = sum_j A[i][j]^2.
cudaError_t ingest_reduce_launch(const float *A, int64_t m, int64_t n, int64_t lda, int wide,
                                 int f64, double *colnorm2, double *scal, int *status,
                                 cudaStream_t s);

// Ingest: alpha = 2^round(log2 ||A||_F), X0 = A_tall / alpha written as
//   xs (same orientation as A): hi (and lo when xs_lo), leading dim ld_s;
//   xt (transposed): hi (and lo when xt_lo), leading dim ld_t;
// in BF16 (f64 = 0) or FP64 (f64 = 1, hi only). Also fills the scalar slots.
cudaError_t ingest_split_launch(const float *A, int64_t m, int64_t n, int64_t lda, float tau,
                                int f64, void *xs_hi, void *xs_lo, int64_t ld_s, void *xt_hi,
                                void *xt_lo, int64_t ld_t, double *scal, int *status,
                                cudaStream_t s);

// Final status: non-finite output norm -> DIVERGED (unless already set), then
// copy the internal status word to the caller's (if any).
cudaError_t finalize_launch(double *scal, int *status, svt_status *user_status, cudaStream_t s);

// Per-matrix record of the grouped memory-bound kernels (device table).
struct AuxRec {
    int64_t m, n;                    // input shape
    int wide, f64;
    double *scal;                    // scalar slots; scal .. scal + zero_words are cleared
    int *status;
    double *colnorm;
    int64_t zero_words;              // 8-byte words from scal to the end of colnorm
    void *xs_hi, *xs_lo;             // same-orientation copy of X0 (hi, lo)
    int64_t ld_s;
    void *xt_hi, *xt_lo;             // transposed copy
    int64_t ld_t;
    int blk_reduce, blk_split;       // first block of this matrix in the grouped grids
};

// Grouped memory-bound kernels over `count` matrices (records and call table in
// device memory; blocks_* = total blocks, i.e. the last record's start + its blocks).
cudaError_t grouped_zero_launch(const AuxRec *recs, int count, cudaStream_t s);
cudaError_t grouped_reduce_launch(const AuxRec *recs, const CallRec *calls, int count,
                                  int blocks_reduce, cudaStream_t s);
cudaError_t grouped_split_launch(const AuxRec *recs, const CallRec *calls, int count,
                                 int blocks_split, cudaStream_t s);
cudaError_t grouped_finalize_launch(const AuxRec *recs, const CallRec *calls, int count,
                                    cudaStream_t s);
// Blocks the grouped reduce / split kernels use for one m x n matrix.
int grouped_reduce_blocks(int64_t m, int64_t n, int wide);
int grouped_split_blocks(int64_t m, int64_t n);

// Host schedule (schedule.cpp).
// coef[3t..3t+2] = (a_t, b_t, c_t); lo_out (nullable) receives the lower end l_t of
// the interval step t was designed for.
int schedule_coeffs(int kind, int iters, double ell0, double delta, double *coef,
                    double *lo_out = nullptr);

// Tensor-map encoders (driver entry point resolved through the runtime).
// Operand loads: BF16, box 64 (K) x box_rows, 128-byte swizzle.
bool encode_bf16_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld,
                     int box_rows);
// e4m3 operand loads (FP8 experiment): box 128 (K) x box_rows, 128-byte swizzle.
bool encode_e4m3_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld,
                     int box_rows);
// Epilogue stores: BF16 (64-byte swizzle) or FP32 (128-byte swizzle), box 32 x 32.
bool encode_store_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld,
                      bool f32);
// Fill mapO / mapT of a problem from its epilogue's outputs where they qualify.
void attach_store_maps(TcProblem &p);

} // namespace svt
