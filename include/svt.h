/*
 * svt.h -- C ABI of libsvt: singular value soft-thresholding without an SVD,
 * on one GB300 GPU (sm_103a).
 *
 * What it computes (Becker, "Singular value soft-thresholding via the polar
 * decomposition"):
 *
 *   Eq. 1:           A_tau = U max(Sigma - tau I, 0) V^T
 *   Proposition 1:   A_tau = 1/2 (A + A S) - tau/2 (P + P S)
 *                    with P = polar(A), S = polar(A^T A - tau^2 I)
 *   (factored form)  A_tau = 1/2 (A - tau P)(I + S)
 *   Footnote:        for n > m, S = polar(A A^T - tau^2 I) and
 *                    A_tau = 1/2 (I + S)(A - tau P)
 *
 * The shift is tau^2 (the paper's code listing, Section 4); the proposition as
 * printed writes tau I, which does not split the spectrum at sigma = tau.
 * P and S are computed by odd-polynomial polar iterations that use only matrix
 * products (Section 1: Newton-Schulz; Section 3: Polar Express), on tensor cores.
 *
 * Conventions shared by every entry point:
 *   - Matrices are row-major FP32 in DEVICE memory; element (i, j) of an m x n
 *     matrix with leading dimension ld is at ptr[i * ld + j]; ld >= n.
 *   - The caller owns every buffer it passes (A, Y, workspace, status words).
 *     The library never frees caller memory and allocates no device memory on
 *     any solve path; all scratch lives in the workspace given to
 *     svt_ctx_create.
 *   - Argument errors are returned synchronously (SVT_ERR_INVALID) before any
 *     launch, like the paper's ValueError on non-2-D input (Section 4).
 *   - Errors found on the device (non-finite input, divergence, a device wait
 *     that ran out of time) are written to the caller's device status word
 *     (svt_status, 4 bytes) when one is given, and are returned by
 *     svt_ctx_sync / svt_serve_poll.
 *   - Streams are cudaStream_t passed as void* (NULL = legacy default stream).
 *   - A context is not thread-safe, except svt_serve_submit / svt_serve_poll,
 *     which may be called from any thread. All solves of one context share its
 *     workspace, so their work must be ordered on the device (one stream, or
 *     streams synchronised by the caller); serving must be idle while
 *     svt_polar / svt_batch run (they return SVT_ERR_BUSY otherwise).
 */
#ifndef SVT_H
#define SVT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SVT_OK = 0,
    SVT_ERR_INVALID = 1,   /* bad argument (null pointer, size, ld, tau, iters) */
    SVT_ERR_OOM = 2,       /* workspace or admission budget too small */
    SVT_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    SVT_ERR_NONFINITE = 4, /* input contains NaN or Inf (found on the device) */
    SVT_ERR_DIVERGED = 5,  /* iteration produced a non-finite value */
    SVT_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up */
    SVT_ERR_NOT_READY = 7, /* serving ticket still pending */
    SVT_ERR_BUSY = 8,      /* serving queue full; or a request too far along to cancel */
    SVT_ERR_UNSUPPORTED = 9, /* size or option outside what this build supports */
    SVT_ERR_CANCELLED = 10 /* serving request cancelled by svt_serve_cancel */
} svt_status;

typedef enum {
    SVT_FP64 = 0, /* every step in FP64 (SIMT); correctness tier, small inputs */
    SVT_FP32 = 1, /* every product FP32-class: three BF16 tensor-core products
                     (hi*hi + hi*lo + lo*hi) with FP32 accumulation */
    SVT_BF16 = 2, /* polynomial steps in BF16 (FP32 accumulation); Gram, polish
                     and combine FP32-class; norms and the tau^2 shift in FP64 */
    SVT_FP8_EXPERIMENTAL = 3 /* no FP8 tier: every entry point but svt_polar_fp8 and
                     svt_workspace_bytes_fp8 returns SVT_ERR_UNSUPPORTED for it. Those two
                     take it as the BF16 tier plus an e4m3 step policy; measured, no policy
                     is both faster and within the BF16 tier's 2e-2: an e4m3 rounding of
                     an early iterate moves the matrix whose polar factor the later steps
                     converge to, they do not undo it */
} svt_precision;

typedef enum {
    SVT_SCHED_AUTO = 0, /* PE5 */
    SVT_SCHED_PE5 = 1,  /* Polar-Express-style minimax odd quintics (Section 3) */
    SVT_SCHED_NS3 = 2   /* cubic Newton-Schulz X (3/2 I - 1/2 X^T X) (Section 1) */
} svt_schedule_kind;

typedef enum {
    SVT_NORM_AUTO = 0, /* GRAM for PE5, FRO for NS3 */
    SVT_NORM_FRO = 1,  /* divide the chain's start by its Frobenius norm */
    SVT_NORM_GRAM = 2  /* divide by ||X0^T X0||_F^(1/2) (>= ||X0||_2, tighter) */
} svt_norm_kind;

typedef enum {
    SVT_MODE_SVT = 0,    /* A_tau (Proposition 1) */
    SVT_MODE_RANK_R = 1  /* Corollary 1: 1/2 (A + A S), the best rank-r
                            approximation when tau lies between sigma_{r+1}
                            and sigma_r; the P chain is skipped */
} svt_mode;

/* Per-solve options. svt_options_default fills the defaults noted here. */
typedef struct {
    int iters;                  /* polynomial steps per chain, >= 0 (default 20) */
    svt_precision prec;         /* default SVT_BF16 */
    svt_schedule_kind schedule; /* default SVT_SCHED_AUTO */
    svt_norm_kind norm;         /* default SVT_NORM_AUTO */
    double ell0;                /* PE5 lower end of the first interval, in (0,1)
                                   (default 1e-3) */
    double delta;               /* PE5 interval widening (default: 0.01 BF16,
                                   1e-4 FP32, 0 FP64); < 0 selects the default */
    int polish;                 /* 1: one cubic Newton-Schulz step per chain in
                                   the FP32-class tier after the iterations
                                   (default 1; ignored for SVT_FP64, which
                                   polishes in FP64) */
    svt_mode mode;              /* default SVT_MODE_SVT */
    int fuse;                   /* 1 (default): all product launches of a solve run as
                                   one persistent launch whose tiles wait on the
                                   problems they read (device-side dependency
                                   counters); 0: one launch per product stage */
    int hp_steps;               /* SVT_BF16 only: number of leading S-chain steps run
                                   in the FP32-class tier (the shifted Gram's small
                                   eigenvalues sigma^2 - tau^2 do not survive BF16
                                   rounding until the iteration has spread them);
                                   -1 (default) = every step whose design interval
                                   starts below 0.1 */
    int tile;                   /* product tiles (BF16 / FP32 tiers, svt_polar_ex):
                                   0 (default) = automatic (svt_autotune's choice
                                   when it ran for this shape); 128 or 256 = one
                                   CTA per 128 x 128 or 128 x 256 tile; 512 = a
                                   cluster of two CTAs per 256 x 256 tile
                                   (tcgen05 cta_group::2, each CTA staging half of
                                   the tile's operands). A grouped batch takes 128
                                   or 256 from its matrices' options (0 or 512:
                                   chosen by a cost model, see svt_autotune_batch);
                                   serving chooses its own tiles. Other values:
                                   SVT_ERR_INVALID */
} svt_options;

typedef struct svt_ctx *svt_ctx_t;

/* One matrix of a batch or one serving request. */
typedef struct {
    const float *A;      /* m x n device, row-major, leading dimension lda */
    int64_t m, n, lda;
    float tau;           /* threshold, finite, >= 0 */
    float *Y;            /* m x n device output, leading dimension ldy */
    int64_t ldy;
    svt_options opt;     /* per-matrix options */
    svt_status *d_status; /* nullable device status word for this matrix */
} svt_matrix;

/* Human-readable name of a status code. Never NULL. */
const char *svt_status_str(svt_status s);

/* Fill *opt with the defaults documented in svt_options. */
void svt_options_default(svt_options *opt);

/*
 * Device workspace one solve of an m x n matrix needs (bytes), for the given
 * options (NULL = defaults). Pure host arithmetic.
 * Errors: SVT_ERR_INVALID on m, n <= 0 or out == NULL.
 */
svt_status svt_workspace_bytes_ex(int64_t m, int64_t n, const svt_options *opt, size_t *out);

/* Same with default options and the given precision. */
svt_status svt_workspace_bytes(int64_t m, int64_t n, svt_precision prec, size_t *out);

/*
 * Create a context on CUDA device `device` that uses the caller's device buffer
 * `workspace` (ws_bytes bytes, 256-byte aligned) for all scratch. The context
 * creates two CUDA streams and a few events and keeps a cache of launch plans;
 * it allocates no device memory.
 * Errors: SVT_ERR_INVALID (null out, misaligned or null workspace with
 * ws_bytes > 0), SVT_ERR_CUDA.
 */
svt_status svt_ctx_create(int device, void *workspace, size_t ws_bytes, svt_ctx_t *out);

/* Stop the serving thread (if started), wait for the context's streams and free
 * the context's host state. The workspace stays the caller's. */
svt_status svt_ctx_destroy(svt_ctx_t ctx);

/*
 * svt_polar: Y = A_tau for one m x n matrix, enqueued on `stream`.
 *   A: m x n FP32 device (lda >= n), read only.  Y: m x n FP32 device (ldy >= n).
 *   A and Y must not overlap. tau: finite, >= 0. iters >= 0.
 *   prec: precision tier (see svt_precision); other options at their defaults.
 *   d_status: nullable device word; receives SVT_OK or a device-side error.
 * Branch: m >= n uses A^T A (n x n Gram); n > m uses A A^T (footnote), computed
 * as the tall problem of A^T with the result transposed back.
 * Returns SVT_OK once all work is enqueued (asynchronous), or a synchronous
 * error: SVT_ERR_INVALID, SVT_ERR_OOM (workspace too small),
 * SVT_ERR_UNSUPPORTED (SVT_FP64 above 4096 in either dimension), SVT_ERR_CUDA.
 */
svt_status svt_polar(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda,
                     float tau, int iters, svt_precision prec, float *Y, int64_t ldy,
                     svt_status *d_status, void *stream);

/* svt_polar with explicit options (NULL = defaults). Same contract. */
svt_status svt_polar_ex(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda,
                        float tau, const svt_options *opt, float *Y, int64_t ldy,
                        svt_status *d_status, void *stream);

/*
 * svt_polar_f64: the FP64 tier's A_tau (Eq. 1 through Proposition 1, every step in
 * FP64) stored in FP64, so that its accuracy is not capped by an FP32 output's
 * rounding (~6e-8 relative).
 *   A: m x n FP32 device (lda >= n), read only. Y: m x n FP64 device, row-major,
 *   leading dimension ldy >= n, not overlapping A. opt: as svt_polar_ex; opt must
 *   not be NULL and opt->prec must be SVT_FP64. Other arguments as svt_polar.
 * Errors: as svt_polar_ex; SVT_ERR_INVALID when opt is NULL or names another tier.
 */
svt_status svt_polar_f64(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda,
                         float tau, const svt_options *opt, double *Y, int64_t ldy,
                         svt_status *d_status, void *stream);

/*
 * svt_batch: A_tau for `count` independent matrices of any sizes, enqueued on
 * `stream`. When all matrices share one option set with the default pipeline
 * (BF16 or FP32 tier, polish on, SVT mode), every product of every matrix (both
 * chains, all stages) runs as ONE persistent launch whose tiles wait on device-side
 * counters only for the earlier products of their own matrix, between grouped
 * ingest and finalize kernels; the sequence is captured once per batch shape
 * signature into a CUDA graph and replayed. Other batches run as per-matrix solves
 * over the context's worker streams. The workspace must hold the sum of the
 * matrices' workspaces plus the launch tables (svt_batch_workspace_bytes).
 * A second call with the same shape signature waits (on the host) until the first
 * call's call table has been consumed.
 * Errors: as svt_polar, checked for every matrix before any launch.
 */
svt_status svt_batch(svt_ctx_t ctx, const svt_matrix *mats, int count, void *stream);

/* Workspace bytes svt_batch needs for these matrices. */
svt_status svt_batch_workspace_bytes(const svt_matrix *mats, int count, size_t *out);

/*
 * Serving (continuous batching). svt_serve_submit copies the request descriptor
 * (A and Y stay caller-owned device memory and must stay valid until the ticket
 * completes) into the admission queue and returns a ticket. A scheduler thread
 * admits queued requests while their workspaces fit in the context's workspace
 * and a slot is free, advances all admitted requests one stage window at a time
 * with one grouped launch per window, and retires finished requests. Requests of
 * at least 8 Mi elements take the large lane instead, one at a time: a fused solve
 * issued as consecutive launches of a few milliseconds each, on every SM while no
 * smaller request is waiting or running and on all but 32 SMs otherwise.
 * Errors: SVT_ERR_INVALID (bad request), SVT_ERR_OOM (request larger than the
 * whole workspace), SVT_ERR_BUSY (queue full).
 */
svt_status svt_serve_submit(svt_ctx_t ctx, const svt_matrix *req, uint64_t *ticket);

/*
 * Poll a ticket: SVT_ERR_NOT_READY while pending; otherwise the request's final
 * status (SVT_OK or the device-side error), with the submit-to-completion
 * latency in milliseconds in *latency_ms (nullable). A completed ticket can be
 * polled again until svt_serve_release.
 */
svt_status svt_serve_poll(svt_ctx_t ctx, uint64_t ticket, double *latency_ms);

/* Forget a completed ticket. SVT_ERR_NOT_READY if still pending. */
svt_status svt_serve_release(svt_ctx_t ctx, uint64_t ticket);

/*
 * Cancel a serving request. A request still in the admission queue is removed at
 * once; one whose stages are being issued window by window is dropped before its
 * next window and retired once its work already on the device has finished; a large
 * request is dropped the same way before its next launch. Either
 * way the ticket then polls as SVT_ERR_CANCELLED and its Y is unspecified (the
 * combine that writes Y may or may not have run). Returns SVT_OK when the request
 * is or will be cancelled, SVT_ERR_BUSY when its remaining work is already on the
 * device (its last stage or launch went out, or it is an FP64-tier large request,
 * issued whole: poll for its result), SVT_ERR_INVALID for an unknown or completed
 * ticket.
 */
svt_status svt_serve_cancel(svt_ctx_t ctx, uint64_t ticket);

/*
 * Per-request records of the serving loop: from this call on, every retired request
 * (completed, failed or cancelled) appends one JSON line to the file at `path`:
 *   {"ticket", "m", "n", "prec", "tau", "iters", "lane" ("small" | "large"),
 *    "queue_ms" (submit to admission), "run_ms" (admission to retirement),
 *    "latency_ms" (submit to retirement), "status"}.
 * path = NULL stops recording. The environment variable SVT_SERVE_METRICS=<path>
 * starts recording when the serving loop starts.
 * Errors: SVT_ERR_INVALID (null ctx, or a file that cannot be opened for appending).
 */
svt_status svt_serve_metrics(svt_ctx_t ctx, const char *path);

/* Wait for all work of the context (svt_polar/svt_batch streams and serving)
 * and return the first device-side error recorded since the last sync. */
svt_status svt_ctx_sync(svt_ctx_t ctx, void *stream);

/*
 * The polynomial schedule the library uses (host arithmetic, no GPU):
 * coefficients (a_t, b_t, c_t) of p_t(x) = a x + b x^3 + c x^5 for t < iters,
 * written to coef[3 t .. 3 t + 2]. kind SVT_SCHED_NS3 gives (1.5, -0.5, 0).
 * PE5: each p_t minimises max |1 - p(x)| over [l_t, (1 + delta) u_t] (Remez),
 * [l_0, u_0] = [ell0, 1], and the next interval is [1 - E_t, 1 + E_t]; once the
 * design interval is narrower than 1e-3 the step is (15/8, -5/4, 3/8).
 * Errors: SVT_ERR_INVALID (iters < 0, coef NULL with iters > 0, ell0 not in (0,1),
 * delta < 0).
 */
svt_status svt_schedule_coeffs(svt_schedule_kind kind, int iters, double ell0, double delta,
                               double *coef);

/*
 * Diagnostic entry point for the tensor-core product kernel (used by the tests):
 *   D = sum_s L_s R_s^T with nseg in {1, 2, 3} segments taken from hi/lo parts:
 *     nseg 1: L_hi R_hi^T
 *     nseg 2: L_hi R_hi^T + L_hi R_lo^T
 *     nseg 3: L_hi R_hi^T + L_hi R_lo^T + L_lo R_hi^T
 *   L parts are M x K BF16 row-major (leading dimension ldl), R parts N x K BF16
 *   row-major (ldr); ldl and ldr multiples of 8, device pointers 16-byte
 *   aligned, unused parts may be NULL. FP32 accumulation in tensor memory; D is
 *   written as FP32 row-major (ldd >= N). sym = 1 computes only the tiles on or
 *   above the diagonal and mirrors them (requires M == N).
 * Errors: SVT_ERR_INVALID, SVT_ERR_CUDA.
 */
svt_status svt_debug_gemm_bf16(svt_ctx_t ctx, int nseg, const void *L_hi, const void *L_lo,
                               const void *R_hi, const void *R_lo, int64_t M, int64_t N,
                               int64_t K, int64_t ldl, int64_t ldr, float *D, int64_t ldd,
                               int sym, void *stream);

/*
 * svt_prox_grad_step: one proximal-gradient step of nuclear-norm regularised
 * matrix completion, the use of singular value soft-thresholding that Section 2
 * names (SVT is the proximal operator of tau ||.||_*):
 *   minimise F(X) = 1/2 ||P_Omega(X - M)||_F^2 + lambda ||X||_*,
 *   Z = X + step P_Omega(M - X);  X <- A_{step lambda}(Z)   (Eq. 1, via svt_polar_ex).
 * The smooth part's gradient has Lipschitz constant 1, so 0 < step <= 1 does not
 * increase F.
 *   X: m x n FP32 device (ldx >= n), the iterate, read and overwritten in place.
 *   M: m x n FP32 device (ldm >= n), the observed matrix (entries off Omega ignored).
 *   mask: m x n bytes device (ldw >= n), nonzero = observed (Omega).
 *   Z: m x n FP32 device scratch (ldz >= n), overlapping none of X, M, mask; holds
 *      the gradient step on return.
 *   step: finite, > 0. lambda: finite, >= 0. opt: as svt_polar_ex (NULL = defaults).
 *   d_status: nullable device word for the solve's device-side status.
 * Asynchronous on `stream`: a memory-bound masked-update kernel, then the solve.
 * Errors (before any launch): SVT_ERR_INVALID (null pointers, sizes, leading
 * dimensions, step, lambda, options, overlapping buffers), SVT_ERR_OOM (the
 * context's workspace is smaller than svt_workspace_bytes_ex(m, n, opt)),
 * SVT_ERR_UNSUPPORTED, SVT_ERR_BUSY (serving active), SVT_ERR_CUDA.
 */
svt_status svt_prox_grad_step(svt_ctx_t ctx, float *X, int64_t ldx, const float *M, int64_t ldm,
                              const uint8_t *mask, int64_t ldw, float *Z, int64_t ldz, int64_t m,
                              int64_t n, float step, float lambda, const svt_options *opt,
                              svt_status *d_status, void *stream);

/*
 * svt_complete: proximal-gradient matrix completion (the problem of
 * svt_prox_grad_step) run as one device-resident loop, with lambda continuation and
 * a stopping test on the iterates; the host issues one graph launch and is not
 * involved again until the run ends.
 *
 * Stage k = 0, 1, ... solves at lambda_k = max(lambda, lambda0 eta^k); the stage
 * with lambda_k == lambda is the last. A stage repeats proximal-gradient steps
 *   Z = X + step P_Omega(M - X);  X <- A_{step lambda_k}(Z)
 * until the relative change rho = ||X_new - X_old||_F / ||P_Omega(M)||_F (FP64,
 * against the data's scale so that it stays meaningful for a zero or nearly zero
 * iterate; 0 when both norms are zero) is <= tol, or until it has run stage_steps
 * steps (stages before the last; 0 = no cap). The run ends when the last stage stops, after max_steps steps in all,
 * or at the first solve whose device-side status is not SVT_OK. At a fixed lambda
 * the step map is non-expansive, so ||X_new - X_old||_F does not grow within a stage,
 * and ||P_Omega(M - X_new)||_2 <= lambda_k + (1 + 1/step) ||X_new - X_old||_F.
 *
 * The loop is a CUDA graph: one conditional WHILE node per stage whose body is the
 * masked gradient step (which also copies X to Xprev), the solve's launches, an FP64
 * reduction of ||X - Xprev||_F^2, and a one-thread kernel that updates
 * *d_stats and decides whether the body runs again. Graphs are cached on the context
 * per argument set (the four most recent); a repeated call relaunches its graph.
 *
 *   X, M, mask, Z: as svt_prox_grad_step (X: the starting point, overwritten with the
 *     result).
 *   Xprev: m x n FP32 device scratch (ldp >= n), overlapping none of X, M, mask, Z.
 *   p: the parameters below. opt: as svt_polar_ex (NULL = defaults).
 *   d_stats: device, 8-byte aligned, written by the run (any earlier contents are
 *     ignored); valid once the stream reaches the end of the run.
 * Asynchronous on `stream`. The context's workspace is in use until the run ends.
 * svt_ctx_launch_count counts the run as one launch.
 * Errors (before any launch): SVT_ERR_INVALID (pointers, sizes, leading dimensions,
 * overlapping buffers, parameters outside the ranges below, more than 64 stages,
 * options), SVT_ERR_OOM (workspace), SVT_ERR_BUSY (serving active),
 * SVT_ERR_UNSUPPORTED (sizes, or a driver without conditional graph nodes),
 * SVT_ERR_CUDA.
 */
typedef struct {
    float lambda;     /* target lambda, finite, >= 0 */
    float lambda0;    /* lambda of the first stage, finite, >= lambda (== lambda: one stage) */
    float eta;        /* stage factor, in (0, 1) when lambda0 > lambda (else ignored) */
    float step;       /* proximal-gradient step, finite, > 0 (<= 1 does not increase F) */
    float tol;        /* relative-change tolerance, finite, >= 0 */
    int max_steps;    /* steps in all stages, >= 0 */
    int stage_steps;  /* steps per stage before the last, >= 0 (0 = no cap) */
} svt_completion_params;

typedef struct {
    int steps;          /* proximal-gradient steps taken */
    int stages;         /* stages entered */
    int stage_steps;    /* steps of the last stage entered */
    int status;         /* SVT_OK, or the first solve's non-OK device-side status */
    int solve_status;   /* device-side status of the last solve */
    int reserved;
    double lambda;      /* lambda of the last step */
    double rel_change;  /* rho of the last step */
    double diff2;       /* reduction accumulator (zero between steps) */
    double data2;       /* ||P_Omega(M)||_F^2 */
} svt_completion_stats;

svt_status svt_complete(svt_ctx_t ctx, float *X, int64_t ldx, const float *M, int64_t ldm,
                        const uint8_t *mask, int64_t ldw, float *Z, int64_t ldz, float *Xprev,
                        int64_t ldp, int64_t m, int64_t n, const svt_completion_params *p,
                        const svt_options *opt, svt_completion_stats *d_stats, void *stream);

/* svt_debug_gemm_bf16 with an explicit tile-width code: 0 = automatic (as
 * svt_debug_gemm_bf16), 128, 256, or 512 (a cluster of two CTAs per 256 x 256
 * tile, tcgen05 cta_group::2). Errors: as above; SVT_ERR_INVALID on another tile. */
svt_status svt_debug_gemm_bf16_ex(svt_ctx_t ctx, int nseg, const void *L_hi, const void *L_lo,
                                  const void *R_hi, const void *R_lo, int64_t M, int64_t N,
                                  int64_t K, int64_t ldl, int64_t ldr, float *D, int64_t ldd,
                                  int sym, int tile, void *stream);

/*
 * FP8 experiment (the lower precision Section 3 weighs for speed): a BF16-tier solve
 * with chosen polynomial steps on e4m3 operands (tcgen05.mma kind::f8f6f4, FP32
 * accumulation). The products that write the operands also write e4m3 copies of them,
 * scaled by powers of two fixed from the iterates' bounds (|entries| <= 1.03 -> x 256,
 * saturated at 448); the BF16 results stay for everything else.
 */
typedef struct {
    uint64_t p_steps;  /* bit t: the P chain's Z = a I + b Y + c Y^2 of step t takes Y^2 from
                          an e4m3 copy of Y = X^T X (quintic steps) */
    uint64_t s_steps;  /* bit t: S-chain step t (t >= 1, a BF16 step: past the leading
                          FP32-class steps; other bits are ignored) runs Y = S^2, Y^2 and
                          S Z on e4m3 operands */
    int s_y2_only;     /* 1: in those S steps only the Y^2 product */
    int reserved;      /* 0 */
} svt_fp8_policy;

/* Workspace svt_polar_fp8 needs: svt_workspace_bytes_ex of the BF16 tier plus one
 * e4m3 k x k copy (k = min(m, n), rows padded) for p_steps != 0 and four for
 * s_steps != 0. Errors: SVT_ERR_INVALID (null out or policy, non-zero reserved, a
 * tier other than SVT_BF16 / SVT_FP8_EXPERIMENTAL), as svt_workspace_bytes_ex. */
svt_status svt_workspace_bytes_fp8(int64_t m, int64_t n, const svt_options *opt,
                                   const svt_fp8_policy *policy, size_t *out);

/* svt_polar_ex with the FP8 policy: opt->prec must be SVT_BF16 or SVT_FP8_EXPERIMENTAL
 * (both: the BF16 tier plus the policy); opt may be NULL (defaults). Same contract
 * otherwise, with the workspace of svt_workspace_bytes_fp8. Errors: as svt_polar_ex;
 * SVT_ERR_INVALID for a null policy, a non-zero reserved field or another tier.
 *
 * Measured on a GB300 (4096^2 inputs, 20 steps): e4m3 in the early steps of either
 * chain leaves the result outside the BF16 tier's 2e-2 (0.24-1.1 in the P chain; the
 * S chain diverges or reaches 4-5 %); Y^2 alone in the last five steps of either chain
 * stays within it (1.01e-2 and 1.07e-2 against 1.00e-2 BF16 on a gapped spectrum) and
 * is about 8 % slower: the products it speeds up are few and the e4m3 copies are extra
 * stores. No policy is faster at the BF16 tier's accuracy. */
svt_status svt_polar_fp8(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda,
                         float tau, const svt_options *opt, const svt_fp8_policy *policy, float *Y,
                         int64_t ldy, svt_status *d_status, void *stream);

/* Diagnostic for the e4m3 product path (used by the tests): D = L R^T with L M x K and
 * R N x K e4m3 bytes, row-major (ldl, ldr in elements, multiples of 16; device pointers
 * 16-byte aligned), FP32 accumulation, D FP32 row-major (ldd >= N); tile as
 * svt_debug_gemm_bf16_ex. Errors: SVT_ERR_INVALID, SVT_ERR_CUDA. */
svt_status svt_debug_gemm_e4m3(svt_ctx_t ctx, const void *L, const void *R, int64_t M, int64_t N,
                               int64_t K, int64_t ldl, int64_t ldr, float *D, int64_t ldd, int tile,
                               void *stream);

/* Failure-path check of the device-side bounded waits: launches the product kernel
 * (fused form) on a one-tile table whose tile waits for its own completion, so the
 * wait runs out (about 2 s); the kernel records SVT_ERR_TIMEOUT in *d_status (device
 * word, initially SVT_OK), releases its resources and returns, and the context stays
 * usable. Overwrites the start of the context's workspace (any later solve restores
 * what it needs). Errors: SVT_ERR_INVALID, SVT_ERR_OOM (a workspace smaller than
 * the one-tile table), SVT_ERR_BUSY, SVT_ERR_CUDA. */
svt_status svt_debug_wait_timeout(svt_ctx_t ctx, svt_status *d_status, void *stream);

/* Number of kernel launches the library has issued on this context so far
 * (host counter; used to report launches per solve). */
uint64_t svt_ctx_launch_count(svt_ctx_t ctx);

/* Host-side fault injection and debug settings of a context (none makes the GPU
 * fault, trap or hang: each turns into an ordinary error status). */
typedef enum {
    /* value N >= 1: the Nth launch-plan build from now on fails with SVT_ERR_OOM
     * (plan builds are where the library allocates host memory: one per new shape
     * and option set); 0 turns it off. */
    SVT_DEBUG_FAIL_PLAN = 1,
    /* value in microseconds: serving admits a request no earlier than this long
     * after its submission (0: off). */
    SVT_DEBUG_ADMIT_DELAY_US = 2,
    /* value in nanoseconds: the product kernel's waits on other tiles' results (its
     * device-side dependency counters) give up after this long instead of 2 s and
     * report SVT_ERR_TIMEOUT in the solve's status; 1 makes any wait that is not
     * already satisfied time out at once. 0 restores the default. Applies to launches
     * issued (or captured into a batch's graph) after the call. */
    SVT_DEBUG_WAIT_LIMIT_NS = 3
} svt_debug_flag;

/* Set one debug setting (see svt_debug_flag). Errors: SVT_ERR_INVALID (null ctx,
 * unknown flag, negative value). */
svt_status svt_ctx_debug(svt_ctx_t ctx, svt_debug_flag flag, int64_t value);

/*
 * The context's autotune results (svt_autotune tile choices) as JSON text, to keep
 * them across contexts and processes:
 *   {"format": 1, "gpu": "<device name>", "sms": <SM count>, "entries": [
 *     {"m", "n", "iters", "prec", "schedule", "norm", "polish", "mode", "hp_steps",
 *      "ell0", "delta", "fuse", "widths": [tile width of each product launch]}, ...]}
 * Entries are keyed by the exact shape and the options that shape the launch
 * sequence (tier included); the file is keyed by the GPU's name and SM count.
 * svt_tuning_export writes at most cap bytes including the terminating NUL into buf
 * (buf may be NULL with cap 0) and the full length (without the NUL) into *len;
 * SVT_ERR_OOM when cap is too small (*len still set).
 * svt_tuning_import merges the entries of such text into the context (later solves
 * of those shapes and options use them); SVT_ERR_INVALID when the text does not
 * parse, is of another format, or was tuned on a GPU of another name or SM count
 * (nothing is imported then).
 */
svt_status svt_tuning_export(svt_ctx_t ctx, char *buf, size_t cap, size_t *len);
svt_status svt_tuning_import(svt_ctx_t ctx, const char *json);

/*
 * Measurement hooks. svt_ctx_profile(ctx, 1) makes every later tensor-core
 * launch of svt_polar / svt_polar_ex on this context record a CUDA event pair
 * on its own stream (0 turns it off; both reset the record).
 * svt_ctx_profile_read waits for the recorded events and returns, since the last
 * reset, the summed device time of those launches (ms), their summed
 * algorithmic flops (2 M N K per product, symmetric products counted at half,
 * hi/lo segments of FP32-class products not counted again) and their number;
 * then resets. Errors: SVT_ERR_INVALID (null argument), SVT_ERR_CUDA.
 */
svt_status svt_ctx_profile(svt_ctx_t ctx, int enable);
svt_status svt_ctx_profile_read(svt_ctx_t ctx, double *tc_ms, double *tc_flops,
                                uint64_t *tc_launches);
/* As svt_ctx_profile_read, plus (nullable) the flops the tensor cores executed in
 * those launches: every hi/lo segment product, whole tiles (the padding and the
 * diagonal tiles of symmetric products) and K rounded up to 64. Their ratio to the
 * algorithmic flops is the cost of the FP32-class products and of the tiling. */
svt_status svt_ctx_profile_read_ex(svt_ctx_t ctx, double *tc_ms, double *tc_flops,
                                   double *tc_tensor_flops, uint64_t *tc_launches);

/*
 * Autotuner for the product kernel's tiles. Runs the svt_polar_ex solve of this A
 * (m x n, lda), tau and options (NULL = defaults) with each tile mode (128 x 128,
 * 128 x 256, and CTA pairs on 256 x 256), once as warm-up and `reps` times timed
 * with CUDA events on `stream`. Fused solves (opt->fuse = 1, the default) keep the
 * mode with the shortest whole solve; unfused solves keep the fastest mode per
 * product launch. The choice is stored in the context; later svt_polar /
 * svt_polar_ex calls with the same shape and options and tile = 0 use it. Y
 * receives A_tau. Synchronises `stream`.
 * Errors: as svt_polar_ex; SVT_ERR_BUSY while serving requests are in flight.
 * The FP64 tier has no tile choice (returns SVT_OK without work).
 */
svt_status svt_autotune(svt_ctx_t ctx, const float *A, int64_t m, int64_t n, int64_t lda,
                        float tau, const svt_options *opt, float *Y, int64_t ldy, int reps,
                        void *stream);

/*
 * svt_autotune_schedule: picks the iteration schedule -- polynomial steps per chain
 * and ell0, the lower end of the first design interval of the Polar-Express-style
 * schedule -- for a class of inputs represented by A, in the tier `opt` names. The
 * paper leaves the iteration count open (maxIts: 11 in its code, 20 suggested, 25 in
 * its timings); this measures the fewest steps that reach a given accuracy.
 *   Reference: one FP32-tier solve of A with 32 steps and ell0 = 1e-3, into Yref.
 *   Candidates: ell0 in {1e-3, 1e-2}; steps 2, 3, 4, 5, 6, 8, 10, 12, 14, 16, 20, 24,
 *   28, 32 up to max_iters, in that order. For each ell0 the first step count whose
 *   deviation ||Y - Yref||_F / ||Yref||_F (FP64 reduction; relative to ||A||_F when
 *   Yref = 0) is <= target; the pick is the fewer steps (ties: ell0 = 1e-3). When no
 *   candidate reaches the target: max_iters with ell0 = 1e-3.
 *   opt: tier (BF16 or FP32) and the other options of the solves being tuned; its
 *     iters, ell0 and schedule are the tuned quantities and are ignored (NULL =
 *     defaults).
 *   target: finite, > 0 (e.g. 2e-2 for the BF16 tier). max_iters: 2 .. 32.
 *   Y, Yref: m x n FP32 device scratch (ldy, ldr >= n), overlapping neither A nor
 *     each other; Y holds the last candidate's result on return.
 *   Outputs: *iters_out, *ell0_out, and *dev_out, the pick's measured deviation.
 * Synchronous: waits for each candidate on `stream`. Allocates 16 bytes of device
 * memory for the reduction during the call (a tuning call, not a solve).
 * Errors: as svt_polar_ex; SVT_ERR_INVALID also for target, max_iters, null outputs,
 * overlapping buffers or the FP64 tier.
 */
svt_status svt_autotune_schedule(svt_ctx_t ctx, const float *A, int64_t m, int64_t n,
                                 int64_t lda, float tau, const svt_options *opt, double target,
                                 int max_iters, float *Y, int64_t ldy, float *Yref, int64_t ldr,
                                 int *iters_out, double *ell0_out, double *dev_out, void *stream);

/*
 * svt_autotune_batch: times the grouped batch `mats` with 128- and 256-wide product
 * tiles (one untimed call each, then `reps` timed svt_batch calls on `stream`) and
 * returns the faster width in *tile_out (and its mean time per batch in *ms_out,
 * nullable). Set svt_options.tile of the batch's matrices to it. The outputs of
 * `mats` are written by every call. Synchronous. Errors: as svt_batch;
 * SVT_ERR_INVALID for count <= 0, reps < 1 or a null tile_out.
 */
svt_status svt_autotune_batch(svt_ctx_t ctx, const svt_matrix *mats, int count, int reps,
                              void *stream, int *tile_out, double *ms_out);

/*
 * svt_polar_noalloc: the svt_polar_ex solve without any workspace from the
 * caller and without allocating device memory. (The paper has no counterpart:
 * this entry point exists for callers, not for the method.)
 *
 * For callers that cannot allocate device memory at call time -- code inside a
 * framework that owns all device allocations through its own pool, loops that
 * must not pay cudaMalloc's implicit synchronisation or risk an out-of-memory
 * failure at run time -- and that have no workspace to lend. Scratch comes from
 * one static device array of SVT_NOALLOC_SCRATCH_BYTES (32 MiB) that every GPU
 * loading the library reserves until the process exits; enough for BF16 and
 * FP32-tier solves up to about 768 x 768 and FP64-tier solves up to 512 x 512.
 *
 *   device: CUDA device to run on (made current for the call, then restored).
 *   A, m, n, lda, tau, opt, Y, ldy, d_status, stream: as svt_polar_ex.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and sets up an internal context; make that first call
 * before any stream capture. The first call for each new shape and option set
 * also builds a launch plan, which allocates a small pinned host buffer
 * (cudaMallocHost, a few KB per product of the solve) that later calls copy the
 * launch table from; that allocation may synchronise the device and is not
 * allowed under capture, so make those calls before any capture as well. The
 * internal context caches up to 64 plans; a call that finds 64 cached waits for
 * the device (cudaDeviceSynchronize) and drops them. All calls share the one
 * array and it keeps the
 * last call's contents (the solve re-initialises what must start at zero), so
 * calls whose GPU work overlaps -- on different streams or from different
 * threads without ordering -- race and corrupt each other's results.
 * Errors: as svt_polar_ex, plus SVT_ERR_UNSUPPORTED when the solve needs more
 * than SVT_NOALLOC_SCRATCH_BYTES (see svt_workspace_bytes_ex) and
 * SVT_ERR_INVALID for a device index outside [0, 64).
 */
#define SVT_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
svt_status svt_polar_noalloc(int device, const float *A, int64_t m, int64_t n, int64_t lda,
                             float tau, const svt_options *opt, float *Y, int64_t ldy,
                             svt_status *d_status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SVT_H */
