/*
 * mg.h - C ABI of the GB300 multigrid library (libmg.so).
 *
 * Solves the 2D periodic pressure-Poisson problem of the paper (Sec. 2.2,
 * Eq. poissoneq; Sec. 3.2, Eq. poisson_ns) on an N x N vertex grid,
 * h = 2 pi / N, with the 5-point operator A = -Lap_h,
 *     (A x)_ij = (4 x_ij - x_i+1,j - x_i-1,j - x_i,j+1 - x_i,j-1) / h^2,
 * periodic in both axes.  A is singular (constants), so the library returns
 * the zero-mean solution of the zero-mean part of f.
 *
 * Method: geometric multigrid V(nu_pre, nu_post) cycles (Fig. 1a; Appendix A,
 * Algorithm 6): red-black Gauss-Seidel smoothing (red = (i + j) even first),
 * residual, full-weighting restriction, recursion on the re-discretised
 * operator, exact pseudo-inverse solve on the coarsest grid, and one of two
 * coarse-to-fine prolongations (Sec. 2.2 and Sec. 3.1; Algorithm 5):
 *   MG_PROLONG_CUBIC - the periodic tensor-product cubic interpolating spline;
 *   MG_PROLONG_SR    - the cubic spline plus a learned super-resolution
 *                      correction s * G(e_c / s), s = max|e_c|, from a
 *                      convolutional generator (weights loaded separately).
 *
 * Precision: MG_PREC_FP64 runs plain FP64 V-cycles.  MG_PREC_MIXED runs FP32
 * V-cycles as the inner solver of FP64 defect correction: r = f - A x in
 * FP64, e ~ A^+ r by `inner_cycles` FP32 V-cycles from e = 0, x += e.
 * Convergence is tested on ||f - A x||_2 / ||f||_2 in FP64 in both modes.
 *
 * Memory layout: every grid is row-major, N x N, contiguous, index i*N + j
 * with j (x) the fast axis.  Pointers named "device or host" may point to
 * device memory or to host memory; host buffers are staged through the
 * context (copies on the context's stream, inside the call).
 *
 * Errors: every call returns an mg_status and never aborts the process.
 * mg_last_error() gives a one-line description of the most recent failure
 * on the calling thread.  Calls on one context are not thread-safe; distinct
 * contexts may be used from distinct threads.
 */
#ifndef MG_H
#define MG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_ctx mg_ctx; /* opaque: owns the level hierarchy and scratch */

typedef enum {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = 1,   /* bad size, pointer or option */
    MG_ERR_OOM = 2,           /* device allocation failed */
    MG_ERR_CUDA = 3,          /* a CUDA runtime call failed; see mg_last_error() */
    MG_ERR_NOT_CONVERGED = 4, /* max_cycles reached; x holds the last iterate */
    MG_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
    MG_ERR_NO_WEIGHTS = 6,    /* MG_PROLONG_SR requested with no weights loaded */
    MG_ERR_BAD_WEIGHTS = 7,   /* weight blob malformed */
    MG_ERR_NONFINITE = 8      /* f (or the iterate) holds NaN or Inf */
} mg_status;

typedef enum { MG_PROLONG_CUBIC = 0, MG_PROLONG_SR = 1 } mg_prolong;
typedef enum { MG_PREC_FP64 = 0, MG_PREC_MIXED = 1 } mg_precision;

typedef struct {
    int outer_iters;      /* FP64 residual evaluations after the first */
    int vcycles;          /* V-cycles run (FP32 in MIXED, FP64 in FP64) */
    double rel_residual;  /* final ||f - A x||_2 / ||f||_2 (FP64) */
    double removed_mean;  /* mean of f that was projected out */
    double update_norm;   /* ||x_k - x_{k-1}||_2 of the last update */
    double time_ms;       /* wall time of the call (host clock) */
    int prolong_used;     /* MG_PROLONG_SR if any V-cycle used SR, else MG_PROLONG_CUBIC */
    int sr_fallback;      /* 1 if SR was dropped for the rest of this solve (an outer
                             step using it did not halve the relative residual) */
    int sr_cycles;        /* V-cycles whose top prolongation was SR */
} mg_solve_info;

/* Create a context for N x N grids with `levels` levels (Fig. 1a hierarchy).
 * N must be a power of two, 8 <= N <= 16384, and the coarsest grid
 * N >> (levels - 1) must be 4, 8 or 16 (it is solved exactly).  Uses the
 * current CUDA device.  *out is set to NULL on failure. */
mg_status mg_setup(int levels, int N, mg_ctx **out);

/* Options (defaults: MG_PREC_MIXED, nu_pre = nu_post = 2, max_cycles = 100,
 * inner_cycles = 2, stream 0).  nu_pre / nu_post are the relaxation counts
 * before and after the coarse correction (Algorithm 6's relaxation step; the
 * smoothing count N_smooth of Sec. 4.2 and Table 1); max_cycles is the
 * iteration cap (Table 1's N_iter).  0 <= nu <= 4.  max_cycles bounds the V-cycles
 * of one mg_solve.  `cuda_stream` is a cudaStream_t (NULL = legacy stream);
 * all work of this context is ordered on it. */
mg_status mg_set_options(mg_ctx *ctx, mg_precision precision, int nu_pre, int nu_post,
                         int max_cycles, void *cuda_stream);
/* FP32 V-cycles per FP64 outer step of MIXED solves.  mg_set_inner_cycles
 * fixes the count (1..16; batched solves and the server always use this
 * count, default 2).  mg_set_adaptive_cycles (the default for single solves
 * with the cubic prolongation: m_max = 3, rho = 0.06) lets every outer step
 * run the smallest m in [1, m_max] with rel * rho^m <= tol, rel the relative
 * residual before the step and rho the expected contraction per V-cycle
 * (m_max <= 4; rho = 0 turns it off; mg_set_inner_cycles also turns it off).
 * The FP32 inner solve cannot reduce the residual by much more than 1e-5 per
 * outer step, which bounds useful m_max. */
mg_status mg_set_inner_cycles(mg_ctx *ctx, int inner_cycles);
mg_status mg_set_adaptive_cycles(mg_ctx *ctx, int m_max, double rho);

/* Execution mode of mg_solve (default 1).  1: the whole solve is one CUDA
 * graph launch - a WHILE conditional node runs the outer steps on the device
 * and a test kernel decides convergence, so the host synchronises once per
 * solve; graphs are recorded on first use per (f, x, prolongation, tol) and
 * cached (up to 4).  In this mode max_cycles is rounded down to a multiple of
 * inner_cycles.  0: a host loop with one residual read-back per outer step
 * (also used while a probe is active). */
mg_status mg_set_graph_execution(mg_ctx *ctx, int enable);

/* Prolongation policy of solves with MG_PROLONG_SR (the hybrid operator
 * choice of Sec. 4.2 and Algorithm 6).  n_gan >= 1: n_gan V-cycles with SR
 * per V-cycle with the cubic spline (n_gan = 1 alternates, INFINITY = SR
 * only); n_gan < 1: 1/n_gan cubic V-cycles per SR V-cycle (>= 1e-6).  V-cycle i
 * (1-based over the solve) uses the first operator (SR when n_gan >= 1, cubic
 * otherwise) when i mod (N + 1) != 0, N = n_gan or 1/n_gan rounded, and the
 * other one otherwise.  s_thres > 0: once the relative residual after an
 * outer step is <= s_thres, every later V-cycle uses the second operator.
 * Independently of the policy, an outer step that used SR and did not halve
 * the relative residual turns SR off for the rest of the solve
 * (mg_solve_info.sr_fallback).  Default: n_gan = INFINITY, s_thres = 0. */
mg_status mg_set_prolong_policy(mg_ctx *ctx, double n_gan, double s_thres);

/* Load super-resolution generator weights (Sec. 2.3, Fig. 1b).  The blob is
 * copied (the caller keeps ownership).  Blob layout: a 64-byte header
 * {magic "MGSRW001", u32 n_feat, u32 n_blocks, u32 n_params, 44 bytes 0}
 * followed by n_params little-endian float32 values in the order
 * in.w, in.b, in.a, then per block w1, b1, a, w2, b2, then up.w, up.b, up.a,
 * out.w, out.b (conv weights [out][in][3][3]).  n_feat must be 64.
 * Returns MG_ERR_BAD_WEIGHTS on any mismatch. */
mg_status mg_load_prolong_weights(mg_ctx *ctx, const void *blob, size_t bytes);

/* Cold starts (Algorithm 6 iterates from an initial guess; the configurations
 * here start from p = 0): with on = 1 the context's solves (mg_solve,
 * mg_two_level_solve) start from x = 0 and never read x, so a host x is not
 * copied to the device.  Mixed solves of N >= 32 with the fused outer step
 * (mg_set_fused_update) take x = 0 in their first residual and first update
 * without reading or zeroing x; other solves zero the device copy, or a
 * device x, first.  The result is bit for bit that of a solve from x = 0.
 * on = 0 (the default): x is the initial guess.  MG_ERR_INVALID_ARG for a
 * null context or other values. */
mg_status mg_set_zero_guess(mg_ctx *ctx, int on);

/* Solve A x = f to ||f - A x||_2 / ||f||_2 <= tol.  f: N*N doubles (device or
 * host), not modified.  x: N*N doubles (device or host), the initial guess on
 * entry (warm start; zeros for a cold start, or any contents after
 * mg_set_zero_guess(ctx, 1)) and the zero-mean solution on return.  info may
 * be NULL.  Returns MG_ERR_NOT_CONVERGED (x = last iterate)
 * if max_cycles V-cycles do not reach tol, MG_ERR_NONFINITE for NaN/Inf. */
mg_status mg_solve(mg_ctx *ctx, const double *f, double *x, double tol, mg_prolong prolong,
                   mg_solve_info *info);

/* One V(nu_pre, nu_post) cycle on A x = f, in place (Algorithm 6).  FP64
 * mode: one FP64 V-cycle on x.  MIXED mode: one defect-correction step with
 * one FP32 V-cycle.  x is not projected to zero mean. */
mg_status mg_vcycle(mg_ctx *ctx, const double *f, double *x, mg_prolong prolong);

/* The paper's two-level configuration (Sec. 4.1; Table 1: N_step = 4, one
 * coarse level 16 times coarser): FP64 defect correction as in mg_solve, each
 * outer step running one FP32 two-level cycle from e = 0 - nu_smooth
 * red-black Gauss-Seidel sweeps on the finest grid, the residual restricted by
 * 2^coarsen_log2 (full weighting applied coarsen_log2 times), coarse_sweeps
 * red-black sweeps of the coarse correction equation from zero (Algorithm 6's
 * coarsest-level relaxation), the coarse correction interpolated back by
 * 2^coarsen_log2 in one step with the periodic cubic spline (B-spline
 * coefficients by a truncated exact inverse filter, then the tensor cubic
 * B-spline at every fine point) and added; no post-smoothing.  MIXED contexts
 * with levels >= coarsen_log2 + 2 and N >> coarsen_log2 >= 64; 0 <= nu_smooth
 * <= 64; 1 <= coarse_sweeps <= 64.  prolong = MG_PROLONG_SR interpolates the
 * correction with the loaded generator instead (Sec. 2.3, Algorithm 5, which
 * applies the generator repeatedly): coarsen_log2 stages, each the cubic
 * spline by 2 plus the generator's correction s G(e / s), s = max|e|; it needs
 * weights (MG_ERR_NO_WEIGHTS), coarsen_log2 <= 8 and N >> coarsen_log2 >= 128;
 * the context's policy (mg_set_prolong_policy) picks SR or cubic per cycle,
 * and an SR cycle that does not reduce the relative residual turns SR off for
 * the rest of the solve (info->sr_fallback).  info->vcycles and
 * info->outer_iters count two-level cycles, info->sr_cycles those with SR;
 * MG_ERR_NOT_CONVERGED after max_cycles with the best x. */
mg_status mg_two_level_solve(mg_ctx *ctx, const double *f, double *x, double tol, int coarsen_log2, int nu_smooth,
                             int coarse_sweeps, int max_cycles, mg_prolong prolong, mg_solve_info *info);

/* Solve B independent problems, ctxs[k] with f[k], x[k], each to tol (the
 * batched form of Algorithm 6 over many right-hand sides; the paper solves
 * grids one at a time).  Contexts may have different N.  When every context
 * is MG_PREC_MIXED with the same nu_pre, nu_post, inner_cycles and
 * max_cycles and all buffers are in device memory, the whole batch runs as
 * one CUDA graph: each V-cycle of the batch is one launch per grid size and
 * direction (every right-hand side with a level of that size takes part) plus
 * one launch for all coarse levels, the FP64 outer steps are one launch each,
 * and a right-hand side stops once it has converged.  With MG_PROLONG_SR
 * (every context loaded with the same weights) the finest transition of each
 * right-hand side whose coarse grid is >= 128 (a multiple of 128) adds the
 * generator's correction (Algorithm 5): one generator launch per layer and
 * grid size serves all right-hand sides of that size, SR on every V-cycle,
 * inner_cycles V-cycles per outer step, and a right-hand side whose outer
 * step did not halve its relative residual drops SR for the rest of its
 * solve (infos[k].sr_fallback); smaller grids use the cubic spline.  The
 * graph is kept for the next call with the same contexts, buffers and
 * prolongation (the stream is the first context's).  Otherwise the problems
 * are solved one after another.  Returns the first non-MG_OK status
 * (MG_ERR_TIMEOUT if a bounded wait of the generator expired); infos (may be
 * NULL) get one entry each. */
mg_status mg_solve_batched(mg_ctx *const *ctxs, const double *const *f, double *const *x, int B,
                           double tol, mg_prolong prolong, mg_solve_info *infos);

/* ---------------------------------------------------------------------
 * Continuous-batching server (mixed precision, cubic prolongation).
 * Requests wait in a FIFO until a slot - a resident level hierarchy plus f
 * and x of the request's size - and the device-memory budget allow
 * admission.  Each mg_server_tick runs one outer step of defect correction
 * (FP64 residual, inner_cycles FP32 V-cycles, FP64 update) for every admitted
 * request as batched launches: new requests start with their first residual
 * while the others continue, and requests that converged are retired (zero-
 * mean projection, the solution copied to x_out, and kept on the device as the
 * warm start of the next request of the same stream_id and N).  Requests thus
 * join and leave between ticks while the rest of the batch keeps running.
 * ------------------------------------------------------------------- */
typedef struct mg_server mg_server;

/* Create a server on the current device.  hbm_budget_bytes bounds the device
 * memory of its slots, warm starts and tables; other arguments as for
 * mg_set_options, except that inner_cycles = 0 (0 <= inner_cycles <= 16)
 * selects adaptive V-cycles per outer step: a request's first step runs 3,
 * each later one the count mg_set_adaptive_cycles' rule (m_max 3, rho 0.06)
 * gives for the relative residual the request is predicted to have, i.e. its
 * last measured one times its own observed contraction per V-cycle to the
 * power of the V-cycles run since; the count depends only on the request's
 * own history, never on the rest of the batch.  Work is ordered on
 * cuda_stream. */
mg_status mg_server_create(size_t hbm_budget_bytes, int nu_pre, int nu_post, int inner_cycles, int max_cycles,
                           double tol, void *cuda_stream, mg_server **out);

/* Queue a request: N x N source f (host or device, read when the request is
 * admitted, so it must stay valid until then), solution written to x_out
 * (host or device, may be NULL) when it retires.  stream_id >= 0 enables warm
 * starts across requests of one stream; -1 means none.  request_id (may be
 * NULL) receives the id that mg_server_poll reports. */
mg_status mg_server_submit(mg_server *srv, int stream_id, int N, const double *f, double *x_out,
                           long long *request_id);

/* Admit what fits, run one outer step for all admitted requests, retire the
 * converged ones.  Synchronous.  Outputs (may be NULL): requests in flight,
 * requests still queued, requests retired by this tick. */
mg_status mg_server_tick(mg_server *srv, int *n_active, int *n_queued, int *n_done);

/* One retired request.  Times are milliseconds on the server's monotonic
 * clock (zero at mg_server_create); info.time_ms = t_finish_ms - t_submit_ms. */
typedef struct mg_server_result {
    long long request_id;
    int stream_id;
    int N;
    mg_status status;
    int pad;
    double t_submit_ms;
    double t_admit_ms;
    double t_finish_ms;
    mg_solve_info info;
} mg_server_result;

/* Pop the oldest retired request into *result (*got = 1), or set *got = 0. */
mg_status mg_server_poll(mg_server *srv, mg_server_result *result, int *got);

void mg_server_destroy(mg_server *srv);

/* ---------------------------------------------------------------------
 * Tile-shape autotuning (no counterpart in the paper: an implementation
 * choice of this library).  The FP32 stencil kernels exist in eight tile
 * variants: tiles of 64 >> (v & 3) rows (64, 32, 16 or 8) by 64 columns; bit 2
 * set = the prolongation's spline passes on pairs of rows / columns with
 * packed FP32x2 instructions (else scalar, one midpoint per work item).  kind 0
 * is the down kernel (sweeps, residual, restriction: variants 0-3 only), kind 1
 * the up kernel (prolongation, correction, sweeps).  Every variant computes
 * the same bits; the choice changes only speed.  The choice is process-wide,
 * per (kind, grid size n, sweep count nu), starts from built-in defaults, and
 * applies to every later solve, batched solve and server tick (cached graphs
 * are re-recorded).
 * ------------------------------------------------------------------- */

/* Time every variant of both kernels on each tile level of ctx (n >= 128)
 * with its nu_pre / nu_post, on the context's stream, and keep the fastest.
 * The context's level buffers are overwritten (not x or f of any solve).  If
 * cache_path is not NULL, entries recorded there for this GPU model are used
 * without timing and new measurements are appended (plain text, one entry per
 * line).  *n_timed (may be NULL) = entries measured.  Synchronous. */
mg_status mg_autotune(mg_ctx *ctx, const char *cache_path, int *n_timed);

/* Programmatic dependent launch between the library's kernels (process-wide;
 * mode 0 = off, the default unless the environment variable MG_LAUNCH_OVERLAP
 * was 1 or 2 at first use).  Mode 1: every kernel is launched with CUDA's
 * programmatic stream serialization and starts by waiting for its
 * predecessor's completion, so the next kernel's blocks are scheduled while
 * the previous grid drains; mode 2: only kernels whose grid has at most 304
 * blocks (about one wave: the coarse levels, the bottom solve, the outer and
 * convergence kernels).  Results are identical in every mode; graphs recorded
 * before a change are re-recorded.  Returns MG_ERR_INVALID_ARG for other
 * modes.  (Measured on GB300: both modes slower for these graphs, hence off.)  Every
 * kernel waits on its predecessors at its start and signals its dependents
 * when each block exits. */
mg_status mg_set_launch_overlap(int enable);
int mg_get_launch_overlap(void);

/* Staging of the smoother's tiles (Algorithm 6, relax / residual / restrict:
 * the down pass of a level, red-black sweeps, residual and full weighting on
 * one shared-memory tile with its halo).  on = 1: single solves stage every
 * interior 64-row tile of an FP32 level with V(2, .) by TMA (tiled 2D copies
 * of the x and b tiles with their halo into shared memory, split there into
 * the red and black arrays); tiles whose halo wraps around the periodic grid
 * keep the 16-byte vector loads.  on = 0 (the default): vector loads for
 * every tile.  Results are identical bit for bit; graphs recorded before a
 * change are re-recorded.  A TMA wait that runs out makes the solve return
 * MG_ERR_TIMEOUT.  MG_ERR_INVALID_ARG for other values. */
mg_status mg_set_tma_tiles(int on);
int mg_get_tma_tiles(void);

/* Launch form of the coarse tail of a single solve's V(2,2) cycle
 * (Algorithm 6's recursion below the 128^2 level: its down pass, the levels
 * <= 64^2 down to the exact coarsest solve and back, its up pass).  on = 1
 * (the default): one launch of a thread-block cluster of 8 CTAs, CTA r taking
 * tile r of the 128^2 level, CTA 0 the bottom V-cycle, the phases ordered by
 * the cluster's hardware barrier; on = 0: three launches.  Results are
 * identical bit for bit; graphs recorded before a change are re-recorded.
 * MG_ERR_INVALID_ARG for other values. */
mg_status mg_set_coarse_cluster(int on);
int mg_get_coarse_cluster(void);

/* Launch form of a mixed solve's outer step (FP64 defect correction: x += e,
 * then r = f - A x for the convergence test and the next step; grids of
 * N >= 32; mixed precision is this library's design, the paper has no
 * counterpart).  on = 1 (the default): the update and the next residual run as
 * one launch that reads x and e once, writes x + e into the other buffer of a
 * pair (the caller's x and a context buffer, alternating each outer step) and
 * forms the residual of x + e from the same loads; the solve's projection
 * writes the caller's x.  on = 0: an update launch and a residual launch.  x,
 * the residuals and every decision are identical bit for bit; the reported
 * update_norm is the same sum in another order (equal to about 1e-15
 * relative).  Graphs recorded before a change are re-recorded.
 * MG_ERR_INVALID_ARG for other values. */
mg_status mg_set_fused_update(int on);
int mg_get_fused_update(void);

/* Where the FP64 V-cycle's cubic prolongation (Sec. 2.2, Algorithm 6's
 * prolongate step) runs its pass along x.  on = 1 (the default): once per
 * level, over the whole coarse error, into a context buffer of (N/2) x N
 * doubles, before the up pass loads the refined rows; on = 0: inside every
 * tile of the up pass, which also refines the 2L - 1 coarse halo rows its
 * pass along y reads (the FP64 filter has L = 28 taps per side).  Results are
 * identical bit for bit; graphs recorded before a change are re-recorded.
 * FP32 V-cycles always refine per tile.  MG_ERR_INVALID_ARG for other
 * values. */
mg_status mg_set_fp64_separate_x_pass(int on);
int mg_get_fp64_separate_x_pass(void);

/* Read or set one table entry (n a power of two >= 128, nu 0..4). */
mg_status mg_get_tile_variant(int kind, int n, int nu, int *variant);
mg_status mg_set_tile_variant(int kind, int n, int nu, int variant);

/* ---------------------------------------------------------------------
 * Training of the SR generator (Sec. 2.3 and Sec. 3.2: the generator learns
 * the fine-grid error from the coarse-grid one).  The trainer holds FP32
 * master weights, Adam moments (beta1 0.9, beta2 0.999, eps 1e-8) and the
 * activations of one batch of `batch` periodic coarse fields of H x W (powers
 * of two >= 8; batch * H * W a multiple of 2048, at most 2^24); every
 * forward and backward convolution runs in the library's own kernels.  When
 * W is a multiple of 128 the 64- and 256-channel convolutions (forward, data
 * gradient, weight gradient) run on the tcgen05 tensor cores by default, with
 * BF16 operands (activations and the FP32 master weights rounded to nearest
 * even) and FP32 accumulation; the thin first and last layers, PReLU, the
 * loss and Adam stay in FP32.  Otherwise, or after
 * mg_trainer_set_tensor_cores(tr, 0), every convolution runs in FP32 on the
 * CUDA cores.
 * Inputs are device arrays: q [batch][H][W] (the normalised coarse error
 * e_c / s), target [batch][2H][2W] (the generator's target, e.g.
 * (e_f - cubic(e_c)) / s), mask [batch][2H][2W] or NULL (per-pixel weights of
 * the loss).  Loss = sum(mask * (y - target)^2) / (batch * 4 * H * W).
 * Calls are synchronous on the default stream.
 * ------------------------------------------------------------------- */
typedef struct mg_trainer mg_trainer;

/* blob: initial weights in the mg_load_prolong_weights layout; lr: Adam step size. */
mg_status mg_trainer_create(int H, int W, int batch, const void *blob, size_t bytes, double lr,
                            mg_trainer **out);
/* y [batch][2H][2W] (device) = G(q) with the current weights. */
mg_status mg_trainer_forward(mg_trainer *tr, const float *q, float *y);
/* Loss (host double, may be NULL) and its gradient with respect to every
 * parameter, written to grad (device, n_params floats in blob order). */
mg_status mg_trainer_gradients(mg_trainer *tr, const float *q, const float *target, const float *mask,
                               float *grad, double *loss);
/* One Adam step on the batch; *loss (may be NULL) = the loss before the step. */
mg_status mg_trainer_step(mg_trainer *tr, const float *q, const float *target, const float *mask,
                          double *loss);
/* Set the Adam learning rate (lr > 0) for the following steps. */
mg_status mg_trainer_set_lr(mg_trainer *tr, double lr);
/* Choose the convolution arithmetic of the following passes (Sec. 3.2 trains
 * the generator; the precision is this library's choice): on != 0 = BF16
 * operands on the tcgen05 tensor cores (MG_ERR_INVALID_ARG unless W is a
 * multiple of 128), 0 = FP32 on the CUDA cores.  A tensor-core pass whose
 * bounded wait on its MMAs runs out makes the call that ran it return
 * MG_ERR_TIMEOUT. */
mg_status mg_trainer_set_tensor_cores(mg_trainer *tr, int on);
/* *on = 1 if the trainer's convolutions run on the tensor cores, else 0. */
mg_status mg_trainer_get_tensor_cores(mg_trainer *tr, int *on);
/* Current weights as a blob (bytes = 64 + 4 * n_params). */
mg_status mg_trainer_get_weights(mg_trainer *tr, void *blob, size_t bytes);
/* Free the trainer and its device memory; NULL is ignored. */
void mg_trainer_destroy(mg_trainer *tr);

/* Free a context: its level hierarchy, graphs, staging buffers, generator
 * weights and streams it created (not a caller's stream); waits for its work
 * first.  NULL is ignored.  (Resource management of this library; the paper
 * has no counterpart.) */
void mg_destroy(mg_ctx *ctx);
/* Name of a status code ("MG_OK", ...); a static string, never NULL.  (Error
 * reporting of this library; the paper has no counterpart.) */
const char *mg_status_string(mg_status status);
/* Text of the last error raised on the calling thread (thread-local; empty
 * when none); valid until the thread's next failing call. */
const char *mg_last_error(void);

/* ---------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper): used by the benchmark to
 * time one kernel kind live inside a solve and to count launches.
 * ------------------------------------------------------------------- */

/* Number of kernels this library has launched in this process so far. */
unsigned long long mg_kernel_launches(void);

/* Record a CUDA event pair around each launch of one kernel kind on the
 * context's stream: 1 = finest-level pre-smoothing/restriction kernel,
 * 2 = finest-level prolongation/post-smoothing kernel, 3 = outer residual
 * (the exact sum of the FP64 iterate's residual), 4 = FP64 update, 5 = the
 * coarse part of an FP32 V-cycle (every
 * launch below the finest level, as one span), 6 = the FP64 update fused with
 * the next outer residual (mg_set_fused_update); 0 disables.  At most
 * `capacity` launches (spans) are recorded until mg_probe_read. */
mg_status mg_probe_kernel(mg_ctx *ctx, int kind, int capacity);

/* Synchronise the context's stream and return the number of recorded
 * launches, their summed device time (ms) and their summed algorithmic
 * bytes (compulsory reads + writes); resets the probe's accumulators. */
mg_status mg_probe_read(mg_ctx *ctx, int *launches, double *total_ms, double *bytes);

/* ---------------------------------------------------------------------
 * Operator-level entry points (device pointers only), for verification of
 * each step against a reference.  dtype: 0 = double, 1 = float.  Grids use
 * the scaled right-hand side b = h^2 * rhs, so that A x = rhs reads
 * 4 x_ij - (sum of 4 neighbours) = b_ij.  Work is ordered on `stream`.
 * ------------------------------------------------------------------- */

/* Pre-smoothing and restriction (Algorithm 6: relax, residual, restrict):
 * x_out = nu red-black sweeps applied to x (x read as 0 if zero_init), then
 * bc = 4 * FW(b - (4 x_out - sum nbrs)), the scaled coarse right-hand side on
 * the n/2 grid.  n: power of two >= 64.  x and x_out must not overlap (the
 * kernel is out of place). */
mg_status mg_op_down(int dtype, int n, const void *x, void *x_out, const void *b, int nu,
                     int zero_init, void *bc, void *stream);

/* Correction and post-smoothing (Algorithm 6: prolongate, correct; Sec. 2.2
 * spline): x_out = nu red-black sweeps applied to x + P ec, P the periodic
 * tensor-product cubic spline from the n/2 grid.  x, x_out distinct. */
mg_status mg_op_up(int dtype, int n, const void *x, void *x_out, const void *b, const void *ec,
                   int nu, void *stream);

/* V-cycles below the top: runs one V(nu1, nu2) cycle on the n x n problem
 * 4x - sum = b (n <= 64, down to a coarsest grid of size `coarsest`),
 * x = 0 on entry if zero_init. */
mg_status mg_op_vcycle(int dtype, int n, int coarsest, void *x, const void *b, int nu1, int nu2,
                       int zero_init, void *stream);

/* Allocation-free variant of mg_op_vcycle (no counterpart in the paper; the
 * paper's method has no memory-management side).  mg_op_vcycle allocates
 * device memory on every call for the coarsest-grid pseudo-inverse; callers
 * that cannot call cudaMalloc use this one instead - for example a solver
 * stepped inside a fixed-rate simulation loop, which cannot take the
 * device-wide synchronisation cudaMalloc implies, or a process whose framework
 * allocator already reserved most device memory, where a raw cudaMalloc fails
 * although the framework holds free blocks.  Same arguments and results as
 * mg_op_vcycle.  The pseudo-inverse is built on the device, on `stream`, into
 * one static device array of 256*256 doubles (512 KiB) that every GPU loading
 * the library keeps until exit, so coarsest must be 4, 8 or 16 and n <= 64;
 * larger sizes return MG_ERR_INVALID_ARG.  No cudaMalloc/cudaFree or other
 * allocating call is made.  Every call made outside stream capture looks up
 * the array's address on the current device (cudaGetSymbolAddress, which
 * allocates nothing) - make one such call before any stream capture - and a
 * call on a capturing stream uses the address the last uncaptured call found
 * (so a capture that spans a cudaDeviceReset needs an uncaptured call after
 * the reset first).  All calls share the array and rewrite it, so calls that
 * overlap on the GPU (unordered streams) race.
 * Asynchronous on `stream`. */
mg_status mg_op_vcycle_static(int dtype, int n, int coarsest, void *x, const void *b, int nu1,
                              int nu2, int zero_init, void *stream);

/* One 3x3 convolution of the SR generator (Sec. 2.3, Fig. 1b) on the tensor
 * cores: BF16 operands, FP32 accumulation, BF16 output.  Activations are
 * channels-last with 64 channels and a one-pixel periodic halo: an H x W grid
 * is (H+2) x (W+2) x 64 bf16, pixel (y, x) at padded (y+1, x+1), halo entries
 * holding the wrapped neighbours (the output's halo is written too).  W must
 * be a multiple of 128.  w_packed: bf16 [groups][9 taps (ky*3+kx)][64 co][64 ci]
 * (groups = 4 for mode 2).  mode 0: out = PReLU(conv(in) + bias) with prelu[64];
 * mode 1: out = skip + conv(in) + bias (residual block end); mode 2 (pixel
 * shuffle): group g computes fine channel c at sub-pixel (g >> 1, g & 1) of a
 * 2H x 2W padded output, out = PReLU_c(conv(in) + bias[g][c]).  bias holds
 * groups x 64 floats.  Synchronous; MG_ERR_TIMEOUT if a bounded wait expired. */
mg_status mg_op_sr_conv(int mode, int H, int W, const void *in, const void *skip, const void *w_packed,
                        const float *bias, const float *prelu, void *out, void *stream);

/* The SR correction s * G(ec / s), s = max|ec|, for a coarse error ec
 * (nc x nc floats, device) with the context's loaded weights, written to out
 * (2nc x 2nc floats, device).  nc a multiple of 128.  Synchronous on the
 * context's stream. */
mg_status mg_op_sr_generator(mg_ctx *ctx, const float *ec, int nc, float *out);

/* One layer of the context's loaded SR generator (Sec. 2.3, Fig. 1b;
 * Appendix A, Algorithm 5) on caller buffers: the production kernels and
 * packed weights of mg_op_sr_generator, which runs layers 0 .. 2 n_blocks + 2
 * in order, for layer-by-layer verification.  Buffers are device memory,
 * activations padded bf16 in the layout of mg_op_sr_conv (halo written).
 *   layer 0: in = ec (nc x nc floats); *s (device float) receives
 *            s = max|ec| (1 when ec = 0); out = PReLU(conv 1 -> 64 of ec / s),
 *            padded coarse.
 *   layers 1 .. 2 n_blocks: residual block k = (layer - 1) / 2; odd layers
 *            out = PReLU(conv(in)), even layers out = skip + conv(in) (skip
 *            the block's input); in, skip, out padded coarse.
 *   layer 2 n_blocks + 1: out = PReLU(pixel_shuffle(conv 64 -> 256 of in)),
 *            in padded coarse, out padded fine ((2nc + 2)^2 x 64).
 *   layer 2 n_blocks + 2: out = s * (conv 64 -> 1 of in), in padded fine,
 *            *s read, out 2nc x 2nc floats.
 * nc a multiple of 128 (the coarse grid).  MG_ERR_INVALID_ARG for a layer
 * out of range or a missing buffer, MG_ERR_NO_WEIGHTS without weights,
 * MG_ERR_TIMEOUT if a bounded wait expired.  Synchronous on the context's
 * stream. */
mg_status mg_op_sr_layer(mg_ctx *ctx, int layer, int nc, const void *in, const void *skip, float *s, void *out);

/* The windowed SR prolongation of Sec. 3.1 and Fig. 2 (Appendix A,
 * Algorithms 1-5) with the context's loaded generator: the coarse field ec
 * (nc x nc floats, device) is normalised by the symmetric logarithm
 * (Algorithm 3: q = sgn(p) (log10|p| - log10 p_min) / (log10 p_max -
 * log10 p_min), magnitudes clamped to [p_min, p_max], 0 kept), cut into
 * 6 x 6 windows whose origins step by 2 (window (a, b) covers rows 2a - 2 ..
 * 2a + 3 and columns 2b - 2 .. 2b + 3, wrapped around the periodic grid),
 * each window goes through the generator alone with zero padding, the
 * central 2 x 2 coarse cells of each (4 x 4 fine points) are kept and
 * stitched, and each kept value g is mapped back (Algorithm 4: sgn(g)
 * 10^(log10 p_min + |g| (log10 p_max - log10 p_min))).  out: 2nc x 2nc
 * floats (device), the prolongation itself (Algorithm 5 has no spline term).
 * nc a power of two >= 32; 0 < p_min < p_max (the paper's interval is
 * [1e-10, 1e-3]).  MG_ERR_NO_WEIGHTS without weights; synchronous on the
 * context's stream. */
mg_status mg_op_sr_windowed(mg_ctx *ctx, const float *ec, int nc, double p_min, double p_max, float *out);

/* Outer residual of FP64 data: s = b - (4x - sum nbrs) with b = h^2 (f - mu)
 * formed in FP64 (so s = h^2 r), written as float to s32 when s32 != NULL;
 * out[0] = sum s^2, out[1] = sum (f - mu)^2 (out: 2 doubles, device).  The
 * stencil sum is exact on the integer pipe and rounded once to float: for
 * n >= 32 with s32, the solver's task-tiled kernel (operands aligned to the
 * largest exponent of the point's 32-column x 8-row task, error under
 * 10 * 2^-59 of that task's largest operand before the rounding); otherwise
 * each point's six operands are aligned to their own largest exponent (error
 * under 6 * 2^-59 of it).  An infinite or NaN operand gives NaN. */
mg_status mg_op_outer_residual(int n, const double *f, const double *x, double mu, float *s32,
                               double *out, void *stream);

/* The library's float <-> double conversions on the integer pipe (used by the
 * outer kernels in place of the FP64-pipe conversion instructions):
 * dir 0: out[i] = (float)in[i] rounded to nearest even, in double, out float;
 * dir 1: out[i] = (double)in[i], in float, out double.  Device arrays of
 * count elements.  Exposed so that tests can compare them bit for bit with
 * the hardware conversion.  Synchronous. */
mg_status mg_op_convert(int dir, size_t count, const void *in, void *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* MG_H */
