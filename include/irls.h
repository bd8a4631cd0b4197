/*
 * irls.h - C ABI of libirls: GPU L1 phase unwrapping by iteratively reweighted least squares
 * (IRLS) with a DCT-preconditioned conjugate gradient inner solver, for NVIDIA GB300 (sm_103a).
 *
 * Method: "Iteratively Reweighted Least Squares for Phase Unwrapping" (arXiv 2401.09961).
 *   - problem (main), Sec. 2: minimise over U the weighted L1 mismatch
 *       sum Cv |U[i+1,j] - U[i,j] - Gv[i,j]| + sum Ch |U[i,j+1] - U[i,j] - Gh[i,j]|
 *     of the wrapped phase differences Gv, Gh of the observed phase X;
 *   - Sec. 3.1: slack variables Vv, Vh with penalty 1/(2 tau), delta-smoothing F_delta, and the
 *     IRLS loop of Alg. 1 (closed-form weights W = sqrt(C^2 V^2 + delta^2), then an approximate
 *     solve of the linear system of Prop. 'linear system' for (U, Vv, Vh), then U -= mean(U));
 *   - Sec. 3.2: the inner solve is the preconditioned CG of Alg. 2;
 *   - Sec. 3.3: the preconditioner is block diagonal; its Laplacian block is a Sylvester
 *     equation solved through the DCT-II eigenbasis of the 1-D Neumann Laplacians.
 *
 * Conventions shared by every entry point
 *   - Images are H x W (H = the paper's N rows, W = the paper's M columns), float32, row-major
 *     and contiguous (element (i, j) at offset i*W + j).  Vertical-edge arrays (Gv, Cv, Vv) are
 *     (H-1) x W row-major; horizontal-edge arrays (Gh, Ch, Vh) are H x (W-1) row-major.
 *   - Pointers named d_* are DEVICE memory on the plan's device; h_* are HOST memory.  The
 *     caller owns every buffer it passes; the library never frees or retains caller pointers
 *     beyond the call (asynchronous calls read/write them until the stream reaches that point).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - Return value: 0 = success; 1 = warning (CG reached cg_max_iter in some outer iteration
 *     without meeting cg_tol); negative = error (IRLS_ERR_*).  No C++ exception crosses the ABI.
 *   - H = 1 or W = 1 is valid: the corresponding edge set is empty.
 *   - A plan is not thread-safe: use one plan per host thread / stream.
 */
#ifndef IRLS_H
#define IRLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------------- */
#define IRLS_OK              0
#define IRLS_WARN_CG_MAX     1   /* CG stopped on cg_max_iter before cg_tol in some outer step */
#define IRLS_ERR_ARG        -1   /* null pointer, tau <= 0, delta <= 0, cg_tol < 0, ...        */
#define IRLS_ERR_SHAPE      -2   /* H < 1, W < 1, or H*W too large                             */
#define IRLS_ERR_NONFINITE  -3   /* NaN or Inf found in X, coherence or the weights            */
#define IRLS_ERR_OOM        -4   /* device allocation failed                                   */
#define IRLS_ERR_BREAKDOWN  -5   /* CG breakdown: rho <= 0 or p^T A p <= 0 with r != 0         */
#define IRLS_ERR_TIMEOUT    -6   /* a bounded device-side wait gave up                         */
#define IRLS_ERR_CUDA       -7   /* a CUDA runtime call failed (see irls_last_cuda_error)      */
#define IRLS_ERR_UNSUPPORTED -8  /* option not available for this shape / device               */

/* ---- precision of the DCT preconditioner (Sec. 3.3 dense products) -------------------- */
#define IRLS_PREC_FP32   0  /* float32 operands, float32 accumulation (SIMT FMA)              */
#define IRLS_PREC_BF16   1  /* bfloat16 operands, float32 accumulation (tcgen05), one pass    */
#define IRLS_PREC_BF16X3 2  /* split bfloat16: x = hi + lo, three tcgen05 products per GEMM   */
                            /* (hi*hi + hi*lo + lo*hi), float32 accumulation                  */
#define IRLS_PREC_FP16   3  /* float16 operands, one tcgen05 product, float32 accumulation;   */
                            /* folded form only (single-image plans, sides >= 256): r_U is   */
                            /* scaled by sqrt(H W) / ||r_U||, each row of the eigenvalue      */
                            /* stage by (mu + lambda_1) / tau, undone by a pre-scaled basis   */
                            /* in the last stage; not for batches or the adjoint              */

/* Form of the preconditioner's Laplacian block (Sec. 3.3).  AUTO, DIRECT and FOLDED choose
 * how the tensor-core precisions run the dense products; FFT replaces the products by fast
 * transforms of the same map. */
#define IRLS_DCT_AUTO   0   /* folded where allowed, else direct                                  */
#define IRLS_DCT_DIRECT 1   /* four full-size products per application                            */
#define IRLS_DCT_FOLDED 2   /* even / odd folded products, half the multiply-adds, all four
                             * stages in one persistent launch; needs precision IRLS_PREC_BF16X3
                             * or IRLS_PREC_FP16 (which always runs it) and H, W >= 256 (odd or
                             * even); otherwise plan creation returns IRLS_ERR_UNSUPPORTED       */
#define IRLS_DCT_FFT    3   /* every orthonormal DCT-II / DCT-III of the map evaluated by a
                             * complex FFT of the same length in float32 on the CUDA cores
                             * (three passes over a float32 plane per application; r_U^T z_U
                             * from the spectrum by Parseval); needs precision IRLS_PREC_FP32,
                             * H a power of two in [64, 8192] or one of 2000, 4000, 8000, and
                             * W a power of two in [64, 16384] or one of 2000, 4000, 8000,
                             * 16000 (the 4000 x M sizes; radix-5 stages);
                             * single-image plans only (batches: IRLS_ERR_UNSUPPORTED).  Not
                             * in the paper, which forms the dense products                      */

/* Inner-solve budget (Sec. 4.3). */
#define IRLS_CG_FIXED 0     /* outer_iters IRLS iterations, each solve capped at cg_max_iter    */
#define IRLS_CG_PAPER 1     /* the adaptive budget m_CG(k) and IRLS stop of Sec. 4.3            */

/* Linear system of each outer step. */
#define IRLS_SYS_FULL  0    /* the (U, Vv, Vh) system of Sec. 3.1 with the block-diagonal
                             * preconditioner of Sec. 3.3 (the paper's method)                    */
#define IRLS_SYS_SCHUR 1    /* the U-only system left after eliminating V (exact algebraically):
                             * S^T Om_v (S U - Gv) + (U T - Gh) Om_h T^T = 0, Om = D/(1 + tau D),
                             * Alg. 2 with the Laplacian block of Sec. 3.3 as the preconditioner,
                             * then V = (D U - G)/(1 + tau D); the stopping rule uses the U-only
                             * residual, so the trajectory differs from IRLS_SYS_FULL unless the
                             * solves converge                                                    */

#define IRLS_MAX_OUTER 256

typedef struct irls_plan_s* irls_plan;   /* opaque: device workspace, DCT bases, device state */
typedef struct irls_tape_s* irls_tape;   /* opaque: checkpoints of a recorded forward solve   */
typedef struct irls_batch_s* irls_batch; /* opaque: a batched solve of many images            */
typedef struct irls_tiled_s* irls_tiled; /* opaque: a tiled solve of one large image          */

/* Solver options.  Defaults (irls_opts_default): tau = 1e-2 and delta = 1e-6 (the paper's
 * model parameters, Sec. 4.4), outer_iters = 20, cg_tol = 1e-6, cg_max_iter = 1000,
 * precision = IRLS_PREC_FP32, flexible_cg = 0, warm_start = 1, dct_form = IRLS_DCT_AUTO,
 * cg_schedule = IRLS_CG_FIXED, cg_m0 = 5, cg_eps_tol = 1e-3, cg_alpha = 1.7 (the values of
 * Sec. 4.3), system = IRLS_SYS_FULL. */
typedef struct {
    float tau;          /* penalty tau of problem (soft constraints), Sec. 3.1; > 0            */
    float delta;        /* smoothing delta of F_delta, Sec. 3.1; > 0                           */
    int   outer_iters;  /* number of IRLS (Alg. 1) iterations; 1 .. IRLS_MAX_OUTER             */
    float cg_tol;       /* stop CG when ||r||_2 <= cg_tol * ||b||_2 (full 3-block residual)     */
    int   cg_max_iter;  /* cap on products with A per outer iteration; >= 0                    */
    int   precision;    /* IRLS_PREC_*                                                         */
    int   flexible_cg;  /* 0: beta = rho_new / rho (Alg. 2); 1: Polak-Ribiere (flexible) beta  */
    int   warm_start;   /* 1: CG starts from the current (U, V); 0: from zero each outer step  */
    int   dct_form;     /* IRLS_DCT_*; FOLDED or FFT where not allowed: IRLS_ERR_UNSUPPORTED   */
    /* IRLS_CG_PAPER (Sec. 4.3): solve k is capped at min(m_CG(k), cg_max_iter), m_CG(0) = cg_m0.
     * For k >= 1, with Delta = (H_delta(x^k, W^{k-1}) - H_delta(x^k, W^k)) / H_delta(x^k,
     * W^{k-1}): Delta > cg_eps_tol keeps m_CG; otherwise the run stops and returns U^k if m_CG
     * was raised at k-1, else m_CG(k) = floor(cg_alpha * m_CG(k-1)).  outer_iters bounds the
     * number of IRLS iterations.  Reaching a planned budget is not a warning; reaching
     * cg_max_iter is.  Single-image solves only (the batched and recorded forms return
     * IRLS_ERR_UNSUPPORTED). */
    int   cg_schedule;  /* IRLS_CG_FIXED or IRLS_CG_PAPER                                      */
    int   cg_m0;        /* m_CG(0) >= 1                                                         */
    float cg_eps_tol;   /* epsilon_tol of Sec. 4.3 (not NaN)                                   */
    float cg_alpha;     /* alpha > 1 of Sec. 4.3                                               */
    int   system;       /* IRLS_SYS_FULL or IRLS_SYS_SCHUR (single-image solves; the batched and
                           recorded forms return IRLS_ERR_UNSUPPORTED for IRLS_SYS_SCHUR)      */
} irls_opts;

/* Per-call statistics (host struct filled by the library). */
typedef struct {
    int    outer_done;                  /* outer iterations completed                         */
    int    cg_total;                    /* sum of CG iterations                               */
    int    status;                      /* status of the call (same code as the return value) */
    int    cg_iters[IRLS_MAX_OUTER];    /* CG iterations (products with A) per outer step     */
    double rel_res[IRLS_MAX_OUTER];     /* final ||r|| / ||b|| of each inner solve            */
    double l1_obj[IRLS_MAX_OUTER];      /* objective of problem (main) at U^{k+1}             */
    double h_delta[IRLS_MAX_OUTER];     /* H_delta(U^{k+1}, V^{k+1}, W^k), problem (alt1)     */
    double f_delta[IRLS_MAX_OUTER];     /* F_delta(U^k, V^k) = H_delta(x^k, W^k) before solve */
    int    cg_cap[IRLS_MAX_OUTER];      /* cap of each inner solve (IRLS_CG_PAPER: m_CG(k))   */
    int    schedule_stop;               /* 1: the Sec. 4.3 rule ended the run before outer_iters;
                                           f_delta[outer_done] then holds the F_delta(x^k) it
                                           read at that iteration                          */
} irls_stats;

/* Fill *opts with the defaults above.  Returns IRLS_ERR_ARG if opts is NULL. */
int irls_opts_default(irls_opts* opts);

/* Bytes of device memory a plan for an H x W image allocates (workspace, DCT bases, state).
 * Returns 0 on invalid arguments. */
size_t irls_workspace_bytes(int H, int W, const irls_opts* opts);

/* Create a plan on the current CUDA device: allocates the workspace and precomputes the
 * eigendecompositions S^T S = P_S L_S P_S^T and T T^T = P_T L_T P_T^T (Sec. 3.3: computed
 * once, kept in memory).  opts may be NULL (defaults).  *out receives the plan.  Synchronous. */
int irls_plan_create(int H, int W, const irls_opts* opts, irls_plan* out);

/* Release a plan and its device memory (synchronises the device first).  NULL is a no-op. */
int irls_plan_destroy(irls_plan plan);

/* Replace the plan's options (same H, W).  `precision` may change only to IRLS_PREC_FP32 or to
 * the precision the plan was created with (IRLS_ERR_UNSUPPORTED otherwise). */
int irls_plan_set_opts(irls_plan plan, const irls_opts* opts);

/* Preconditioner form the plan runs with its current options: IRLS_DCT_FOLDED or
 * IRLS_DCT_DIRECT for the tensor-core precisions, IRLS_DCT_FFT for the fast-transform form,
 * IRLS_DCT_AUTO for IRLS_PREC_FP32 with dense products (float32 SIMT GEMMs, no tensor cores);
 * IRLS_ERR_ARG for a NULL plan.  The paper has no counterpart (an implementation
 * choice of this library). */
int irls_plan_dct_form(irls_plan plan);

/* Tile shapes of the CG direction and update kernels (Alg. 2's two stencil passes per
 * iteration, both bound by HBM bandwidth): image rows per thread block, 8 to 64 for a plan
 * (defaults 24 and 32; batches: one of 8, 16, 24, 32, see irls_batch_set_tiles).  They change
 * the block decomposition, so results change within rounding (the reductions' summation order
 * follows the blocks), never the method.  irls_plan_set_tiles sets them (0 keeps a value;
 * anything outside 8..64 is IRLS_ERR_ARG); irls_plan_get_tiles reads the values in use.
 * irls_plan_autotune times, for each kernel, 8, 16, 24 and 32 rows and the row counts that make
 * the kernel's launch the fewest whole waves on this device with at most 32 and at most 64 rows
 * a block (when those counts are other ones),
 * on the plan's workspace (ten launches each, after two warm-up launches, CUDA events on
 * `stream`), and keeps the fastest; h_ms (NULL allowed) receives eight mean times in ms:
 * direction for 8, 16, 24, 32 rows, then update.  It overwrites the plan's scratch planes and
 * state: call it between solves, not between a forward record and its backward sweep.
 * Synchronous with respect to the host.  No counterpart in the paper (an implementation choice
 * of this library). */
int irls_plan_set_tiles(irls_plan plan, int dir_rows, int upd_rows);

/* Test hook for failure detection: with on = 1, every stage-2 tile of the plan's folded
 * preconditioner launch waits for a row panel count one higher than the panel ever reaches.
 * Each such wait gives up after its bounded budget (about 2 s); the launch then finishes with
 * every image's state marked IRLS_ERR_TIMEOUT and stopped, its tensor memory freed, and the
 * context usable; a solve returns IRLS_ERR_TIMEOUT.  on = 0 restores the normal tables (the
 * next solve is unaffected).  IRLS_ERR_UNSUPPORTED when the plan does not run the folded form.
 * Not for production use. */
int irls_debug_stall_fold(irls_plan plan, int on);

/* The folded preconditioner's persistent-launch work list (Sec. 3.3's four dense products in
 * even / odd folded form, every tile of every stage in one list), as the launch's set-up builds
 * it for n_img images of sizes H[t] x W[t] (host arrays) run by `pairs` CTA pairs, without any
 * device work: for checking the schedule on a host without a GPU.  Writes the item count, the
 * panel counter count and the launch's item capacity (all host pointers, non-NULL); with rec
 * non-NULL and rec_items >= the item count, also IRLS_FOLD_SCHED_INTS ints per item in list
 * order:
 *   0 stage (0-3), 1 image, 2 tile within its problem, 3 first output row, 4 first column,
 *   5 columns, 6 k-blocks per operand set, 7 two operand sets, 8 half-width split,
 *   9 counter the tile completes (-1: none; each CTA of the pair adds one),
 *   10 dependency count, 11-18 counters waited for (-1 unused), 19-26 counts waited for,
 *   27 last tile of its pair in the image's stage-2 run, 28 r^T z slots of the image,
 *   29-31 the problem's M, N, K, 32 the problem (index among its stage's problems, images in
 *   order: 2 per image in stages 0 and 2, 4 in stage 1, 1 in stage 3).
 * Pair p runs items p, p + pairs, p + 2 pairs, ... in order.  IRLS_ERR_ARG for a NULL pointer,
 * n_img < 1, pairs < 1 or rec_items too small (the counts are still written); IRLS_ERR_SHAPE
 * for a side below 256 (the folded form's minimum) or above 32768.  Not for production use. */
#define IRLS_FOLD_SCHED_INTS 33
int irls_debug_fold_schedule(int n_img, const int* H, const int* W, int pairs, int* n_items,
                             int* n_ctr, int* cap_items, int* rec, int rec_items);
int irls_plan_get_tiles(irls_plan plan, int* dir_rows, int* upd_rows);
int irls_plan_autotune(irls_plan plan, float* h_ms, void* stream);

/* Simple form: unwrap d_X (H x W) into d_U (H x W, zero mean) with weights from d_coherence
 * (H x W, may be NULL for uniform weights), delta = eps, the given number of IRLS iterations
 * and CG tolerance, and the remaining options at their defaults (tau = 1e-2).  Edge weights from
 * coherence: Cv[i,j] = (coh[i,j] + coh[i+1,j]) / 2, Ch[i,j] = (coh[i,j] + coh[i,j+1]) / 2.
 * Synchronises `stream` before returning, so the status covers device-side failures. */
int irls_unwrap(const float* d_X, const float* d_coherence, int H, int W, float eps,
                int outer_iters, float cg_tol, float* d_U, void* stream);

/* Full form (Alg. 1 with Alg. 2).  d_Cv ((H-1) x W) and d_Ch (H x (W-1)), when both non-NULL,
 * are the edge weights and take precedence over d_coherence (as in the paper's unwrap(),
 * Sec. 4.4).  d_Vv / d_Vh may be NULL; when non-NULL they receive the final slacks.  When
 * d_U_init is non-NULL, (d_U_init, d_Vv, d_Vh) are the starting iterate (a restart point; the
 * default start is U = 0, V = -G as in Alg. 1).  h_stats may be NULL.  The call is
 * synchronous with respect to the host (it polls the device-side CG stopping flag). */
int irls_unwrap_ex(irls_plan plan, const float* d_X, const float* d_coherence,
                   const float* d_Cv, const float* d_Ch, const float* d_U_init,
                   float* d_U, float* d_Vv, float* d_Vh, irls_stats* h_stats, void* stream);

/* Batched solve: ntiles independent images of their own sizes H[t] x W[t] (non-square allowed),
 * each unwrapped as by irls_unwrap_ex with the options `opts`, with one GPU launch per phase of
 * Alg. 1 / Alg. 2 for all images together (the stencil kernels over the union of the images'
 * blocks, the preconditioner over all images' tiles: one launch for the folded form, one
 * grouped tensor-core GEMM per DCT stage for the direct form).  Each image keeps its own CG scalars and stopping test: an image whose CG run has
 * stopped drops out of later launches of the same outer step (its blocks return at once).  The
 * inner CG iterations are replayed from CUDA graphs captured once per batch.  Precision must be
 * IRLS_PREC_BF16X3 or IRLS_PREC_BF16 (IRLS_ERR_UNSUPPORTED for IRLS_PREC_FP32).
 * irls_batch_create allocates the workspace of all images and the DCT bases (one set per
 * distinct side length); irls_unwrap_batched_ex runs a batch on arrays of ntiles device pointers
 * d_X[t], d_coherence[t] (the array may be NULL for uniform weights; entries may be NULL),
 * d_U[t]; per_tile (nullable) receives ntiles statistics.  Synchronous with respect to the host;
 * `stream` is ordered before and after the batch.  irls_unwrap_batched is create + run +
 * destroy in one call.  irls_batch_uses_graphs returns 1 once the CG chunk graphs exist.
 * Preconditioner form: with dct_form IRLS_DCT_AUTO the batch runs the folded form (one
 * persistent CTA-pair launch over every image's tiles of all four stages, plus one fold of
 * r_U) when every image allows it (IRLS_PREC_BF16X3, sides >= 256), else the direct
 * grouped form;
 * IRLS_DCT_FOLDED where some image does not allow it is IRLS_ERR_UNSUPPORTED.  An image's
 * results do not depend on the batch it runs in: they equal, bit for bit, a single-image plan
 * in the same form.  irls_batch_dct_form returns IRLS_DCT_FOLDED or IRLS_DCT_DIRECT. */
int irls_batch_create(int ntiles, const int* H, const int* W, const irls_opts* opts,
                      irls_batch* out);
int irls_batch_destroy(irls_batch batch);
int irls_unwrap_batched_ex(irls_batch batch, const float* const* d_X,
                           const float* const* d_coherence, float* const* d_U,
                           irls_stats* per_tile, void* stream);
int irls_unwrap_batched(int ntiles, const int* H, const int* W, const float* const* d_X,
                        const float* const* d_coherence, float* const* d_U, const irls_opts* opts,
                        irls_stats* per_tile, void* stream);
int irls_batch_uses_graphs(irls_batch batch);
int irls_batch_dct_form(irls_batch batch);

/* Tiled unwrapping of one large image: the paper leaves very large images to future work
 * (Sec. 5, after the 4000 x M study of Sec. 4.5); this is that step built on the batched form.
 * The H x W image is cut into overlapping tiles of min(tile, H) x min(tile, W) pixels: along a
 * side of n pixels the tiles start at 0, tile - overlap, 2 (tile - overlap), ... while a tile
 * ends before n, and one more tile ends flush at n (one tile when n <= tile).  All tiles are
 * solved as one batch (irls_batch_create with `opts`; the batched form's precision rules
 * apply).  Each tile's solution is then shifted by a constant c_t: for every pair of
 * neighbouring tiles (next column or next row of tiles) d_ts is the mean of U_t - U_s over
 * their overlap, taken again over the pixels within pi of that first mean; c minimises
 * sum n_ts (c_s - c_t - d_ts)^2 (n_ts: the pixels of that second mean) with c_0 = 0.  Each
 * pixel of d_U takes U_t + c_t from the tile whose core holds it (consecutive tiles split their
 * overlap at (start of the next + end of this) / 2, rounded down), and d_U is made zero-mean.
 *   irls_tiled_create: 1 <= overlap < tile (IRLS_ERR_ARG otherwise); allocates the
 *     batch and the tiles' inputs and outputs (3 floats per tile pixel).  Synchronous.
 *   irls_tiled_info: the number of tiles, their height and width and the neighbour pairs
 *     (host pointers, non-NULL).  irls_tiled_batch: the underlying batch (for its tile shapes
 *     and autotuning; owned by the tiled handle).
 *   irls_unwrap_tiled: d_X, d_coherence (NULL: uniform weights) and d_U are H x W device
 *     arrays; per_tile (nullable) receives n_tiles statistics and h_constants (nullable)
 *     n_tiles constants.  Synchronous with respect to the host; the status is the batch's.
 * No paper counterpart for the stitching rule (the paper states no procedure). */
int irls_tiled_create(int H, int W, int tile, int overlap, const irls_opts* opts,
                      irls_tiled* out);
int irls_tiled_destroy(irls_tiled tiled);
int irls_tiled_info(irls_tiled tiled, int* n_tiles, int* tile_h, int* tile_w, int* n_pairs);
int irls_tiled_batch(irls_tiled tiled, irls_batch* batch);
int irls_unwrap_tiled(irls_tiled tiled, const float* d_X, const float* d_coherence, float* d_U,
                      irls_stats* per_tile, double* h_constants, void* stream);

/* Tile shapes of the batched CG direction and update launches (one value per batch, the same
 * meaning and allowed values as irls_plan_set_tiles; defaults 24 and 32).  An image's blocks,
 * and so its results, are those of a single-image plan with the same tile shapes.
 * irls_batch_autotune times each allowed value of each kernel over the whole batch (ten
 * launches each after two warm-up launches, CUDA events) and keeps the fastest; h_ms as for
 * irls_plan_autotune.  Both overwrite the batch's scratch and states: call them between runs;
 * the CG chunk graphs are captured again on the next run.  Ordered after `stream`; synchronous
 * with respect to the host. */
int irls_batch_set_tiles(irls_batch batch, int dir_rows, int upd_rows);
int irls_batch_get_tiles(irls_batch batch, int* dir_rows, int* upd_rows);
int irls_batch_autotune(irls_batch batch, float* h_ms, void* stream);

/* Forward solve that records what the adjoint needs (the reverse sweep below):
 * the wrapped gradients G and weights C it used, and V^k of every outer step k = 0..K (the
 * weights W^k = sqrt(C^2 (V^k)^2 + delta^2) of Alg. 1 are recomputed from them), K+5 pairs of
 * planes allocated by the library.  Arguments as in irls_unwrap_ex (no restart point).
 * *tape receives the record; release it with irls_tape_free.  The plan must outlive the tape;
 * other solves on the plan between recording and the backward call are allowed (the tape
 * keeps its own copies).  Synchronous like irls_unwrap_ex. */
int irls_unwrap_forward_record(irls_plan plan, const float* d_X, const float* d_coherence,
                               const float* d_Cv, const float* d_Ch, float* d_U, irls_tape* tape,
                               irls_stats* h_stats, void* stream);

/* Reverse sweep: given d_dL_dU (H x W), writes d_dL_dX (H x W) and, when the forward used a
 * coherence map, d_dL_dcoh (H x W; pass NULL to skip; NULL is required when explicit Cv/Ch were
 * given).  Model: each outer step is its converged solve x^{k+1} = A_k^+ b (Sec. 3.1-3.2), so
 * step k costs one PCG solve with the same symmetric A_k (same preconditioner, tolerance and
 * cap as the plan) plus the chain through D^k = C^2 / W^k(V^k); the wrap has derivative 1
 * almost everywhere.  h_stats (nullable) receives the CG iterations of each adjoint solve
 * (reverse order).  Uses the plan's workspace; synchronous. */
int irls_unwrap_backward(irls_tape tape, const float* d_dL_dU, float* d_dL_dX, float* d_dL_dcoh,
                         irls_stats* h_stats, void* stream);

/* Release a tape (synchronises the device first).  NULL is a no-op. */
int irls_tape_free(irls_tape tape);

/* One application of the Laplacian block of the preconditioner (Sec. 3.3, Sylvester equation
 * S^T S Z + Z T T^T = tau R solved in the DCT eigenbasis, zero-frequency coefficient set to 0):
 * d_Z = P_S [(P_S^T (tau d_R) P_T) / (l_i + m_j)] P_T^T, both H x W, in the plan's precision.
 * Asynchronous on `stream`. */
int irls_precond_laplacian(irls_plan plan, const float* d_R, float* d_Z, void* stream);

/* One product with the matrix A of Sec. 3.2 (eq. 'matrix-soft-constraints'):
 *   q_U  = (S^T S U + U T T^T - S^T Vv - Vh T^T) / tau
 *   q_Vv = Dv o Vv + (Vv - S U) / tau,    q_Vh = Dh o Vh + (Vh - U T) / tau
 * with Dv = d_Dv ((H-1) x W), Dh = d_Dh (H x (W-1)) and tau from the plan's options.
 * Runs the same update kernel as the CG loop.  Asynchronous on `stream`. */
int irls_apply_A(irls_plan plan, const float* d_U, const float* d_Vv, const float* d_Vh,
                 const float* d_Dv, const float* d_Dh, float* d_qU, float* d_qVv, float* d_qVh,
                 void* stream);

/* "Rounded IRLS" (Sec. 4.5): moves an unwrapped image d_U (H x W, the plan's shape) to the
 * nearest image 2pi-congruent to the input phase d_X.  The global offset of U is free (the model
 * is shift invariant), so U is first aligned with X by the circular mean
 * c = arg sum exp(i (U - X)) (FP64 sums); then, per pixel in float32 (one rounded operation at a
 * time), K = rint(((U - c) - X) / 2pi) and U_round = X + 2pi K.  d_Uround (float, H x W) and d_K
 * (int32, H x W) may each be NULL; h_offset (host, nullable) receives c.  Uses the plan's
 * device state (not during a solve on another stream).  Synchronous. */
int irls_round_congruent(irls_plan plan, const float* d_U, const float* d_X, float* d_Uround,
                         int* d_K, double* h_offset, void* stream);

/* Best-shift error of Sec. 4.5 against a reference unwrapping d_Xu (H x W):
 * alpha = mean(Xu - U) (FP64), E = (Xu - U) - alpha (float32, d_E nullable), and the RMS of E
 * (FP64).  h_alpha, h_rms: host, nullable.  Synchronous. */
int irls_best_shift_error(irls_plan plan, const float* d_U, const float* d_Xu, float* d_E,
                          double* h_alpha, double* h_rms, void* stream);

/* Allocation-free Laplacian preconditioner.  The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory - plug-ins whose host framework owns every
 * device byte through its own allocator, and latency-critical code that must never meet
 * cudaMalloc's implicit device synchronisation or an out-of-memory failure after start-up.
 * It computes what irls_precond_laplacian computes with IRLS_PREC_FP32, d_Z = L^+ (tau d_R), but
 * needs no plan and allocates nothing: the DCT bases and intermediates live in one fixed
 * 1.84 MB buffer compiled into the library (every GPU that loads the library holds it until the
 * process exits), sized for H, W <= IRLS_NOALLOC_MAX_SIDE.
 *   d_R, d_Z  H x W float32 device arrays, row-major and contiguous, owned by the caller;
 *   tau       > 0 (the penalty of the plan-based form);
 *   returns   IRLS_ERR_SHAPE if H or W is < 1 or > IRLS_NOALLOC_MAX_SIDE, IRLS_ERR_ARG for a
 *             null pointer or tau <= 0, IRLS_ERR_UNSUPPORTED if the current device's ordinal is
 *             64 or more, IRLS_ERR_CUDA if a launch fails; asynchronous on stream.
 * The first call on a device looks up the buffer's device address (cudaGetSymbolAddress) with
 * that device current and keeps it for the life of the process; make that first call before any
 * stream capture, and do not call the entry point on a device after cudaDeviceReset in the same
 * process (the reset unloads the module, and the kept address would be stale).  All calls share the one
 * buffer and each call rewrites every part of it that it reads, so nothing needs clearing
 * between calls - but calls that overlap on the GPU (other streams or host threads without
 * ordering between them) race on the buffer and corrupt each other's results. */
#define IRLS_NOALLOC_MAX_SIDE 256
int irls_precond_laplacian_noalloc(const float* d_R, float* d_Z, int H, int W, float tau,
                                   void* stream);

/* Live profiler (for measurement tools).  When on, every solve on this plan records a CUDA
 * event pair around each kernel launch on the solve's stream and accumulates the elapsed time
 * per kernel class; turning it on (or off) clears the totals.  Classes, in order:
 *   0 gradients/weights/||b|| (once per solve)   1 reweight + initial residual (per outer)
 *   2 search direction + p^T A p (per CG iter)    3 CG update x, r (per CG iter)
 *   4 Laplacian preconditioner (all its launches) 5 end-of-outer reductions and U -= mean
 * irls_plan_profile copies min(n, classes) totals (milliseconds) and launch counts and returns
 * the number of classes (6); launches skipped on the device after CG stopped are counted too. */
int irls_plan_set_profiling(irls_plan plan, int on);
int irls_plan_profile(irls_plan plan, double* ms, long long* launches, int n);

/* Human-readable text for a status code (static storage). */
const char* irls_status_string(int status);

/* The CUDA error code behind the last IRLS_ERR_CUDA returned on this host thread (0 if none). */
int irls_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IRLS_H */
