// Internal declarations shared by the libirls translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <vector>

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define IRLS_HAVE_NVTX 1
#else
#define IRLS_HAVE_NVTX 0
#endif

#include "../../include/irls.h"

namespace irls {

// A named NVTX range over the host thread's span of a phase, so that Nsight tools can attribute
// and filter the kernels launched in it (e.g. ncu --nvtx --nvtx-include "irls_unwrap/irls_pcg/").
// Without an attached tool each push and pop is a no-op call; without the NVTX headers in the
// toolkit the ranges are compiled out.
struct TraceRange {
#if IRLS_HAVE_NVTX
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
#else
    explicit TraceRange(const char*) {}
#endif
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

constexpr int kMaxOuter = IRLS_MAX_OUTER;

// Device-side error bits, OR-ed into DevState::status.
enum : int {
    ST_NONFINITE = 1,
    ST_BREAKDOWN = 2,
    ST_TIMEOUT = 4,
    ST_CGMAX = 8,
};

// Scalars of the IRLS / PCG state that never leave the device during a solve (Alg. 1, Alg. 2).
// All reductions are FP64; every kernel that produces one finishes it in its last block.
struct DevState {
    double rho;      // r^T z of the current iterate
    double alpha;    // rho / p^T A p
    double beta;     // ratio that forms the next search direction
    double pq;       // p^T A p
    double rr;       // ||r||^2 after the last update
    double bb;       // ||b||^2
    double rz_v;     // V-block part of r^T z (from the kernel that produced r)
    double rz_old;   // r_{l+1}^T z_l (Polak-Ribiere numerator term)
    double mean_u;   // mean of U at the end of an outer step
    double rel;      // ||r|| / ||b|| after the last update
    double rnorm_u;  // ||r_U||_2 (used to scale the fp16 preconditioner input)
    double pad0;
    int done;        // the current CG run has stopped
    int iter;        // CG iterations of the current run
    int p_fresh;     // the next search direction is p = z (start of a CG run)
    int status;      // OR of ST_* bits
    int outer;       // outer iterations completed
    int cg_total;
    unsigned int counter;   // last-block-done ticket for the deterministic reductions
    int pbuf;        // which ping-pong buffer holds the newest search direction
    int stop_next;   // a stop found inside a launch whose tiles still test done (set at its end)
    int cg_iters[kMaxOuter];
    double rel_res[kMaxOuter];
    double l1_obj[kMaxOuter];
    double h_delta[kMaxOuter];
    double f_delta[kMaxOuter];
    double aux[4];   // post-processing results: circular offset, best shift, sum of E^2
    double adj_scale;  // adjoint sweep: factor of the cotangent held in the residual planes
    double adj_step;   // adjoint sweep: ||xbar|| of the current reverse step
};

// Image-shaped planes.  Every plane is H rows x ld floats (ld a multiple of 32); the vertical
// edge planes use rows 0..H-2 and the horizontal ones columns 0..W-2; the unused row / column
// and the pitch padding are kept at zero by every kernel.
struct Planes {
    float* U;  float* Vv;  float* Vh;          // iterate x = (U, Vv, Vh)
    float* rU; float* rVv; float* rVh;         // residual r = b - A x
    float* pU[2]; float* pVv[2]; float* pVh[2];// search directions (ping-pong)
    float* zU;                                 // Laplacian-block preconditioner output
    float* dv; float* dh;                      // D = C^2 / W
    float* Wv; float* Wh;                      // W of the current outer step
    float* Gv; float* Gh;                      // wrapped gradients
    float* Cv; float* Ch;                      // edge weights
};

struct StencilArgs {
    int H, W, ld;
    float tau, inv_tau, delta;
    double tol2;        // cg_tol^2
    int cg_max;
    int cap_warn;       // 1: a run ended by cg_max short of the tolerance sets ST_CGMAX
    int flexible;
    int warm_start;
    int cur;            // which pU/pVv/pVh buffer holds the newest direction
    // optional bf16 emission of r_U for the tensor-core preconditioner
    void* r16;          // Hp x Wp (row-major, pitch Wp) or nullptr: bf16(r_U)
    void* r16lo;        // same shape or nullptr: bf16(r_U - bf16(r_U)) for split precision
    int ld16;
    int prec;           // IRLS_PREC_*
    // image rows per block of the CG direction and update kernels, set per plan by
    // irls_plan_set_tiles / irls_plan_autotune (single images: kMinTileRows .. kMaxTileRows;
    // batches: one of kTileRows); rw_rows / fin_rows: the reweighting and finalize kernels'
    // (aux_rows of the image's size; 0: the update kernel's; the launchers fill in the count
    // they dispatch)
    int dir_rows, upd_rows;
    int rw_rows, fin_rows;
    int sdir_rows, supd_rows;   // U-only system's direction and update kernels (0: 24)
};

// Image rows per block the CG direction and update kernels are built for, and the defaults
// (measured fastest at 4096 x 4096).
constexpr int kTileRows[4] = {8, 16, 24, 32};
constexpr int kDefaultDirRows = 24, kDefaultUpdRows = 32;
constexpr int kMinTileRows = 8, kMaxTileRows = 64;
inline bool tile_rows_ok(int r) { return r == 8 || r == 16 || r == 24 || r == 32; }
inline bool plan_rows_ok(int r) { return r >= kMinTileRows && r <= kMaxTileRows; }

// DCT-preconditioner resources owned by a plan.
struct DctPlan {
    int H, W, Hp, Wp;
    int prec;
    float tau;
    // fp32 bases: P_N (Hp x Hp) with P_N[i][k], its transpose, and the same for M (may alias N)
    float *PN, *PNT, *PM, *PMT;
    float *lamN, *lamM;     // eigenvalues, padded with zeros
    float *T1, *T2;         // fp32 intermediates (Wp x Hp each, reused)
    // bfloat16 copies for the tensor-core path (the *lo parts only in split precision)
    void *PN16, *PNT16, *PM16, *PMT16;
    void *PN16lo, *PNT16lo, *PM16lo, *PMT16lo;
    void *R16, *S16a, *S16b;        // bf16 input and intermediates (hi parts)
    void *R16lo, *S16alo, *S16blo;  // lo parts
    int split;
    int umma_ok;
    // folded (even/odd) form for H, W multiples of 256: half-size products on r_U(j) +- r_U(W-1-j)
    int fold;                  // folded form in use
    int fold_ready;            // folded form built (memory, bases)
    void *Re, *Relo, *Ro, *Rolo;   // folded residual, H x W/2 each
    void* fold_host;               // host-side record of the folded form (owned)
    // fast-transform form (float32 FFTs on the CUDA cores; power-of-two sides)
    int fft;                       // in use
    int fft_ready;                 // twiddle tables built
    float2 *fftTwN, *fftTtN;       // exp(-2 pi i m / H), exp(-i pi k / 2H)
    float2 *fftTwM, *fftTtM;       // the same for W
    alignas(64) unsigned char tmap_storage[2048];   // TMA descriptors of the four stages
};

// One image of a batched solve: its planes, arguments, device state, reduction scratch and
// inputs, and where its blocks start in the two stencil launch grids (one column per thread:
// "strip"; four columns per thread: "vec").  Kept in device memory as an array over images.
struct TileRec {
    Planes P;
    StencilArgs a;
    DevState* st;
    double* partials;
    const float* X;
    const float* coh;
    int sblk0, sgx, sgy;
    int vblk0, vgx, vgy;       // direction kernel's blocks
    int ublk0, ugy;            // update kernel's blocks (same columns, its own rows per block)
    int rblk0, rgy;            // reweighting kernel's blocks (same columns, a.rw_rows rows)
    int fblk0, fgy;            // finalize kernel's blocks (same columns, a.fin_rows rows)
};

// Tensor-core preconditioner of a batched solve, with the DCT bases cached per distinct side
// length.  Direct form: per-stage device arrays of grouped-GEMM problems (one per image and
// stage) and the images' bf16 copies of r_U (written by the update kernel).  Folded form
// (fold = 1): one problem table holding each image's nine problems of the four stages, the
// fused launch's work list and panel counters, and the images' fold records (the fold of r_U
// runs as its own batched launch).
struct BatchDctPlan {
    int T = 0, prec = 0, split = 0, fold = 0;
    float tau = 0.f;
    void* d_tiles[4] = {nullptr, nullptr, nullptr, nullptr};   // direct: problems per stage
    int total_ctas[4] = {0, 0, 0, 0};                         // direct: CTAs per stage
    void* d_frec = nullptr;             // folded: T fold records
    int frec_blocks = 0;
    int n_sm = 0;
    // folded: the fused launch's problem table, work list and panel counters
    void* d_probs = nullptr;
    void* d_items = nullptr;
    void* d_ctr = nullptr;
    void* d_sts = nullptr;
    int n_probs = 0, n_items = 0, n_ctr = 0, pairs = 0, n_st = 0, honour_stop = 1;
    std::vector<void*> r16, r16lo;
    std::vector<int> ld16;
};

// ---- launchers (stencil kernels, irls_kernels.cu) -----------------------------------------
cudaError_t launch_init(const float* X, const float* coh, const float* Cv_in, const float* Ch_in,
                        const float* U0, const float* Vv0, const float* Vh0, const Planes& P,
                        const StencilArgs& a, DevState* st, double* partials, cudaStream_t s);
cudaError_t launch_bnorm(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                         cudaStream_t s);
cudaError_t launch_norm_u(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                          cudaStream_t s);
cudaError_t launch_reweight_residual(const Planes& P, const StencilArgs& a, DevState* st,
                                     double* partials, cudaStream_t s);
cudaError_t launch_direction_pap(const Planes& P, const StencilArgs& a, DevState* st,
                                 double* partials, cudaStream_t s);
cudaError_t launch_update(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                          cudaStream_t s);
cudaError_t launch_finalize(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                            cudaStream_t s);
cudaError_t launch_copy_out(const float* src, int rows, int cols, int ld, float* dst,
                            cudaStream_t s);
cudaError_t launch_copy_in(const float* src, int rows, int cols, float* dst, int ld,
                           cudaStream_t s);
cudaError_t launch_matvec_via_update(const Planes& P, const StencilArgs& a, DevState* st,
                                     double* partials, cudaStream_t s);
cudaError_t launch_emit16(const float* src, int H, int W, int ld, void* r16, void* r16lo, int ld16,
                         cudaStream_t s);
int stencil_grid_blocks(int H, int W);
// rows per block that make a launch of the single-image kernel (0 direction, 1 update,
// 2 reweighting, 3 finalize, 4 and 5 the U-only system's direction and update) on an H x W image a whole number of waves on the current device,
// between kMinTileRows and `max_rows` (0 when no count in that range does)
int wave_rows(int kernel, int H, int W, int max_rows);
// rows per block of the reweighting (kernel 2) or finalize (kernel 3) launch for an H x W image:
// the count of the fewest whole waves up to kMaxTileRows rows, else kDefaultUpdRows.  A single-image plan and a batch
// both take it, so that they sum in the same order.
int aux_rows(int kernel, int H, int W);
// adjoint sweep (reverse over the outer steps)
cudaError_t launch_record_step(DevState* st, cudaStream_t s);
cudaError_t launch_adj_init(const Planes& P, const StencilArgs& a, const float* dLdU, DevState* st,
                            double* partials, cudaStream_t s);
cudaError_t launch_adj_setup_schur(const Planes& P, const StencilArgs& a, const float* Vkv,
                                   const float* Vkh, const float* Cv, const float* Ch,
                                   DevState* st, double* partials, cudaStream_t s);
cudaError_t launch_adj_recover_v(const Planes& P, const StencilArgs& a, const DevState* st,
                                 cudaStream_t s);
cudaError_t launch_adj_norm(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                            cudaStream_t s);
cudaError_t launch_adj_accumulate(const Planes& P, const StencilArgs& a, const float* Vkv,
                                  const float* Vkh, const float* Vnv, const float* Vnh,
                                  const float* Cv, const float* Ch, float* Gbv, float* Gbh,
                                  float* Cbv, float* Cbh, const DevState* st, cudaStream_t s);
cudaError_t launch_adj_final(const Planes& P, const StencilArgs& a, const float* Gbv,
                             const float* Gbh, const float* Cbv, const float* Cbh, float* dX,
                             float* dcoh, const DevState* st, cudaStream_t s);

// batched launches over a device array of TileRec (one launch for all images; images whose CG
// run has stopped return at once)
void strip_dims(int H, int W, int& gx, int& gy);
void vec_dims(int H, int W, int dir_rows, int upd_rows, int& gx, int& gy_dir, int& gy_upd);
cudaError_t launch_init_batched(const TileRec* recs, int T, int total_strip, cudaStream_t s);
cudaError_t launch_bnorm_batched(const TileRec* recs, int T, int total_strip, cudaStream_t s);
cudaError_t launch_reweight_batched(const TileRec* recs, int T, int total_rw, cudaStream_t s);
cudaError_t launch_direction_batched(const TileRec* recs, int T, int total_vec, int rows,
                                     cudaStream_t s);
cudaError_t launch_update_batched(const TileRec* recs, int T, int total_upd, int rows,
                                  cudaStream_t s);
cudaError_t launch_finalize_batched(const TileRec* recs, int T, int total_strip, int total_fin,
                                    cudaStream_t s);
cudaError_t launch_count_active(const DevState* states, int T, int* out, cudaStream_t s);

// ---- DCT preconditioner (dct.cu) ------------------------------------------------------------
size_t dct_bytes(int H, int W, int prec);
cudaError_t dct_setup(DctPlan& d, int H, int W, int prec, float tau, char* mem);
// z_U = L^+ (tau r_U) from the plane rU (pitch ld) into zU (pitch ld).  `st` (never null)
// receives error flags; with reduce_rho the last GEMM also forms rho = r_U^T z_U + st->rz_v
// and the next beta (Alg. 2).  With skip_if_done the launches return at once once CG stopped.
void dct_release(DctPlan& d);
// zeroes the folded form's launch counters (recovery after a launch that timed out)
cudaError_t dct_reset(const DctPlan& d, cudaStream_t s);
// test hook: the folded launch's dependency waits run out (IRLS_ERR_TIMEOUT path)
bool dct_stall(DctPlan& d, int on);
// host-only: the fused folded launch's work list, kFoldSchedInts ints per item (dct_umma.cu)
constexpr int kFoldSchedInts = IRLS_FOLD_SCHED_INTS;
bool fold_schedule(const int* H, const int* W, int T, int pairs, int& n_items, int& n_ctr,
                   int& cap_items, std::vector<int>& rec);
cudaError_t launch_schur_reweight(const Planes& P, const StencilArgs& a, DevState* st,
                                  double* partials, cudaStream_t s);
cudaError_t launch_schur_direction(const Planes& P, const StencilArgs& a, DevState* st,
                                   double* partials, cudaStream_t s);
cudaError_t launch_schur_update(const Planes& P, const StencilArgs& a, DevState* st,
                                double* partials, cudaStream_t s);
cudaError_t launch_schur_recover_v(const Planes& P, const StencilArgs& a, cudaStream_t s);
cudaError_t launch_round_congruent(const float* U, const float* X, size_t n, DevState* st,
                                   double* partials, int max_blocks, float* Ur, int* K,
                                   cudaStream_t s);
cudaError_t launch_best_shift(const float* U, const float* Xu, size_t n, DevState* st,
                              double* partials, int max_blocks, float* E, cudaStream_t s);
cudaError_t dct_apply(const DctPlan& d, const float* rU, float* zU, int ld, DevState* st,
                      int reduce_rho, const StencilArgs& a, double* partials, int skip_if_done,
                      cudaStream_t s);
int dct_max_blocks(int H, int W);
size_t dct_rho_slots(int H, int W);
// fast-transform form (dct_fft.cu): shapes it takes, its table memory, its widest grid-reduced
// launch, set-up and application (same contract as dct_apply, float32 only)
bool fft_dct_supported(int H, int W);
size_t fft_dct_bytes(int H, int W);
int fft_dct_max_blocks(int H, int W);
cudaError_t fft_dct_setup(DctPlan& d, char* mem);
cudaError_t fft_dct_apply(const DctPlan& d, const float* rU, float* zU, int ld, DevState* st,
                          int reduce_rho, const StencilArgs& a, double* partials, int skip_if_done,
                          cudaStream_t s);
// batched form (dct_umma.cu): memory for T images of sizes H[t] x W[t], set-up, application
bool foldable(int H, int W, int split);
size_t batch_dct_bytes(const int* H, const int* W, int T, int prec, int fold);
cudaError_t batch_dct_setup(BatchDctPlan& bd, const int* H, const int* W, int T, int prec,
                            int fold, float tau, int flexible, char* mem, const float* const* rU,
                            float* const* zU, const int* ld, DevState* states,
                            double* const* partials);
cudaError_t batch_dct_apply(const BatchDctPlan& bd, cudaStream_t s);
cudaError_t batch_dct_reset(const BatchDctPlan& bd, cudaStream_t s);

}  // namespace irls
