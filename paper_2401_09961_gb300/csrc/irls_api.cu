// Host driver and C ABI of libirls (see include/irls.h).
//
// A plan owns one device allocation that is carved into the image planes, the device-resident
// PCG state, the reduction scratch and the DCT bases.  A solve runs Alg. 1 of arXiv 2401.09961:
// per outer step one reweighting/residual pass, then PCG iterations (Alg. 2) whose scalars
// (alpha, beta, rho, the stopping flag) stay on the device.  The host only issues kernels in
// chunks and polls the device stopping flag through pinned memory, one chunk behind, so the GPU
// never idles waiting for the host.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "irls_internal.cuh"

using namespace irls;

namespace {

thread_local int g_last_cuda = 0;

}  // namespace

namespace irls {
void set_last_cuda_error(int code) { g_last_cuda = code; }
}  // namespace irls

namespace {

constexpr int kPlanes = 21;
constexpr int kChunk = 8;

struct Fail {};

inline void ck(cudaError_t e) {
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        throw Fail{};
    }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int row_pitch(int W) { return (W + 31) / 32 * 32; }

bool opts_valid(const irls_opts& o) {
    if (!(o.tau > 0.f) || !(o.delta > 0.f) || !std::isfinite(o.tau) || !std::isfinite(o.delta))
        return false;
    if (!(o.cg_tol >= 0.f)) return false;
    if (o.outer_iters < 0 || o.outer_iters > IRLS_MAX_OUTER) return false;
    if (o.cg_max_iter < 0) return false;
    if (o.precision < IRLS_PREC_FP32 || o.precision > IRLS_PREC_FP16) return false;
    if (o.dct_form < IRLS_DCT_AUTO || o.dct_form > IRLS_DCT_FFT) return false;
    if (o.cg_schedule != IRLS_CG_FIXED && o.cg_schedule != IRLS_CG_PAPER) return false;
    if (o.system != IRLS_SYS_FULL && o.system != IRLS_SYS_SCHUR) return false;
    if (o.cg_schedule == IRLS_CG_PAPER &&
        (o.cg_m0 < 1 || !(o.cg_alpha > 1.f) || std::isnan(o.cg_eps_tol)))
        return false;
    return true;
}

bool shape_valid(int H, int W) {
    if (H < 1 || W < 1) return false;
    if ((long long)H * (long long)row_pitch(W) > (1LL << 31)) return false;
    return true;
}

struct Layout {
    size_t plane_bytes, planes, state, partials, dct, total;
    int max_blocks;
};

// reduction slots: eight per block of the widest grid-reduced launch, or the folded
// preconditioner's per-tile slots
size_t partial_count(int H, int W, int max_blocks) {
    return std::max((size_t)8 * max_blocks, dct_rho_slots(H, W));
}

Layout layout(int H, int W, int prec) {
    Layout L{};
    const int ld = row_pitch(W);
    L.plane_bytes = align_up((size_t)H * ld * sizeof(float), 256);
    L.planes = 0;
    L.state = L.planes + kPlanes * L.plane_bytes;
    L.partials = L.state + align_up(sizeof(DevState), 256);
    L.max_blocks = std::max({stencil_grid_blocks(H, W), dct_max_blocks(H, W),
                             fft_dct_max_blocks(H, W)});
    L.dct = L.partials + align_up(partial_count(H, W, L.max_blocks) * sizeof(double), 1024);
    L.total = L.dct + align_up(dct_bytes(H, W, prec), 1024) + 1024;
    return L;
}

int status_to_code(int st) {
    if (st & ST_NONFINITE) return IRLS_ERR_NONFINITE;
    if (st & ST_BREAKDOWN) return IRLS_ERR_BREAKDOWN;
    if (st & ST_TIMEOUT) return IRLS_ERR_TIMEOUT;
    if (st & ST_CGMAX) return IRLS_WARN_CG_MAX;
    return IRLS_OK;
}

// Kernel classes timed by the optional live profiler (CUDA events on the solve's stream).
enum ProfClass : int {
    PC_INIT = 0, PC_REWEIGHT, PC_DIRECTION, PC_UPDATE, PC_DCT, PC_FINALIZE, PC_N
};

// Records an event pair around each profiled launch and folds the elapsed times in once the
// stream has passed them (the solve already waits on chunk boundaries, so draining adds no
// synchronisation of its own).
struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> free_ev;
    struct Pair { int cls; cudaEvent_t a, b; };
    std::vector<Pair> pend;
    double ms[PC_N] = {0};
    long long n[PC_N] = {0};

    cudaEvent_t get() {
        if (free_ev.empty()) {
            cudaEvent_t e;
            ck(cudaEventCreate(&e));
            return e;
        }
        cudaEvent_t e = free_ev.back();
        free_ev.pop_back();
        return e;
    }
    cudaEvent_t begin(cudaStream_t s) {
        if (!on) return nullptr;
        cudaEvent_t e = get();
        ck(cudaEventRecord(e, s));
        return e;
    }
    void end(int cls, cudaEvent_t a, cudaStream_t s) {
        if (!on) return;
        cudaEvent_t b = get();
        ck(cudaEventRecord(b, s));
        pend.push_back({cls, a, b});
    }
    // fold in every pair recorded before `upto` pairs (all of them complete)
    void drain(size_t upto) {
        upto = std::min(upto, pend.size());
        for (size_t i = 0; i < upto; ++i) {
            float t = 0.f;
            ck(cudaEventElapsedTime(&t, pend[i].a, pend[i].b));
            ms[pend[i].cls] += t;
            n[pend[i].cls] += 1;
            free_ev.push_back(pend[i].a);
            free_ev.push_back(pend[i].b);
        }
        pend.erase(pend.begin(), pend.begin() + upto);
    }
    void reset() {
        for (int i = 0; i < PC_N; ++i) { ms[i] = 0; n[i] = 0; }
    }
    ~Profiler() {
        for (auto& p : pend) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
        for (auto e : free_ev) cudaEventDestroy(e);
    }
};

}  // namespace

struct irls_plan_s {
    int H = 0, W = 0, ld = 0, dev = 0;
    irls_opts opts{};
    int prec_alloc = 0;
    char* mem = nullptr;
    Layout L{};
    Planes P{};
    DevState* st = nullptr;
    double* partials = nullptr;
    DctPlan dct{};
    int* h_flag = nullptr;     // pinned, 2 slots
    double* h_pair = nullptr;  // pinned, 2 doubles: H_delta values read by the Sec. 4.3 rule
    std::vector<int> caps;     // cap of each inner solve of the last run
    int schedule_stop = 0;
    int dir_rows = 0, upd_rows = 0;   // stencil tile shapes (0: the defaults)
    int rw_rows = 0, fin_rows = 0;    // reweighting and finalize rows (aux_rows of H, W)
    int sdir_rows = 0, supd_rows = 0; // U-only direction and update rows (whole waves, or 0)
    cudaEvent_t ev[2] = {nullptr, nullptr};
    Profiler prof;
};

// Checkpoints of a recorded forward solve for the adjoint sweep: the wrapped gradients and edge
// weights it used, V^k of every outer step (W^k = sqrt(C^2 (V^k)^2 + delta^2) is recomputed
// from them), and the adjoint accumulators.  Planes share the plan's pitch.
struct irls_tape_s {
    irls_plan_s* plan = nullptr;
    int H = 0, W = 0, ld = 0, K = 0, has_coh = 0;
    float tau = 0.f, delta = 0.f;
    char* mem = nullptr;
    size_t plane_bytes = 0;
    float *Gv = nullptr, *Gh = nullptr, *Cv = nullptr, *Ch = nullptr;
    std::vector<float*> Vv, Vh;
    float *Gbv = nullptr, *Gbh = nullptr, *Cbv = nullptr, *Cbh = nullptr;
};

namespace {

StencilArgs make_args(const irls_plan_s* p) {
    StencilArgs a{};
    a.H = p->H; a.W = p->W; a.ld = p->ld;
    a.tau = p->opts.tau;
    a.inv_tau = 1.0f / p->opts.tau;
    a.delta = p->opts.delta;
    a.tol2 = (double)p->opts.cg_tol * (double)p->opts.cg_tol;
    a.cg_max = p->opts.cg_max_iter;
    a.cap_warn = 1;
    a.flexible = p->opts.flexible_cg;
    a.warm_start = p->opts.warm_start;
    a.prec = p->opts.precision;
    a.r16 = (p->opts.precision != IRLS_PREC_FP32) ? p->dct.R16 : nullptr;
    // the residual carries a lo part when the first product splits its data operand
    a.r16lo = (p->opts.precision == IRLS_PREC_BF16X3 && (p->dct.split & 2)) ? p->dct.R16lo
                                                                             : nullptr;
    // the folded form makes its own bf16 operands from r_U (sums and differences of mirrored
    // columns), so the stencil kernels emit none
    if ((p->opts.precision == IRLS_PREC_BF16X3 || p->opts.precision == IRLS_PREC_FP16) &&
        p->dct.fold)
        a.r16 = a.r16lo = nullptr;
    a.ld16 = p->dct.Wp;
    a.dir_rows = p->dir_rows ? p->dir_rows : kDefaultDirRows;
    a.upd_rows = p->upd_rows ? p->upd_rows : kDefaultUpdRows;
    // the reweighting and finalize kernels take rows of their own, a function of the image's
    // size that a batch uses as well (so both sum in the same order)
    a.rw_rows = p->rw_rows;
    a.fin_rows = p->fin_rows;
    a.sdir_rows = p->sdir_rows;
    a.supd_rows = p->supd_rows;
    return a;
}

// Folded preconditioner on or off for the given options; false when IRLS_DCT_FOLDED is asked for
// and the plan has no folded form (a shape or precision that does not allow it).
bool select_dct_form(irls_plan_s* p, const irls_opts& o) {
    // the fast-transform form computes in float32 and takes power-of-two sides
    if (o.dct_form == IRLS_DCT_FFT) {
        if (o.precision != IRLS_PREC_FP32 || !p->dct.fft_ready) return false;
        p->dct.fft = 1;
        p->dct.fold = 0;
        return true;
    }
    p->dct.fft = 0;
    const bool ready = p->dct.fold_ready &&
                       (o.precision == IRLS_PREC_BF16X3 || o.precision == IRLS_PREC_FP16);
    if (o.dct_form == IRLS_DCT_FOLDED && !ready) return false;
    // float16 runs in the folded form only
    if (o.precision == IRLS_PREC_FP16 && (!ready || o.dct_form == IRLS_DCT_DIRECT)) return false;
    p->dct.fold = ready && o.dct_form != IRLS_DCT_DIRECT;
    return true;
}

void destroy_plan(irls_plan_s* p) {
    if (!p) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->dev);
    cudaDeviceSynchronize();
    dct_release(p->dct);
    if (p->mem) cudaFree(p->mem);
    if (p->h_flag) cudaFreeHost(p->h_flag);
    if (p->h_pair) cudaFreeHost(p->h_pair);
    for (auto& e : p->ev)
        if (e) cudaEventDestroy(e);
    cudaSetDevice(cur);
    delete p;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ck(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Copies the device statistics into *stats (if given) and returns the device status bits.
int fetch_stats(irls_plan_s* p, cudaStream_t s, irls_stats* stats) {
    DevState* st = p->st;
    if (stats) {
        DevState h;
        ck(cudaMemcpyAsync(&h, st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        std::memset(stats, 0, sizeof(*stats));
        stats->outer_done = h.outer;
        stats->cg_total = h.cg_total;
        const int n = std::min(h.outer, IRLS_MAX_OUTER);
        for (int k = 0; k < n; ++k) {
            stats->cg_cap[k] = k < (int)p->caps.size() ? p->caps[k] : 0;
            stats->cg_iters[k] = h.cg_iters[k];
            stats->rel_res[k] = h.rel_res[k];
            stats->l1_obj[k] = h.l1_obj[k];
            stats->h_delta[k] = h.h_delta[k];
            stats->f_delta[k] = h.f_delta[k];
        }
        stats->schedule_stop = p->schedule_stop;
        // the rule's last input: F_delta(x^k) at the iteration where it stopped the run
        if (p->schedule_stop && n < IRLS_MAX_OUTER) stats->f_delta[n] = h.f_delta[n];
        stats->status = status_to_code(h.status);
        return h.status;
    }
    ck(cudaMemcpyAsync(&p->h_flag[0], &st->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    return p->h_flag[0];
}

// PCG iterations (Alg. 2) after the first preconditioner application of a run: issued in chunks,
// the device stopping flag polled one chunk behind.
void run_cg(irls_plan_s* p, const StencilArgs& a, DevState* st, cudaStream_t s,
            bool schur_system = false) {
    Profiler& pf = p->prof;
    cudaEvent_t t0;
    int issued = 0, slot = 0;
    bool pending = false;
    size_t mark[2] = {0, 0};
    while (issued < a.cg_max) {
        const int n = std::min(kChunk, a.cg_max - issued);
        const bool schur = schur_system || p->opts.system == IRLS_SYS_SCHUR;
        for (int c = 0; c < n; ++c) {
            t0 = pf.begin(s);
            if (schur) ck(launch_schur_direction(p->P, a, st, p->partials, s));
            else ck(launch_direction_pap(p->P, a, st, p->partials, s));
            pf.end(PC_DIRECTION, t0, s);
            t0 = pf.begin(s);
            if (schur) ck(launch_schur_update(p->P, a, st, p->partials, s));
            else ck(launch_update(p->P, a, st, p->partials, s));
            pf.end(PC_UPDATE, t0, s);
            t0 = pf.begin(s);
            ck(dct_apply(p->dct, p->P.rU, p->P.zU, p->ld, st, 1, a, p->partials, 1, s));
            pf.end(PC_DCT, t0, s);
        }
        issued += n;
        ck(cudaMemcpyAsync(&p->h_flag[slot], &st->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        ck(cudaEventRecord(p->ev[slot], s));
        mark[slot] = pf.pend.size();
        if (pending) {
            ck(cudaEventSynchronize(p->ev[slot ^ 1]));
            pf.drain(mark[slot ^ 1]);
            mark[slot] -= std::min(mark[slot], mark[slot ^ 1]);
            if (p->h_flag[slot ^ 1]) break;
        }
        pending = true;
        slot ^= 1;
    }
}

void copy_plane(float* dst, const float* src, size_t bytes, cudaStream_t s) {
    ck(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s));
}

// Runs the whole of Alg. 1 on the plan's workspace; returns the device status bits.  With a
// tape, G, C and V^0 .. V^K are checkpointed for the adjoint sweep.
int run_solve(irls_plan_s* p, const float* X, const float* coh, const float* Cv, const float* Ch,
              const float* U0, const float* Vv0, const float* Vh0, cudaStream_t s,
              irls_stats* stats, irls_tape_s* tape = nullptr) {
    TraceRange trace("irls_unwrap");
    const StencilArgs a = make_args(p);
    DevState* st = p->st;
    Profiler& pf = p->prof;
    const size_t pb = p->L.plane_bytes;
    cudaEvent_t t0;
    {
        TraceRange r("irls_init");
        ck(cudaMemsetAsync(st, 0, sizeof(DevState), s));
        ck(dct_reset(p->dct, s));
        t0 = pf.begin(s);
        ck(launch_init(X, coh, Cv, Ch, U0, Vv0, Vh0, p->P, a, st, p->partials, s));
        ck(launch_bnorm(p->P, a, st, p->partials, s));
        pf.end(PC_INIT, t0, s);
    }
    // stop early on invalid input
    ck(cudaMemcpyAsync(&p->h_flag[0], &st->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    pf.drain(pf.pend.size());
    if (p->h_flag[0] & ST_NONFINITE) return p->h_flag[0];
    if (tape) {
        copy_plane(tape->Gv, p->P.Gv, pb, s); copy_plane(tape->Gh, p->P.Gh, pb, s);
        copy_plane(tape->Cv, p->P.Cv, pb, s); copy_plane(tape->Ch, p->P.Ch, pb, s);
        copy_plane(tape->Vv[0], p->P.Vv, pb, s); copy_plane(tape->Vh[0], p->P.Vh, pb, s);
    }

    // inner-solve budget: fixed, or the adaptive rule of Sec. 4.3
    const bool sched = p->opts.cg_schedule == IRLS_CG_PAPER;
    int m_cg = p->opts.cg_m0;
    bool raised = false;
    p->caps.assign(p->opts.outer_iters, 0);
    p->schedule_stop = 0;
    const bool schur = p->opts.system == IRLS_SYS_SCHUR;
    for (int k = 0; k < p->opts.outer_iters; ++k) {
        TraceRange r_outer("irls_outer");
        t0 = pf.begin(s);
        {
            TraceRange r("irls_reweight");
            if (schur) ck(launch_schur_reweight(p->P, a, st, p->partials, s));
            else ck(launch_reweight_residual(p->P, a, st, p->partials, s));
        }
        pf.end(PC_REWEIGHT, t0, s);
        StencilArgs ak = a;
        if (sched) {
            if (k >= 1 && k < IRLS_MAX_OUTER) {
                // Delta_{k-1,k} from H_delta(x^k, W^{k-1}) (the previous finalize) and
                // H_delta(x^k, W^k) = F_delta(x^k) (this reweight)
                ck(cudaMemcpyAsync(&p->h_pair[0], &st->h_delta[k - 1], sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
                ck(cudaMemcpyAsync(&p->h_pair[1], &st->f_delta[k], sizeof(double),
                                   cudaMemcpyDeviceToHost, s));
                ck(cudaStreamSynchronize(s));
                const double hp = p->h_pair[0], hk = p->h_pair[1];
                const double d = (hp - hk) / hp;
                if (d > (double)p->opts.cg_eps_tol) {
                    raised = false;
                } else if (raised) {
                    p->schedule_stop = 1;   // return U^k
                    break;
                } else {
                    m_cg = (int)std::floor((double)p->opts.cg_alpha * (double)m_cg);
                    raised = true;
                }
            }
            ak.cg_max = std::min(m_cg, p->opts.cg_max_iter);
            // a planned budget is not a warning; the hard cap is
            ak.cap_warn = ak.cg_max >= p->opts.cg_max_iter ? 1 : 0;
        }
        p->caps[k] = ak.cg_max;
        {
            TraceRange r("irls_pcg");
            t0 = pf.begin(s);
            ck(dct_apply(p->dct, p->P.rU, p->P.zU, p->ld, st, 1, ak, p->partials, 1, s));
            pf.end(PC_DCT, t0, s);
            run_cg(p, ak, st, s);
        }
        t0 = pf.begin(s);
        {
            TraceRange r("irls_finalize");
            if (schur) ck(launch_schur_recover_v(p->P, ak, s));
            ck(launch_finalize(p->P, ak, st, p->partials, s));
        }
        pf.end(PC_FINALIZE, t0, s);
        if (tape) {
            copy_plane(tape->Vv[k + 1], p->P.Vv, pb, s);
            copy_plane(tape->Vh[k + 1], p->P.Vh, pb, s);
        }
    }
    if (pf.on) {
        ck(cudaStreamSynchronize(s));
        pf.drain(pf.pend.size());
    }
    return fetch_stats(p, s, stats);
}

std::mutex g_simple_mu;

}  // namespace

// A batched solve: T images of their own sizes, one launch per phase for all of them.
struct irls_batch_s {
    int T = 0, dev = 0;
    irls_opts opts{};
    std::vector<int> H, W, ld;
    char* mem = nullptr;
    std::vector<TileRec> recs;
    TileRec* d_recs = nullptr;
    DevState* states = nullptr;
    int total_strip = 0, total_vec = 0, total_upd = 0, total_rw = 0, total_fin = 0;
    int dir_rows = kDefaultDirRows, upd_rows = kDefaultUpdRows;   // stencil tile shapes
    BatchDctPlan dct;
    int* d_count = nullptr;          // device, 2 slots
    int* h_count = nullptr;          // pinned, 2 slots
    cudaStream_t stream = nullptr;   // internal stream (capturable)
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaEvent_t join = nullptr;
    cudaGraphExec_t chunk[2] = {nullptr, nullptr};
    int chunk_iters = 0;
    bool graphs_tried = false;
};

namespace {

void destroy_batch(irls_batch_s* b) {
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(b->dev);
    cudaDeviceSynchronize();
    for (auto& g : b->chunk)
        if (g) cudaGraphExecDestroy(g);
    if (b->mem) cudaFree(b->mem);
    if (b->h_count) cudaFreeHost(b->h_count);
    for (auto& e : b->ev)
        if (e) cudaEventDestroy(e);
    if (b->join) cudaEventDestroy(b->join);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaSetDevice(cur);
    delete b;
}

// Each image's blocks in the batched direction and update launches for the batch's tile shapes
// (host records; uploaded with the image pointers at the start of every run).
void layout_vec_blocks(irls_batch_s* b) {
    int vblk = 0, ublk = 0, rblk = 0, fblk = 0;
    for (int t = 0; t < b->T; ++t) {
        TileRec& r = b->recs[t];
        vec_dims(b->H[t], b->W[t], b->dir_rows, b->upd_rows, r.vgx, r.vgy, r.ugy);
        r.vblk0 = vblk;
        r.ublk0 = ublk;
        r.rblk0 = rblk;
        r.fblk0 = fblk;
        r.rgy = (b->H[t] + r.a.rw_rows - 1) / r.a.rw_rows;
        r.fgy = (b->H[t] + r.a.fin_rows - 1) / r.a.fin_rows;
        vblk += r.vgx * r.vgy;
        ublk += r.vgx * r.ugy;
        rblk += r.vgx * r.rgy;
        fblk += r.vgx * r.fgy;
    }
    b->total_vec = vblk;
    b->total_upd = ublk;
    b->total_rw = rblk;
    b->total_fin = fblk;
}

// The CG chunk graphs bake in the launches' grids and kernels: captured again on the next run.
void drop_graphs(irls_batch_s* b) {
    for (auto& g : b->chunk)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    b->graphs_tried = false;
}

// one chunk of n batched CG iterations followed by the count of images still iterating
void issue_chunk(irls_batch_s* b, int n, int slot, cudaStream_t s) {
    for (int c = 0; c < n; ++c) {
        ck(launch_direction_batched(b->d_recs, b->T, b->total_vec, b->dir_rows, s));
        ck(launch_update_batched(b->d_recs, b->T, b->total_upd, b->upd_rows, s));
        ck(batch_dct_apply(b->dct, s));
    }
    ck(launch_count_active(b->states, b->T, b->d_count + slot, s));
}

// Captures the full-size chunk once per batch (two graphs: one per count slot); eager launches
// are used if capture is unavailable.
void prepare_graphs(irls_batch_s* b) {
    if (b->graphs_tried) return;
    b->graphs_tried = true;
    b->chunk_iters = kChunk;
    for (int slot = 0; slot < 2; ++slot) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        bool ok = true;
        try {
            issue_chunk(b, kChunk, slot, b->stream);
        } catch (Fail&) {
            ok = false;
        }
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (!ok || e != cudaSuccess || !g) {
            cudaGetLastError();
            if (g) cudaGraphDestroy(g);
            for (auto& x : b->chunk)
                if (x) { cudaGraphExecDestroy(x); x = nullptr; }
            return;
        }
        e = cudaGraphInstantiate(&b->chunk[slot], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            for (auto& x : b->chunk)
                if (x) { cudaGraphExecDestroy(x); x = nullptr; }
            return;
        }
    }
}

int run_batch(irls_batch_s* b, const float* const* X, const float* const* coh, float* const* U,
              irls_stats* stats, cudaStream_t user) {
    TraceRange trace("irls_batch_unwrap");
    const int T = b->T;
    cudaStream_t s = b->stream;
    // order after the caller's stream
    ck(cudaEventRecord(b->join, user));
    ck(cudaStreamWaitEvent(s, b->join, 0));
    for (int t = 0; t < T; ++t) {
        b->recs[t].X = X[t];
        b->recs[t].coh = coh ? coh[t] : nullptr;
    }
    ck(cudaMemcpyAsync(b->d_recs, b->recs.data(), (size_t)T * sizeof(TileRec),
                       cudaMemcpyHostToDevice, s));
    ck(cudaMemsetAsync(b->states, 0, (size_t)T * sizeof(DevState), s));
    ck(batch_dct_reset(b->dct, s));
    ck(launch_init_batched(b->d_recs, T, b->total_strip, s));
    ck(launch_bnorm_batched(b->d_recs, T, b->total_strip, s));
    std::vector<DevState> h(T);
    ck(cudaMemcpyAsync(h.data(), b->states, (size_t)T * sizeof(DevState), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    int bad = 0;
    for (int t = 0; t < T; ++t) bad |= h[t].status & ST_NONFINITE;
    if (bad) return ST_NONFINITE;
    prepare_graphs(b);
    for (int k = 0; k < b->opts.outer_iters; ++k) {
        TraceRange r_outer("irls_outer");
        ck(launch_reweight_batched(b->d_recs, T, b->total_rw, s));
        {
            TraceRange r_pcg("irls_pcg");
            ck(batch_dct_apply(b->dct, s));
            int issued = 0, slot = 0;
            bool pending = false;
            while (issued < b->opts.cg_max_iter) {
                const int n = std::min(kChunk, b->opts.cg_max_iter - issued);
                if (n == kChunk && b->chunk[slot])
                    ck(cudaGraphLaunch(b->chunk[slot], s));
                else
                    issue_chunk(b, n, slot, s);
                issued += n;
                ck(cudaMemcpyAsync(&b->h_count[slot], b->d_count + slot, sizeof(int),
                                   cudaMemcpyDeviceToHost, s));
                ck(cudaEventRecord(b->ev[slot], s));
                if (pending) {
                    ck(cudaEventSynchronize(b->ev[slot ^ 1]));
                    if (b->h_count[slot ^ 1] == 0) break;
                }
                pending = true;
                slot ^= 1;
            }
        }
        TraceRange r_fin("irls_finalize");
        ck(launch_finalize_batched(b->d_recs, T, b->total_strip, b->total_fin, s));
    }
    for (int t = 0; t < T; ++t)
        ck(launch_copy_out(b->recs[t].P.U, b->H[t], b->W[t], b->ld[t], U[t], s));
    ck(cudaMemcpyAsync(h.data(), b->states, (size_t)T * sizeof(DevState), cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    int all = 0;
    for (int t = 0; t < T; ++t) {
        all |= h[t].status;
        if (stats) {
            irls_stats& o = stats[t];
            std::memset(&o, 0, sizeof(o));
            o.outer_done = h[t].outer;
            o.cg_total = h[t].cg_total;
            const int n = std::min(h[t].outer, IRLS_MAX_OUTER);
            for (int q = 0; q < n; ++q) {
                o.cg_iters[q] = h[t].cg_iters[q];
                o.rel_res[q] = h[t].rel_res[q];
                o.l1_obj[q] = h[t].l1_obj[q];
                o.h_delta[q] = h[t].h_delta[q];
                o.f_delta[q] = h[t].f_delta[q];
            }
            o.status = status_to_code(h[t].status);
        }
    }
    return all;
}

}  // namespace

extern "C" {

int irls_opts_default(irls_opts* o) {
    if (!o) return IRLS_ERR_ARG;
    o->tau = 1e-2f;
    o->delta = 1e-6f;
    o->outer_iters = 20;
    o->cg_tol = 1e-6f;
    o->cg_max_iter = 1000;
    o->precision = IRLS_PREC_FP32;
    o->flexible_cg = 0;
    o->warm_start = 1;
    o->dct_form = IRLS_DCT_AUTO;
    o->cg_schedule = IRLS_CG_FIXED;
    o->cg_m0 = 5;
    o->cg_eps_tol = 1e-3f;
    o->cg_alpha = 1.7f;
    o->system = IRLS_SYS_FULL;
    return IRLS_OK;
}

size_t irls_workspace_bytes(int H, int W, const irls_opts* opts) {
    irls_opts o;
    irls_opts_default(&o);
    if (opts) o = *opts;
    if (!shape_valid(H, W) || !opts_valid(o)) return 0;
    return layout(H, W, o.precision).total;
}

int irls_plan_create(int H, int W, const irls_opts* opts, irls_plan* out) {
    if (!out) return IRLS_ERR_ARG;
    *out = nullptr;
    irls_opts o;
    irls_opts_default(&o);
    if (opts) o = *opts;
    if (!opts_valid(o)) return IRLS_ERR_ARG;
    if (!shape_valid(H, W)) return IRLS_ERR_SHAPE;
    // the fast-transform form's precision and lengths are known before any device work
    if (o.dct_form == IRLS_DCT_FFT &&
        (o.precision != IRLS_PREC_FP32 || !fft_dct_supported(H, W)))
        return IRLS_ERR_UNSUPPORTED;
    irls_plan_s* p = new (std::nothrow) irls_plan_s();
    if (!p) return IRLS_ERR_OOM;
    try {
        ck(cudaGetDevice(&p->dev));
        p->H = H; p->W = W; p->ld = row_pitch(W);
        p->rw_rows = aux_rows(2, H, W);
        p->fin_rows = aux_rows(3, H, W);
        p->sdir_rows = wave_rows(4, H, W, kMaxTileRows);
        p->supd_rows = wave_rows(5, H, W, kMaxTileRows);
        p->opts = o;
        p->prec_alloc = o.precision;
        p->L = layout(H, W, o.precision);
        cudaError_t e = cudaMalloc(&p->mem, p->L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p->mem = nullptr;
            destroy_plan(p);
            return IRLS_ERR_OOM;
        }
        ck(cudaMemset(p->mem, 0, p->L.total));
        float* f[kPlanes];
        for (int i = 0; i < kPlanes; ++i)
            f[i] = reinterpret_cast<float*>(p->mem + p->L.planes + (size_t)i * p->L.plane_bytes);
        Planes& P = p->P;
        int q = 0;
        P.U = f[q++]; P.Vv = f[q++]; P.Vh = f[q++];
        P.rU = f[q++]; P.rVv = f[q++]; P.rVh = f[q++];
        for (int b = 0; b < 2; ++b) { P.pU[b] = f[q++]; P.pVv[b] = f[q++]; P.pVh[b] = f[q++]; }
        P.zU = f[q++];
        P.dv = f[q++]; P.dh = f[q++];
        P.Wv = f[q++]; P.Wh = f[q++];
        P.Gv = f[q++]; P.Gh = f[q++];
        P.Cv = f[q++]; P.Ch = f[q++];
        p->st = reinterpret_cast<DevState*>(p->mem + p->L.state);
        p->partials = reinterpret_cast<double*>(p->mem + p->L.partials);
        ck(dct_setup(p->dct, H, W, o.precision, o.tau, p->mem + p->L.dct));
        if (!select_dct_form(p, o)) {
            destroy_plan(p);
            return IRLS_ERR_UNSUPPORTED;
        }
        ck(cudaHostAlloc(&p->h_flag, 2 * sizeof(int), cudaHostAllocDefault));
        ck(cudaHostAlloc(&p->h_pair, 2 * sizeof(double), cudaHostAllocDefault));
        for (auto& ev : p->ev) ck(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        ck(cudaDeviceSynchronize());
    } catch (Fail&) {
        destroy_plan(p);
        return IRLS_ERR_CUDA;
    }
    *out = p;
    return IRLS_OK;
}

int irls_plan_dct_form(irls_plan p) {
    if (!p) return IRLS_ERR_ARG;
    if (p->dct.fft) return IRLS_DCT_FFT;
    if (p->opts.precision == IRLS_PREC_FP32) return IRLS_DCT_AUTO;
    return p->dct.fold ? IRLS_DCT_FOLDED : IRLS_DCT_DIRECT;
}

int irls_debug_stall_fold(irls_plan p, int on) {
    if (!p) return IRLS_ERR_ARG;
    return dct_stall(p->dct, on) ? IRLS_OK : IRLS_ERR_UNSUPPORTED;
}

int irls_debug_fold_schedule(int n_img, const int* H, const int* W, int pairs, int* n_items,
                             int* n_ctr, int* cap_items, int* rec, int rec_items) {
    if (n_img < 1 || pairs < 1 || !H || !W || !n_items || !n_ctr || !cap_items)
        return IRLS_ERR_ARG;
    for (int t = 0; t < n_img; ++t)
        if (H[t] < 256 || W[t] < 256 || H[t] > 32768 || W[t] > 32768) return IRLS_ERR_SHAPE;
    try {
        std::vector<int> r;
        int ni = 0, nc = 0, cap = 0;
        if (!fold_schedule(H, W, n_img, pairs, ni, nc, cap, r)) return IRLS_ERR_SHAPE;
        *n_items = ni;
        *n_ctr = nc;
        *cap_items = cap;
        if (!rec) return IRLS_OK;
        if (rec_items < ni) return IRLS_ERR_ARG;
        std::copy(r.begin(), r.end(), rec);
        return IRLS_OK;
    } catch (...) {
        return IRLS_ERR_OOM;
    }
}

int irls_plan_set_tiles(irls_plan p, int dir_rows, int upd_rows) {
    if (!p) return IRLS_ERR_ARG;
    if ((dir_rows != 0 && !plan_rows_ok(dir_rows)) || (upd_rows != 0 && !plan_rows_ok(upd_rows)))
        return IRLS_ERR_ARG;
    if (dir_rows) p->dir_rows = dir_rows;
    if (upd_rows) p->upd_rows = upd_rows;
    return IRLS_OK;
}

int irls_plan_get_tiles(irls_plan p, int* dir_rows, int* upd_rows) {
    if (!p || !dir_rows || !upd_rows) return IRLS_ERR_ARG;
    const StencilArgs a = make_args(p);
    *dir_rows = a.dir_rows;
    *upd_rows = a.upd_rows;
    return IRLS_OK;
}

int irls_plan_autotune(irls_plan p, float* h_ms, void* stream) {
    if (!p) return IRLS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = IRLS_OK;
    try {
        DeviceGuard g(p->dev);
        ck(cudaEventCreate(&e0));
        ck(cudaEventCreate(&e1));
        StencilArgs a = make_args(p);
        // a run that never stops on its own: the kernels do their full traffic every launch
        a.cg_max = 1 << 30;
        a.tol2 = -1.0;
        a.cap_warn = 0;
        constexpr int kWarm = 2, kReps = 10;
        // candidates: the fixed row counts, then for each kernel the counts that make its
        // launch the fewest whole waves with at most 32 and at most 64 rows a block (where they
        // are not among the others)
        int cand[2][6];
        int ncand[2];
        for (int k = 0; k < 2; ++k) {
            for (int i = 0; i < 4; ++i) cand[k][i] = kTileRows[i];
            ncand[k] = 4;
            for (int cap : {32, kMaxTileRows}) {
                const int w = wave_rows(k, p->H, p->W, cap);
                bool seen = (w == 0);
                for (int i = 0; i < ncand[k]; ++i) seen |= (cand[k][i] == w);
                if (!seen) cand[k][ncand[k]++] = w;
            }
        }
        float ms[2][6];
        for (int k = 0; k < 2; ++k)
            for (int i = 0; i < ncand[k]; ++i) {
                StencilArgs b = a;
                if (k == 0) b.dir_rows = cand[k][i];
                else b.upd_rows = cand[k][i];
                float tot = 0.f;
                for (int r = 0; r < kWarm + kReps; ++r) {
                    // a fresh state per launch (a stopped run's kernels return at once)
                    ck(cudaMemsetAsync(p->st, 0, sizeof(DevState), s));
                    ck(cudaEventRecord(e0, s));
                    if (k == 0) ck(launch_direction_pap(p->P, b, p->st, p->partials, s));
                    else ck(launch_update(p->P, b, p->st, p->partials, s));
                    ck(cudaEventRecord(e1, s));
                    ck(cudaEventSynchronize(e1));
                    float t = 0.f;
                    ck(cudaEventElapsedTime(&t, e0, e1));
                    if (r >= kWarm) tot += t;
                }
                ms[k][i] = tot / kReps;
            }
        int bd = 0, bu = 0;
        for (int i = 1; i < ncand[0]; ++i)
            if (ms[0][i] < ms[0][bd]) bd = i;
        for (int i = 1; i < ncand[1]; ++i)
            if (ms[1][i] < ms[1][bu]) bu = i;
        p->dir_rows = cand[0][bd];
        p->upd_rows = cand[1][bu];
        if (h_ms)
            for (int k = 0; k < 2; ++k)
                for (int i = 0; i < 4; ++i) h_ms[4 * k + i] = ms[k][i];
        ck(cudaMemsetAsync(p->st, 0, sizeof(DevState), s));
        ck(cudaStreamSynchronize(s));
    } catch (Fail&) {
        rc = IRLS_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

int irls_plan_destroy(irls_plan p) {
    destroy_plan(p);
    return IRLS_OK;
}

int irls_plan_set_opts(irls_plan p, const irls_opts* opts) {
    if (!p || !opts) return IRLS_ERR_ARG;
    if (!opts_valid(*opts)) return IRLS_ERR_ARG;
    if (opts->precision != p->opts.precision && opts->precision != IRLS_PREC_FP32 &&
        opts->precision != p->prec_alloc)
        return IRLS_ERR_UNSUPPORTED;
    if (!select_dct_form(p, *opts)) return IRLS_ERR_UNSUPPORTED;
    if (opts->tau != p->opts.tau) {
        p->dct.tau = opts->tau;
    }
    p->opts = *opts;
    p->dct.prec = opts->precision;
    return IRLS_OK;
}

int irls_unwrap_ex(irls_plan p, const float* X, const float* coh, const float* Cv,
                   const float* Ch, const float* U0, float* U, float* Vv, float* Vh,
                   irls_stats* stats, void* stream) {
    if (!p || !X || !U) return IRLS_ERR_ARG;
    if ((Cv == nullptr) != (Ch == nullptr)) return IRLS_ERR_ARG;
    if (U0 && ((p->H > 1 && !Vv) || (p->W > 1 && !Vh))) return IRLS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int status = 0;
    try {
        DeviceGuard g(p->dev);
        status = run_solve(p, X, coh, Cv, Ch, U0, U0 ? Vv : nullptr, U0 ? Vh : nullptr, s, stats);
        if (status & ST_NONFINITE) {
            if (stats) stats->status = IRLS_ERR_NONFINITE;
            return IRLS_ERR_NONFINITE;
        }
        ck(launch_copy_out(p->P.U, p->H, p->W, p->ld, U, s));
        if (Vv) ck(launch_copy_out(p->P.Vv, p->H - 1, p->W, p->ld, Vv, s));
        if (Vh) ck(launch_copy_out(p->P.Vh, p->H, p->W - 1, p->ld, Vh, s));
        ck(cudaStreamSynchronize(s));
    } catch (Fail&) {
        return IRLS_ERR_CUDA;
    }
    return status_to_code(status);
}

int irls_unwrap_forward_record(irls_plan p, const float* X, const float* coh, const float* Cv,
                               const float* Ch, float* U, irls_tape* out, irls_stats* stats,
                               void* stream) {
    if (!p || !X || !U || !out) return IRLS_ERR_ARG;
    *out = nullptr;
    if ((Cv == nullptr) != (Ch == nullptr)) return IRLS_ERR_ARG;
    // the adjoint differentiates through converged inner solves: no planned budgets; its
    // right-hand sides carry no norm for the float16 scale
    if (p->opts.cg_schedule != IRLS_CG_FIXED || p->opts.system != IRLS_SYS_FULL ||
        p->opts.precision == IRLS_PREC_FP16)
        return IRLS_ERR_UNSUPPORTED;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    irls_tape_s* t = new (std::nothrow) irls_tape_s();
    if (!t) return IRLS_ERR_OOM;
    int status = 0;
    try {
        DeviceGuard g(p->dev);
        t->plan = p;
        t->H = p->H; t->W = p->W; t->ld = p->ld;
        t->K = p->opts.outer_iters;
        t->has_coh = (coh != nullptr && Cv == nullptr) ? 1 : 0;
        t->tau = p->opts.tau;
        t->delta = p->opts.delta;
        t->plane_bytes = p->L.plane_bytes;
        const size_t nplanes = 8 + 2 * (size_t)(t->K + 1);
        if (cudaMalloc(&t->mem, nplanes * t->plane_bytes) != cudaSuccess) {
            cudaGetLastError();
            delete t;
            return IRLS_ERR_OOM;
        }
        float* f[64 + 2 * IRLS_MAX_OUTER];
        for (size_t i = 0; i < nplanes; ++i)
            f[i] = reinterpret_cast<float*>(t->mem + i * t->plane_bytes);
        size_t q = 0;
        t->Gv = f[q++]; t->Gh = f[q++]; t->Cv = f[q++]; t->Ch = f[q++];
        t->Gbv = f[q++]; t->Gbh = f[q++]; t->Cbv = f[q++]; t->Cbh = f[q++];
        for (int k = 0; k <= t->K; ++k) { t->Vv.push_back(f[q++]); t->Vh.push_back(f[q++]); }
        status = run_solve(p, X, coh, Cv, Ch, nullptr, nullptr, nullptr, s, stats, t);
        if (status & ST_NONFINITE) {
            cudaStreamSynchronize(s);
            cudaFree(t->mem);
            delete t;
            if (stats) stats->status = IRLS_ERR_NONFINITE;
            return IRLS_ERR_NONFINITE;
        }
        ck(launch_copy_out(p->P.U, p->H, p->W, p->ld, U, s));
        ck(cudaStreamSynchronize(s));
    } catch (Fail&) {
        if (t->mem) cudaFree(t->mem);
        delete t;
        return IRLS_ERR_CUDA;
    }
    *out = t;
    return status_to_code(status);
}

int irls_unwrap_backward(irls_tape t, const float* dLdU, float* dLdX, float* dLdcoh,
                         irls_stats* stats, void* stream) {
    if (!t || !dLdU || !dLdX) return IRLS_ERR_ARG;
    if (dLdcoh && !t->has_coh) return IRLS_ERR_ARG;
    irls_plan_s* p = t->plan;
    if (!p || p->H != t->H || p->W != t->W) return IRLS_ERR_ARG;
    if (p->opts.tau != t->tau || p->opts.delta != t->delta) return IRLS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int status = 0;
    try {
        DeviceGuard g(p->dev);
        const StencilArgs a = make_args(p);
        DevState* st = p->st;
        const size_t pb = t->plane_bytes;
        ck(cudaMemsetAsync(st, 0, sizeof(DevState), s));
        ck(dct_reset(p->dct, s));
        for (float* z : {t->Gbv, t->Gbh, t->Cbv, t->Cbh}) ck(cudaMemsetAsync(z, 0, pb, s));
        TraceRange trace("irls_backward");
        ck(launch_adj_init(p->P, a, dLdU, st, p->partials, s));
        for (int k = t->K - 1; k >= 0; --k) {
            TraceRange r_step("irls_backward_step");
            // lambda = A_k^+ xbar through the U-only system (V eliminated exactly), for the
            // step's cotangent normalised to unit norm (its factor kept in FP64 on the device)
            ck(launch_adj_norm(p->P, a, st, p->partials, s));
            ck(launch_adj_setup_schur(p->P, a, t->Vv[k], t->Vh[k], t->Cv, t->Ch, st,
                                      p->partials, s));
            ck(dct_apply(p->dct, p->P.rU, p->P.zU, p->ld, st, 1, a, p->partials, 1, s));
            run_cg(p, a, st, s, true);
            ck(launch_adj_recover_v(p->P, a, st, s));
            ck(launch_record_step(st, s));
            ck(launch_adj_accumulate(p->P, a, t->Vv[k], t->Vh[k], t->Vv[k + 1], t->Vh[k + 1],
                                     t->Cv, t->Ch, t->Gbv, t->Gbh, t->Cbv, t->Cbh, st, s));
        }
        ck(launch_adj_final(p->P, a, t->Gbv, t->Gbh, t->Cbv, t->Cbh, dLdX, dLdcoh, st, s));
        status = fetch_stats(p, s, stats);
    } catch (Fail&) {
        return IRLS_ERR_CUDA;
    }
    return status_to_code(status);
}

int irls_tape_free(irls_tape t) {
    if (!t) return IRLS_OK;
    if (t->mem) {
        cudaDeviceSynchronize();
        cudaFree(t->mem);
    }
    delete t;
    return IRLS_OK;
}

int irls_unwrap(const float* X, const float* coh, int H, int W, float eps, int outer_iters,
                float cg_tol, float* U, void* stream) {
    if (!X || !U) return IRLS_ERR_ARG;
    if (!shape_valid(H, W)) return IRLS_ERR_SHAPE;
    irls_opts o;
    irls_opts_default(&o);
    o.delta = eps;
    o.outer_iters = outer_iters;
    o.cg_tol = cg_tol;
    if (!opts_valid(o)) return IRLS_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_simple_mu);
    irls_plan p = nullptr;
    int rc = irls_plan_create(H, W, &o, &p);
    if (rc != IRLS_OK) return rc;
    rc = irls_unwrap_ex(p, X, coh, nullptr, nullptr, nullptr, U, nullptr, nullptr, nullptr, stream);
    irls_plan_destroy(p);
    return rc;
}

int irls_batch_create(int ntiles, const int* H, const int* W, const irls_opts* opts,
                      irls_batch* out) {
    if (!out || !H || !W || ntiles < 1) return IRLS_ERR_ARG;
    *out = nullptr;
    irls_opts o;
    irls_opts_default(&o);
    if (opts) o = *opts;
    if (!opts_valid(o)) return IRLS_ERR_ARG;
    if (o.precision == IRLS_PREC_FP32 || o.precision == IRLS_PREC_FP16) return IRLS_ERR_UNSUPPORTED;
    if (o.cg_schedule != IRLS_CG_FIXED) return IRLS_ERR_UNSUPPORTED;  // images run in lockstep
    if (o.system != IRLS_SYS_FULL) return IRLS_ERR_UNSUPPORTED;
    for (int t = 0; t < ntiles; ++t)
        if (!shape_valid(H[t], W[t])) return IRLS_ERR_SHAPE;
    // folded preconditioner when every image allows it (split precision, sides >= 256, odd or even)
    bool all_fold = true;
    for (int t = 0; t < ntiles; ++t)
        all_fold &= foldable(H[t], W[t], o.precision == IRLS_PREC_BF16X3 ? 1 : 0);
    if (o.dct_form == IRLS_DCT_FOLDED && !all_fold) return IRLS_ERR_UNSUPPORTED;
    if (o.dct_form == IRLS_DCT_FFT) return IRLS_ERR_UNSUPPORTED;   // single-image plans only
    const int fold = all_fold && o.dct_form != IRLS_DCT_DIRECT ? 1 : 0;
    irls_batch_s* b = new (std::nothrow) irls_batch_s();
    if (!b) return IRLS_ERR_OOM;
    try {
        ck(cudaGetDevice(&b->dev));
        const int T = ntiles;
        b->T = T;
        b->opts = o;
        b->H.assign(H, H + T);
        b->W.assign(W, W + T);
        std::vector<size_t> plane_bytes(T), part_bytes(T);
        size_t total = 0;
        for (int t = 0; t < T; ++t) {
            const int ld = row_pitch(W[t]);
            b->ld.push_back(ld);
            plane_bytes[t] = align_up((size_t)H[t] * ld * sizeof(float), 256);
            const int nb = std::max(stencil_grid_blocks(H[t], W[t]), dct_max_blocks(H[t], W[t]));
            part_bytes[t] = align_up(partial_count(H[t], W[t], nb) * sizeof(double), 256);
            total += kPlanes * plane_bytes[t] + part_bytes[t];
        }
        const size_t state_off = align_up(total, 1024);
        const size_t recs_off = align_up(state_off + (size_t)T * sizeof(DevState), 1024);
        const size_t count_off = align_up(recs_off + (size_t)T * sizeof(TileRec), 256);
        const size_t dct_off = align_up(count_off + 256, 1024);
        const size_t all = dct_off + batch_dct_bytes(H, W, T, o.precision, fold);
        if (cudaMalloc(&b->mem, all) != cudaSuccess) {
            cudaGetLastError();
            b->mem = nullptr;
            destroy_batch(b);
            return IRLS_ERR_OOM;
        }
        ck(cudaMemset(b->mem, 0, all));
        b->states = reinterpret_cast<DevState*>(b->mem + state_off);
        b->d_recs = reinterpret_cast<TileRec*>(b->mem + recs_off);
        b->d_count = reinterpret_cast<int*>(b->mem + count_off);
        b->recs.resize(T);
        std::vector<const float*> rU(T);
        std::vector<float*> zU(T);
        std::vector<double*> parts(T);
        size_t off = 0;
        for (int t = 0; t < T; ++t) {
            float* f[kPlanes];
            for (int i = 0; i < kPlanes; ++i)
                f[i] = reinterpret_cast<float*>(b->mem + off + (size_t)i * plane_bytes[t]);
            off += kPlanes * plane_bytes[t];
            parts[t] = reinterpret_cast<double*>(b->mem + off);
            off += part_bytes[t];
            TileRec& r = b->recs[t];
            Planes& P = r.P;
            int q = 0;
            P.U = f[q++]; P.Vv = f[q++]; P.Vh = f[q++];
            P.rU = f[q++]; P.rVv = f[q++]; P.rVh = f[q++];
            for (int bb = 0; bb < 2; ++bb) { P.pU[bb] = f[q++]; P.pVv[bb] = f[q++]; P.pVh[bb] = f[q++]; }
            P.zU = f[q++];
            P.dv = f[q++]; P.dh = f[q++];
            P.Wv = f[q++]; P.Wh = f[q++];
            P.Gv = f[q++]; P.Gh = f[q++];
            P.Cv = f[q++]; P.Ch = f[q++];
            rU[t] = P.rU;
            zU[t] = P.zU;
            r.st = b->states + t;
            r.partials = parts[t];
        }
        ck(batch_dct_setup(b->dct, H, W, T, o.precision, fold, o.tau, o.flexible_cg,
                           b->mem + dct_off,
                           rU.data(), zU.data(), b->ld.data(), b->states, parts.data()));
        int sblk = 0, vblk = 0, ublk = 0;
        for (int t = 0; t < T; ++t) {
            TileRec& r = b->recs[t];
            StencilArgs& a = r.a;
            a = StencilArgs{};
            a.H = H[t]; a.W = W[t]; a.ld = b->ld[t];
            a.tau = o.tau; a.inv_tau = 1.0f / o.tau; a.delta = o.delta;
            a.tol2 = (double)o.cg_tol * (double)o.cg_tol;
            a.cg_max = o.cg_max_iter;
            a.cap_warn = 1;
            a.flexible = o.flexible_cg;
            a.warm_start = o.warm_start;
            a.prec = o.precision;
            a.rw_rows = aux_rows(2, H[t], W[t]);
            a.fin_rows = aux_rows(3, H[t], W[t]);
            // the direct form reads the update kernel's bf16 copy of r_U; the folded form folds
            // r_U itself
            if (!fold) {
                a.r16 = b->dct.r16[t];
                a.r16lo = b->dct.split ? b->dct.r16lo[t] : nullptr;
                a.ld16 = b->dct.ld16[t];
            }
            strip_dims(H[t], W[t], r.sgx, r.sgy);
            r.sblk0 = sblk;
            sblk += r.sgx * r.sgy;
        }
        b->total_strip = sblk;
        layout_vec_blocks(b);
        ck(cudaMemcpy(b->d_recs, b->recs.data(), (size_t)T * sizeof(TileRec), cudaMemcpyHostToDevice));
        ck(cudaHostAlloc(&b->h_count, 2 * sizeof(int), cudaHostAllocDefault));
        for (auto& e : b->ev) ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ck(cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming));
        ck(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        ck(cudaDeviceSynchronize());
    } catch (Fail&) {
        destroy_batch(b);
        return IRLS_ERR_CUDA;
    }
    *out = b;
    return IRLS_OK;
}

int irls_batch_destroy(irls_batch b) {
    destroy_batch(b);
    return IRLS_OK;
}

int irls_batch_dct_form(irls_batch b) {
    if (!b) return IRLS_ERR_ARG;
    return b->dct.fold ? IRLS_DCT_FOLDED : IRLS_DCT_DIRECT;
}

int irls_batch_set_tiles(irls_batch b, int dir_rows, int upd_rows) {
    if (!b) return IRLS_ERR_ARG;
    if ((dir_rows != 0 && !tile_rows_ok(dir_rows)) || (upd_rows != 0 && !tile_rows_ok(upd_rows)))
        return IRLS_ERR_ARG;
    const int d = dir_rows ? dir_rows : b->dir_rows, u = upd_rows ? upd_rows : b->upd_rows;
    if (d == b->dir_rows && u == b->upd_rows) return IRLS_OK;
    try {
        DeviceGuard g(b->dev);
        ck(cudaStreamSynchronize(b->stream));
        b->dir_rows = d;
        b->upd_rows = u;
        layout_vec_blocks(b);
        ck(cudaMemcpy(b->d_recs, b->recs.data(), (size_t)b->T * sizeof(TileRec),
                      cudaMemcpyHostToDevice));
        drop_graphs(b);
    } catch (Fail&) {
        return IRLS_ERR_CUDA;
    }
    return IRLS_OK;
}

int irls_batch_get_tiles(irls_batch b, int* dir_rows, int* upd_rows) {
    if (!b || !dir_rows || !upd_rows) return IRLS_ERR_ARG;
    *dir_rows = b->dir_rows;
    *upd_rows = b->upd_rows;
    return IRLS_OK;
}

int irls_batch_autotune(irls_batch b, float* h_ms, void* stream) {
    if (!b) return IRLS_ERR_ARG;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = IRLS_OK;
    try {
        DeviceGuard g(b->dev);
        cudaStream_t s = b->stream;
        ck(cudaEventRecord(b->join, static_cast<cudaStream_t>(stream)));
        ck(cudaStreamWaitEvent(s, b->join, 0));
        ck(cudaEventCreate(&e0));
        ck(cudaEventCreate(&e1));
        constexpr int kWarm = 2, kReps = 10;
        float ms[2][4];
        const int d0 = b->dir_rows, u0 = b->upd_rows;
        for (int k = 0; k < 2; ++k)
            for (int i = 0; i < 4; ++i) {
                b->dir_rows = k == 0 ? kTileRows[i] : d0;
                b->upd_rows = k == 1 ? kTileRows[i] : u0;
                layout_vec_blocks(b);
                ck(cudaMemcpyAsync(b->d_recs, b->recs.data(), (size_t)b->T * sizeof(TileRec),
                                   cudaMemcpyHostToDevice, s));
                float tot = 0.f;
                for (int r = 0; r < kWarm + kReps; ++r) {
                    // fresh states per launch (a stopped image's blocks return at once)
                    ck(cudaMemsetAsync(b->states, 0, (size_t)b->T * sizeof(DevState), s));
                    ck(cudaEventRecord(e0, s));
                    if (k == 0)
                        ck(launch_direction_batched(b->d_recs, b->T, b->total_vec, b->dir_rows, s));
                    else
                        ck(launch_update_batched(b->d_recs, b->T, b->total_upd, b->upd_rows, s));
                    ck(cudaEventRecord(e1, s));
                    ck(cudaEventSynchronize(e1));
                    float t = 0.f;
                    ck(cudaEventElapsedTime(&t, e0, e1));
                    if (r >= kWarm) tot += t;
                }
                ms[k][i] = tot / kReps;
            }
        int bd = 0, bu = 0;
        for (int i = 1; i < 4; ++i) {
            if (ms[0][i] < ms[0][bd]) bd = i;
            if (ms[1][i] < ms[1][bu]) bu = i;
        }
        b->dir_rows = kTileRows[bd];
        b->upd_rows = kTileRows[bu];
        layout_vec_blocks(b);
        ck(cudaMemcpyAsync(b->d_recs, b->recs.data(), (size_t)b->T * sizeof(TileRec),
                           cudaMemcpyHostToDevice, s));
        ck(cudaMemsetAsync(b->states, 0, (size_t)b->T * sizeof(DevState), s));
        ck(cudaStreamSynchronize(s));
        drop_graphs(b);
        if (h_ms)
            for (int k = 0; k < 2; ++k)
                for (int i = 0; i < 4; ++i) h_ms[4 * k + i] = ms[k][i];
    } catch (Fail&) {
        rc = IRLS_ERR_CUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

int irls_batch_uses_graphs(irls_batch b) {
    if (!b) return IRLS_ERR_ARG;
    return (b->chunk[0] && b->chunk[1]) ? 1 : 0;
}

int irls_unwrap_batched_ex(irls_batch b, const float* const* X, const float* const* coh,
                           float* const* U, irls_stats* per_tile, void* stream) {
    if (!b || !X || !U) return IRLS_ERR_ARG;
    for (int t = 0; t < b->T; ++t)
        if (!X[t] || !U[t]) return IRLS_ERR_ARG;
    int status = 0;
    try {
        DeviceGuard g(b->dev);
        status = run_batch(b, X, coh, U, per_tile, static_cast<cudaStream_t>(stream));
        if (status & ST_NONFINITE) return IRLS_ERR_NONFINITE;
        // the caller's stream waits for the batch
        ck(cudaEventRecord(b->join, b->stream));
        ck(cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), b->join, 0));
    } catch (Fail&) {
        return IRLS_ERR_CUDA;
    }
    return status_to_code(status);
}

int irls_unwrap_batched(int ntiles, const int* H, const int* W, const float* const* X,
                        const float* const* coh, float* const* U, const irls_opts* opts,
                        irls_stats* per_tile, void* stream) {
    irls_batch b = nullptr;
    int rc = irls_batch_create(ntiles, H, W, opts, &b);
    if (rc != IRLS_OK) return rc;
    rc = irls_unwrap_batched_ex(b, X, coh, U, per_tile, stream);
    irls_batch_destroy(b);
    return rc;
}

int irls_precond_laplacian(irls_plan p, const float* R, float* Z, void* stream) {
    if (!p || !R || !Z) return IRLS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    try {
        DeviceGuard g(p->dev);
        StencilArgs a = make_args(p);
        ck(cudaMemsetAsync(p->P.rU, 0, p->L.plane_bytes, s));
        ck(launch_copy_in(R, p->H, p->W, p->P.rU, p->ld, s));
        if (a.r16) ck(launch_emit16(p->P.rU, p->H, p->W, p->ld, a.r16, a.r16lo, a.ld16, s));
        // the float16 form scales its input by ||r_U||, which no solve kernel produced here
        if (p->opts.precision == IRLS_PREC_FP16)
            ck(launch_norm_u(p->P, a, p->st, p->partials, s));
        ck(dct_reset(p->dct, s));
        ck(dct_apply(p->dct, p->P.rU, p->P.zU, p->ld, p->st, 0, a, p->partials, 0, s));
        ck(launch_copy_out(p->P.zU, p->H, p->W, p->ld, Z, s));
    } catch (Fail&) {
        return IRLS_ERR_CUDA;
    }
    return IRLS_OK;
}

int irls_round_congruent(irls_plan p, const float* U, const float* X, float* Ur, int* K,
                         double* offset, void* stream) {
    if (!p || !U || !X) return IRLS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    try {
        DeviceGuard g(p->dev);
        const size_t n = (size_t)p->H * p->W;
        ck(cudaMemsetAsync(&p->st->counter, 0, sizeof(unsigned int), s));
        ck(launch_round_congruent(U, X, n, p->st, p->partials, p->L.max_blocks, Ur, K, s));
        double h = 0.0;
        ck(cudaMemcpyAsync(p->h_pair, &p->st->aux[0], sizeof(double), cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        h = p->h_pair[0];
        if (offset) *offset = h;
    } catch (Fail&) {
        return IRLS_ERR_CUDA;
    }
    return IRLS_OK;
}

int irls_best_shift_error(irls_plan p, const float* U, const float* Xu, float* E, double* alpha,
                          double* rms, void* stream) {
    if (!p || !U || !Xu) return IRLS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    try {
        DeviceGuard g(p->dev);
        const size_t n = (size_t)p->H * p->W;
        ck(cudaMemsetAsync(&p->st->counter, 0, sizeof(unsigned int), s));
        ck(launch_best_shift(U, Xu, n, p->st, p->partials, p->L.max_blocks, E, s));
        ck(cudaMemcpyAsync(p->h_pair, &p->st->aux[1], 2 * sizeof(double), cudaMemcpyDeviceToHost,
                           s));
        ck(cudaStreamSynchronize(s));
        if (alpha) *alpha = p->h_pair[0];
        if (rms) *rms = std::sqrt(p->h_pair[1] / (double)n);
    } catch (Fail&) {
        return IRLS_ERR_CUDA;
    }
    return IRLS_OK;
}

int irls_apply_A(irls_plan p, const float* U, const float* Vv, const float* Vh, const float* Dv,
                 const float* Dh, float* qU, float* qVv, float* qVh, void* stream) {
    if (!p || !U || !qU) return IRLS_ERR_ARG;
    if (p->H > 1 && (!Vv || !Dv || !qVv)) return IRLS_ERR_ARG;
    if (p->W > 1 && (!Vh || !Dh || !qVh)) return IRLS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    try {
        DeviceGuard g(p->dev);
        StencilArgs a = make_args(p);
        const Planes& P = p->P;
        const size_t pb = p->L.plane_bytes;
        float* zero[] = {P.U, P.Vv, P.Vh, P.rU, P.rVv, P.rVh, P.pU[0], P.pVv[0], P.pVh[0], P.dv, P.dh};
        for (float* z : zero) ck(cudaMemsetAsync(z, 0, pb, s));
        ck(launch_copy_in(U, p->H, p->W, P.pU[0], p->ld, s));
        if (p->H > 1) {
            ck(launch_copy_in(Vv, p->H - 1, p->W, P.pVv[0], p->ld, s));
            ck(launch_copy_in(Dv, p->H - 1, p->W, P.dv, p->ld, s));
        }
        if (p->W > 1) {
            ck(launch_copy_in(Vh, p->H, p->W - 1, P.pVh[0], p->ld, s));
            ck(launch_copy_in(Dh, p->H, p->W - 1, P.dh, p->ld, s));
        }
        ck(launch_matvec_via_update(P, a, p->st, p->partials, s));
        ck(launch_copy_out(P.rU, p->H, p->W, p->ld, qU, s));
        if (p->H > 1) ck(launch_copy_out(P.rVv, p->H - 1, p->W, p->ld, qVv, s));
        if (p->W > 1) ck(launch_copy_out(P.rVh, p->H, p->W - 1, p->ld, qVh, s));
    } catch (Fail&) {
        return IRLS_ERR_CUDA;
    }
    return IRLS_OK;
}

int irls_plan_set_profiling(irls_plan p, int on) {
    if (!p) return IRLS_ERR_ARG;
    p->prof.on = on != 0;
    p->prof.reset();
    return IRLS_OK;
}

int irls_plan_profile(irls_plan p, double* ms, long long* launches, int n) {
    if (!p || n < 0 || (n > 0 && (!ms || !launches))) return IRLS_ERR_ARG;
    for (int i = 0; i < n && i < PC_N; ++i) {
        ms[i] = p->prof.ms[i];
        launches[i] = p->prof.n[i];
    }
    return PC_N;
}

const char* irls_status_string(int status) {
    switch (status) {
        case IRLS_OK: return "ok";
        case IRLS_WARN_CG_MAX: return "warning: CG stopped on cg_max_iter before reaching cg_tol";
        case IRLS_ERR_ARG: return "invalid argument";
        case IRLS_ERR_SHAPE: return "invalid shape";
        case IRLS_ERR_NONFINITE: return "non-finite input";
        case IRLS_ERR_OOM: return "device out of memory";
        case IRLS_ERR_BREAKDOWN: return "CG breakdown (non-positive curvature or rho)";
        case IRLS_ERR_TIMEOUT: return "device-side wait timed out";
        case IRLS_ERR_CUDA: return "CUDA runtime error";
        case IRLS_ERR_UNSUPPORTED: return "unsupported option";
        default: return "unknown status";
    }
}

int irls_last_cuda_error(void) { return g_last_cuda; }

}  // extern "C"
