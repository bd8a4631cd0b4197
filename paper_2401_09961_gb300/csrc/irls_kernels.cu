// Stencil kernels of the IRLS / PCG path (Alg. 1, Alg. 2 of arXiv 2401.09961).
//
// Every kernel walks the image in strips: a block of 128 threads owns 128 consecutive columns
// and kRows consecutive rows; each thread owns one column and marches down its rows, keeping
// the previous / next row in registers.  Horizontal neighbours come from warp shuffles, and
// the two columns beyond a warp's edge are read directly by its edge lanes.  Loads and stores
// of a warp are 128-byte rows, so every plane is read or written once per pass.
//
// The edge quantities used throughout are the rows of B x (proof of the existence theorem,
// Sec. 3.1):  y_v = S p_U - p_Vv  and  y_h = p_U T - p_Vh.  With them
//     A p = ( (S^T y_v + y_h T^T) / tau ,  D_v p_Vv - y_v / tau ,  D_h p_Vh - y_h / tau )
// (eq. 'matrix-soft-constraints'), and p^T A p = sum (y_v^2 + y_h^2) / tau + D p_V^2.
#include <algorithm>

#include "irls_internal.cuh"
#include "reduce.cuh"

namespace irls {

namespace {

constexpr int kThreads = 128;
constexpr int kRows = 16;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool finite(float x) { return isfinite(x); }

// Wrapped phase difference in [-pi, pi), one correctly rounded float32 operation at a time
// (Sec. 2, "mod 2 pi"): k = floor((t + pi) / 2pi), result = t - (2pi * k).
__device__ __forceinline__ float wrap_pi(float t) {
    const float kPi = 3.14159265358979323846f;
    const float kTwoPi = 6.28318530717958647692f;
    float k = floorf(__fdiv_rn(__fadd_rn(t, kPi), kTwoPi));
    return __fsub_rn(t, __fmul_rn(kTwoPi, k));
}

__device__ __forceinline__ int strip_rows(int H, int i0) { return min(i0 + kRows, H); }

// ------------------------------------------------------------------------------------------
// Wrapped gradients, edge weights and the starting iterate (Sec. 2; Alg. 1 initialisation)
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_init(const float* __restrict__ X, const float* __restrict__ coh, const float* __restrict__ Cv_in,
       const float* __restrict__ Ch_in, const float* __restrict__ U0, const float* __restrict__ Vv0,
       const float* __restrict__ Vh0, Planes P, StencilArgs a, DevState* st) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    int bad = 0;
    if (j < W) {
        for (int i = i0; i < i1; ++i) {
            const size_t o = (size_t)i * ld + j;
            const bool hv = i + 1 < H, hh = j + 1 < W;
            const float x = X[(size_t)i * W + j];
            bad |= !finite(x);
            float gv = 0.f, gh = 0.f;
            if (hv) gv = wrap_pi(__fsub_rn(X[(size_t)(i + 1) * W + j], x));
            if (hh) gh = wrap_pi(__fsub_rn(X[(size_t)i * W + j + 1], x));
            float cv = 0.f, ch = 0.f;
            if (Cv_in != nullptr && Ch_in != nullptr) {
                if (hv) cv = Cv_in[(size_t)i * W + j];
                if (hh) ch = Ch_in[(size_t)i * (W - 1) + j];
            } else if (coh != nullptr) {
                const float c0 = coh[(size_t)i * W + j];
                bad |= !finite(c0);
                if (hv) cv = 0.5f * (c0 + coh[(size_t)(i + 1) * W + j]);
                if (hh) ch = 0.5f * (c0 + coh[(size_t)i * W + j + 1]);
            } else {
                cv = hv ? 1.f : 0.f;
                ch = hh ? 1.f : 0.f;
            }
            bad |= !finite(cv) | !finite(ch) | (cv < 0.f) | (ch < 0.f);
            P.Gv[o] = gv; P.Gh[o] = gh; P.Cv[o] = cv; P.Ch[o] = ch;
            if (U0 != nullptr) {
                const float u = U0[(size_t)i * W + j];
                const float vv = hv ? Vv0[(size_t)i * W + j] : 0.f;
                const float vh = hh ? Vh0[(size_t)i * (W - 1) + j] : 0.f;
                bad |= !finite(u) | !finite(vv) | !finite(vh);
                P.U[o] = u; P.Vv[o] = vv; P.Vh[o] = vh;
            } else {
                P.U[o] = 0.f; P.Vv[o] = -gv; P.Vh[o] = -gh;     // V^0 = S U^0 - G with U^0 = 0
            }
        }
    }
    if (bad) atomicOr(&st->status, ST_NONFINITE);
}

// ||b||^2 with b = ((S^T Gv + Gh T^T)/tau, -Gv/tau, -Gh/tau)  (Sec. 3.2, definition of B1..B3)
__global__ void __launch_bounds__(kThreads)
k_bnorm(Planes P, StencilArgs a, DevState* st, double* partials) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    float acc = 0.f;
    if (j < W) {
        for (int i = i0; i < i1; ++i) {
            const size_t o = (size_t)i * ld + j;
            const float gv = P.Gv[o], gh = P.Gh[o];
            const float gv_up = i > 0 ? P.Gv[o - ld] : 0.f;
            const float gh_l = j > 0 ? P.Gh[o - 1] : 0.f;
            const float bu = a.inv_tau * (gv_up - gv + gh_l - gh);
            acc += bu * bu + a.inv_tau * a.inv_tau * (gv * gv + gh * gh);
        }
    }
    double v[1] = {(double)acc}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) st->bb = tot[0];
}

// ------------------------------------------------------------------------------------------
// Start of an outer step: reweighting (Alg. 1, closed form W = sqrt(C^2 V^2 + delta^2)),
// D = C^2 / W, and the initial CG residual r = b - A x of the warm start (Alg. 2).
//   with e_v = S U - Vv - Gv and e_h = U T - Vh - Gh:
//   r_U = -(S^T e_v + e_h T^T) / tau,   r_V = e / tau - D o V.
// A cold start (warm_start = 0) uses x = 0, i.e. r = b, and zeroes the iterate.
// Also F_delta(x^k) = sum W + ||e||^2 / (2 tau)  (= H_delta(x^k, W^k)).
// ------------------------------------------------------------------------------------------
// bfloat16 copy of r_U for the tensor-core preconditioner; with a lo plane the value is split
// as hi = bf16(v), lo = bf16(v - hi) (split precision).
__device__ __forceinline__ void emit16(void* r16, void* r16lo, int ld16, int i, int j, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    static_cast<__nv_bfloat16*>(r16)[(size_t)i * ld16 + j] = h;
    if (r16lo != nullptr)
        static_cast<__nv_bfloat16*>(r16lo)[(size_t)i * ld16 + j] =
            __float2bfloat16_rn(v - __bfloat162float(h));
}

__global__ void __launch_bounds__(kThreads)
k_reweight_residual(Planes P, StencilArgs a, DevState* st, double* partials) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    const bool col = j < W, hh = j + 1 < W;
    const float it = a.inv_tau, d2 = a.delta * a.delta;
    const bool warm = a.warm_start != 0;
    float rr = 0.f, rzv = 0.f, fd = 0.f, ru2 = 0.f;
    float uc = col ? P.U[(size_t)i0 * ld + j] : 0.f;
    float ev_prev = 0.f;          // residual-edge e_v of the row above
    if (col && i0 > 0) {
        const size_t o = (size_t)(i0 - 1) * ld + j;
        ev_prev = warm ? (uc - P.U[o] - P.Vv[o] - P.Gv[o]) : -P.Gv[o];
    }
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j;
        const bool hv = i + 1 < H;
        float vv = 0.f, vh = 0.f, cv = 0.f, ch = 0.f, gv = 0.f, gh = 0.f, un = 0.f;
        if (col) {
            vv = P.Vv[o]; vh = P.Vh[o]; cv = P.Cv[o]; ch = P.Ch[o]; gv = P.Gv[o]; gh = P.Gh[o];
            if (hv) un = P.U[o + ld];
        }
        float ur = __shfl_down_sync(kFull, uc, 1);
        if (lane == 31 && col && hh) ur = P.U[o + 1];
        // edge residuals at the iterate x^k
        const float evk = (col && hv) ? (un - uc - vv - gv) : 0.f;
        const float ehk = (col && hh) ? (ur - uc - vh - gh) : 0.f;
        // edge residuals of the CG starting point
        const float ev = warm ? evk : ((col && hv) ? -gv : 0.f);
        const float eh = warm ? ehk : ((col && hh) ? -gh : 0.f);
        float eh_l = __shfl_up_sync(kFull, eh, 1);
        if (lane == 0) {
            eh_l = 0.f;
            if (col && j > 0)
                eh_l = warm ? (uc - P.U[o - 1] - P.Vh[o - 1] - P.Gh[o - 1]) : -P.Gh[o - 1];
        }
        if (col) {
            float wv = 0.f, wh = 0.f, dv = 0.f, dh = 0.f;
            if (hv) { wv = sqrtf(cv * cv * vv * vv + d2); dv = cv * cv / wv; }
            if (hh) { wh = sqrtf(ch * ch * vh * vh + d2); dh = ch * ch / wh; }
            const float xvv = warm ? vv : 0.f, xvh = warm ? vh : 0.f;
            const float ru = -it * (ev_prev - ev + eh_l - eh);
            const float rv = it * ev - dv * xvv;
            const float rh = it * eh - dh * xvh;
            P.Wv[o] = wv; P.Wh[o] = wh; P.dv[o] = dv; P.dh[o] = dh;
            P.rU[o] = ru; P.rVv[o] = rv; P.rVh[o] = rh;
            if (!warm) { P.U[o] = 0.f; P.Vv[o] = 0.f; P.Vh[o] = 0.f; }
            if (a.r16 != nullptr) emit16(a.r16, a.r16lo, a.ld16, i, j, ru);
            rr += ru * ru + rv * rv + rh * rh;
            ru2 += ru * ru;
            rzv += rv * rv / (dv + it) + rh * rh / (dh + it);
            fd += wv + wh + 0.5f * it * (evk * evk + ehk * ehk);
        }
        ev_prev = ev;
        uc = un;
    }
    double v[4] = {(double)rr, (double)rzv, (double)fd, (double)ru2}, tot[4];
    if (grid_reduce<4>(v, partials, &st->counter, tot) && threadIdx.x == 0) {
        st->rr = tot[0];
        st->rz_v = tot[1];
        st->rnorm_u = sqrt(tot[3]);
        const double rel = st->bb > 0.0 ? sqrt(tot[0] / st->bb) : 0.0;
        st->rel = rel;
        st->iter = 0;
        st->p_fresh = 1;
        st->done = (rel * rel <= a.tol2 || a.cg_max <= 0 || st->bb <= 0.0) ? 1 : 0;
        const int k = st->outer;
        if (k < kMaxOuter) st->f_delta[k] = tot[2];
    }
}

// ------------------------------------------------------------------------------------------
// Search direction and curvature (Alg. 2): p_new = z + beta p_old with z_U from the Laplacian
// block and z_V = r_V / (D + 1/tau) (the diagonal blocks of the preconditioner, Sec. 3.3);
// p^T A p = sum (y_v^2 + y_h^2) / tau + D p_V^2; alpha = rho / p^T A p.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_direction_pap(Planes P, StencilArgs a, DevState* st, double* partials) {
    if (st->done) return;
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    const bool col = j < W, hh = j + 1 < W;
    const float it = a.inv_tau;
    const int cur = st->pbuf, nxt = cur ^ 1;
    const bool fresh = st->p_fresh != 0;
    const float beta = fresh ? 0.f : (float)st->beta;
    const float* __restrict__ pUo = P.pU[cur];
    const float* __restrict__ pVvo = P.pVv[cur];
    const float* __restrict__ pVho = P.pVh[cur];
    float* __restrict__ pUn = P.pU[nxt];
    float* __restrict__ pVvn = P.pVv[nxt];
    float* __restrict__ pVhn = P.pVh[nxt];
    const float* __restrict__ zU = P.zU;

    float cu = 0.f, cvv = 0.f, cvh = 0.f, cdv = 0.f, cdh = 0.f;
    if (col) {
        const size_t o = (size_t)i0 * ld + j;
        cu = fresh ? zU[o] : zU[o] + beta * pUo[o];
        cdv = P.dv[o]; cdh = P.dh[o];
        cvv = P.rVv[o] / (cdv + it);
        cvh = P.rVh[o] / (cdh + it);
        if (!fresh) { cvv += beta * pVvo[o]; cvh += beta * pVho[o]; }
    }
    float acc = 0.f;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j;
        const bool hv = i + 1 < H;
        float nu = 0.f, nvv = 0.f, nvh = 0.f, ndv = 0.f, ndh = 0.f;
        if (col && hv) {
            const size_t on = o + ld;
            nu = fresh ? zU[on] : zU[on] + beta * pUo[on];
            if (i + 1 < i1) {
                ndv = P.dv[on]; ndh = P.dh[on];
                nvv = P.rVv[on] / (ndv + it);
                nvh = P.rVh[on] / (ndh + it);
                if (!fresh) { nvv += beta * pVvo[on]; nvh += beta * pVho[on]; }
            }
        }
        float ur = __shfl_down_sync(kFull, cu, 1);
        if (lane == 31 && col && hh) ur = fresh ? zU[o + 1] : zU[o + 1] + beta * pUo[o + 1];
        if (col) {
            pUn[o] = cu; pVvn[o] = cvv; pVhn[o] = cvh;
            const float yh = hh ? (ur - cu - cvh) : 0.f;
            const float yv = hv ? (nu - cu - cvv) : 0.f;
            acc += it * (yh * yh + yv * yv) + cdv * cvv * cvv + cdh * cvh * cvh;
        }
        cu = nu; cvv = nvv; cvh = nvh; cdv = ndv; cdh = ndh;
    }
    double v[1] = {(double)acc}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot) && threadIdx.x == 0) {
        const double pq = tot[0];
        st->pq = pq;
        st->pbuf = nxt;
        st->p_fresh = 0;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->alpha = 0.0;
            if (st->rr > 0.0) st->status |= ST_BREAKDOWN;
            st->done = 1;
        } else {
            st->alpha = st->rho / pq;
        }
    }
}

// ------------------------------------------------------------------------------------------
// CG update (Alg. 2): x += alpha p, r -= alpha A p with A p recomputed from p (the stencil of
// eq. 'matrix-soft-constraints'), then ||r||^2, r_V^T z_V (z_V = r_V / (D + 1/tau)) and, for the
// flexible variant, r_new^T z_old.  Stops the run when ||r|| <= cg_tol ||b|| or on cg_max.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_update(Planes P, StencilArgs a, DevState* st, double* partials) {
    if (st->done) return;
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    const bool col = j < W, hh = j + 1 < W;
    const float it = a.inv_tau;
    const int cur = st->pbuf;
    const float alpha = (float)st->alpha;
    const bool flex = a.flexible != 0;
    const float* __restrict__ pU = P.pU[cur];
    const float* __restrict__ pVv = P.pVv[cur];
    const float* __restrict__ pVh = P.pVh[cur];

    float cu = 0.f, cvv = 0.f, cvh = 0.f, yv_prev = 0.f;
    if (col) {
        const size_t o = (size_t)i0 * ld + j;
        cu = pU[o]; cvv = pVv[o]; cvh = pVh[o];
        if (i0 > 0) yv_prev = cu - pU[o - ld] - pVv[o - ld];
    }
    float rr = 0.f, rzv = 0.f, rzo = 0.f, ru2 = 0.f;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j;
        const bool hv = i + 1 < H;
        float nu = 0.f, nvv = 0.f, nvh = 0.f;
        if (col && hv) {
            nu = pU[o + ld];
            if (i + 1 < i1) { nvv = pVv[o + ld]; nvh = pVh[o + ld]; }
        }
        const float yv = (col && hv) ? (nu - cu - cvv) : 0.f;
        float ur = __shfl_down_sync(kFull, cu, 1);
        if (lane == 31 && col && hh) ur = pU[o + 1];
        const float yh = (col && hh) ? (ur - cu - cvh) : 0.f;
        float yh_l = __shfl_up_sync(kFull, yh, 1);
        if (lane == 0) yh_l = (col && j > 0) ? (cu - pU[o - 1] - pVh[o - 1]) : 0.f;
        if (col) {
            const float dv = P.dv[o], dh = P.dh[o];
            const float qu = it * (yv_prev - yv + yh_l - yh);
            const float qv = dv * cvv - it * yv;
            const float qh = dh * cvh - it * yh;
            P.U[o] += alpha * cu;
            P.Vv[o] += alpha * cvv;
            P.Vh[o] += alpha * cvh;
            const float ru0 = P.rU[o], rv0 = P.rVv[o], rh0 = P.rVh[o];
            const float ru = ru0 - alpha * qu, rv = rv0 - alpha * qv, rh = rh0 - alpha * qh;
            P.rU[o] = ru; P.rVv[o] = rv; P.rVh[o] = rh;
            const float iv = 1.f / (dv + it), ih = 1.f / (dh + it);
            rr += ru * ru + rv * rv + rh * rh;
            ru2 += ru * ru;
            rzv += rv * rv * iv + rh * rh * ih;
            if (flex) rzo += ru * P.zU[o] + (rv * rv0) * iv + (rh * rh0) * ih;
            if (a.r16 != nullptr) emit16(a.r16, a.r16lo, a.ld16, i, j, ru);
        }
        yv_prev = yv;
        cu = nu; cvv = nvv; cvh = nvh;
    }
    double v[4] = {(double)rr, (double)rzv, (double)rzo, (double)ru2}, tot[4];
    if (grid_reduce<4>(v, partials, &st->counter, tot) && threadIdx.x == 0) {
        st->rr = tot[0];
        st->rz_v = tot[1];
        st->rz_old = tot[2];
        st->rnorm_u = sqrt(tot[3]);
        const int itn = st->iter + 1;
        st->iter = itn;
        const double rel = st->bb > 0.0 ? sqrt(tot[0] / st->bb) : 0.0;
        st->rel = rel;
        if (rel * rel <= a.tol2 || itn >= a.cg_max || !isfinite(rel)) st->done = 1;
        if (!isfinite(rel)) st->status |= ST_NONFINITE;
    }
}

// ------------------------------------------------------------------------------------------
// End of an outer step: sum U (for U -= mean(U), Prop. 'minimising (alt1)'), the objective of
// problem (main) and H_delta(x^{k+1}, W^k) of problem (alt1); then record the statistics.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_finalize_reduce(Planes P, StencilArgs a, DevState* st, double* partials) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    const double it = 1.0 / (double)a.tau, d2 = (double)a.delta * (double)a.delta;
    // FP64 evaluation: the difference of two float32 values is exact in double, so the edge
    // residuals of the objective carry no cancellation error of their own
    double su = 0.0, l1 = 0.0, hd = 0.0;
    if (j < W) {
        for (int i = i0; i < i1; ++i) {
            const size_t o = (size_t)i * ld + j;
            const double u = P.U[o];
            su += u;
            if (i + 1 < H) {
                const double e = ((double)P.U[o + ld] - u) - (double)P.Gv[o];
                const double c = P.Cv[o], v = P.Vv[o], w = P.Wv[o];
                l1 += c * fabs(e);
                const double pe = e - v;
                hd += 0.5 * ((c * c * v * v + d2) / w + w) + 0.5 * it * pe * pe;
            }
            if (j + 1 < W) {
                const double e = ((double)P.U[o + 1] - u) - (double)P.Gh[o];
                const double c = P.Ch[o], v = P.Vh[o], w = P.Wh[o];
                l1 += c * fabs(e);
                const double pe = e - v;
                hd += 0.5 * ((c * c * v * v + d2) / w + w) + 0.5 * it * pe * pe;
            }
        }
    }
    double v[3] = {su, l1, hd}, tot[3];
    if (grid_reduce<3>(v, partials, &st->counter, tot) && threadIdx.x == 0) {
        st->mean_u = tot[0] / ((double)H * (double)W);
        const int k = st->outer;
        if (k < kMaxOuter) {
            st->l1_obj[k] = tot[1];
            st->h_delta[k] = tot[2];
            st->cg_iters[k] = st->iter;
            st->rel_res[k] = st->rel;
        }
        st->cg_total += st->iter;
        if (st->iter >= a.cg_max && st->rel * st->rel > a.tol2) st->status |= ST_CGMAX;
        st->outer = k + 1;
    }
}

__global__ void __launch_bounds__(kThreads)
k_subtract_mean(float* U, int H, int W, int ld, const DevState* st) {
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    if (j >= W) return;
    const float m = (float)st->mean_u;
    for (int i = i0; i < i1; ++i) U[(size_t)i * ld + j] -= m;
}

__global__ void k_copy_out(const float* __restrict__ src, int rows, int cols, int ld,
                           float* __restrict__ dst) {
    const size_t n = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t r = t / cols, c = t % cols;
        dst[t] = src[r * ld + c];
    }
}

__global__ void k_copy_in(const float* __restrict__ src, int rows, int cols,
                          float* __restrict__ dst, int ld) {
    const size_t n = (size_t)rows * cols;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x) {
        const size_t r = t / cols, c = t % cols;
        dst[r * ld + c] = src[t];
    }
}

__global__ void k_emit16(const float* __restrict__ src, int H, int W, int ld, void* r16, void* r16lo,
                         int ld16) {
    const size_t n = (size_t)H * W;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
         t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / W), j = (int)(t % W);
        emit16(r16, r16lo, ld16, i, j, src[(size_t)i * ld + j]);
    }
}

__global__ void k_prepare_matvec(DevState* st) {
    st->done = 0;
    st->iter = 0;
    st->alpha = -1.0;
    st->pbuf = 0;
    st->bb = 1.0;
}

dim3 strip_grid(int H, int W) { return dim3((W + kThreads - 1) / kThreads, (H + kRows - 1) / kRows); }

}  // namespace

int stencil_grid_blocks(int H, int W) {
    dim3 g = strip_grid(H, W);
    return (int)(g.x * g.y);
}

cudaError_t launch_init(const float* X, const float* coh, const float* Cv_in, const float* Ch_in,
                        const float* U0, const float* Vv0, const float* Vh0, const Planes& P,
                        const StencilArgs& a, DevState* st, double* partials, cudaStream_t s) {
    (void)partials;
    k_init<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(X, coh, Cv_in, Ch_in, U0, Vv0, Vh0, P, a, st);
    return cudaGetLastError();
}

cudaError_t launch_bnorm(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                         cudaStream_t s) {
    k_bnorm<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_reweight_residual(const Planes& P, const StencilArgs& a, DevState* st,
                                     double* partials, cudaStream_t s) {
    k_reweight_residual<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_direction_pap(const Planes& P, const StencilArgs& a, DevState* st,
                                 double* partials, cudaStream_t s) {
    k_direction_pap<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_update(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                          cudaStream_t s) {
    k_update<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                            cudaStream_t s) {
    k_finalize_reduce<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, st, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_subtract_mean<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P.U, a.H, a.W, a.ld, st);
    return cudaGetLastError();
}

cudaError_t launch_copy_out(const float* src, int rows, int cols, int ld, float* dst,
                            cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const size_t n = (size_t)rows * cols;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 8192);
    k_copy_out<<<blocks, 256, 0, s>>>(src, rows, cols, ld, dst);
    return cudaGetLastError();
}

cudaError_t launch_copy_in(const float* src, int rows, int cols, float* dst, int ld,
                           cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    const size_t n = (size_t)rows * cols;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 8192);
    k_copy_in<<<blocks, 256, 0, s>>>(src, rows, cols, dst, ld);
    return cudaGetLastError();
}

cudaError_t launch_emit16(const float* src, int H, int W, int ld, void* r16, void* r16lo, int ld16,
                         cudaStream_t s) {
    const size_t n = (size_t)H * W;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 8192);
    k_emit16<<<blocks, 256, 0, s>>>(src, H, W, ld, r16, r16lo, ld16);
    return cudaGetLastError();
}

cudaError_t launch_matvec_via_update(const Planes& P, const StencilArgs& a, DevState* st,
                                     double* partials, cudaStream_t s) {
    k_prepare_matvec<<<1, 1, 0, s>>>(st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    StencilArgs b = a;
    b.flexible = 0;
    b.r16 = nullptr;
    b.r16lo = nullptr;
    b.cg_max = 1 << 30;
    b.tol2 = -1.0;
    k_update<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, b, st, partials);
    return cudaGetLastError();
}

}  // namespace irls
