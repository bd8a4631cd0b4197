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
constexpr double kBreakdownRel = 1e-3;

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

// ||r||^2 without the mean of r_U: in exact arithmetic r stays in the range of A (App. B), which
// excludes constant U; the constant that float32 rounding of the telescoping sums adds to r_U is
// invisible to the preconditioner (its zero-frequency coefficient is dropped) and to A, so it is
// left out of the stopping test.
__device__ __forceinline__ double range_part(double rr, double sum_ru, int H, int W) {
    const double n = (double)H * (double)W;
    return fmax(rr - sum_ru * sum_ru / n, 0.0);
}

// ------------------------------------------------------------------------------------------
// Wrapped gradients, edge weights and the starting iterate (Sec. 2; Alg. 1 initialisation)
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void k_init_body(const float* __restrict__ X, const float* __restrict__ coh, const float* __restrict__ Cv_in,
       const float* __restrict__ Ch_in, const float* __restrict__ U0, const float* __restrict__ Vv0,
       const float* __restrict__ Vh0, Planes P, StencilArgs a, DevState* st, const Blk& blk) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blk.bx * kThreads + threadIdx.x;
    const int i0 = blk.by * kRows, i1 = strip_rows(H, i0);
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

__global__ void __launch_bounds__(kThreads)
k_init(const float* __restrict__ X, const float* __restrict__ coh, const float* __restrict__ Cv_in,
       const float* __restrict__ Ch_in, const float* __restrict__ U0, const float* __restrict__ Vv0,
       const float* __restrict__ Vh0, Planes P, StencilArgs a, DevState* st) {
    k_init_body(X, coh, Cv_in, Ch_in, U0, Vv0, Vh0, P, a, st, single_blk());
}

// ||b||^2 with b = ((S^T Gv + Gh T^T)/tau, -Gv/tau, -Gh/tau)  (Sec. 3.2, definition of B1..B3)
__device__ __forceinline__ void k_bnorm_body(Planes P, StencilArgs a, DevState* st, double* partials, const Blk& blk) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blk.bx * kThreads + threadIdx.x;
    const int i0 = blk.by * kRows, i1 = strip_rows(H, i0);
    CSum acc;
    if (j < W) {
        for (int i = i0; i < i1; ++i) {
            const size_t o = (size_t)i * ld + j;
            const float gv = P.Gv[o], gh = P.Gh[o];
            const float gv_up = i > 0 ? P.Gv[o - ld] : 0.f;
            const float gh_l = j > 0 ? P.Gh[o - 1] : 0.f;
            const float bu = a.inv_tau * (gv_up - gv + gh_l - gh);
            acc.add(bu * bu + a.inv_tau * a.inv_tau * (gv * gv + gh * gh));
        }
    }
    double v[1] = {acc.value()}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) st->bb = tot[0];
}

__global__ void __launch_bounds__(kThreads)
k_bnorm(Planes P, StencilArgs a, DevState* st, double* partials) {
    k_bnorm_body(P, a, st, partials, single_blk());
}

// ||r_U|| of the residual plane (deterministic grid reduction) into the state: the norm the
// float16 preconditioner scales its input by, for a residual no solve kernel has produced.
__global__ void __launch_bounds__(kThreads)
k_norm_u(Planes P, StencilArgs a, DevState* st, double* partials) {
    const Blk blk = single_blk();
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blk.bx * kThreads + threadIdx.x;
    const int i0 = blk.by * kRows, i1 = strip_rows(H, i0);
    CSum acc;
    if (j < W)
        for (int i = i0; i < i1; ++i) {
            const float r = P.rU[(size_t)i * ld + j];
            acc.add(r * r);
        }
    double v[1] = {acc.value()}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0)
        st->rnorm_u = sqrt(tot[0]);
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

// ------------------------------------------------------------------------------------------
// The two per-iteration kernels work on float4 lanes: a thread owns 4 consecutive columns, a
// warp 128 and a block of 128 threads 512, so each warp moves 512-byte rows; the next row's
// loads are issued before the current row's stores (all plane pointers are __restrict__).
// Columns at or beyond W are zero in every plane; they are computed like the others (their
// values stay zero) and only the edge masks hh[] exclude the edges that do not exist.
// ------------------------------------------------------------------------------------------
constexpr int kVec = 4;
// rows per block of the float4-lane kernels, measured at 4096 x 4096 (16, 24 and 32 tried):
// direction 24, update 32; the U-only kernels 24
constexpr int kDirRows = kDefaultDirRows;
constexpr int kUpdRows = kDefaultUpdRows;
constexpr int kSchurRows = 24;

__device__ __forceinline__ void ld4(const float* __restrict__ p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void st4(float* __restrict__ p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}


// Start of an outer step (see the comment above emit16), on float4 lanes (the update kernel's
// columns per block, rows a.rw_rows): a thread owns four columns; the horizontal neighbour of its last column
// comes from the next lane (lane 31 loads it), the horizontal edge left of its first column from
// the previous lane (lane 0 recomputes it).  Padding columns (>= W) get no W, D or r.
template <int ROWS>
__device__ __forceinline__ void k_reweight_residual_body(Planes P, StencilArgs a, DevState* st,
                                                         double* partials, const Blk& blk) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j0 = (blk.bx * kThreads + threadIdx.x) * kVec;
    const int lane = threadIdx.x & 31;
    const int R = ROWS > 0 ? ROWS : a.rw_rows;   // 0: the row count of the launch's arguments
    const int i0 = blk.by * R, i1 = min(i0 + R, H);
    const bool act = j0 < W;
    const float it = a.inv_tau, d2 = a.delta * a.delta;
    const bool warm = a.warm_start != 0;
    // not __restrict__: a cold start zeroes the iterate through P in the same pass
    const float* U = P.U;
    const float* Vv = P.Vv;
    const float* Vh = P.Vh;
    const float* __restrict__ Gv = P.Gv;
    const float* __restrict__ Gh = P.Gh;
    bool col[kVec], hh[kVec];
#pragma unroll
    for (int e = 0; e < kVec; ++e) {
        col[e] = j0 + e < W;
        hh[e] = j0 + e + 1 < W;
    }
    CSum rr, rzv, fd, ru2, su;
    float uc[4] = {0, 0, 0, 0}, evp[4] = {0, 0, 0, 0};   // this row's U; e_v of the row above
    if (act) {
        ld4(U + (size_t)i0 * ld + j0, uc);
        if (i0 > 0) {
            const size_t o = (size_t)(i0 - 1) * ld + j0;
            float uu[4], vu[4], gu[4];
            ld4(U + o, uu); ld4(Vv + o, vu); ld4(Gv + o, gu);
#pragma unroll
            for (int e = 0; e < 4; ++e) evp[e] = warm ? (uc[e] - uu[e] - vu[e] - gu[e]) : -gu[e];
        }
    }
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j0;
        const bool hv = i + 1 < H;
        float vv[4] = {0, 0, 0, 0}, vh[4] = {0, 0, 0, 0}, cv[4] = {0, 0, 0, 0};
        float ch[4] = {0, 0, 0, 0}, gv[4] = {0, 0, 0, 0}, gh[4] = {0, 0, 0, 0};
        float un[4] = {0, 0, 0, 0};
        if (act) {
            ld4(Vv + o, vv); ld4(Vh + o, vh); ld4(P.Cv + o, cv); ld4(P.Ch + o, ch);
            ld4(Gv + o, gv); ld4(Gh + o, gh);
            if (hv) ld4(U + o + ld, un);
        }
        float ur = __shfl_down_sync(kFull, uc[0], 1);
        if (lane == 31) ur = (act && j0 + kVec < W) ? U[o + kVec] : 0.f;
        const float pr[4] = {uc[1], uc[2], uc[3], ur};
        // edge residuals at the iterate x^k, and of the CG starting point
        float evk[4], ehk[4], ev[4], eh[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            evk[e] = hv ? (un[e] - uc[e] - vv[e] - gv[e]) : 0.f;
            ehk[e] = hh[e] ? (pr[e] - uc[e] - vh[e] - gh[e]) : 0.f;
            ev[e] = warm ? evk[e] : (hv ? -gv[e] : 0.f);
            eh[e] = warm ? ehk[e] : (hh[e] ? -gh[e] : 0.f);
        }
        float ehl = __shfl_up_sync(kFull, eh[3], 1);
        if (lane == 0) {
            ehl = 0.f;
            if (act && j0 > 0)
                ehl = warm ? (uc[0] - U[o - 1] - Vh[o - 1] - Gh[o - 1]) : -Gh[o - 1];
        }
        const float el[4] = {ehl, eh[0], eh[1], eh[2]};
        if (act) {
            float wv[4], wh[4], dv[4], dh[4], ru[4], rv[4], rh[4];
            float prr = 0.f, pru2 = 0.f, psu = 0.f, przv = 0.f, pfd = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool ve = hv && col[e];
                wv[e] = ve ? sqrtf(cv[e] * cv[e] * vv[e] * vv[e] + d2) : 0.f;
                dv[e] = ve ? cv[e] * cv[e] / wv[e] : 0.f;
                wh[e] = hh[e] ? sqrtf(ch[e] * ch[e] * vh[e] * vh[e] + d2) : 0.f;
                dh[e] = hh[e] ? ch[e] * ch[e] / wh[e] : 0.f;
                const float xvv = warm ? vv[e] : 0.f, xvh = warm ? vh[e] : 0.f;
                // r = b - A x with the cancelling terms carried as hi + lo pairs
                float h, l;
                sum4_scaled(-it, evp[e], -ev[e], el[e], -eh[e], h, l);
                ru[e] = __fadd_rn(h, l);
                diff_prod(dv[e], xvv, it, ev[e], h, l);
                rv[e] = -__fadd_rn(h, l);
                diff_prod(dh[e], xvh, it, eh[e], h, l);
                rh[e] = -__fadd_rn(h, l);
                prr += ru[e] * ru[e] + rv[e] * rv[e] + rh[e] * rh[e];
                pru2 += ru[e] * ru[e];
                psu += ru[e];
                przv += rv[e] * rv[e] / (dv[e] + it) + rh[e] * rh[e] / (dh[e] + it);
                pfd += wv[e] + wh[e] + 0.5f * it * (evk[e] * evk[e] + ehk[e] * ehk[e]);
            }
            st4(P.Wv + o, wv); st4(P.Wh + o, wh); st4(P.dv + o, dv); st4(P.dh + o, dh);
            st4(P.rU + o, ru); st4(P.rVv + o, rv); st4(P.rVh + o, rh);
            if (!warm) {
                const float z[4] = {0.f, 0.f, 0.f, 0.f};
                st4(P.U + o, z); st4(P.Vv + o, z); st4(P.Vh + o, z);
            }
            if (a.r16 != nullptr) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (col[e]) emit16(a.r16, a.r16lo, a.ld16, i, j0 + e, ru[e]);
            }
            rr.add(prr);
            ru2.add(pru2);
            su.add(psu);
            rzv.add(przv);
            fd.add(pfd);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            evp[e] = ev[e];
            uc[e] = un[e];
        }
    }
    double v[5] = {rr.value(), rzv.value(), fd.value(), ru2.value(), su.value()}, tot[5];
    if (grid_reduce<5>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        const double rr_range = range_part(tot[0], tot[4], a.H, a.W);
        st->rr = rr_range;
        st->rz_v = tot[1];
        st->rnorm_u = sqrt(tot[3]);
        const double rel = st->bb > 0.0 ? sqrt(rr_range / st->bb) : 0.0;
        st->rel = rel;
        st->iter = 0;
        st->p_fresh = 1;
        st->done = (rel * rel <= a.tol2 || a.cg_max <= 0 || st->bb <= 0.0) ? 1 : 0;
        const int k = st->outer;
        if (k < kMaxOuter) st->f_delta[k] = tot[2];
    }
}

template <int ROWS>
__global__ void __launch_bounds__(kThreads)
k_reweight_residual(Planes P, StencilArgs a, DevState* st, double* partials) {
    k_reweight_residual_body<ROWS>(P, a, st, partials, single_blk());
}

// ------------------------------------------------------------------------------------------
// Search direction and curvature (Alg. 2): p_new = z + beta p_old with z_U from the Laplacian
// block and z_V = r_V / (D + 1/tau) (the diagonal blocks of the preconditioner, Sec. 3.3);
// p^T A p = sum (y_v^2 + y_h^2) / tau + D p_V^2; alpha = rho / p^T A p.
// ------------------------------------------------------------------------------------------
template <int ROWS>
__device__ __forceinline__ void k_direction_pap_body(Planes P, StencilArgs a, DevState* st, double* partials, const Blk& blk) {
    if (st->done) return;
    const int H = a.H, W = a.W, ld = a.ld;
    const int j0 = (blk.bx * kThreads + threadIdx.x) * kVec;
    const int lane = threadIdx.x & 31;
    const int R = ROWS > 0 ? ROWS : a.dir_rows;   // 0: the row count of the launch's arguments
    const int i0 = blk.by * R, i1 = min(i0 + R, H);
    const bool act = j0 < W;
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
    const float* __restrict__ rVv = P.rVv;
    const float* __restrict__ rVh = P.rVh;
    const float* __restrict__ Dv = P.dv;
    const float* __restrict__ Dh = P.dh;
    bool hh[kVec];
#pragma unroll
    for (int e = 0; e < kVec; ++e) hh[e] = j0 + e + 1 < W;

    // direction at (row, j0..j0+3): U part only, or all three parts with the diagonals; lane 31
    // also forms the U part at column j0 + 4 (the next warp's first column: its right neighbour),
    // loaded with the rest of the row two rows ahead of its use
    auto dir_u = [&](size_t o, float (&pu)[4], float& rh) {
        float z[4];
        ld4(zU + o, z);
        if (fresh) {
#pragma unroll
            for (int e = 0; e < 4; ++e) pu[e] = z[e];
        } else {
            float q[4];
            ld4(pUo + o, q);
#pragma unroll
            for (int e = 0; e < 4; ++e) pu[e] = z[e] + beta * q[e];
        }
        rh = 0.f;
        if (lane == 31 && j0 + kVec < W) {
            const float zr = zU[o + kVec];
            rh = fresh ? zr : zr + beta * pUo[o + kVec];
        }
    };
    auto dir_v = [&](size_t o, float (&pvv)[4], float (&pvh)[4], float (&dv)[4], float (&dh)[4]) {
        float r1[4], r2[4];
        ld4(Dv + o, dv); ld4(Dh + o, dh); ld4(rVv + o, r1); ld4(rVh + o, r2);
        if (fresh) {
#pragma unroll
            for (int e = 0; e < 4; ++e) { pvv[e] = r1[e] / (dv[e] + it); pvh[e] = r2[e] / (dh[e] + it); }
        } else {
            float q1[4], q2[4];
            ld4(pVvo + o, q1); ld4(pVho + o, q2);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                pvv[e] = r1[e] / (dv[e] + it) + beta * q1[e];
                pvh[e] = r2[e] / (dh[e] + it) + beta * q2[e];
            }
        }
    };

    float cu[4] = {0, 0, 0, 0}, cvv[4] = {0, 0, 0, 0}, cvh[4] = {0, 0, 0, 0};
    float cdv[4] = {0, 0, 0, 0}, cdh[4] = {0, 0, 0, 0};
    float nu[4] = {0, 0, 0, 0}, nvv[4] = {0, 0, 0, 0}, nvh[4] = {0, 0, 0, 0};
    float ndv[4] = {0, 0, 0, 0}, ndh[4] = {0, 0, 0, 0};
    float rcu = 0.f, rnu = 0.f;
    if (act) {
        const size_t o = (size_t)i0 * ld + j0;
        dir_u(o, cu, rcu);
        dir_v(o, cvv, cvh, cdv, cdh);
        if (i0 + 1 < H) {
            dir_u(o + ld, nu, rnu);
            if (i0 + 1 < i1) dir_v(o + ld, nvv, nvh, ndv, ndh);
        }
    }
    CSum acc;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j0;
        const bool hv = i + 1 < H;
        // direction of row i + 2 (its U part closes row i + 1's vertical edges)
        float mu[4] = {0, 0, 0, 0}, mvv[4] = {0, 0, 0, 0}, mvh[4] = {0, 0, 0, 0};
        float mdv[4] = {0, 0, 0, 0}, mdh[4] = {0, 0, 0, 0};
        float rmu = 0.f;
        if (act && i + 1 < i1 && i + 2 < H) {
            dir_u(o + 2 * (size_t)ld, mu, rmu);
            if (i + 2 < i1) dir_v(o + 2 * (size_t)ld, mvv, mvh, mdv, mdh);
        }
        float right = __shfl_down_sync(kFull, cu[0], 1);
        if (lane == 31) right = rcu;
        if (act) {
            st4(pUn + o, cu); st4(pVvn + o, cvv); st4(pVhn + o, cvh);
            const float pr[4] = {cu[1], cu[2], cu[3], right};
            float row = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float yh = hh[e] ? (pr[e] - cu[e] - cvh[e]) : 0.f;
                const float yv = hv ? (nu[e] - cu[e] - cvv[e]) : 0.f;
                row += it * (yh * yh + yv * yv) + cdv[e] * cvv[e] * cvv[e] + cdh[e] * cvh[e] * cvh[e];
            }
            acc.add(row);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            cu[e] = nu[e]; cvv[e] = nvv[e]; cvh[e] = nvh[e]; cdv[e] = ndv[e]; cdh[e] = ndh[e];
            nu[e] = mu[e]; nvv[e] = mvv[e]; nvh[e] = mvh[e]; ndv[e] = mdv[e]; ndh[e] = mdh[e];
        }
        rcu = rnu;
        rnu = rmu;
    }
    double v[1] = {acc.value()}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        const double pq = tot[0];
        st->pq = pq;
        st->pbuf = nxt;
        st->p_fresh = 0;
        if (!(pq > 0.0) || !isfinite(pq)) {
            // non-positive curvature: a breakdown unless rounding has already brought the
            // residual to the attainable accuracy
            st->alpha = 0.0;
            if (st->rel > kBreakdownRel || !isfinite(pq)) st->status |= ST_BREAKDOWN;
            st->done = 1;
        } else {
            st->alpha = st->rho / pq;
        }
    }
}

template <int ROWS>
__global__ void __launch_bounds__(kThreads)
k_direction_pap(Planes P, StencilArgs a, DevState* st, double* partials) {
    k_direction_pap_body<ROWS>(P, a, st, partials, single_blk());
}

// ------------------------------------------------------------------------------------------
// CG update (Alg. 2): x += alpha p, r -= alpha A p with A p recomputed from p (the stencil of
// eq. 'matrix-soft-constraints'), then ||r||^2, r_V^T z_V (z_V = r_V / (D + 1/tau)) and, for the
// flexible variant, r_new^T z_old.  Stops the run when ||r|| <= cg_tol ||b|| or on cg_max.
// ------------------------------------------------------------------------------------------
template <int ROWS>
__device__ __forceinline__ void k_update_body(Planes P, StencilArgs a, DevState* st, double* partials, const Blk& blk) {
    if (st->done) return;
    const int H = a.H, W = a.W, ld = a.ld;
    const int j0 = (blk.bx * kThreads + threadIdx.x) * kVec;
    const int lane = threadIdx.x & 31;
    const int R = ROWS > 0 ? ROWS : a.upd_rows;   // 0: the row count of the launch's arguments
    const int i0 = blk.by * R, i1 = min(i0 + R, H);
    const bool act = j0 < W;
    const float it = a.inv_tau;
    const int cur = st->pbuf;
    const float alpha = (float)st->alpha;
    const bool flex = a.flexible != 0;
    const float* __restrict__ pU = P.pU[cur];
    const float* __restrict__ pVv = P.pVv[cur];
    const float* __restrict__ pVh = P.pVh[cur];
    const float* __restrict__ Dv = P.dv;
    const float* __restrict__ Dh = P.dh;
    const float* __restrict__ Zu = P.zU;
    float* __restrict__ U = P.U;
    float* __restrict__ Vv = P.Vv;
    float* __restrict__ Vh = P.Vh;
    float* __restrict__ rU = P.rU;
    float* __restrict__ rVv = P.rVv;
    float* __restrict__ rVh = P.rVh;
    bool hh[kVec];
#pragma unroll
    for (int e = 0; e < kVec; ++e) hh[e] = j0 + e + 1 < W;

    float cu[4] = {0, 0, 0, 0}, cvv[4] = {0, 0, 0, 0}, cvh[4] = {0, 0, 0, 0};
    float nu[4] = {0, 0, 0, 0}, nvv[4] = {0, 0, 0, 0}, nvh[4] = {0, 0, 0, 0};
    float yvp[4] = {0, 0, 0, 0};
    if (act) {
        const size_t o = (size_t)i0 * ld + j0;
        ld4(pU + o, cu); ld4(pVv + o, cvv); ld4(pVh + o, cvh);
        if (i0 > 0) {
            float q[4], w[4];
            ld4(pU + o - ld, q); ld4(pVv + o - ld, w);
#pragma unroll
            for (int e = 0; e < 4; ++e) yvp[e] = cu[e] - q[e] - w[e];
        }
        if (i0 + 1 < H) {
            ld4(pU + o + ld, nu);
            if (i0 + 1 < i1) { ld4(pVv + o + ld, nvv); ld4(pVh + o + ld, nvh); }
        }
    }
    CSum rr, rzv, rzo, ru2, su;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j0;
        const bool hv = i + 1 < H;
        float dv[4] = {0, 0, 0, 0}, dh[4] = {0, 0, 0, 0}, u[4] = {0, 0, 0, 0};
        float vv[4] = {0, 0, 0, 0}, vh[4] = {0, 0, 0, 0};
        float r0[4] = {0, 0, 0, 0}, r1[4] = {0, 0, 0, 0}, r2[4] = {0, 0, 0, 0};
        float z[4] = {0, 0, 0, 0};
        float mu[4] = {0, 0, 0, 0}, mvv[4] = {0, 0, 0, 0}, mvh[4] = {0, 0, 0, 0};
        if (act) {
            ld4(Dv + o, dv); ld4(Dh + o, dh);
            ld4(U + o, u); ld4(Vv + o, vv); ld4(Vh + o, vh);
            ld4(rU + o, r0); ld4(rVv + o, r1); ld4(rVh + o, r2);
            if (flex) ld4(Zu + o, z);
            if (i + 1 < i1 && i + 2 < H) {
                ld4(pU + o + 2 * (size_t)ld, mu);
                if (i + 2 < i1) { ld4(pVv + o + 2 * (size_t)ld, mvv); ld4(pVh + o + 2 * (size_t)ld, mvh); }
            }
        }
        float yv[4], yh[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) yv[e] = hv ? (nu[e] - cu[e] - cvv[e]) : 0.f;
        float right = __shfl_down_sync(kFull, cu[0], 1);
        if (lane == 31) right = (act && j0 + kVec < W) ? pU[o + kVec] : 0.f;
        const float pr[4] = {cu[1], cu[2], cu[3], right};
#pragma unroll
        for (int e = 0; e < 4; ++e) yh[e] = hh[e] ? (pr[e] - cu[e] - cvh[e]) : 0.f;
        float left = __shfl_up_sync(kFull, yh[3], 1);
        if (lane == 0) left = (act && j0 > 0) ? (cu[0] - pU[o - 1] - pVh[o - 1]) : 0.f;
        const float yl[4] = {left, yh[0], yh[1], yh[2]};
        if (act) {
            float n0[4], n1[4], n2[4];
            float prr = 0.f, pru2 = 0.f, psu = 0.f, przv = 0.f, przo = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                // A p with its cancelling terms as hi + lo pairs, subtracted from r with one
                // rounding each (the residual is far smaller than the terms near convergence)
                float quh, qul, qvh, qvl, qhh, qhl;
                sum4_scaled(it, yvp[e], -yv[e], yl[e], -yh[e], quh, qul);
                diff_prod(dv[e], cvv[e], it, yv[e], qvh, qvl);
                diff_prod(dh[e], cvh[e], it, yh[e], qhh, qhl);
                u[e] += alpha * cu[e];
                vv[e] += alpha * cvv[e];
                vh[e] += alpha * cvh[e];
                n0[e] = __fmaf_rn(-alpha, qul, __fmaf_rn(-alpha, quh, r0[e]));
                n1[e] = __fmaf_rn(-alpha, qvl, __fmaf_rn(-alpha, qvh, r1[e]));
                n2[e] = __fmaf_rn(-alpha, qhl, __fmaf_rn(-alpha, qhh, r2[e]));
                const float iv = 1.f / (dv[e] + it), ih = 1.f / (dh[e] + it);
                prr += n0[e] * n0[e] + n1[e] * n1[e] + n2[e] * n2[e];
                pru2 += n0[e] * n0[e];
                psu += n0[e];
                przv += n1[e] * n1[e] * iv + n2[e] * n2[e] * ih;
                if (flex) przo += n0[e] * z[e] + (n1[e] * r1[e]) * iv + (n2[e] * r2[e]) * ih;
            }
            rr.add(prr);
            ru2.add(pru2);
            su.add(psu);
            rzv.add(przv);
            if (flex) rzo.add(przo);
            st4(U + o, u); st4(Vv + o, vv); st4(Vh + o, vh);
            st4(rU + o, n0); st4(rVv + o, n1); st4(rVh + o, n2);
            if (a.r16 != nullptr) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (j0 + e < W) emit16(a.r16, a.r16lo, a.ld16, i, j0 + e, n0[e]);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            yvp[e] = yv[e];
            cu[e] = nu[e]; cvv[e] = nvv[e]; cvh[e] = nvh[e];
            nu[e] = mu[e]; nvv[e] = mvv[e]; nvh[e] = mvh[e];
        }
    }
    double v[5] = {rr.value(), rzv.value(), rzo.value(), ru2.value(), su.value()}, tot[5];
    if (grid_reduce<5>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        const double rr_range = range_part(tot[0], tot[4], a.H, a.W);
        st->rr = rr_range;
        st->rz_v = tot[1];
        st->rz_old = tot[2];
        st->rnorm_u = sqrt(tot[3]);
        const int itn = st->iter + 1;
        st->iter = itn;
        const double rel = st->bb > 0.0 ? sqrt(rr_range / st->bb) : 0.0;
        st->rel = rel;
        if (rel * rel <= a.tol2 || itn >= a.cg_max || !isfinite(rel)) st->done = 1;
        if (!isfinite(rel)) st->status |= ST_NONFINITE;
    }
}

template <int ROWS>
__global__ void __launch_bounds__(kThreads)
k_update(Planes P, StencilArgs a, DevState* st, double* partials) {
    k_update_body<ROWS>(P, a, st, partials, single_blk());
}

// ------------------------------------------------------------------------------------------
// End of an outer step: sum U (for U -= mean(U), Prop. 'minimising (alt1)'), the objective of
// problem (main) and H_delta(x^{k+1}, W^k) of problem (alt1); then record the statistics.
// ------------------------------------------------------------------------------------------
// On float4 lanes (the update kernel's columns per block, rows a.fin_rows).  Per edge in
// float32: the difference U_{i+1} - U_i and its residual e = (U_{i+1} - U_i) - G are formed with
// two-sums, so e is exact up to one rounding of itself; C |e| and the H_delta term are each one
// or two roundings of themselves, and all sums are compensated per thread, then FP64 across
// threads.
__device__ __forceinline__ float edge_residual(float un, float u, float g) {
    float d, dl, e, el;
    two_sum(un, -u, d, dl);
    two_sum(d, -g, e, el);
    return __fadd_rn(e, __fadd_rn(el, dl));
}

template <int ROWS>
__device__ __forceinline__ void k_finalize_reduce_body(Planes P, StencilArgs a, DevState* st,
                                                       double* partials, const Blk& blk) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j0 = (blk.bx * kThreads + threadIdx.x) * kVec;
    const int lane = threadIdx.x & 31;
    const int R = ROWS > 0 ? ROWS : a.fin_rows;   // 0: the row count of the launch's arguments
    const int i0 = blk.by * R, i1 = min(i0 + R, H);
    const bool act = j0 < W;
    const float it = a.inv_tau, d2 = a.delta * a.delta;
    const float* __restrict__ U = P.U;
    bool hh[kVec];
#pragma unroll
    for (int e = 0; e < kVec; ++e) hh[e] = j0 + e + 1 < W;
    CSum su, l1, hd;
    float uc[4] = {0, 0, 0, 0};
    if (act) ld4(U + (size_t)i0 * ld + j0, uc);
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j0;
        const bool hv = i + 1 < H;
        float un[4] = {0, 0, 0, 0}, gv[4] = {0, 0, 0, 0}, gh[4] = {0, 0, 0, 0};
        float cv[4] = {0, 0, 0, 0}, ch[4] = {0, 0, 0, 0}, vv[4] = {0, 0, 0, 0};
        float vh[4] = {0, 0, 0, 0}, wv[4] = {0, 0, 0, 0}, wh[4] = {0, 0, 0, 0};
        if (act) {
            if (hv) {
                ld4(U + o + ld, un); ld4(P.Gv + o, gv); ld4(P.Cv + o, cv); ld4(P.Vv + o, vv);
                ld4(P.Wv + o, wv);
            }
            ld4(P.Gh + o, gh); ld4(P.Ch + o, ch); ld4(P.Vh + o, vh); ld4(P.Wh + o, wh);
        }
        float ur = __shfl_down_sync(kFull, uc[0], 1);
        if (lane == 31) ur = (act && j0 + kVec < W) ? U[o + kVec] : 0.f;
        const float pr[4] = {uc[1], uc[2], uc[3], ur};
        if (act) {
            float psu = 0.f, pl1 = 0.f, phd = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                psu += uc[e];
                if (hv && j0 + e < W) {
                    const float r = edge_residual(un[e], uc[e], gv[e]);
                    pl1 += cv[e] * fabsf(r);
                    const float pe = r - vv[e];
                    phd += 0.5f * ((cv[e] * cv[e] * vv[e] * vv[e] + d2) / wv[e] + wv[e]) +
                           0.5f * it * pe * pe;
                }
                if (hh[e]) {
                    const float r = edge_residual(pr[e], uc[e], gh[e]);
                    pl1 += ch[e] * fabsf(r);
                    const float pe = r - vh[e];
                    phd += 0.5f * ((ch[e] * ch[e] * vh[e] * vh[e] + d2) / wh[e] + wh[e]) +
                           0.5f * it * pe * pe;
                }
            }
            su.add(psu);
            l1.add(pl1);
            hd.add(phd);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) uc[e] = un[e];
    }
    double v[3] = {su.value(), l1.value(), hd.value()}, tot[3];
    if (grid_reduce<3>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        st->mean_u = tot[0] / ((double)H * (double)W);
        const int k = st->outer;
        if (k < kMaxOuter) {
            st->l1_obj[k] = tot[1];
            st->h_delta[k] = tot[2];
            st->cg_iters[k] = st->iter;
            st->rel_res[k] = st->rel;
        }
        st->cg_total += st->iter;
        if (a.cap_warn && st->iter >= a.cg_max && st->rel * st->rel > a.tol2)
            st->status |= ST_CGMAX;
        st->outer = k + 1;
    }
}

template <int ROWS>
__global__ void __launch_bounds__(kThreads)
k_finalize_reduce(Planes P, StencilArgs a, DevState* st, double* partials) {
    k_finalize_reduce_body<ROWS>(P, a, st, partials, single_blk());
}

// U -= mean(U) with the mean the finalize kernel formed (Prop. 'minimising (alt1)').
__device__ __forceinline__ void k_subtract_mean_body(float* U, int H, int W, int ld, const DevState* st, const Blk& blk) {
    const int j = blk.bx * kThreads + threadIdx.x;
    const int i0 = blk.by * kRows, i1 = strip_rows(H, i0);
    if (j >= W) return;
    const float m = (float)st->mean_u;
    for (int i = i0; i < i1; ++i) U[(size_t)i * ld + j] -= m;
}

__global__ void __launch_bounds__(kThreads)
k_subtract_mean(float* U, int H, int W, int ld, const DevState* st) {
    k_subtract_mean_body(U, H, W, ld, st, single_blk());
}

// ------------------------------------------------------------------------------------------
// Adjoint of the IRLS map through converged inner solves (reverse sweep over the outer steps).
// Step k takes the checkpointed V^k, V^{k+1}, the solve's result lambda = A_k^+ xbar (in the
// iterate planes) and accumulates
//   Gbar_v += (S lambda_U - lambda_Vv) / tau,  Gbar_h += (lambda_U T - lambda_Vh) / tau
//   Dbar    = -lambda_V o V^{k+1}
//   Cbar   += Dbar o (2 C / W - C^3 (V^k)^2 / W^3)
// and writes the next right-hand side xbar = (0, Dbar o (-C^4 V^k / W^3)) into the residual
// planes (W^k = sqrt(C^2 (V^k)^2 + delta^2), D^k = C^2 / W^k: Alg. 1's reweighting).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void k_user_mean_body(const float* __restrict__ src, int H, int W, DevState* st, double* partials, const Blk& blk) {
    const int j = blk.bx * kThreads + threadIdx.x;
    const int i0 = blk.by * kRows, i1 = strip_rows(H, i0);
    CSum acc;
    if (j < W)
        for (int i = i0; i < i1; ++i) acc.add(src[(size_t)i * W + j]);
    double v[1] = {acc.value()}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0)
        st->mean_u = tot[0] / ((double)H * (double)W);
}

__global__ void __launch_bounds__(kThreads)
k_user_mean(const float* __restrict__ src, int H, int W, DevState* st, double* partials) {
    k_user_mean_body(src, H, W, st, partials, single_blk());
}

// xbar^K = (dL/dU - mean, 0, 0) into the residual planes, with factor 1.
//
// Scaling of the sweep: the cotangent shrinks by about the same factor at every reverse step (by
// 1e-7 per step on the 1024^2 workload's law: 1e-89 after 15 steps), far below float32's range.
// The residual planes therefore hold xbar' with xbar = adj_scale * xbar' (adj_scale in FP64);
// each step solves with xbar' / ||xbar'|| and multiplies what it accumulates by the running
// factor, so no plane ever underflows (contributions below float32's range become 0, as they
// would in float32 arithmetic of the unscaled sweep).
__global__ void __launch_bounds__(kThreads)
k_adj_init(Planes P, StencilArgs a, const float* __restrict__ dLdU, DevState* st) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) st->adj_scale = 1.0;
    if (j >= W) return;
    const float m = (float)st->mean_u;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j;
        P.rU[o] = dLdU[(size_t)i * W + j] - m;
        P.rVv[o] = 0.f;
        P.rVh[o] = 0.f;
    }
}

// The adjoint solve A_k lambda = xbar through the U-only (Schur) system: its V rows give
//   lambda_V = (tau xbar_V + S lambda_U) / (1 + tau D)     per edge,
// and the U row becomes L_Om lambda_U = f with Om = D / (1 + tau D) and
//   f = xbar_U + S^T (xbar_Vv / (1 + tau Dv)) + (xbar_Vh / (1 + tau Dh)) T^T.
// The elimination is exact; it keeps lambda_V accurate edge by edge where D is large (the
// weights of nearly consistent edges, D ~ C^2 / delta), where a float32 solve of the full
// system resolves lambda_V only to the rounding of the largest component, which the next
// reverse step amplifies by up to 1 / delta.  Set-up: W, D from the checkpoint V^k, f into
// r_U (xbar_V stays in r_Vv, r_Vh for the recovery), lambda = 0, the stopping scale ||f||.
__device__ __forceinline__ float adj_wd(float c, float v, float d2, float& w) {
    w = sqrtf(c * c * v * v + d2);
    return c * c / w;
}

// ||xbar'|| of a reverse step into st->adj_step, and the step's factor adj_scale * ||xbar'||
// into st->adj_scale (the factor of this step's solution and of the next cotangent).
__global__ void __launch_bounds__(kThreads)
k_adj_norm(Planes P, StencilArgs a, DevState* st, double* partials) {
    const Blk blk = single_blk();
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blk.bx * kThreads + threadIdx.x;
    const int i0 = blk.by * kRows, i1 = strip_rows(H, i0);
    CSum acc;
    if (j < W)
        for (int i = i0; i < i1; ++i) {
            const size_t o = (size_t)i * ld + j;
            const float u = P.rU[o], v = P.rVv[o], h = P.rVh[o];
            acc.add(u * u + v * v + h * h);
        }
    double v[1] = {acc.value()}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        const double s = sqrt(tot[0]);
        st->adj_step = s;
        st->adj_scale = st->adj_scale * s;
    }
}

__global__ void __launch_bounds__(kThreads)
k_adj_setup_schur(Planes P, StencilArgs a, const float* __restrict__ Vkv,
                  const float* __restrict__ Vkh, const float* __restrict__ Cv,
                  const float* __restrict__ Ch, DevState* st, double* partials) {
    const Blk blk = single_blk();
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blk.bx * kThreads + threadIdx.x;
    const int i0 = blk.by * kRows, i1 = strip_rows(H, i0);
    const float tau = a.tau, d2 = a.delta * a.delta;
    // the step's right-hand side normalised: xbar' / ||xbar'||
    const double sn = st->adj_step;
    const float inv = sn > 0.0 ? (float)(1.0 / sn) : 0.f;
    CSum rr, su;
    if (j < W) {
        for (int i = i0; i < i1; ++i) {
            const size_t o = (size_t)i * ld + j;
            float wv = 0.f, wh = 0.f, dv = 0.f, dh = 0.f, gv = 0.f, gh = 0.f, gvu = 0.f, ghl = 0.f;
            if (i + 1 < H) {
                dv = adj_wd(Cv[o], Vkv[o], d2, wv);
                gv = inv * P.rVv[o] / (1.f + tau * dv);
            }
            if (j + 1 < W) {
                dh = adj_wd(Ch[o], Vkh[o], d2, wh);
                gh = inv * P.rVh[o] / (1.f + tau * dh);
            }
            if (i > 0) {
                float w;
                gvu = inv * P.rVv[o - ld] / (1.f + tau * adj_wd(Cv[o - ld], Vkv[o - ld], d2, w));
            }
            if (j > 0) {
                float w;
                ghl = inv * P.rVh[o - 1] / (1.f + tau * adj_wd(Ch[o - 1], Vkh[o - 1], d2, w));
            }
            P.Wv[o] = wv; P.Wh[o] = wh; P.dv[o] = dv; P.dh[o] = dh;
            P.U[o] = 0.f; P.Vv[o] = 0.f; P.Vh[o] = 0.f;
            float h, l;
            sum4_scaled(1.f, gvu, -gv, ghl, -gh, h, l);
            const float f = __fadd_rn(inv * P.rU[o], __fadd_rn(h, l));
            P.rU[o] = f;
            if (a.r16 != nullptr) emit16(a.r16, a.r16lo, a.ld16, i, j, f);
            rr.add(f * f);
            su.add(f);
        }
    }
    double v[2] = {rr.value(), su.value()}, tot[2];
    if (grid_reduce<2>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        const double rr_range = range_part(tot[0], tot[1], a.H, a.W);
        st->rr = rr_range;
        st->rz_v = 0.0;
        st->rz_old = 0.0;
        st->rnorm_u = sqrt(tot[0]);
        st->bb = rr_range;
        st->rel = rr_range > 0.0 ? 1.0 : 0.0;
        st->iter = 0;
        st->p_fresh = 1;
        st->done = (rr_range <= 0.0 || a.cg_max <= 0) ? 1 : 0;
    }
}

// lambda_V = (tau xbar_V + S lambda_U) / (1 + tau D) after the U-only adjoint solve, with the
// step's normalised right-hand side xbar' / ||xbar'||
__global__ void __launch_bounds__(kThreads)
k_adj_recover_v(Planes P, StencilArgs a, const DevState* st) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    if (j >= W) return;
    const double sn = st->adj_step;
    const float tau = a.tau * (sn > 0.0 ? (float)(1.0 / sn) : 0.f);
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j;
        const float u = P.U[o];
        if (i + 1 < H)
            P.Vv[o] = (tau * P.rVv[o] + (P.U[o + ld] - u)) / (1.f + a.tau * P.dv[o]);
        if (j + 1 < W)
            P.Vh[o] = (tau * P.rVh[o] + (P.U[o + 1] - u)) / (1.f + a.tau * P.dh[o]);
    }
}

__global__ void __launch_bounds__(kThreads)
k_adj_accumulate(Planes P, StencilArgs a, const float* __restrict__ Vkv,
                 const float* __restrict__ Vkh, const float* __restrict__ Vnv,
                 const float* __restrict__ Vnh, const float* __restrict__ Cv,
                 const float* __restrict__ Ch, float* __restrict__ Gbv, float* __restrict__ Gbh,
                 float* __restrict__ Cbv, float* __restrict__ Cbh, const DevState* st) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    const float d2 = a.delta * a.delta;
    // the step's factor: lambda = F lambda'' for the normalised solve (float32: 0 once the
    // contribution is below float32's range)
    const float F = (float)st->adj_scale;
    const float it = a.inv_tau * F;
    if (j >= W) return;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j;
        const float lu = P.U[o];
        float nv = 0.f, nh = 0.f;
        if (i + 1 < H) {
            const float lv = P.Vv[o];
            Gbv[o] += it * ((P.U[o + ld] - lu) - lv);
            const float c = Cv[o], v = Vkv[o];
            const float w = sqrtf(c * c * v * v + d2);
            const float w3 = w * w * w;
            const float db = -lv * Vnv[o];
            Cbv[o] += F * db * (2.f * c / w - c * c * c * v * v / w3);
            nv = db * (-(c * c * c * c) * v / w3);
        }
        if (j + 1 < W) {
            const float lh = P.Vh[o];
            Gbh[o] += it * ((P.U[o + 1] - lu) - lh);
            const float c = Ch[o], v = Vkh[o];
            const float w = sqrtf(c * c * v * v + d2);
            const float w3 = w * w * w;
            const float db = -lh * Vnh[o];
            Cbh[o] += F * db * (2.f * c / w - c * c * c * v * v / w3);
            nh = db * (-(c * c * c * c) * v / w3);
        }
        P.rU[o] = 0.f;
        P.rVv[o] = nv;
        P.rVh[o] = nh;
    }
}

// dL/dX = S^T Gbar_v + Gbar_h T^T with Gbar -= Vbar^0 (V^0 = -G), and dL/dcoherence from the
// averaging Cv = (coh_i + coh_i+1) / 2, both written with pitch W.
__global__ void __launch_bounds__(kThreads)
k_adj_final(Planes P, StencilArgs a, const float* __restrict__ Gbv, const float* __restrict__ Gbh,
            const float* __restrict__ Cbv, const float* __restrict__ Cbh, float* __restrict__ dX,
            float* __restrict__ dcoh, const DevState* st) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    if (j >= W) return;
    const float F = (float)st->adj_scale;   // factor of the cotangent left in the planes
    auto gv = [&](size_t o) { return Gbv[o] - F * P.rVv[o]; };
    auto gh = [&](size_t o) { return Gbh[o] - F * P.rVh[o]; };
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j;
        float x = 0.f, c = 0.f;
        if (i > 0) { x += gv(o - ld); c += 0.5f * Cbv[o - ld]; }
        if (i + 1 < H) { x -= gv(o); c += 0.5f * Cbv[o]; }
        if (j > 0) { x += gh(o - 1); c += 0.5f * Cbh[o - 1]; }
        if (j + 1 < W) { x -= gh(o); c += 0.5f * Cbh[o]; }
        dX[(size_t)i * W + j] = x;
        if (dcoh != nullptr) dcoh[(size_t)i * W + j] = c;
    }
}

// ------------------------------------------------------------------------------------------
// Batched launches: one grid over the blocks of every image; each block finds its image by a
// binary search over the images' first-block indices and runs the single-image body with its
// own coordinates, state and scratch.
// ------------------------------------------------------------------------------------------
// grid of a batched launch: the strip kernels, the direction kernel, the update kernel
// and the reweighting and finalize kernels (the direction kernel's columns, their own rows)
enum GridKind : int { GK_STRIP = 0, GK_DIR = 1, GK_UPD = 2, GK_RW = 3, GK_FIN = 4 };

__device__ __forceinline__ int grid_blk0(const TileRec& r, int kind) {
    switch (kind) {
        case GK_STRIP: return r.sblk0;
        case GK_DIR: return r.vblk0;
        case GK_UPD: return r.ublk0;
        case GK_RW: return r.rblk0;
        default: return r.fblk0;
    }
}

__device__ __forceinline__ int find_tile(const TileRec* __restrict__ r, int T, int bid, int kind) {
    int lo = 0, hi = T - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (grid_blk0(r[mid], kind) <= bid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ Blk tile_blk(const TileRec& r, int bid, int kind) {
    Blk b;
    const int gx = kind == GK_STRIP ? r.sgx : r.vgx;
    const int gy = kind == GK_STRIP ? r.sgy : kind == GK_DIR ? r.vgy : kind == GK_UPD ? r.ugy
                 : kind == GK_RW ? r.rgy : r.fgy;
    const int local = bid - grid_blk0(r, kind);
    b.bx = local % gx;
    b.by = local / gx;
    b.nblk = (unsigned)(gx * gy);
    b.bid = (unsigned)local;
    return b;
}

__global__ void __launch_bounds__(kThreads) kb_init(const TileRec* __restrict__ recs, int T) {
    const TileRec& r = recs[find_tile(recs, T, blockIdx.x, GK_STRIP)];
    k_init_body(r.X, r.coh, nullptr, nullptr, nullptr, nullptr, nullptr, r.P, r.a, r.st,
                tile_blk(r, blockIdx.x, GK_STRIP));
}

__global__ void __launch_bounds__(kThreads) kb_bnorm(const TileRec* __restrict__ recs, int T) {
    const TileRec& r = recs[find_tile(recs, T, blockIdx.x, GK_STRIP)];
    k_bnorm_body(r.P, r.a, r.st, r.partials, tile_blk(r, blockIdx.x, GK_STRIP));
}

// the reweighting and finalize kernels run each image with its own row count (a.rw_rows,
// a.fin_rows: the same function of the image's size as in a single-image plan)
__global__ void __launch_bounds__(kThreads) kb_reweight(const TileRec* __restrict__ recs, int T) {
    const TileRec& r = recs[find_tile(recs, T, blockIdx.x, GK_RW)];
    k_reweight_residual_body<0>(r.P, r.a, r.st, r.partials, tile_blk(r, blockIdx.x, GK_RW));
}

template <int ROWS>
__global__ void __launch_bounds__(kThreads) kb_direction(const TileRec* __restrict__ recs, int T) {
    const TileRec& r = recs[find_tile(recs, T, blockIdx.x, GK_DIR)];
    k_direction_pap_body<ROWS>(r.P, r.a, r.st, r.partials, tile_blk(r, blockIdx.x, GK_DIR));
}

template <int ROWS>
__global__ void __launch_bounds__(kThreads) kb_update(const TileRec* __restrict__ recs, int T) {
    const TileRec& r = recs[find_tile(recs, T, blockIdx.x, GK_UPD)];
    k_update_body<ROWS>(r.P, r.a, r.st, r.partials, tile_blk(r, blockIdx.x, GK_UPD));
}

__global__ void __launch_bounds__(kThreads) kb_finalize(const TileRec* __restrict__ recs, int T) {
    const TileRec& r = recs[find_tile(recs, T, blockIdx.x, GK_FIN)];
    k_finalize_reduce_body<0>(r.P, r.a, r.st, r.partials, tile_blk(r, blockIdx.x, GK_FIN));
}

__global__ void __launch_bounds__(kThreads) kb_subtract_mean(const TileRec* __restrict__ recs, int T) {
    const TileRec& r = recs[find_tile(recs, T, blockIdx.x, GK_STRIP)];
    k_subtract_mean_body(r.P.U, r.a.H, r.a.W, r.a.ld, r.st, tile_blk(r, blockIdx.x, GK_STRIP));
}

// number of images whose CG run has not stopped
__global__ void k_count_active(const DevState* __restrict__ states, int T, int* out) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) c += states[t].done ? 0 : 1;
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) *out = cnt;
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

// statistics of one adjoint solve: CG iterations and final relative residual
__global__ void k_record_step(DevState* st) {
    const int k = st->outer;
    if (k < kMaxOuter) {
        st->cg_iters[k] = st->iter;
        st->rel_res[k] = st->rel;
    }
    st->cg_total += st->iter;
    st->outer = k + 1;
}

// ------------------------------------------------------------------------------------------
// U-only (Schur complement) form of the same linear system.  The V rows of the system of
// Sec. 3.1 give V = (D U - G) / (1 + tau D) edge by edge; the U row becomes
//     L_Om U = f,   L_Om U = S^T (Om_v o S U) + (Om_h o U T) T^T,
//     f = S^T (Om_v o Gv) + (Om_h o Gh) T^T,   Om = D / (1 + tau D)
// solved by Alg. 2 with the Laplacian block of Sec. 3.3 as the preconditioner.  The planes dv,
// dh keep D (Om is formed where it is used); the CG state and stopping rule are those of the
// (U, V) form with r = r_U only (r_V, z_V and their products are zero).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float omega_of(float d, float tau) { return d / (1.f + tau * d); }

// Start of an outer step: W = sqrt(C^2 V^2 + delta^2), D = C^2 / W, the Schur right-hand side
// f and its norm, the initial residual r = f - L_Om U^k (warm start) or f (cold start), and
// F_delta(x^k) (the same statistic as the (U, V) form).
__device__ __forceinline__ void k_schur_reweight_body(Planes P, StencilArgs a, DevState* st,
                                                      double* partials, const Blk& blk) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blk.bx * kThreads + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int i0 = blk.by * kRows, i1 = strip_rows(H, i0);
    const bool col = j < W, hh = j + 1 < W;
    const float it = a.inv_tau, tau = a.tau, d2 = a.delta * a.delta;
    const bool warm = a.warm_start != 0;
    // vertical edge (i, j): omega and the edge terms Om (S U - Gv) and Om Gv
    auto vedge = [&](int i, float& flux, float& fg) {
        const size_t o = (size_t)i * ld + j;
        const float cv = P.Cv[o], vv = P.Vv[o], gv = P.Gv[o];
        const float wv = sqrtf(cv * cv * vv * vv + d2);
        const float om = omega_of(cv * cv / wv, tau);
        const float su = warm ? (P.U[o + ld] - P.U[o]) : 0.f;
        flux = om * (su - gv);
        fg = om * gv;
    };
    CSum rr, bb, fd, su_r;
    float uc = col ? P.U[(size_t)i0 * ld + j] : 0.f;
    float flux_up = 0.f, fg_up = 0.f;   // vertical edge (i - 1, j)
    if (col && i0 > 0) vedge(i0 - 1, flux_up, fg_up);
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
        float wv = 0.f, wh = 0.f, dv = 0.f, dh = 0.f;
        if (col && hv) { wv = sqrtf(cv * cv * vv * vv + d2); dv = cv * cv / wv; }
        if (col && hh) { wh = sqrtf(ch * ch * vh * vh + d2); dh = ch * ch / wh; }
        const float ov = omega_of(dv, tau), oh = omega_of(dh, tau);
        const float sv = (col && hv && warm) ? (un - uc) : 0.f;
        const float sh = (col && hh && warm) ? (ur - uc) : 0.f;
        const float flux_v = (col && hv) ? ov * (sv - gv) : 0.f;
        const float flux_h = (col && hh) ? oh * (sh - gh) : 0.f;
        const float fgv = (col && hv) ? ov * gv : 0.f;
        const float fgh = (col && hh) ? oh * gh : 0.f;
        float flux_l = __shfl_up_sync(kFull, flux_h, 1);
        float fg_l = __shfl_up_sync(kFull, fgh, 1);
        if (lane == 0) {
            flux_l = 0.f;
            fg_l = 0.f;
            if (col && j > 0) {
                const float c = P.Ch[o - 1], v = P.Vh[o - 1], g = P.Gh[o - 1];
                const float w = sqrtf(c * c * v * v + d2);
                const float om = omega_of(c * c / w, tau);
                const float s = warm ? (uc - P.U[o - 1]) : 0.f;
                flux_l = om * (s - g);
                fg_l = om * g;
            }
        }
        if (col) {
            // r = -(S^T flux_v + flux_h T^T),  f = S^T (Om Gv) + (Om Gh) T^T
            const float ru = -(flux_up - flux_v + flux_l - flux_h);
            const float fu = fg_up - fgv + fg_l - fgh;
            P.Wv[o] = wv; P.Wh[o] = wh; P.dv[o] = dv; P.dh[o] = dh;
            P.rU[o] = ru;
            if (!warm) P.U[o] = 0.f;
            if (a.r16 != nullptr) emit16(a.r16, a.r16lo, a.ld16, i, j, ru);
            rr.add(ru * ru);
            su_r.add(ru);
            bb.add(fu * fu);
            // F_delta(x^k) with the edge residuals S U - V - G at the iterate
            const float evk = hv ? (un - uc - vv - gv) : 0.f;
            const float ehk = hh ? (ur - uc - vh - gh) : 0.f;
            fd.add(wv + wh + 0.5f * it * (evk * evk + ehk * ehk));
        }
        flux_up = flux_v;
        fg_up = fgv;
        uc = un;
    }
    double v[4] = {rr.value(), bb.value(), fd.value(), su_r.value()}, tot[4];
    if (grid_reduce<4>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        const double rr_range = range_part(tot[0], tot[3], a.H, a.W);
        st->rr = rr_range;
        st->bb = tot[1];
        st->rz_v = 0.0;
        st->rz_old = 0.0;
        st->rnorm_u = sqrt(tot[0]);
        const double rel = st->bb > 0.0 ? sqrt(rr_range / st->bb) : 0.0;
        st->rel = rel;
        st->iter = 0;
        st->p_fresh = 1;
        st->done = (rel * rel <= a.tol2 || a.cg_max <= 0 || st->bb <= 0.0) ? 1 : 0;
        const int k = st->outer;
        if (k < kMaxOuter) st->f_delta[k] = tot[2];
    }
}

__global__ void __launch_bounds__(kThreads)
k_schur_reweight(Planes P, StencilArgs a, DevState* st, double* partials) {
    k_schur_reweight_body(P, a, st, partials, single_blk());
}

// p = z + beta p_old and p^T L_Om p = sum Om_v (S p)^2 + Om_h (p T)^2; alpha = rho / p^T L p.
template <int ROWS>
__global__ void __launch_bounds__(kThreads)
k_schur_direction(Planes P, StencilArgs a, DevState* st, double* partials) {
    const Blk blk = single_blk();
    if (st->done) return;
    const int H = a.H, W = a.W, ld = a.ld;
    const int j0 = (blk.bx * kThreads + threadIdx.x) * kVec;
    const int lane = threadIdx.x & 31;
    const int R = ROWS > 0 ? ROWS : a.sdir_rows;   // 0: the row count of the launch's arguments
    const int i0 = blk.by * R, i1 = min(i0 + R, H);
    const bool act = j0 < W;
    const float tau = a.tau;
    const int cur = st->pbuf, nxt = cur ^ 1;
    const bool fresh = st->p_fresh != 0;
    const float beta = fresh ? 0.f : (float)st->beta;
    const float* __restrict__ pUo = P.pU[cur];
    float* __restrict__ pUn = P.pU[nxt];
    const float* __restrict__ zU = P.zU;
    const float* __restrict__ Dv = P.dv;
    const float* __restrict__ Dh = P.dh;
    bool hh[kVec];
#pragma unroll
    for (int e = 0; e < kVec; ++e) hh[e] = j0 + e + 1 < W;
    // p_U of a row (and, in lane 31, at column j0 + 4: the right neighbour), two rows ahead
    auto dir_u = [&](size_t o, float (&pu)[4], float& rh) {
        float z[4];
        ld4(zU + o, z);
        if (fresh) {
#pragma unroll
            for (int e = 0; e < 4; ++e) pu[e] = z[e];
        } else {
            float q[4];
            ld4(pUo + o, q);
#pragma unroll
            for (int e = 0; e < 4; ++e) pu[e] = z[e] + beta * q[e];
        }
        rh = 0.f;
        if (lane == 31 && j0 + kVec < W) {
            const float zr = zU[o + kVec];
            rh = fresh ? zr : zr + beta * pUo[o + kVec];
        }
    };
    float cu[4] = {0, 0, 0, 0}, nu[4] = {0, 0, 0, 0};
    float dv[4] = {0, 0, 0, 0}, dh[4] = {0, 0, 0, 0};   // D of the current row, one row ahead
    float rcu = 0.f, rnu = 0.f;
    if (act) {
        const size_t o = (size_t)i0 * ld + j0;
        dir_u(o, cu, rcu);
        ld4(Dv + o, dv);
        ld4(Dh + o, dh);
        if (i0 + 1 < H) dir_u(o + ld, nu, rnu);
    }
    CSum acc;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j0;
        const bool hv = i + 1 < H;
        float mu[4] = {0, 0, 0, 0}, ndv[4] = {0, 0, 0, 0}, ndh[4] = {0, 0, 0, 0};
        float rmu = 0.f;
        if (act && i + 1 < i1) {
            ld4(Dv + o + ld, ndv);
            ld4(Dh + o + ld, ndh);
            if (i + 2 < H) dir_u(o + 2 * (size_t)ld, mu, rmu);
        }
        float right = __shfl_down_sync(kFull, cu[0], 1);
        if (lane == 31) right = rcu;
        if (act) {
            st4(pUn + o, cu);
            const float pr[4] = {cu[1], cu[2], cu[3], right};
            float row = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float yh = hh[e] ? (pr[e] - cu[e]) : 0.f;
                const float yv = hv ? (nu[e] - cu[e]) : 0.f;
                row += omega_of(dv[e], tau) * yv * yv + omega_of(dh[e], tau) * yh * yh;
            }
            acc.add(row);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            cu[e] = nu[e];
            nu[e] = mu[e];
            dv[e] = ndv[e];
            dh[e] = ndh[e];
        }
        rcu = rnu;
        rnu = rmu;
    }
    double v[1] = {acc.value()}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        const double pq = tot[0];
        st->pq = pq;
        st->pbuf = nxt;
        st->p_fresh = 0;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->alpha = 0.0;
            if (st->rel > kBreakdownRel || !isfinite(pq)) st->status |= ST_BREAKDOWN;
            st->done = 1;
        } else {
            st->alpha = st->rho / pq;
        }
    }
}

// U += alpha p, r -= alpha L_Om p, ||r||^2 (range part), r_new^T z_old for the flexible ratio.
template <int ROWS>
__global__ void __launch_bounds__(kThreads)
k_schur_update(Planes P, StencilArgs a, DevState* st, double* partials) {
    const Blk blk = single_blk();
    if (st->done) return;
    const int H = a.H, W = a.W, ld = a.ld;
    const int j0 = (blk.bx * kThreads + threadIdx.x) * kVec;
    const int lane = threadIdx.x & 31;
    const int R = ROWS > 0 ? ROWS : a.supd_rows;   // 0: the row count of the launch's arguments
    const int i0 = blk.by * R, i1 = min(i0 + R, H);
    const bool act = j0 < W;
    const float tau = a.tau;
    const int cur = st->pbuf;
    const float alpha = (float)st->alpha;
    const bool flex = a.flexible != 0;
    const float* __restrict__ pU = P.pU[cur];
    const float* __restrict__ Dv = P.dv;
    const float* __restrict__ Dh = P.dh;
    const float* __restrict__ Zu = P.zU;
    float* __restrict__ U = P.U;
    float* __restrict__ rU = P.rU;
    bool hh[kVec];
#pragma unroll
    for (int e = 0; e < kVec; ++e) hh[e] = j0 + e + 1 < W;
    float cu[4] = {0, 0, 0, 0}, nu[4] = {0, 0, 0, 0};
    float yvp[4] = {0, 0, 0, 0};   // Om_v (S p) on the vertical edge above
    if (act) {
        const size_t o = (size_t)i0 * ld + j0;
        ld4(pU + o, cu);
        if (i0 > 0) {
            float q[4], d[4];
            ld4(pU + o - ld, q);
            ld4(Dv + o - ld, d);
#pragma unroll
            for (int e = 0; e < 4; ++e) yvp[e] = omega_of(d[e], tau) * (cu[e] - q[e]);
        }
        if (i0 + 1 < H) ld4(pU + o + ld, nu);
    }
    // the row's own data and its neighbour halos (lane 31: p_U at column j0 + 4; lane 0: p_U
    // and D_h at column j0 - 1), loaded one row ahead of their use
    struct SRow {
        float dv[4], dh[4], u[4], r0[4], z[4];
        float rgt, lpu, ldh;
    };
    auto load_row = [&](size_t o, SRow& d) {
        ld4(Dv + o, d.dv);
        ld4(Dh + o, d.dh);
        ld4(U + o, d.u);
        ld4(rU + o, d.r0);
        if (flex) ld4(Zu + o, d.z);
        d.rgt = d.lpu = d.ldh = 0.f;
        if (lane == 31 && j0 + kVec < W) d.rgt = pU[o + kVec];
        if (lane == 0 && j0 > 0) {
            d.lpu = pU[o - 1];
            d.ldh = Dh[o - 1];
        }
    };
    SRow rc;
    if (act) load_row((size_t)i0 * ld + j0, rc);
    CSum rr, rzo, su;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j0;
        const bool hv = i + 1 < H;
        float mu[4] = {0, 0, 0, 0};
        SRow rn;
        if (act) {
            if (i + 1 < i1) load_row(o + ld, rn);
            if (i + 1 < i1 && i + 2 < H) ld4(pU + o + 2 * (size_t)ld, mu);
        }
        float (&dv)[4] = rc.dv, (&dh)[4] = rc.dh, (&u)[4] = rc.u, (&r0)[4] = rc.r0, (&z)[4] = rc.z;
        float yv[4], yh[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) yv[e] = hv ? omega_of(dv[e], tau) * (nu[e] - cu[e]) : 0.f;
        float right = __shfl_down_sync(kFull, cu[0], 1);
        if (lane == 31) right = rc.rgt;
        const float pr[4] = {cu[1], cu[2], cu[3], right};
#pragma unroll
        for (int e = 0; e < 4; ++e) yh[e] = hh[e] ? omega_of(dh[e], tau) * (pr[e] - cu[e]) : 0.f;
        float left = __shfl_up_sync(kFull, yh[3], 1);
        if (lane == 0) left = (act && j0 > 0) ? omega_of(rc.ldh, tau) * (cu[0] - rc.lpu) : 0.f;
        const float yl[4] = {left, yh[0], yh[1], yh[2]};
        if (act) {
            float n0[4];
            float prr = 0.f, psu = 0.f, przo = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                // (L_Om p) = S^T (Om_v S p) + (Om_h p T) T^T at this pixel
                const float q = yvp[e] - yv[e] + yl[e] - yh[e];
                u[e] += alpha * cu[e];
                n0[e] = r0[e] - alpha * q;
                prr += n0[e] * n0[e];
                psu += n0[e];
                if (flex) przo += n0[e] * z[e];
            }
            rr.add(prr);
            su.add(psu);
            if (flex) rzo.add(przo);
            st4(U + o, u);
            st4(rU + o, n0);
            if (a.r16 != nullptr) {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (j0 + e < W) emit16(a.r16, a.r16lo, a.ld16, i, j0 + e, n0[e]);
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            yvp[e] = yv[e];
            cu[e] = nu[e];
            nu[e] = mu[e];
        }
        rc = rn;
    }
    double v[3] = {rr.value(), rzo.value(), su.value()}, tot[3];
    if (grid_reduce<3>(v, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        const double rr_range = range_part(tot[0], tot[2], a.H, a.W);
        st->rr = rr_range;
        st->rz_v = 0.0;
        st->rz_old = tot[1];
        st->rnorm_u = sqrt(tot[0]);
        const int itn = st->iter + 1;
        st->iter = itn;
        const double rel = st->bb > 0.0 ? sqrt(rr_range / st->bb) : 0.0;
        st->rel = rel;
        if (rel * rel <= a.tol2 || itn >= a.cg_max || !isfinite(rel)) st->done = 1;
        if (!isfinite(rel)) st->status |= ST_NONFINITE;
    }
}

// After the solve: V = (D U - G) / (1 + tau D) on every edge (the V rows of the system).
__global__ void __launch_bounds__(kThreads)
k_schur_recover_v(Planes P, StencilArgs a) {
    const int H = a.H, W = a.W, ld = a.ld;
    const int j = blockIdx.x * kThreads + threadIdx.x;
    const int i0 = blockIdx.y * kRows, i1 = strip_rows(H, i0);
    if (j >= W) return;
    for (int i = i0; i < i1; ++i) {
        const size_t o = (size_t)i * ld + j;
        const float u = P.U[o];
        if (i + 1 < H) P.Vv[o] = (P.U[o + ld] - u - P.Gv[o]) / (1.f + a.tau * P.dv[o]);
        if (j + 1 < W) P.Vh[o] = (P.U[o + 1] - u - P.Gh[o]) / (1.f + a.tau * P.dh[o]);
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

dim3 vec_grid(int H, int W, int rows) {
    return dim3((W + kThreads * kVec - 1) / (kThreads * kVec), (H + rows - 1) / rows);
}

}  // namespace

void strip_dims(int H, int W, int& gx, int& gy) {
    dim3 g = strip_grid(H, W);
    gx = (int)g.x;
    gy = (int)g.y;
}

void vec_dims(int H, int W, int dir_rows, int upd_rows, int& gx, int& gy_dir, int& gy_upd) {
    dim3 g = vec_grid(H, W, dir_rows);
    gx = (int)g.x;
    gy_dir = (int)g.y;
    gy_upd = (int)vec_grid(H, W, upd_rows).y;
}

cudaError_t launch_init_batched(const TileRec* recs, int T, int total, cudaStream_t s) {
    kb_init<<<total, kThreads, 0, s>>>(recs, T);
    return cudaGetLastError();
}

cudaError_t launch_bnorm_batched(const TileRec* recs, int T, int total, cudaStream_t s) {
    kb_bnorm<<<total, kThreads, 0, s>>>(recs, T);
    return cudaGetLastError();
}

cudaError_t launch_reweight_batched(const TileRec* recs, int T, int total_rw, cudaStream_t s) {
    kb_reweight<<<total_rw, kThreads, 0, s>>>(recs, T);
    return cudaGetLastError();
}

cudaError_t launch_direction_batched(const TileRec* recs, int T, int total, int rows,
                                     cudaStream_t s) {
    switch (rows) {
        case 8: kb_direction<8><<<total, kThreads, 0, s>>>(recs, T); break;
        case 16: kb_direction<16><<<total, kThreads, 0, s>>>(recs, T); break;
        case 24: kb_direction<24><<<total, kThreads, 0, s>>>(recs, T); break;
        case 32: kb_direction<32><<<total, kThreads, 0, s>>>(recs, T); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_update_batched(const TileRec* recs, int T, int total, int rows,
                                  cudaStream_t s) {
    switch (rows) {
        case 8: kb_update<8><<<total, kThreads, 0, s>>>(recs, T); break;
        case 16: kb_update<16><<<total, kThreads, 0, s>>>(recs, T); break;
        case 24: kb_update<24><<<total, kThreads, 0, s>>>(recs, T); break;
        case 32: kb_update<32><<<total, kThreads, 0, s>>>(recs, T); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize_batched(const TileRec* recs, int T, int total, int total_fin,
                                    cudaStream_t s) {
    kb_finalize<<<total_fin, kThreads, 0, s>>>(recs, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kb_subtract_mean<<<total, kThreads, 0, s>>>(recs, T);
    return cudaGetLastError();
}

cudaError_t launch_count_active(const DevState* states, int T, int* out, cudaStream_t s) {
    k_count_active<<<1, 256, 0, s>>>(states, T, out);
    return cudaGetLastError();
}

int wave_rows(int kernel, int H, int W, int max_rows) {
    static const void* const fn[6] = {(const void*)k_direction_pap<0>, (const void*)k_update<0>,
                                      (const void*)k_reweight_residual<0>,
                                      (const void*)k_finalize_reduce<0>,
                                      (const void*)k_schur_direction<0>,
                                      (const void*)k_schur_update<0>};
    if (kernel < 0 || kernel > 5 || H < 1 || W < 1) return 0;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn[kernel], kThreads, 0) !=
            cudaSuccess || sms < 1 || per < 1)
        return 0;
    const int gx = (int)vec_grid(H, W, kMinTileRows).x;
    const long long slots = (long long)sms * per;
    // the fewest waves k whose row strips (k slots / gx of them) need at most max_rows rows each
    for (int k = 1; k <= 64; ++k) {
        const long long strips = k * slots / gx;
        if (strips < 1) continue;
        const int r = (int)((H + strips - 1) / strips);
        if (r > max_rows) continue;
        if (r < kMinTileRows) return 0;
        return r;
    }
    return 0;
}

int aux_rows(int kernel, int H, int W) {
    const int r = wave_rows(kernel, H, W, kMaxTileRows);
    return r ? r : kDefaultUpdRows;
}

int stencil_grid_blocks(int H, int W) {
    dim3 g = strip_grid(H, W), v = vec_grid(H, W, std::min({kDirRows, kUpdRows, kSchurRows,
                                                           kTileRows[0]}));
    return (int)std::max(g.x * g.y, v.x * v.y);
}

namespace {

// The direction and update kernels for a runtime row count (one of kTileRows; the defaults
// otherwise).
template <template <int> class K, typename... Args>
cudaError_t launch_rows(int rows, int H, int W, cudaStream_t s, Args... args) {
    switch (rows) {
        case 8: K<8>::go(vec_grid(H, W, 8), s, args...); break;
        case 16: K<16>::go(vec_grid(H, W, 16), s, args...); break;
        case 24: K<24>::go(vec_grid(H, W, 24), s, args...); break;
        case 32: K<32>::go(vec_grid(H, W, 32), s, args...); break;
        default:
            // any other count in range: the runtime-rows instance (the count travels in the
            // kernel's arguments)
            if (!plan_rows_ok(rows)) return cudaErrorInvalidValue;
            K<0>::go(vec_grid(H, W, rows), s, args...);
            break;
    }
    return cudaGetLastError();
}


template <int R>
struct DirK {
    static void go(dim3 g, cudaStream_t s, Planes P, StencilArgs a, DevState* st, double* pa) {
        k_direction_pap<R><<<g, kThreads, 0, s>>>(P, a, st, pa);
    }
};

template <int R>
struct UpdK {
    static void go(dim3 g, cudaStream_t s, Planes P, StencilArgs a, DevState* st, double* pa) {
        k_update<R><<<g, kThreads, 0, s>>>(P, a, st, pa);
    }
};

template <int R>
struct RwK {
    static void go(dim3 g, cudaStream_t s, Planes P, StencilArgs a, DevState* st, double* pa) {
        k_reweight_residual<R><<<g, kThreads, 0, s>>>(P, a, st, pa);
    }
};

template <int R>
struct FinK {
    static void go(dim3 g, cudaStream_t s, Planes P, StencilArgs a, DevState* st, double* pa) {
        k_finalize_reduce<R><<<g, kThreads, 0, s>>>(P, a, st, pa);
    }
};

int rows_or(int r, int dflt) { return plan_rows_ok(r) ? r : dflt; }

}  // namespace

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

cudaError_t launch_norm_u(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                          cudaStream_t s) {
    k_norm_u<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_reweight_residual(const Planes& P, const StencilArgs& a, DevState* st,
                                     double* partials, cudaStream_t s) {
    StencilArgs b = a;
    b.rw_rows = plan_rows_ok(a.rw_rows) ? a.rw_rows : rows_or(a.upd_rows, kUpdRows);
    return launch_rows<RwK>(b.rw_rows, a.H, a.W, s, P, b, st, partials);
}

cudaError_t launch_direction_pap(const Planes& P, const StencilArgs& a, DevState* st,
                                 double* partials, cudaStream_t s) {
    StencilArgs b = a;
    b.dir_rows = rows_or(a.dir_rows, kDirRows);
    return launch_rows<DirK>(b.dir_rows, a.H, a.W, s, P, b, st, partials);
}

cudaError_t launch_update(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                          cudaStream_t s) {
    StencilArgs b = a;
    b.upd_rows = rows_or(a.upd_rows, kUpdRows);
    return launch_rows<UpdK>(b.upd_rows, a.H, a.W, s, P, b, st, partials);
}

cudaError_t launch_schur_reweight(const Planes& P, const StencilArgs& a, DevState* st,
                                  double* partials, cudaStream_t s) {
    k_schur_reweight<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, st, partials);
    return cudaGetLastError();
}

// U-only CG kernels: the plan's whole-wave row counts (a.sdir_rows, a.supd_rows), else 24 rows
cudaError_t launch_schur_direction(const Planes& P, const StencilArgs& a, DevState* st,
                                   double* partials, cudaStream_t s) {
    const int rows = plan_rows_ok(a.sdir_rows) ? a.sdir_rows : kSchurRows;
    if (rows == kSchurRows)
        k_schur_direction<kSchurRows><<<vec_grid(a.H, a.W, rows), kThreads, 0, s>>>(P, a, st,
                                                                                   partials);
    else
        k_schur_direction<0><<<vec_grid(a.H, a.W, rows), kThreads, 0, s>>>(P, a, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_schur_update(const Planes& P, const StencilArgs& a, DevState* st,
                                double* partials, cudaStream_t s) {
    const int rows = plan_rows_ok(a.supd_rows) ? a.supd_rows : kSchurRows;
    if (rows == kSchurRows)
        k_schur_update<kSchurRows><<<vec_grid(a.H, a.W, rows), kThreads, 0, s>>>(P, a, st,
                                                                                partials);
    else
        k_schur_update<0><<<vec_grid(a.H, a.W, rows), kThreads, 0, s>>>(P, a, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_schur_recover_v(const Planes& P, const StencilArgs& a, cudaStream_t s) {
    k_schur_recover_v<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                            cudaStream_t s) {
    StencilArgs b = a;
    b.fin_rows = plan_rows_ok(a.fin_rows) ? a.fin_rows : rows_or(a.upd_rows, kUpdRows);
    cudaError_t e = launch_rows<FinK>(b.fin_rows, a.H, a.W, s, P, b, st, partials);
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

cudaError_t launch_record_step(DevState* st, cudaStream_t s) {
    k_record_step<<<1, 1, 0, s>>>(st);
    return cudaGetLastError();
}

cudaError_t launch_adj_init(const Planes& P, const StencilArgs& a, const float* dLdU, DevState* st,
                            double* partials, cudaStream_t s) {
    k_user_mean<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(dLdU, a.H, a.W, st, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_init<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, dLdU, st);
    return cudaGetLastError();
}

cudaError_t launch_adj_setup_schur(const Planes& P, const StencilArgs& a, const float* Vkv,
                                   const float* Vkh, const float* Cv, const float* Ch,
                                   DevState* st, double* partials, cudaStream_t s) {
    k_adj_setup_schur<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, Vkv, Vkh, Cv, Ch, st,
                                                                 partials);
    return cudaGetLastError();
}

cudaError_t launch_adj_recover_v(const Planes& P, const StencilArgs& a, const DevState* st,
                                 cudaStream_t s) {
    k_adj_recover_v<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, st);
    return cudaGetLastError();
}

cudaError_t launch_adj_norm(const Planes& P, const StencilArgs& a, DevState* st, double* partials,
                            cudaStream_t s) {
    k_adj_norm<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, st, partials);
    return cudaGetLastError();
}

cudaError_t launch_adj_accumulate(const Planes& P, const StencilArgs& a, const float* Vkv,
                                  const float* Vkh, const float* Vnv, const float* Vnh,
                                  const float* Cv, const float* Ch, float* Gbv, float* Gbh,
                                  float* Cbv, float* Cbh, const DevState* st, cudaStream_t s) {
    k_adj_accumulate<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, Vkv, Vkh, Vnv, Vnh, Cv, Ch,
                                                               Gbv, Gbh, Cbv, Cbh, st);
    return cudaGetLastError();
}

cudaError_t launch_adj_final(const Planes& P, const StencilArgs& a, const float* Gbv,
                             const float* Gbh, const float* Cbv, const float* Cbh, float* dX,
                             float* dcoh, const DevState* st, cudaStream_t s) {
    k_adj_final<<<strip_grid(a.H, a.W), kThreads, 0, s>>>(P, a, Gbv, Gbh, Cbv, Cbh, dX, dcoh, st);
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
    return launch_update(P, b, st, partials, s);
}

}  // namespace irls
