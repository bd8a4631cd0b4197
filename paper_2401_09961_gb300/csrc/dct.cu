// Laplacian block of the preconditioner (Sec. 3.3 of arXiv 2401.09961):
//   S^T S Z + Z T T^T = tau R   solved as   Z = P_S [ (P_S^T tau R P_T) / (l_i + m_j) ] P_T^T
// with the zero-frequency coefficient set to 0 (the pseudo-inverse choice of Appendix B).
// P_S, P_T are the orthonormal DCT-II eigenvector matrices of the 1-D Neumann Laplacians, built
// once per plan from the closed form P[i][k] = c_k cos(pi k (2i+1) / 2N).
//
// The four dense products are all computed as "TN" GEMMs C[m][n] = sum_k A[m][k] B[n][k] with
// both operands K-contiguous; stages 1 and 3 store their result transposed so that the next
// stage again contracts over a contiguous index:
//   stage 1: T1[l][i] = sum_j R[i][j]  PMT[l][j]        ( = (R P_T)^T )
//   stage 2: T2[l][k] = tau sum_i T1[l][i] PNT[k][i] / (m_l + l_k)   ( = (P_S^T R P_T)^T / eig )
//   stage 3: T1[i][l] = sum_k T2[l][k] PN[i][k]         ( = P_S Z' , stored transposed back)
//   stage 4: Z[i][j]  = sum_l T1[i][l] PM[j][l]         ( = P_S Z' P_T^T )
// The last stage can also reduce rho = r_U^T z_U + r_V^T z_V and form the next CG ratio beta.
#include <algorithm>

#include "irls_internal.cuh"
#include "reduce.cuh"

namespace irls {

cudaError_t umma_dct_apply(const DctPlan& d, const float* rU, float* zU, int ld, DevState* st,
                           int reduce_rho, const StencilArgs& a, double* partials,
                           int skip_if_done, cudaStream_t s);
size_t umma_dct_bytes(int H, int W, int prec);
cudaError_t umma_dct_setup(DctPlan& d, char* mem);
void umma_dct_release(DctPlan& d);
cudaError_t umma_dct_reset(const DctPlan& d, cudaStream_t s);
bool umma_dct_stall(DctPlan& d, int on);

namespace {

constexpr int BM = 128, BN = 128, BK = 8;

enum Epi : int { EPI_TRANS = 0, EPI_EIG = 1, EPI_ZU = 2, EPI_ZU_RHO = 3 };

struct EpiArgs {
    float* C;          // output
    int ldc;
    int vm, vn;        // valid extents (EPI_EIG: W, H; EPI_ZU: H, W)
    const float* lam_m;
    const float* lam_n;
    float scale;       // tau (EPI_EIG)
    const float* rU;   // EPI_ZU_RHO: residual plane, pitch ldc
    DevState* st;
    double* partials;
    int flexible;
};

// C[m][n] = sum_k A[m][k] B[n][k], M and N multiples of 128; A rows >= a_rows and k >= K read 0.
template <int EPI>
__global__ void __launch_bounds__(256)
k_gemm_tn_f32(const float* __restrict__ A, int lda, int a_rows, const float* __restrict__ B,
              int ldb, int K, EpiArgs ep, int skip_if_done) {
    if (skip_if_done && ep.st != nullptr && ep.st->done) return;
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    // loader mapping: 128 rows x 8 k per operand; thread -> (row, 4 consecutive k)
    const int lr = tid >> 1, lk = (tid & 1) * 4;
    const bool arow = (m0 + lr) < a_rows;
    const float* Ap = A + (size_t)(m0 + lr) * lda;
    const float* Bp = B + (size_t)(n0 + lr) * ldb;

    auto load4 = [&](const float* p, bool rowok, int k, float (&r)[4]) {
        if (rowok && k + 3 < K) {
            float4 v = *reinterpret_cast<const float4*>(p + k);
            r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) r[c] = (rowok && k + c < K) ? p[k + c] : 0.f;
        }
    };

    float ra[4], rb[4];
    load4(Ap, arow, lk, ra);
    load4(Bp, true, lk, rb);
#pragma unroll
    for (int c = 0; c < 4; ++c) { As[0][lk + c][lr] = ra[c]; Bs[0][lk + c][lr] = rb[c]; }
    __syncthreads();

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

    const int nk = (K + BK - 1) / BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            load4(Ap, arow, (kt + 1) * BK + lk, ra);
            load4(Bp, true, (kt + 1) * BK + lk, rb);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (kt + 1 < nk) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                As[buf ^ 1][lk + c][lr] = ra[c];
                Bs[buf ^ 1][lk + c][lr] = rb[c];
            }
        }
        __syncthreads();
    }

    CSum part;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        float row = 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            const float v = acc[i][j];
            if constexpr (EPI == EPI_TRANS) {
                ep.C[(size_t)n * ep.ldc + m] = v;
            } else if constexpr (EPI == EPI_EIG) {
                float o = 0.f;
                if (m < ep.vm && n < ep.vn && (m | n) != 0) o = ep.scale * v / (ep.lam_m[m] + ep.lam_n[n]);
                ep.C[(size_t)m * ep.ldc + n] = o;
            } else {
                if (m < ep.vm && n < ep.vn) {
                    ep.C[(size_t)m * ep.ldc + n] = v;
                    if constexpr (EPI == EPI_ZU_RHO) row += ep.rU[(size_t)m * ep.ldc + n] * v;
                }
            }
        }
        if constexpr (EPI == EPI_ZU_RHO) part.add(row);
    }
    if constexpr (EPI == EPI_ZU_RHO) {
        double vv[1] = {part.value()}, tot[1];
        const Blk blk = single_blk();
        if (grid_reduce<1>(vv, ep.partials, &ep.st->counter, tot, blk.nblk, blk.bid) && tid == 0) {
            DevState* st = ep.st;
            const double rho_new = tot[0] + st->rz_v;
            if (!(rho_new > 0.0) || !isfinite(rho_new)) {
                // rho <= 0 is a breakdown unless the residual is already at the accuracy
                // rounding allows (relative 1e-3 and below)
                if (st->rel > 1e-3 || !isfinite(rho_new)) st->status |= ST_BREAKDOWN;
                st->done = 1;
            } else if (st->p_fresh) {
                st->rho = rho_new;
                st->beta = 0.0;
            } else {
                const double num = ep.flexible ? rho_new - st->rz_old : rho_new;
                st->beta = num / st->rho;
                st->rho = rho_new;
            }
        }
    }
}

// P[i][k] = c_k cos(pi k (2i+1) / (2N)) and its transpose, zero-padded to Np x Np.  The
// argument is reduced exactly in integers before the FP64 cospi.
__global__ void k_build_basis(float* P, float* PT, __nv_bfloat16* P16, __nv_bfloat16* PT16, int N,
                              int Np) {
    const size_t total = (size_t)Np * Np;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / Np), k = (int)(t % Np);
        double v = 0.0;
        if (i < N && k < N) {
            const long long m = ((long long)(2 * i + 1) * k) % (4LL * N);
            const double ck = k == 0 ? sqrt(1.0 / N) : sqrt(2.0 / N);
            v = ck * cospi((double)m / (2.0 * N));
        }
        if (P) P[(size_t)i * Np + k] = (float)v;
        if (PT) PT[(size_t)k * Np + i] = (float)v;
        if (P16) P16[(size_t)i * Np + k] = __double2bfloat16(v);
        if (PT16) PT16[(size_t)k * Np + i] = __double2bfloat16(v);
    }
}

// Eigenvalues l_k = 2 - 2 cos(pi k / N) = 4 sin^2(pi k / 2N) of S^T S (Sec. 3.3), zero-padded.
__global__ void k_build_lambda(float* lam, int N, int Np) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Np; k += gridDim.x * blockDim.x) {
        double v = 0.0;
        if (k < N) {
            const double s = sinpi((double)k / (2.0 * N));
            v = 4.0 * s * s;
        }
        lam[k] = (float)v;
    }
}

inline int rup(int x, int m) { return (x + m - 1) / m * m; }

template <int EPI>
cudaError_t gemm(const float* A, int lda, int a_rows, const float* B, int ldb, int M, int N, int K,
                 const EpiArgs& ep, int skip, cudaStream_t s) {
    dim3 grid(N / BN, M / BM);
    k_gemm_tn_f32<EPI><<<grid, 256, 0, s>>>(A, lda, a_rows, B, ldb, K, ep, skip);
    return cudaGetLastError();
}

}  // namespace

int dct_max_blocks(int H, int W) { return (rup(H, 128) / 128) * (rup(W, 128) / 128); }

size_t dct_bytes(int H, int W, int prec) {
    const size_t Hp = rup(H, 128), Wp = rup(W, 128);
    size_t n = 2 * Hp * Hp + Hp + Wp + 2 * Hp * Wp;
    if (H != W) n += 2 * Wp * Wp;
    size_t bytes = n * sizeof(float) + 4096;
    if (prec != IRLS_PREC_FP32) bytes += umma_dct_bytes(H, W, prec);
    return bytes + fft_dct_bytes(H, W);   // the fast-transform tables at the tail
}

cudaError_t dct_setup(DctPlan& d, int H, int W, int prec, float tau, char* mem) {
    d.H = H; d.W = W; d.Hp = rup(H, 128); d.Wp = rup(W, 128); d.prec = prec; d.tau = tau;
    const size_t Hp = d.Hp, Wp = d.Wp;
    float* f = reinterpret_cast<float*>(mem);
    d.PN = f; f += Hp * Hp;
    d.PNT = f; f += Hp * Hp;
    if (H != W) { d.PM = f; f += Wp * Wp; d.PMT = f; f += Wp * Wp; }
    else { d.PM = d.PN; d.PMT = d.PNT; }
    d.lamN = f; f += Hp;
    d.lamM = (H != W) ? f : d.lamN;
    f += Wp;
    d.T1 = f; f += Hp * Wp;
    d.T2 = f; f += Hp * Wp;
    k_build_basis<<<1024, 256>>>(d.PN, d.PNT, nullptr, nullptr, H, d.Hp);
    if (H != W) k_build_basis<<<1024, 256>>>(d.PM, d.PMT, nullptr, nullptr, W, d.Wp);
    k_build_lambda<<<8, 256>>>(d.lamN, H, d.Hp);
    if (H != W) k_build_lambda<<<8, 256>>>(d.lamM, W, d.Wp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    d.umma_ok = 0;
    d.fft = 0;
    {
        char* mt = mem + (dct_bytes(H, W, prec) - fft_dct_bytes(H, W));
        mt = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(mt) + 255) & ~uintptr_t(255));
        if ((e = fft_dct_setup(d, mt)) != cudaSuccess) return e;
    }
    if (prec != IRLS_PREC_FP32) {
        char* m16 = mem + (dct_bytes(H, W, IRLS_PREC_FP32) - fft_dct_bytes(H, W) - 4096);
        m16 = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(m16) + 1023) & ~uintptr_t(1023));
        e = umma_dct_setup(d, m16);
    }
    return e;
}

void dct_release(DctPlan& d) { umma_dct_release(d); }
cudaError_t dct_reset(const DctPlan& d, cudaStream_t s) { return umma_dct_reset(d, s); }
bool dct_stall(DctPlan& d, int on) { return umma_dct_stall(d, on); }

cudaError_t dct_apply(const DctPlan& d, const float* rU, float* zU, int ld, DevState* st,
                      int reduce_rho, const StencilArgs& a, double* partials, int skip_if_done,
                      cudaStream_t s) {
    if (d.fft) return fft_dct_apply(d, rU, zU, ld, st, reduce_rho, a, partials, skip_if_done, s);
    if (d.prec != IRLS_PREC_FP32)
        return umma_dct_apply(d, rU, zU, ld, st, reduce_rho, a, partials, skip_if_done, s);
    const int H = d.H, W = d.W, Hp = d.Hp, Wp = d.Wp;
    cudaError_t e;
    EpiArgs ep{};
    ep.st = st;
    ep.partials = partials;
    ep.flexible = a.flexible;
    // stage 1: T1[l][i] = sum_j R[i][j] PMT[l][j]
    ep.C = d.T1; ep.ldc = Hp;
    e = gemm<EPI_TRANS>(rU, ld, H, d.PMT, Wp, Hp, Wp, W, ep, skip_if_done, s);
    if (e != cudaSuccess) return e;
    // stage 2: T2[l][k] = tau sum_i T1[l][i] PNT[k][i] / (m_l + l_k), (0,0) -> 0
    ep.C = d.T2; ep.ldc = Hp; ep.vm = W; ep.vn = H; ep.lam_m = d.lamM; ep.lam_n = d.lamN;
    ep.scale = d.tau;
    e = gemm<EPI_EIG>(d.T1, Hp, Wp, d.PNT, Hp, Wp, Hp, H, ep, skip_if_done, s);
    if (e != cudaSuccess) return e;
    // stage 3: T1[i][l] = sum_k T2[l][k] PN[i][k]
    ep.C = d.T1; ep.ldc = Wp;
    e = gemm<EPI_TRANS>(d.T2, Hp, Wp, d.PN, Hp, Wp, Hp, H, ep, skip_if_done, s);
    if (e != cudaSuccess) return e;
    // stage 4: Z[i][j] = sum_l T1[i][l] PM[j][l]
    ep.C = zU; ep.ldc = ld; ep.vm = H; ep.vn = W; ep.rU = rU;
    if (reduce_rho)
        e = gemm<EPI_ZU_RHO>(d.T1, Wp, Hp, d.PM, Wp, Hp, Wp, W, ep, skip_if_done, s);
    else
        e = gemm<EPI_ZU>(d.T1, Wp, Hp, d.PM, Wp, Hp, Wp, W, ep, skip_if_done, s);
    return e;
}

// Floats of scratch that dct_apply_fp32_scratch needs for an H x W image.
size_t dct_scratch_floats(int H, int W) {
    const size_t Hp = rup(H, 128), Wp = rup(W, 128);
    size_t n = 2 * Hp * Hp + Hp + 3 * Hp * Wp;
    if (H != W) n += 2 * Wp * Wp + Wp;
    return n;
}

// The float32 Laplacian preconditioner on caller-provided scratch: builds the DCT bases into
// `work`, copies R into a 128-aligned pitch, runs the four products and writes Z (pitch W).
// Every scratch element that is read is written earlier in the same call.
cudaError_t dct_apply_fp32_scratch(const float* R, float* Z, int H, int W, float tau, float* work,
                                   cudaStream_t s) {
    const int Hp = rup(H, 128), Wp = rup(W, 128);
    float* f = work;
    float* PN = f; f += (size_t)Hp * Hp;
    float* PNT = f; f += (size_t)Hp * Hp;
    float *PM = PN, *PMT = PNT;
    if (H != W) { PM = f; f += (size_t)Wp * Wp; PMT = f; f += (size_t)Wp * Wp; }
    float* lamN = f; f += Hp;
    float* lamM = lamN;
    if (H != W) { lamM = f; f += Wp; }
    float* T1 = f; f += (size_t)Hp * Wp;
    float* T2 = f; f += (size_t)Hp * Wp;
    float* Rp = f;
    k_build_basis<<<256, 256, 0, s>>>(PN, PNT, nullptr, nullptr, H, Hp);
    if (H != W) k_build_basis<<<256, 256, 0, s>>>(PM, PMT, nullptr, nullptr, W, Wp);
    k_build_lambda<<<2, 256, 0, s>>>(lamN, H, Hp);
    if (H != W) k_build_lambda<<<2, 256, 0, s>>>(lamM, W, Wp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = launch_copy_in(R, H, W, Rp, Wp, s)) != cudaSuccess) return e;
    EpiArgs ep{};
    ep.C = T1; ep.ldc = Hp;
    if ((e = gemm<EPI_TRANS>(Rp, Wp, H, PMT, Wp, Hp, Wp, W, ep, 0, s)) != cudaSuccess) return e;
    ep.C = T2; ep.ldc = Hp; ep.vm = W; ep.vn = H; ep.lam_m = lamM; ep.lam_n = lamN; ep.scale = tau;
    if ((e = gemm<EPI_EIG>(T1, Hp, Wp, PNT, Hp, Wp, Hp, H, ep, 0, s)) != cudaSuccess) return e;
    ep.C = T1; ep.ldc = Wp;
    if ((e = gemm<EPI_TRANS>(T2, Hp, Wp, PN, Hp, Wp, Hp, H, ep, 0, s)) != cudaSuccess) return e;
    ep.C = Z; ep.ldc = W; ep.vm = H; ep.vn = W;
    return gemm<EPI_ZU>(T1, Wp, Hp, PM, Wp, Hp, Wp, W, ep, 0, s);
}

}  // namespace irls
