// Tensor-core form of the Laplacian preconditioner block (Sec. 3.3 of arXiv 2401.09961): the
// four dense products P_S^T R P_T and P_S Z' P_T^T on sm_103a tcgen05 tensor cores, bfloat16
// (or float16) operands with float32 accumulation in tensor memory.
//
// Every stage is a "TN" GEMM  D[m][n] = sum_k A[m][k] B[n][k]  with both operands K-contiguous,
// arranged so that each stage's output is again K-contiguous for the next one:
//   stage 1: T1[l][i] = sum_j PMT[l][j] R[i][j]                     (= (R P_T)^T)
//   stage 2: T2[l][k] = tau sum_i T1[l][i] PNT[k][i] / (m_l + l_k)  (= ((P_S^T R P_T) / eig)^T)
//   stage 3: T3[i][l] = sum_k PN[i][k] T2[l][k]                     (= P_S Z')
//   stage 4: Z[i][j]  = sum_l T3[i][l] PM[j][l]                     (= P_S Z' P_T^T)
//
// Two forms share the building blocks below.  The direct form (any side; operands padded to
// multiples of 128) and the grouped batched form run one output tile per CTA, structured as
// follows.  The folded form (sides >= 256) runs one persistent CTA-pair kernel over all four
// stages (k2_fold_fused, tcgen05.mma.cta_group::2, further down), with half the multiply-adds.
//
// Kernel structure of the direct form (one 128 x BN output tile per CTA, 128 threads):
//   warp 0 lane 0  TMA producer: cp.async.bulk.tensor 2-D loads (128-byte swizzle) of the
//                  128 x 64 A tile and the BN x 64 B tile into a ring of shared-memory stages,
//                  each guarded by a full / empty mbarrier pair;
//   warp 1 lane 0  MMA issuer: 4 x tcgen05.mma (K = 16 each) per stage into a 128 x BN fp32
//                  accumulator in tensor memory, tcgen05.commit frees the stage;
//   warp 2         allocates / frees the tensor-memory columns;
//   all 4 warps    epilogue: tcgen05.ld of their 32 accumulator lanes, fused scaling
//                  (eigenvalue divide, zero-frequency drop), conversion and store; the last stage
//                  also reduces r_U^T z_U and forms the CG ratio beta (Alg. 2).
// Every mbarrier wait is bounded by a clock budget; on expiry the kernel flags ST_TIMEOUT, stops
// the CG run, releases its tensor memory and returns.
//
// Split precision (IRLS_PREC_BF16X3): every float32 operand x is carried as two bfloat16 parts,
// hi = bf16(x) and lo = bf16(x - hi), and each product is formed as
// A_hi B_hi + A_hi B_lo + A_lo B_hi in the same float32 accumulator (the dropped A_lo B_lo term
// and the residual of the split are below 2^-16 relative).  A single bfloat16 pass rounds at
// 2^-9, and that error, leaked into the lowest frequencies by the forward transform, is
// amplified by tau / (l_i + m_j) (about 1e4 at 4096 x 4096): the inner CG then stalls.
//
// Float16 (IRLS_PREC_FP16, folded form only): one product per multiply-add on float16 operands
// (rounding 2^-11).  Its range is kept by scales known before each stage runs: the residual by
// sqrt(H W) / ||r_U||, stage 2's coefficient rows by (m_l + l_1) / tau (l_1 the smallest nonzero
// eigenvalue of the other side), which cancels the division's growth, and stage 4's basis by
// the inverse; see UEpiArgs.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "irls_internal.cuh"
#include "reduce.cuh"

namespace irls {

namespace {

constexpr int UBM = 128, UBK = 64;
constexpr int kUThreads = 128;
constexpr long long kWaitBudget = 4000000000LL;   // clock64 cycles (about 2 s at 2 GHz)

enum UEpi : int {
    UE_STORE16 = 0, UE_EIG16 = 1, UE_ZU = 2, UE_ZU_RHO = 3,
    // folded (even/odd) forms, two accumulators
    UE_FOLD16 = 4,        // out+ = acc0 + mirror(acc1), out- = acc0 - mirror(acc1)
    UE_UNFOLD16 = 5,      // row m: acc0 + acc1, row mrows-1-m: acc0 - acc1
    UE_UNFOLDZ = 6,       // col n: acc0 + acc1, col mcols-1-n: acc0 - acc1 (fp32)
    UE_EIG16_RHO = 8      // EIG16, plus r^T z formed from the spectral coefficients
};

struct UEpiArgs {
    void* C;             // bf16 output (STORE16 / EIG16) or float output (ZU)
    void* C_lo;          // bf16 low part of a split output, or null
    void* C2;            // second bf16 output (FOLD16: the differences)
    void* C2_lo;
    int ldc;
    int mrows, mcols;    // mirror extents (UNFOLD16: rows; UNFOLDZ: columns)
    int keep_origin;     // EIG16: keep the (0, 0) coefficient (a folded block that is not DC)
    int vm, vn;          // valid extents of the output
    const float* lam_m;
    const float* lam_n;
    float scale;
    const float* rU;     // residual plane (ZU_RHO), pitch ldc
    DevState* st;        // never null: error flags; rho / beta for ZU_RHO
    double* partials;
    int flexible;
    int skip_if_done;
    // EIG16_RHO in the CTA-pair kernels: the index of this problem's first tile among its
    // image's tiles, and the image's tile count (its problems are consecutive in the table)
    int rho_base, rho_count;
    // FOLD16 with an odd number of B rows: the middle row pairs with itself (its sum is the row
    // itself, not twice it); -1 otherwise
    int mid;
    // float16 operands (folded form): bf16 stores become float16 stores; stage 2 writes its
    // coefficients scaled per row by (mu_m + lam1) / tau (lam1: the smallest nonzero eigenvalue
    // of the other side), which cancels the division's growth; stage 4 (whose basis is scaled
    // by the inverse) undoes the residual's scale sqrt(H W) / ||r_U|| (inv_sqrt_n = 1/sqrt(H W))
    int f16;
    float lam1, inv_sqrt_n;
};

// 1 / (the residual's float16 scale) of the current application: ||r_U|| / sqrt(H W), or 1 for
// r_U = 0.  The kernel that produced r_U set ||r_U||; it does not change during the application.
__device__ __forceinline__ float f16_inv_scale(const UEpiArgs& ep) {
    const double rn = *(volatile const double*)&ep.st->rnorm_u;
    return rn > 0.0 ? (float)(rn * (double)ep.inv_sqrt_n) : 1.f;
}

template <int BN, int SA, int SB>
struct UCfg {
    static constexpr int kABytes = UBM * UBK * 2;             // one bf16 part of the A tile
    static constexpr int kBBytes = BN * UBK * 2;              // one bf16 part of the B tile
    static constexpr int kStageBytes = SA * kABytes + SB * kBBytes;
    static constexpr int kStages = (200 * 1024) / kStageBytes > 8 ? 8 : (200 * 1024) / kStageBytes;
    static constexpr int kSmem = kStages * kStageBytes + 1024 + 256;
    static constexpr uint32_t kTmemCols = BN;
    // instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A bf16 (7-9 = 1), B bf16
    // (10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
    static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                       ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(UBM >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on the given phase parity; false if the budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    if (mbar_try_wait(a, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(a, parity)) {
        if (clock64() - t0 > kWaitBudget) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns of tensor memory into 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with 128-byte swizzling:
// rows of 128 bytes, 8-row atoms 1024 bytes apart (stride byte offset), descriptor version 1,
// layout code 2 (SWIZZLE_128B).  The leading byte offset is unused for this layout.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr);

// The same for a tile written with 64-byte swizzling (rows of 64 bytes = 32 bf16 of K, 8-row
// atoms 512 bytes apart, layout code 4).
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

template <int KB>
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t saddr) {
    static_assert(KB == 64 || KB == 32, "K per stage");
    if constexpr (KB == 64) return desc_sw128(saddr);
    else return desc_sw64(saddr);
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
}

// 32 consecutive values of one row as bf16 (hi) and, with a lo plane, bf16(v - hi)
__device__ __forceinline__ void store_row32(void* hi, void* lo, size_t off, const float (&v)[32]) {
    uint4* dh = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(hi) + off);
    if (lo == nullptr) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4 w;
            w.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
            w.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
            w.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
            w.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
            dh[q] = w;
        }
        return;
    }
    uint4* dl = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(lo) + off);
    float h[32], l[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
        h[t] = __bfloat162float(__float2bfloat16_rn(v[t]));
        l[t] = v[t] - h[t];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint4 w, wl;
        w.x = pack_bf16(h[8 * q + 0], h[8 * q + 1]);
        w.y = pack_bf16(h[8 * q + 2], h[8 * q + 3]);
        w.z = pack_bf16(h[8 * q + 4], h[8 * q + 5]);
        w.w = pack_bf16(h[8 * q + 6], h[8 * q + 7]);
        wl.x = pack_bf16(l[8 * q + 0], l[8 * q + 1]);
        wl.y = pack_bf16(l[8 * q + 2], l[8 * q + 3]);
        wl.z = pack_bf16(l[8 * q + 4], l[8 * q + 5]);
        wl.w = pack_bf16(l[8 * q + 6], l[8 * q + 7]);
        dh[q] = w;
        dl[q] = wl;
    }
}

// rho = r_U^T z_U + r_V^T z_V and the CG ratio beta (Alg. 2), by the last block of the launch.
// `defer`: a launch whose later tiles still test the stop flag records the stop in stop_next,
// which the launch's last CTA moves to done once every tile has run.
__device__ __forceinline__ void finish_rho(const UEpiArgs& ep, double rz_u, bool defer = false) {
    DevState* st = ep.st;
    const double rho_new = rz_u + st->rz_v;
    if (!(rho_new > 0.0) || !isfinite(rho_new)) {
        // rho <= 0 is a breakdown unless the residual is already at the accuracy rounding
        // allows (relative 1e-3 and below)
        if (st->rel > 1e-3 || !isfinite(rho_new)) st->status |= ST_BREAKDOWN;
        if (defer) st->stop_next = 1;
        else st->done = 1;
    } else if (st->p_fresh) {
        st->rho = rho_new;
        st->beta = 0.0;
    } else {
        const double num = ep.flexible ? rho_new - st->rz_old : rho_new;
        st->beta = num / st->rho;
        st->rho = rho_new;
    }
}

// Epilogue of one 128 x BN output tile of the one-tile-per-CTA kernels (the direct form and the
// grouped batched form), for the accumulator row this thread holds: tl is the tensor-memory
// address of its lane at the accumulator's first column, m its output row, n0 the tile's first
// column.  ZU_RHO adds this thread's share of r^T z to `part`.
template <int BN, int EPI>
__device__ __forceinline__ void epi_tile(uint32_t tl, const UEpiArgs& ep, int m, int n0,
                                         CSum& part, int c_begin = 0, int c_end = BN / 32) {
#pragma unroll 1
    for (int c = c_begin; c < c_end; ++c) {
        uint32_t r[32];
        tmem_ld32(tl + (uint32_t)(c * 32), r);
        const int nb = n0 + c * 32;
        static_assert(EPI == UE_STORE16 || EPI == UE_EIG16 || EPI == UE_ZU || EPI == UE_ZU_RHO,
                      "one-tile-per-CTA kernels: direct-form epilogues");
        if constexpr (EPI == UE_STORE16 || EPI == UE_EIG16) {
            float v[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) v[t] = __uint_as_float(r[t]);
            if constexpr (EPI == UE_EIG16) {
                const bool rowok = m < ep.vm;
                const float lm = rowok ? ep.lam_m[m] : 0.f;
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const int n = nb + t;
                    const bool keep = rowok && n < ep.vn && (ep.keep_origin || (m | n) != 0);
                    v[t] = keep ? __fdividef(ep.scale * v[t], lm + __ldg(&ep.lam_n[n])) : 0.f;
                }
            }
            uint4* dst = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(ep.C) +
                                                  (size_t)m * ep.ldc + nb);
            if (ep.C_lo == nullptr) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint4 w;
                    w.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
                    w.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
                    w.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
                    w.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
                    dst[q] = w;
                }
            } else {
                uint4* dlo = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(ep.C_lo) +
                                                      (size_t)m * ep.ldc + nb);
                float lo[32];
#pragma unroll
                for (int t = 0; t < 32; ++t) {
                    const float h = __bfloat162float(__float2bfloat16_rn(v[t]));
                    lo[t] = v[t] - h;
                    v[t] = h;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint4 w, wl;
                    w.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
                    w.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
                    w.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
                    w.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
                    wl.x = pack_bf16(lo[8 * q + 0], lo[8 * q + 1]);
                    wl.y = pack_bf16(lo[8 * q + 2], lo[8 * q + 3]);
                    wl.z = pack_bf16(lo[8 * q + 4], lo[8 * q + 5]);
                    wl.w = pack_bf16(lo[8 * q + 6], lo[8 * q + 7]);
                    dst[q] = w;
                    dlo[q] = wl;
                }
            }
        } else {
            if (m < ep.vm) {
                float* out = static_cast<float*>(ep.C) + (size_t)m * ep.ldc;
                const float* rr = ep.rU + (size_t)m * ep.ldc;
                if (nb + 32 <= ep.vn) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float4 w = make_float4(__uint_as_float(r[4 * q]),
                                               __uint_as_float(r[4 * q + 1]),
                                               __uint_as_float(r[4 * q + 2]),
                                               __uint_as_float(r[4 * q + 3]));
                        reinterpret_cast<float4*>(out + nb)[q] = w;
                        if constexpr (EPI == UE_ZU_RHO) {
                            const float4 x = reinterpret_cast<const float4*>(rr + nb)[q];
                            part.add(x.x * w.x + x.y * w.y + x.z * w.z + x.w * w.w);
                        }
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 32; ++t) {
                        if (nb + t < ep.vn) {
                            const float z = __uint_as_float(r[t]);
                            out[nb + t] = z;
                            if constexpr (EPI == UE_ZU_RHO) part.add(rr[nb + t] * z);
                        }
                    }
                }
            }
        }
    }
}

// Per-warp shared-memory block for the coalesced epilogue: 32 rows x 32 columns (padded).
struct WarpScratch {
    float v[32][33];
};

// Each lane holds one row of a 32 x 32 block (32 consecutive columns); after this call row r is
// readable as s.v[r][column] by any lane of the warp.
__device__ __forceinline__ void scr_put(WarpScratch& s, const float (&v)[32]) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 32; ++t) s.v[lane][t] = v[t];
    __syncwarp();
}

// The block in `s` as bf16 (hi) and, with a lo plane, bf16(x - hi): two rows per instruction,
// each lane one bf16 pair, row r of the block at element offset row_off(r) + col0; rows at or
// beyond nrows are not written.
template <typename RowOff>
__device__ __forceinline__ void scr_store16(const WarpScratch& s, void* hi, void* lo, int col0,
                                            RowOff row_off, int nrows = 32, int f16 = 0) {
    const int lane = threadIdx.x & 31;
    const int rsub = lane >> 4, col = 2 * (lane & 15);
#pragma unroll 4
    for (int rr = 0; rr < 32; rr += 2) {
        const int row = rr + rsub;
        if (row >= nrows) continue;
        const float x0 = s.v[row][col], x1 = s.v[row][col + 1];
        const size_t off = row_off(row) + col0 + col;
        if (f16) {   // float16, one part
            *reinterpret_cast<__half2*>(static_cast<__half*>(hi) + off) = __floats2half2_rn(x0, x1);
            continue;
        }
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(hi) + off) = h;
        if (lo) {
            const float2 hf = __bfloat1622float2(h);
            *reinterpret_cast<__nv_bfloat162*>(static_cast<__nv_bfloat16*>(lo) + off) =
                __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
        }
    }
}

// The block in `s` as float32 rows at out + row_off(r) + col0 (four rows per instruction, one
// float4 per lane); with rU, adds rU . z over the block to `part`.  Only rows < nrows and block
// columns in [c_lo, c_hi) are written.  row_off(r) must be a multiple of 4 floats; groups that
// are partial, or not 16-byte aligned (col0 not a multiple of 4: the mirrored columns of an
// image whose width is not a multiple of 4), go element by element.
template <typename RowOff>
__device__ __forceinline__ void scr_store32(const WarpScratch& s, float* out, const float* rU,
                                            int col0, RowOff row_off, CSum& part, int nrows = 32,
                                            int c_lo = 0, int c_hi = 32) {
    const int lane = threadIdx.x & 31;
    const int rsub = lane >> 3, col = 4 * (lane & 7);
    const bool full = (col0 & 3) == 0 && col >= c_lo && col + 4 <= c_hi;
#pragma unroll 2
    for (int rr = 0; rr < 32; rr += 4) {
        const int row = rr + rsub;
        if (row >= nrows) continue;
        const size_t off = row_off(row) + col0 + col;
        if (full) {
            const float4 z = make_float4(s.v[row][col], s.v[row][col + 1], s.v[row][col + 2],
                                         s.v[row][col + 3]);
            *reinterpret_cast<float4*>(out + off) = z;
            if (rU) {
                const float4 x = *reinterpret_cast<const float4*>(rU + off);
                part.add(x.x * z.x + x.y * z.y + x.z * z.z + x.w * z.w);
            }
        } else {
            for (int e = 0; e < 4; ++e) {
                if (col + e < c_lo || col + e >= c_hi) continue;
                const float z = s.v[row][col + e];
                out[off + e] = z;
                if (rU) part.add(rU[off + e] * z);
            }
        }
    }
}

// Epilogue of the persistent kernels: as epi_tile, for the warp's 32 accumulator rows starting
// at output row m0w (this lane's row is m0w + lane), with coalesced stores through `s`.
template <int BN, int EPI>
__device__ __forceinline__ void epi_tile_t(uint32_t tl, const UEpiArgs& ep, int m0w, int n0,
                                           CSum& part, int c_begin, int c_end, WarpScratch& s) {
    const int lane = threadIdx.x & 31;
    const int m = m0w + lane;
    const size_t ldc = (size_t)ep.ldc;
    auto rows = [&](int r) { return (size_t)(m0w + r) * ldc; };
#pragma unroll 1
    for (int c = c_begin; c < c_end; ++c) {
        uint32_t r[32];
        tmem_ld32(tl + (uint32_t)(c * 32), r);
        const int nb = n0 + c * 32;
        if constexpr (EPI == UE_FOLD16) {
            // acc1 holds the mirrored tile: its column BN-1-x pairs with acc0's column x
            uint32_t r1[32];
            tmem_ld32(tl + (uint32_t)BN + (uint32_t)((BN / 32 - 1 - c) * 32), r1);
            float pl[32], mi[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                const float a = __uint_as_float(r[t]), b = __uint_as_float(r1[31 - t]);
                // columns beyond the half side (padding of a ragged half) are zero
                const bool ok = nb + t < ep.vn;
                const bool self = nb + t == ep.mid;
                pl[t] = ok ? (self ? a : a + b) : 0.f;
                mi[t] = ok && !self ? a - b : 0.f;
            }
            scr_put(s, pl);
            scr_store16(s, ep.C, ep.C_lo, nb, rows, 32, ep.f16);
            scr_put(s, mi);
            scr_store16(s, ep.C2, ep.C2_lo, nb, rows, 32, ep.f16);
        } else if constexpr (EPI == UE_UNFOLD16) {
            uint32_t r1[32];
            tmem_ld32(tl + (uint32_t)BN + (uint32_t)(c * 32), r1);
            float pl[32], mi[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                const float a = __uint_as_float(r[t]), b = __uint_as_float(r1[t]);
                pl[t] = a + b;
                mi[t] = a - b;
            }
            // rows at or beyond the half side (padding) have no mirror partner: not written
            const int nr = min(max(ep.vm - m0w, 0), 32);
            scr_put(s, pl);
            scr_store16(s, ep.C, ep.C_lo, nb, rows, nr, ep.f16);
            scr_put(s, mi);
            const int mr = ep.mrows - 1 - m0w;
            scr_store16(s, ep.C, ep.C_lo, nb, [&](int rr) { return (size_t)(mr - rr) * ldc; }, nr,
                        ep.f16);
        } else if constexpr (EPI == UE_UNFOLDZ) {
            uint32_t r1[32];
            tmem_ld32(tl + (uint32_t)BN + (uint32_t)(c * 32), r1);
            const int mb = ep.mcols - 32 - nb;   // first column of the mirrored 32
            const float us = ep.f16 ? f16_inv_scale(ep) : 1.f;
            float pl[32], mi[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) {
                pl[t] = (__uint_as_float(r[t]) + __uint_as_float(r1[t])) * us;            // nb + t
                mi[t] = (__uint_as_float(r[31 - t]) - __uint_as_float(r1[31 - t])) * us;  // mb + t
            }
            const float* rr = nullptr;   // r^T z is formed in stage 2
            // rows beyond the image and columns beyond the half side (padding) are not written;
            // the mirrored block holds column nb + t at position 31 - t
            const int nr = min(max(ep.vm - m0w, 0), 32);
            const int nc = min(max(ep.vn - nb, 0), 32);
            scr_put(s, pl);
            scr_store32(s, static_cast<float*>(ep.C), rr, nb, rows, part, nr, 0, nc);
            scr_put(s, mi);
            scr_store32(s, static_cast<float*>(ep.C), rr, mb, rows, part, nr, 32 - nc, 32);
        } else if constexpr (EPI == UE_STORE16 || EPI == UE_EIG16 || EPI == UE_EIG16_RHO) {
            float v[32];
#pragma unroll
            for (int t = 0; t < 32; ++t) v[t] = __uint_as_float(r[t]);
            if constexpr (EPI == UE_EIG16 || EPI == UE_EIG16_RHO) {
                const bool rowok = m < ep.vm;
                const float lm = rowok ? ep.lam_m[m] : 0.f;
#pragma unroll
                // float16: the row's coefficients times (lm + lam1) / tau (see UEpiArgs)
                const float rs = ep.f16 ? __fdividef(lm + ep.lam1, ep.scale) : 1.f;
                float q4 = 0.f;
                for (int t = 0; t < 32; ++t) {
                    const int n = nb + t;
                    const bool keep = rowok && n < ep.vn && (ep.keep_origin || (m | n) != 0);
                    const float f = v[t];
                    const float g = keep ? __fdividef(ep.scale * f, lm + __ldg(&ep.lam_n[n])) : 0.f;
                    v[t] = g * rs;
                    // r^T z = sum over frequencies of F * (tau F / eig) (P_N, P_M orthogonal);
                    // with float16 F and G carry the residual's scale, removed when rho is formed;
                    // partials of four frequencies go into the compensated sum
                    if constexpr (EPI == UE_EIG16_RHO) {
                        q4 += f * g;
                        if ((t & 3) == 3) {
                            part.add(q4);
                            q4 = 0.f;
                        }
                    }
                }
            }
            scr_put(s, v);
            scr_store16(s, ep.C, ep.C_lo, nb, rows, 32, ep.f16);
        } else {
            static_assert(EPI == UE_STORE16, "persistent kernels: folded and eigenvalue forms");
        }
    }
}

template <int BN, int EPI, int SA, int SB, int DUAL = 0>
__device__ __forceinline__ void umma_body(const CUtensorMap* tmA0, const CUtensorMap* tmA1,
                                          const CUtensorMap* tmB0, const CUtensorMap* tmB1,
                                          int K, const UEpiArgs& ep_ref, int m0, int n0,
                                          unsigned nblk, unsigned bid,
                                          const CUtensorMap* tmA2 = nullptr,
                                          const CUtensorMap* tmA3 = nullptr,
                                          const CUtensorMap* tmB2 = nullptr,
                                          const CUtensorMap* tmB3 = nullptr, int n0b1 = 0) {
    // DUAL: a second operand set (A2/A3, B2/B3 at B row n0b1) accumulates into TMEM columns
    // [BN, 2 BN); its K loop follows the first one through the same shared-memory ring
    using C = UCfg<BN, SA, SB>;
    constexpr uint32_t kCols = DUAL ? 2 * C::kTmemCols : C::kTmemCols;
    // a register copy: the epilogue's stores could alias a table in global memory, which would
    // force a reload of every argument after each store
    const UEpiArgs ep = ep_ref;
    if (ep.skip_if_done && ep.st->done) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::kStages * C::kStageBytes);
    uint64_t* empty = full + C::kStages;
    uint64_t* accf = empty + C::kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accf + 1);
    __shared__ int s_err;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = K / UBK;
    const int nkt = DUAL ? 2 * nkb : nkb;

    if (threadIdx.x == 0) {
        s_err = 0;
        for (int s = 0; s < C::kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accf, 1);
        fence_mbar_init();
    }
    if (warp == 2) tmem_alloc(tmem_slot, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            for (int kb = 0; kb < nkt; ++kb) {
                const int s = kb % C::kStages;
                const uint32_t ph = (uint32_t)(kb / C::kStages) & 1u;
                if (kb >= C::kStages && !mbar_wait(&empty[s], ph ^ 1u)) {
                    atomicExch(&s_err, 1);
                    break;
                }
                const bool second = DUAL && kb >= nkb;
                const int kc = (second ? kb - nkb : kb) * UBK;
                const int nb0 = second ? n0b1 : n0;
                uint8_t* sa = smem + s * C::kStageBytes;
                uint8_t* sb = sa + SA * C::kABytes;
                mbar_expect_tx(&full[s], C::kStageBytes);
                tma_load_2d(sa, second ? tmA2 : tmA0, &full[s], kc, m0);
                if constexpr (SA == 2)
                    tma_load_2d(sa + C::kABytes, second ? tmA3 : tmA1, &full[s], kc, m0);
                tma_load_2d(sb, second ? tmB2 : tmB0, &full[s], kc, nb0);
                if constexpr (SB == 2)
                    tma_load_2d(sb + C::kBBytes, second ? tmB3 : tmB1, &full[s], kc, nb0);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            for (int kb = 0; kb < nkt; ++kb) {
                const int s = kb % C::kStages;
                const uint32_t ph = (uint32_t)(kb / C::kStages) & 1u;
                if (!mbar_wait(&full[s], ph)) {
                    atomicExch(&s_err, 1);
                    break;
                }
                tc_fence_after();
                const bool second = DUAL && kb >= nkb;
                const int kk = second ? kb - nkb : kb;
                const uint32_t td = tmem + (second ? (uint32_t)BN : 0u);
                const uint32_t sa = smem_u32(smem + s * C::kStageBytes);
                const uint32_t sb = sa + SA * C::kABytes;
                const uint64_t da = desc_sw128(sa), db = desc_sw128(sb);
                const uint64_t dal = desc_sw128(sa + C::kABytes), dbl = desc_sw128(sb + C::kBBytes);
#pragma unroll
                for (int j = 0; j < UBK / 16; ++j) {   // K = 16 per MMA: +32 bytes (= 2 in >> 4)
                    if constexpr (SB == 2) umma_bf16(td, da + 2 * j, dbl + 2 * j, C::kIdesc, (kk | j) != 0);
                    if constexpr (SA == 2)
                        umma_bf16(td, dal + 2 * j, db + 2 * j, C::kIdesc, SB == 2 || (kk | j) != 0);
                    umma_bf16(td, da + 2 * j, db + 2 * j, C::kIdesc, SA == 2 || SB == 2 || (kk | j) != 0);
                }
                umma_commit(&empty[s]);
            }
            umma_commit(accf);
        }
        __syncwarp();
    }

    // ---- epilogue ----
    const bool ok = mbar_wait(accf, 0);
    tc_fence_after();
    __syncthreads();
    const bool good = ok && (*(volatile int*)&s_err == 0);
    if (!good && threadIdx.x == 0) {
        atomicOr(&ep.st->status, ST_TIMEOUT);
        ep.st->done = 1;
    }
    const int m = m0 + warp * 32 + lane;
    CSum part;
    if (good) epi_tile<BN, EPI>(tmem + ((uint32_t)(warp * 32) << 16), ep, m, n0, part);
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        tmem_dealloc(tmem, kCols);
    }
    if constexpr (EPI == UE_ZU_RHO) {
        double vv[1] = {part.value()}, tot[1];
        if (grid_reduce<1>(vv, ep.partials, &ep.st->counter, tot, nblk, bid) && threadIdx.x == 0)
            finish_rho(ep, tot[0]);
    }
}

template <int BN, int EPI, int SA, int SB>
__global__ void __launch_bounds__(kUThreads, 1)
k_umma_gemm(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
            const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
            int K, UEpiArgs ep) {
    umma_body<BN, EPI, SA, SB>(&tmA0, &tmA1, &tmB0, &tmB1, K, ep, blockIdx.y * UBM, blockIdx.x * BN,
                               gridDim.x * gridDim.y, blockIdx.x + gridDim.x * blockIdx.y);
}

// One problem of a grouped GEMM launch: its TMA descriptors (in global memory), shape,
// epilogue arguments and the index of its first CTA in the launch.
struct GemmTile {
    CUtensorMap a0, a1, b0, b1;
    CUtensorMap a2, a3, b2, b3;   // second operand set (dual-accumulator stages)
    UEpiArgs ep;
    int M, N, K;
    int blk0, gx;
    int mirror_b1;                // second set's B rows mirrored: nb_rows - n0 - 128
    int nb_rows;
    int epi, dual;                // fused folded launch: the problem's epilogue and operand sets
    CUtensorMap bh0, bh1, bh2, bh3;   // two-set problems: B maps with 64-row boxes (half tiles)
};

// Grouped GEMM: one launch over the output tiles of every problem (BN = 128).  A CTA finds its
// problem by a binary search over the first-CTA indices; problems whose CG run has stopped
// return at once (the per-problem convergence mask).
template <int EPI, int SA, int SB, int DUAL = 0>
__global__ void __launch_bounds__(kUThreads, 1)
kb_umma_gemm(const GemmTile* __restrict__ tiles, int T) {
    int lo = 0, hi = T - 1;
    const int bid = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tiles[mid].blk0 <= bid) lo = mid; else hi = mid - 1;
    }
    const GemmTile& g = tiles[lo];
    const int local = bid - g.blk0;
    const int m0 = (local / g.gx) * UBM, n0 = (local % g.gx) * 128;
    umma_body<128, EPI, SA, SB, DUAL>(&g.a0, &g.a1, &g.b0, &g.b1, g.K, g.ep, m0, n0,
                                      (unsigned)((g.M / UBM) * g.gx), (unsigned)local, &g.a2,
                                      &g.a3, &g.b2, &g.b3,
                                      g.mirror_b1 ? g.nb_rows - n0 - 128 : n0);
}

// ------------------------------------------------------------------------------------------
// helpers of the persistent (CTA-pair) form
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up as soon as another role of the CTA has flagged an error.
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, int* err) {
    const uint32_t a = smem_u32(bar);
    if (mbar_try_wait(a, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(a, parity)) {
        if (*(volatile int*)err) return false;
        if (clock64() - t0 > kWaitBudget) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// Arrive-and-wait of the CTA's epilogue warps on an mbarrier (count = epilogue warps), bounded;
// `n` counts the uses so far (the phase parity).  False on timeout or another role's error.
__device__ __forceinline__ bool epi_sync(uint64_t* bar, int& n, int* err) {
    const int lane = threadIdx.x & 31;
    int ok = 1;
    __syncwarp();
    if (lane == 0) {
        mbar_arrive(bar);
        ok = mbar_wait_or_abort(bar, (uint32_t)n & 1u, err);
    }
    ++n;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Persistent, warp-specialised grouped GEMM (128 x 128 tiles, split operands: hi + lo parts of
// A and B).  gridDim.x CTAs (at most one per SM) walk the output tiles of every problem of the
// launch, CTA c taking tiles c, c + gridDim.x, ...:
//   warp 0 lane 0   TMA producer: the k-blocks of the CTA's tiles through the shared-memory ring;
//   warp 1 lane 0   MMA issuer into one of two tensor-memory accumulator buffers, alternating
//                   per tile, so that one tile's epilogue overlaps the next tile's products;
//                   warp 1 also owns the tensor-memory allocation;
//   warps 2..5      epilogue: warp w drains accumulator lanes 32 (w mod 4) .. + 31 of a buffer,
//                   then frees it for the MMA issuer.
// DUAL problems accumulate a second operand set in the next BN columns of the same buffer.
// Every wait is bounded and gives up once any role has flagged an error; before exit the
// producer waits (bounded) for its copies in flight and the issuer for its MMAs.  The ZU_RHO
// forms need a launch with a single problem: the r^T z reduction runs over the whole grid.
// ------------------------------------------------------------------------------------------
// CTA-pair form: tcgen05.mma.cta_group::2 over two SMs of a TPC
// ------------------------------------------------------------------------------------------
// A pair of CTAs (a cluster of two) computes 256-row output tiles: each CTA stages its own 128
// rows of A and its half of B's rows, the even CTA issues M = 256 MMAs that read both CTAs'
// shared memory, and each CTA's tensor memory receives its own 128 accumulator rows.  Per SM
// this halves the B bytes streamed per multiply-add against the one-SM form.
constexpr int k2EpiWarps = 8;
constexpr int k2Threads = 64 + 32 * k2EpiWarps;

// Every MMA is M = 256 (two CTAs), N = 256: each CTA stages 128 rows of A and 128 rows of B.
// Measured on this part, N = 128 MMAs keep the tensor pipe busy at most ~77 % of the time and
// N = 256 ones ~99 %, so two-operand-set (DUAL) problems use two N = 256 accumulators (all 512
// tensor-memory columns, one buffer) instead of two N = 128 ones (double-buffered).
template <int DUAL, int SETN = 256>
struct Q2Cfg {
    static constexpr int kBRows = SETN / 2;            // B rows per CTA (per operand set)
    static constexpr int kABytes = UBM * UBK * 2;      // one bf16 part of this CTA's A rows
    static constexpr int kBBytes = kBRows * UBK * 2;
    static constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
    static constexpr int kStages = (192 * 1024) / kStageBytes > 8 ? 8 : (192 * 1024) / kStageBytes;
    // ring, 1024-byte alignment slack, barriers (256 bytes), the epilogue warps' scratch
    static constexpr int kSmem =
        kStages * kStageBytes + 1024 + 256 + k2EpiWarps * (int)sizeof(WarpScratch);
    static constexpr uint32_t kAcc = DUAL ? 2 * SETN : SETN;   // tensor-memory columns per buffer
    static constexpr int kBufs = 512 / kAcc;
    // kind::f16, D f32, A and B bf16 K-major, N = SETN, M = 256
    static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                       ((uint32_t)(SETN >> 3) << 17) |
                                       ((uint32_t)(256 >> 4) << 24);
};

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// shared::cluster address of the same shared-memory offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA load into this CTA's shared memory that signals an mbarrier of either CTA of the pair
__device__ __forceinline__ void tma_load_2d_pair(void* dst, const CUtensorMap* map,
                                                 uint32_t bar_cluster, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void umma_bf16_pair(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                               uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// arrive on the mbarrier at this offset in both CTAs once the issuer's MMAs so far complete
__device__ __forceinline__ void umma_commit_pair(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
        " [%0], %1;" ::"r"(smem_u32(bar)),
        "h"((uint16_t)3)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
                 : "memory");
}

// Tensor memory of both CTAs of the pair, allocated and released collectively (one warp of each
// CTA issues the instruction; both receive the same column address).
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// Persistent CTA-pair kernels.  Pair p (CTAs 2p, 2p+1) takes the 256-row tiles p,
// p + gridDim.x / 2, ... of its work list.  Warp roles in each CTA:
//   warp 0 lane 0   TMA producer: this CTA's A and B rows of each k-block through the
//                   shared-memory ring (the even CTA's full barriers count both CTAs' bytes);
//   warp 1          tensor-memory allocation (both CTAs, collectively); in the even CTA lane 0
//                   also issues the MMAs, into one of the accumulator buffers, so that one
//                   tile's epilogue overlaps the next tile's products where two buffers fit;
//   warps 2..9      epilogue: two warps per accumulator lane quarter split the columns and drain
//                   their CTA's 128 accumulator rows, then release the buffer.
// Per operand set:
//   non-DUAL: one M = 256, N = 256 accumulator, two buffers; CTA r stages B rows n0 + 128 r, or
//             for a mirrored problem rows n0 (even CTA) and nb_rows - n0 - 128 (odd CTA), so
//             that accumulator columns [128, 256) hold the mirrored tile;
//   DUAL:     two M = 256, N = 256 accumulators (operand sets) in one 512-column buffer.
// The even CTA's full barriers count both CTAs' bytes; the issuer's commits arrive in both CTAs;
// both CTAs' epilogue warps release an accumulator buffer on the even CTA's barrier.  All waits
// are bounded; the two CTAs take every branch that has a cluster barrier together.
// ------------------------------------------------------------------------------------------
// Folded preconditioner as one persistent launch: the four stages' tiles in one work list
// ------------------------------------------------------------------------------------------
// A stage's tile reads row panels of the previous stage's output (stage 2 a 256-row panel of
// T1, stage 3 a panel of two T2 blocks, stage 4 the rows of T3 that its Z rows fold from).  Each
// tile that produces such rows adds one per CTA to its panel's counter once its stores are
// visible; a tile waits until the panels it reads are complete before its first copy.  The work
// list holds every stage's tiles in stage order (a producer always before its consumers), pair p
// takes items p, p + P, ..., so the first unfinished item can always run: with all P pairs
// resident the launch cannot deadlock (and every wait is bounded regardless).
constexpr int kMaxDeps = 8;

struct FoldItem {
    const DevState* st;   // the image's state (stop flag)
    int skip;             // the problem honours the stop flag
    int prob, local;      // problem (index into the launch's problem table) and its tile
    int m0, n0;           // first output row (even CTA) and column of the tile
    int nb1;              // first B row the odd CTA stages
    int nkb, dual;        // k-blocks per operand set, operand sets - 1
    int half;             // a two-set tile of half width (N = 128 per set, one accumulator buffer)
    int epi;
    int sig;              // counter this tile completes (one add per CTA), or -1
    int ndep;
    int rho_end;          // stage 2: this pair's last tile of the image's stage-2 range
    int rho_nslot;        // stage 2: CTA flushes that complete the image's r^T z
    int dep[kMaxDeps];    // counters the tile waits for ...
    int need[kMaxDeps];   // ... and the counts that mean complete
};

// Bounded acquire-wait until every counter the item reads has reached its count (all counters
// loaded together: one round trip when they are complete); false on timeout or another role's
// error.
__device__ __forceinline__ bool wait_deps(const FoldItem& f, const unsigned* ctr, int* err) {
    auto ready = [&]() {
        unsigned v[kMaxDeps];
#pragma unroll
        for (int d = 0; d < kMaxDeps; ++d)
            if (d < f.ndep)
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];"
                             : "=r"(v[d])
                             : "l"(ctr + f.dep[d])
                             : "memory");
        bool ok = true;
#pragma unroll
        for (int d = 0; d < kMaxDeps; ++d)
            if (d < f.ndep) ok &= v[d] >= (unsigned)f.need[d];
        return ok;
    };
    if (ready()) return true;
    const long long t0 = clock64();
    while (!ready()) {
        __nanosleep(128);
        if (*(volatile int*)err) return false;
        if (clock64() - t0 > kWaitBudget) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ bool item_live(const FoldItem& f, const DevState*& st, bool& live) {
    if (f.st != st) {
        st = f.st;
        live = !(f.skip && *(volatile const int*)&f.st->done);
    }
    return live;
}

// Generic-proxy stores of other SMs (acquired above) become visible to this thread's TMA loads.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <int EBN, int EPI>
__device__ __forceinline__ void fused_epi(uint32_t tl, const UEpiArgs& ep, int m0w, int n0,
                                          CSum& part, int half, WarpScratch& s) {
    constexpr int kChunks = EBN / 32;
    epi_tile_t<EBN, EPI>(tl, ep, m0w, n0, part, half * (kChunks / 2), (half + 1) * (kChunks / 2), s);
}

// Persistent CTA-pair kernel over the fused work list, with the warp roles and operand sets
// described above; every MMA is M = 256, N = 256 (N = 128 per set for a half-width tile).  An
// item with one operand set uses one 256-column accumulator buffer (two buffers alternate); an
// item with two sets uses both (512 columns).  ctr[0 .. n_ctr) are the panel counters and
// ctr[n_ctr] counts exited CTAs: the last CTA to exit zeroes them for the next launch and applies
// deferred stops.  sts[0 .. n_st) are the images' states; honour_stop: every problem skips a
// stopped image.  f16: float16 operands, one product per multiply-add (no lo parts).
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(k2Threads, 1)
k2_fold_fused(const GemmTile* __restrict__ probs, const FoldItem* __restrict__ items,
              int n_items, unsigned* __restrict__ ctr, int n_ctr, DevState* const* __restrict__ sts,
              int n_st, int honour_stop, int f16) {
    using C = Q2Cfg<0, 256>;
    static_assert(Q2Cfg<1, 256>::kStageBytes == C::kStageBytes, "one ring for both forms");
    constexpr int S = C::kStages;
    constexpr uint32_t kCols = 512, kBuf = 256;
    // N = 128 per operand set (half-width two-set tiles), otherwise as C::kIdesc
    constexpr uint32_t kIdescHalf = (C::kIdesc & ~(0x3Fu << 17)) | ((uint32_t)(128 >> 3) << 17);
    // float16 operands: A and B format fields 0 (float16) instead of 1 (bf16)
    constexpr uint32_t kFmtBits = (7u << 7) | (7u << 10);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~static_cast<uintptr_t>(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * C::kStageBytes);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;     // [2] accumulator buffer ready (both CTAs)
    uint64_t* tempty = tfull + 2;    // [2] accumulator buffer drained (even CTA: all epilogue
                                     //     warps of both CTAs)
    uint64_t* drain = tempty + 2;
    uint64_t* epibar = drain + 1;    // the CTA's epilogue warps
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(epibar + 1);
    WarpScratch* scratch = reinterpret_cast<WarpScratch*>(smem + S * C::kStageBytes + 256);
    __shared__ int s_err;
    __shared__ int s_skip;
    __shared__ int s_last;
    __shared__ int s_exit;
    __shared__ double s_tot[k2EpiWarps];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank();
    {
        // no image's stop flag changes during the launch (stops found here are deferred)
        int live = honour_stop ? 0 : 1;
        for (int i = threadIdx.x; i < n_st && !live; i += blockDim.x)
            live = *(volatile const int*)&sts[i]->done ? 0 : 1;
        live = __syncthreads_or(live);
        if (threadIdx.x == 0) s_skip = live ? 0 : 1;
    }
    if (threadIdx.x == 0) {
        s_err = 0;
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 2 * k2EpiWarps);
        }
        mbar_init(drain, 1);
        mbar_init(epibar, k2EpiWarps);
        fence_mbar_init();
    }
    cluster_sync_all();
    bool skip;
    {
        // both CTAs of the pair skip, or neither
        int peer;
        asm volatile("ld.shared::cluster.u32 %0, [%1];"
                     : "=r"(peer)
                     : "r"(mapa_shared(smem_u32(&s_skip), rank ^ 1u))
                     : "memory");
        skip = (s_skip | peer) != 0;
    }
    cluster_sync_all();
    if (!skip) {
        if (warp == 1) tmem_alloc_pair(tmem_slot, kCols);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        const uint32_t tmem = *tmem_slot;
        const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
        const DevState* lst = nullptr;
        bool llive = true;

        if (warp == 0) {
            if (lane == 0) {
                const uint32_t full0 = mapa_shared(smem_u32(full), 0);
                int it = 0;
                bool bad = false;
                // the next item's record is fetched while this item's copies are issued
                FoldItem f;
                if (pair < n_items) f = items[pair];
                for (int t = pair; t < n_items && !bad; t += npairs) {
                    FoldItem fn;
                    if (t + npairs < n_items) fn = items[t + npairs];
                    if (!item_live(f, lst, llive)) {
                        f = fn;
                        continue;
                    }
                    const GemmTile& g = probs[f.prob];
                    // the rows this tile reads are complete (other SMs' stores, then a proxy fence
                    // so that the tensor copies below observe them)
                    if (f.ndep > 0) {
                        if (!wait_deps(f, ctr, &s_err)) {
                            bad = true;
                            break;
                        }
                        fence_proxy_async_global();
                    }
                    const int dual = f.dual, half = f.half;
                    const int m0 = f.m0 + 128 * (int)rank;
                    const int nb = rank == 0 ? f.n0 : f.nb1;
                    const int nkb = f.nkb, nkt = dual ? 2 * nkb : nkb;
                    // a half-width tile stages 64 B rows per CTA instead of 128; float16 operands have
                    // one part (no lo planes)
                    const uint32_t parts = f16 ? 1u : 2u;
                    const uint32_t tx = 2u * parts * (C::kABytes + (half ? C::kBBytes / 2 : C::kBBytes));
                    for (int kb = 0; kb < nkt; ++kb, ++it) {
                        const int s = it % S;
                        const uint32_t ph = (uint32_t)(it / S) & 1u;
                        if (it >= S && !mbar_wait_or_abort(&empty[s], ph ^ 1u, &s_err)) {
                            bad = true;
                            break;
                        }
                        const bool second = dual && kb >= nkb;
                        const int kc = (second ? kb - nkb : kb) * UBK;
                        uint8_t* sa = smem + s * C::kStageBytes;
                        uint8_t* sb = sa + 2 * C::kABytes;
                        if (rank == 0) mbar_expect_tx(&full[s], tx);
                        const uint32_t fb = full0 + 8u * (uint32_t)s;
                        tma_load_2d_pair(sa, second ? &g.a2 : &g.a0, fb, kc, m0);
                        const CUtensorMap* bm0 = half ? (second ? &g.bh2 : &g.bh0)
                                                      : (second ? &g.b2 : &g.b0);
                        tma_load_2d_pair(sb, bm0, fb, kc, nb);
                        if (!f16) {
                            tma_load_2d_pair(sa + C::kABytes, second ? &g.a3 : &g.a1, fb, kc, m0);
                            const CUtensorMap* bm1 = half ? (second ? &g.bh3 : &g.bh1)
                                                          : (second ? &g.b3 : &g.b1);
                            tma_load_2d_pair(sb + C::kBBytes, bm1, fb, kc, nb);
                        }
                    }
                    f = fn;
                }
                if (rank == 0) {
                    for (int j = it - S < 0 ? 0 : it - S; j < it; ++j)
                        if (!mbar_wait(&full[j % S], (uint32_t)(j / S) & 1u)) atomicExch(&s_err, 1);
                } else if (bad) {
                    const long long t0 = clock64();
                    while (clock64() - t0 < (1LL << 22)) {
                    }
                }
            }
            __syncwarp();
        } else if (warp == 1) {
            if (rank == 0 && lane == 0) {
                int it = 0, nbuf = 0;
                int use[2] = {0, 0};
                bool bad = false;
                FoldItem f;
                if (pair < n_items) f = items[pair];
                for (int t = pair; t < n_items && !bad; t += npairs) {
                    FoldItem fn;
                    if (t + npairs < n_items) fn = items[t + npairs];
                    if (!item_live(f, lst, llive)) {
                        f = fn;
                        continue;
                    }
                    const int dual = f.dual, half = f.half;
                    const bool two = dual && !half;   // both accumulator buffers
                    const int b0 = two ? 0 : nbuf, nbu = two ? 2 : 1;
                    if (!two) nbuf ^= 1;
                    const uint32_t idesc = (half ? kIdescHalf : C::kIdesc) & (f16 ? ~kFmtBits : ~0u);
                    const uint32_t set1 = half ? 128u : kBuf;
                    for (int k = 0; k < nbu && !bad; ++k) {
                        const int b = b0 + k;
                        if (use[b] >= 1 &&
                            !mbar_wait_or_abort(&tempty[b], (uint32_t)(use[b] - 1) & 1u, &s_err))
                            bad = true;
                        ++use[b];
                    }
                    if (bad) break;
                    tc_fence_after();
                    const uint32_t base = tmem + (uint32_t)b0 * kBuf;
                    const int nkb = f.nkb, nkt = dual ? 2 * nkb : nkb;
                    for (int kb = 0; kb < nkt; ++kb, ++it) {
                        const int s = it % S;
                        const uint32_t ph = (uint32_t)(it / S) & 1u;
                        if (!mbar_wait_or_abort(&full[s], ph, &s_err)) {
                            bad = true;
                            break;
                        }
                        tc_fence_after();
                        const bool second = dual && kb >= nkb;
                        const int kk = second ? kb - nkb : kb;
                        const uint32_t td = base + (second ? set1 : 0u);
                        const uint32_t sa = smem_u32(smem + s * C::kStageBytes);
                        const uint32_t sb = sa + 2 * C::kABytes;
                        const uint64_t da = desc_sw128(sa), db = desc_sw128(sb);
                        const uint64_t dal = desc_sw128(sa + C::kABytes);
                        const uint64_t dbl = desc_sw128(sb + C::kBBytes);
    #pragma unroll
                        if (f16) {
#pragma unroll
                            for (int q = 0; q < UBK / 16; ++q)   // one float16 product per K = 16
                                umma_bf16_pair(td, da + 2 * q, db + 2 * q, idesc, (kk | q) != 0);
                        } else {
#pragma unroll
                            for (int q = 0; q < UBK / 16; ++q) {   // K = 16 per MMA: +32 bytes
                                umma_bf16_pair(td, da + 2 * q, dbl + 2 * q, idesc, (kk | q) != 0);
                                umma_bf16_pair(td, dal + 2 * q, db + 2 * q, idesc, 1u);
                                umma_bf16_pair(td, da + 2 * q, db + 2 * q, idesc, 1u);
                            }
                        }
                        umma_commit_pair(&empty[s]);
                    }
                    if (!bad)
                        for (int k = 0; k < nbu; ++k) umma_commit_pair(&tfull[b0 + k]);
                    f = fn;
                }
                umma_commit_pair(drain);
            }
            __syncwarp();
        } else {
            const int q = warp & 3, half = (warp - 2) >> 2;
            const uint32_t te0 = mapa_shared(smem_u32(tempty), 0);
            int nbuf = 0, nsync = 0;
            int use[2] = {0, 0};
            CSum part;
            for (int t = pair; t < n_items; t += npairs) {
                const FoldItem& f = items[t];
                if (!item_live(f, lst, llive)) continue;
                const GemmTile& g = probs[f.prob];
                const bool two = f.dual && !f.half;
                const int b0 = two ? 0 : nbuf, nbu = two ? 2 : 1;
                if (!two) nbuf ^= 1;
                int ok = 1;
                for (int k = 0; k < nbu; ++k) {
                    const int b = b0 + k;
                    if (lane == 0 && ok)
                        ok = mbar_wait_or_abort(&tfull[b], (uint32_t)use[b] & 1u, &s_err);
                    ++use[b];
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) break;
                tc_fence_after();
                const int m0 = f.m0 + 128 * (int)rank;
                const int n0 = f.n0;
                const UEpiArgs ep = g.ep;
                const uint32_t tl = tmem + (uint32_t)b0 * kBuf + ((uint32_t)(q * 32) << 16);
                WarpScratch& sc = scratch[warp - 2];
                switch (f.epi) {
                    case UE_FOLD16:
                        fused_epi<128, UE_FOLD16>(tl, ep, m0 + q * 32, n0, part, half, sc);
                        break;
                    case UE_EIG16:
                        fused_epi<256, UE_EIG16>(tl, ep, m0 + q * 32, n0, part, half, sc);
                        break;
                    case UE_EIG16_RHO:
                        fused_epi<256, UE_EIG16_RHO>(tl, ep, m0 + q * 32, n0, part, half, sc);
                        break;
                    case UE_UNFOLD16:
                        if (f.half)
                            fused_epi<128, UE_UNFOLD16>(tl, ep, m0 + q * 32, n0, part, half, sc);
                        else
                            fused_epi<256, UE_UNFOLD16>(tl, ep, m0 + q * 32, n0, part, half, sc);
                        break;
                    default:
                        if (f.half)
                            fused_epi<128, UE_UNFOLDZ>(tl, ep, m0 + q * 32, n0, part, half, sc);
                        else
                            fused_epi<256, UE_UNFOLDZ>(tl, ep, m0 + q * 32, n0, part, half, sc);
                        break;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    for (int k = 0; k < nbu; ++k) mbar_arrive_cluster(te0 + 8u * (uint32_t)(b0 + k));
                if (f.epi == UE_EIG16_RHO) {
                    // r^T z of an image, in an order fixed by the image's own tile numbering (the same
                    // alone or in a batch): each epilogue warp stores its sum over the tile into slot
                    // ((tile, CTA), warp); at the end of its run of the image's stage-2 tiles (marked
                    // by the host) a CTA counts itself done, and the CTA that completes the count adds
                    // all the image's slots and forms rho and beta
                    double v = part.value();
                    part = CSum();
    #pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                    if (lane == 0)
                        ep.partials[((ep.rho_base + f.local) * 2 + (int)rank) * k2EpiWarps +
                                    (warp - 2)] = v;
                    if (f.rho_end) {
                        if (lane == 0) __threadfence();
                        if (!epi_sync(epibar, nsync, &s_err)) break;
                        if (warp == 2 && lane == 0) {
                            const unsigned prev = atomicAdd(&ep.st->counter, 1u);
                            s_last = prev == (unsigned)f.rho_nslot - 1u;
                        }
                        if (!epi_sync(epibar, nsync, &s_err)) break;
                        if (s_last) {
                            __threadfence();
                            const int n = ep.rho_count * 2 * k2EpiWarps;
                            const int e = threadIdx.x - 64;
                            double tot = 0.0;
                            for (int i = e; i < n; i += 32 * k2EpiWarps)
                                tot += __ldcg(&ep.partials[i]);
    #pragma unroll
                            for (int o = 16; o > 0; o >>= 1)
                                tot += __shfl_down_sync(0xffffffffu, tot, o);
                            if (lane == 0) s_tot[warp - 2] = tot;
                            if (!epi_sync(epibar, nsync, &s_err)) break;
                            if (warp == 2 && lane == 0) {
                                double sum = 0.0;
                                for (int w = 0; w < k2EpiWarps; ++w) sum += s_tot[w];
                                if (ep.f16) {
                                    const double us = (double)f16_inv_scale(ep);
                                    sum *= us * us;
                                }
                                finish_rho(ep, sum, true);
                                ep.st->counter = 0u;
                            }
                        }
                    }
                }
                if (f.sig >= 0) {
                    // this CTA's rows of the tile are stored: the epilogue warps' barrier orders
                    // every lane's stores before one release-add (cumulative) per CTA
                    if (!epi_sync(epibar, nsync, &s_err)) break;
                    if (warp == 2 && lane == 0)
                        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctr[f.sig])
                                     : "memory");
                }
            }
        }

        // every MMA of the pair has completed before the tensor memory is released
        if (warp == 1 && lane == 0 && !mbar_wait(drain, 0)) atomicExch(&s_err, 1);
        tc_fence_before();
        __syncthreads();
        if (warp == 1) {
            tc_fence_after();
            tmem_dealloc_pair(tmem, kCols);
        }
    }
    __syncthreads();
    if (*(volatile int*)&s_err) {
        // a wait gave up: every image of the launch stops with the timeout status
        for (int i = threadIdx.x; i < n_st; i += blockDim.x) {
            atomicOr(&sts[i]->status, ST_TIMEOUT);
            sts[i]->done = 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_exit = atomicAdd(&ctr[n_ctr], 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (s_exit) {
        // every other CTA has exited: reset the counters and apply the stops found in the launch
        __threadfence();
        for (int i = threadIdx.x; i < n_ctr; i += blockDim.x) ctr[i] = 0u;
        for (int i = threadIdx.x; i < n_st; i += blockDim.x) {
            DevState* sti = sts[i];
            if (sti->stop_next) {
                sti->done = 1;
                sti->stop_next = 0;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) ctr[n_ctr] = 0u;
    }
    cluster_sync_all();
}

__global__ void k_build_basis16(__nv_bfloat16* P16, __nv_bfloat16* PT16, __nv_bfloat16* P16lo,
                                __nv_bfloat16* PT16lo, int N, int Np) {
    const size_t total = (size_t)Np * Np;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / Np), k = (int)(t % Np);
        double v = 0.0;
        if (i < N && k < N) {
            const long long mm = ((long long)(2 * i + 1) * k) % (4LL * N);
            const double ck = k == 0 ? sqrt(1.0 / N) : sqrt(2.0 / N);
            v = ck * cospi((double)mm / (2.0 * N));
        }
        const __nv_bfloat16 h = __double2bfloat16(v);
        P16[(size_t)i * Np + k] = h;
        PT16[(size_t)k * Np + i] = h;
        if (P16lo) {
            const __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
            P16lo[(size_t)i * Np + k] = l;
            PT16lo[(size_t)k * Np + i] = l;
        }
    }
}

// Even / odd halves of the DCT basis of side n (n even), h = n / 2:
//   Pe[a][b] = P[a][2b], Po[a][b] = P[a][2b+1] (a, b < h), their transposes, and the eigenvalues
//   permuted to (even indices, odd indices).  P[n-1-a][k] = (-1)^k P[a][k] makes these enough.
// Stored hp x hp (hp >= h, pitch hp) with zeros outside the h x h block; lamP[par * hp + b].
__global__ void k_build_fold16(__nv_bfloat16* Pe, __nv_bfloat16* Po, __nv_bfloat16* PeT,
                               __nv_bfloat16* PoT, __nv_bfloat16* Pelo, __nv_bfloat16* Polo,
                               __nv_bfloat16* PeTlo, __nv_bfloat16* PoTlo, float* lamP, int n,
                               int hp, int f16) {
    // spatial half: (n + 1) / 2 rows (for odd n the middle row is its own mirror); frequencies:
    // (n + 1) / 2 even ones, n / 2 odd ones.  On the middle row every odd-frequency entry is
    // exactly 0 (P[(n-1)/2][k] = (-1)^k P[(n-1)/2][k]), so the two mirrored writes of that row in
    // the inverse stages carry the same value.
    const int hs = (n + 1) / 2;
    const size_t total = (size_t)hp * hp;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / hp), b = (int)(t % hp);
        for (int par = 0; par < 2; ++par) {
            const int k = 2 * b + par;
            double v = 0.0;
            if (a < hs && k < n && !(par == 1 && 2 * a + 1 == n)) {
                const long long mm = ((long long)(2 * a + 1) * k) % (4LL * n);
                const double ck = k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
                v = ck * cospi((double)mm / (2.0 * n));
            }
            __nv_bfloat16* P = par ? Po : Pe;
            __nv_bfloat16* PT = par ? PoT : PeT;
            if (f16) {   // float16, one part (the lo planes stay unused)
                const __half hh = __double2half(v);
                reinterpret_cast<__half*>(P)[(size_t)a * hp + b] = hh;
                reinterpret_cast<__half*>(PT)[(size_t)b * hp + a] = hh;
                continue;
            }
            const __nv_bfloat16 hv = __double2bfloat16(v);
            const __nv_bfloat16 lv = __double2bfloat16(v - (double)__bfloat162float(hv));
            P[(size_t)a * hp + b] = hv;
            PT[(size_t)b * hp + a] = hv;
            __nv_bfloat16* Pl = par ? Polo : Pelo;
            __nv_bfloat16* PTl = par ? PoTlo : PeTlo;
            if (Pl) {
                Pl[(size_t)a * hp + b] = lv;
                PTl[(size_t)b * hp + a] = lv;
            }
        }
        if (a == 0) {
            for (int par = 0; par < 2; ++par) {
                double lam = 0.0;
                if (2 * b + par < n) {
                    const double sn = sinpi((double)(2 * b + par) / (2.0 * n));
                    lam = 4.0 * sn * sn;
                }
                lamP[par * hp + b] = (float)lam;
            }
        }
    }
}

// Folded residual: Re[i][j] = r[i][j] + r[i][W-1-j], Ro[i][j] = r[i][j] - r[i][W-1-j] (j < W/2),
// each split into bf16 hi + lo, pitch ldo (columns W/2 .. ldo-1 are left alone: zero).  W a
// multiple of 8: four columns per thread, the float4 at j and the float4 ending at W-1-j
// (reversed; the pitch ld is a multiple of 4 floats); otherwise one column per thread.
// One image's even / odd column folds of r_U for the folded preconditioner (hi and lo bf16
// parts, row pitch ldo): Re[i][j'] = r[i][j'] + r[i][W-1-j'], Ro[i][j'] = r[i][j'] - r[i][W-1-j'],
// j' < W/2.  Each element is formed on its own, so the result does not depend on the launch.
struct FoldRRec {
    const float* rU;
    int ld, H, W, ldo;
    __nv_bfloat16 *Re, *Relo, *Ro, *Rolo;
    const DevState* st;
    int blk0, nblk;   // the image's blocks in a batched launch
    int f16;          // float16 planes (Re, Ro only), scaled by sqrt(H W) / ||r_U||
    float inv_sqrt_n;
};

__device__ __forceinline__ void fold_r_body(const FoldRRec& f, int bid, int nblk) {
    const float* __restrict__ rU = f.rU;
    const int ld = f.ld, H = f.H, W = f.W, ldo = f.ldo;
    if (f.f16) {
        const double rn = f.st->rnorm_u;
        const float sc = rn > 0.0 ? (float)(1.0 / (rn * (double)f.inv_sqrt_n)) : 1.f;
        __half* __restrict__ Eh = reinterpret_cast<__half*>(f.Re);
        __half* __restrict__ Oh = reinterpret_cast<__half*>(f.Ro);
        const int h = (W + 1) / 2;
        const size_t total = (size_t)H * h;
        for (size_t t = bid * (size_t)blockDim.x + threadIdx.x; t < total;
             t += (size_t)nblk * blockDim.x) {
            const int i = (int)(t / h), j = (int)(t % h);
            const bool self = 2 * j + 1 == W;
            const float a = rU[(size_t)i * ld + j];
            const float b = self ? 0.f : rU[(size_t)i * ld + (W - 1 - j)];
            const size_t off = (size_t)i * ldo + j;
            Eh[off] = __float2half_rn((a + b) * sc);
            Oh[off] = __float2half_rn(self ? 0.f : (a - b) * sc);
        }
        return;
    }
    __nv_bfloat16* __restrict__ Re = f.Re;
    __nv_bfloat16* __restrict__ Relo = f.Relo;
    __nv_bfloat16* __restrict__ Ro = f.Ro;
    __nv_bfloat16* __restrict__ Rolo = f.Rolo;
    if (W % 8 != 0) {
        // (W + 1) / 2 columns: for odd W the middle column is its own mirror (sum: the column
        // itself; difference: 0)
        const int h = (W + 1) / 2;
        const size_t total = (size_t)H * h;
        for (size_t t = bid * (size_t)blockDim.x + threadIdx.x; t < total;
             t += (size_t)nblk * blockDim.x) {
            const int i = (int)(t / h), j = (int)(t % h);
            const bool self = 2 * j + 1 == W;
            const float a = rU[(size_t)i * ld + j];
            const float b = self ? 0.f : rU[(size_t)i * ld + (W - 1 - j)];
            const float se = a + b, so = self ? 0.f : a - b;
            const __nv_bfloat16 eh = __float2bfloat16_rn(se), oh = __float2bfloat16_rn(so);
            const size_t off = (size_t)i * ldo + j;
            Re[off] = eh;
            Ro[off] = oh;
            if (Relo) {
                Relo[off] = __float2bfloat16_rn(se - __bfloat162float(eh));
                Rolo[off] = __float2bfloat16_rn(so - __bfloat162float(oh));
            }
        }
        return;
    }
    const int h4 = W / 8;
    const size_t total = (size_t)H * h4;
    for (size_t t = bid * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)nblk * blockDim.x) {
        const int i = (int)(t / h4), j = (int)(t % h4) * 4;
        const float4 a = *reinterpret_cast<const float4*>(rU + (size_t)i * ld + j);
        const float4 bm = *reinterpret_cast<const float4*>(rU + (size_t)i * ld + (W - 4 - j));
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {bm.w, bm.z, bm.y, bm.x};   // r[W-1-j-k], k = 0..3
        float e[4], o[4], el[4], ol[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float se = av[k] + bv[k], so = av[k] - bv[k];
            e[k] = __bfloat162float(__float2bfloat16_rn(se));
            o[k] = __bfloat162float(__float2bfloat16_rn(so));
            el[k] = se - e[k];
            ol[k] = so - o[k];
        }
        const size_t off = (size_t)i * ldo + j;
        *reinterpret_cast<uint2*>(Re + off) = make_uint2(pack_bf16(e[0], e[1]), pack_bf16(e[2], e[3]));
        *reinterpret_cast<uint2*>(Ro + off) = make_uint2(pack_bf16(o[0], o[1]), pack_bf16(o[2], o[3]));
        if (Relo) {
            *reinterpret_cast<uint2*>(Relo + off) =
                make_uint2(pack_bf16(el[0], el[1]), pack_bf16(el[2], el[3]));
            *reinterpret_cast<uint2*>(Rolo + off) =
                make_uint2(pack_bf16(ol[0], ol[1]), pack_bf16(ol[2], ol[3]));
        }
    }
}

__global__ void k_fold_r(FoldRRec f, int skip_if_done) {
    if (skip_if_done && f.st->done) return;
    fold_r_body(f, blockIdx.x, gridDim.x);
}

// Batched: each image's blocks fold its own r_U; images whose CG run has stopped return at once.
__global__ void k_fold_r_batched(const FoldRRec* __restrict__ recs, int T) {
    int lo = 0, hi = T - 1;
    const int bid = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (recs[mid].blk0 <= bid) lo = mid; else hi = mid - 1;
    }
    const FoldRRec f = recs[lo];
    if (f.st->done) return;
    fold_r_body(f, bid - f.blk0, f.nblk);
}

// blocks of one image's fold (a grid-stride loop over rows x quads, at most 8192 blocks)
int fold_r_blocks(int H, int W, int f16 = 0) {
    const size_t n = (size_t)H * ((W % 8 == 0 && !f16) ? W / 8 : (W + 1) / 2);
    return (int)std::min<size_t>((n + 255) / 256, 8192);
}

// Float16 form, stage 4's B operand: the even / odd basis halves of side W with column (frequency)
// k scaled by tau / (mu_k + lam1), the inverse of the row scale stage 2 gives its coefficients
// (mu_k: this side's eigenvalues, lam1: the other side's smallest nonzero one).  P4e[a][b] for
// frequency 2b, P4o[a][b] for 2b + 1, hp x hp, zero outside the valid block.  Largest entry about
// sqrt(2 / W) tau / lam1 (~ 4e2 at 4096 x 4096): within float16.
__global__ void k_build_fold_stage4_f16(__half* P4e, __half* P4o, int n, int hp, double lam1,
                                        double tau) {
    const int hs = (n + 1) / 2;
    const size_t total = (size_t)hp * hp;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t / hp), b = (int)(t % hp);
        for (int par = 0; par < 2; ++par) {
            const int k = 2 * b + par;
            double v = 0.0;
            if (a < hs && k < n && !(par == 1 && 2 * a + 1 == n)) {
                const long long mm = ((long long)(2 * a + 1) * k) % (4LL * n);
                const double ck = k == 0 ? sqrt(1.0 / n) : sqrt(2.0 / n);
                const double sn = sinpi((double)k / (2.0 * n));
                v = ck * cospi((double)mm / (2.0 * n)) * tau / (4.0 * sn * sn + lam1);
            }
            (par ? P4o : P4e)[(size_t)a * hp + b] = __double2half(v);
        }
    }
}

// ------------------------------------------------------------------------------------------
// host side: TMA descriptors and launches
// ------------------------------------------------------------------------------------------
struct StageMaps {
    CUtensorMap a0, a1, b0, b1;
};
struct TmapSet {
    StageMaps st[4];
};
static_assert(sizeof(TmapSet) <= sizeof(((DctPlan*)nullptr)->tmap_storage), "tmap storage");

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// row-major bf16 matrix rows x cols (cols contiguous), box = 64 columns x box_rows rows
// kb = 64: box 64 columns with 128-byte swizzling; kb = 32: box 32 columns, 64-byte swizzling
bool make_map(CUtensorMap* m, const void* ptr, int rows, int cols, int box_rows, int kb = UBK) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)kb, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    kb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// output tile width: 256 for single-pass stages when N allows it; stages with a split operand
// use 128 so that at least three shared-memory stages fit
int pick_bn(int N, bool split) { return (!split && N % 256 == 0) ? 256 : 128; }

// per-stage split configuration: bit 2s = A operand of stage s carried as hi + lo, bit 2s+1 = B
bool split_a(int mask, int s) { return (mask >> (2 * s)) & 1; }
bool split_b(int mask, int s) { return (mask >> (2 * s + 1)) & 1; }

template <int BN, int EPI, int SA, int SB>
cudaError_t launch_one(const StageMaps& m, int M, int N, int K, const UEpiArgs& ep,
                       cudaStream_t s) {
    using C = UCfg<BN, SA, SB>;
    dim3 grid(N / BN, M / UBM);
    k_umma_gemm<BN, EPI, SA, SB><<<grid, kUThreads, C::kSmem, s>>>(m.a0, m.a1, m.b0, m.b1, K, ep);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_stage(const StageMaps& m, int M, int N, int K, bool sa, bool sb,
                         const UEpiArgs& ep, cudaStream_t s) {
    if (sa && sb) return launch_one<128, EPI, 2, 2>(m, M, N, K, ep, s);
    if (sa) return launch_one<128, EPI, 2, 1>(m, M, N, K, ep, s);
    if (sb) return launch_one<128, EPI, 1, 2>(m, M, N, K, ep, s);
    if (pick_bn(N, false) == 256) return launch_one<256, EPI, 1, 1>(m, M, N, K, ep, s);
    return launch_one<128, EPI, 1, 1>(m, M, N, K, ep, s);
}

inline size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <int BN, int SA, int SB>
cudaError_t set_attrs() {
    const int sm = UCfg<BN, SA, SB>::kSmem;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_umma_gemm<BN, UE_STORE16, SA, SB>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_umma_gemm<BN, UE_EIG16, SA, SB>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_umma_gemm<BN, UE_ZU, SA, SB>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_umma_gemm<BN, UE_ZU_RHO, SA, SB>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

}  // namespace

// The folded form pairs mirrored rows and columns (for an odd side the middle one pairs with
// itself); halves that are not multiples of 256 are padded to them.  Below 256 per side the
// padding would dominate: the direct form runs there.  `tc`: a precision the folded form runs in
// (split bf16 or float16).
bool foldable(int H, int W, int tc) {
    return tc && H >= 256 && W >= 256;
}

// padded extents of the folded operands: the halves and the full height, multiples of 256
struct FoldDims {
    int hN, hM, hNp, hMp, Hp;
};
// hN, hM: the spatial half sides, (n + 1) / 2 (odd n: the middle row / column counted once)
FoldDims fold_dims(int H, int W) {
    FoldDims f;
    f.hN = (H + 1) / 2;
    f.hM = (W + 1) / 2;
    f.hNp = (int)rup(f.hN, 256);
    f.hMp = (int)rup(f.hM, 256);
    f.Hp = (int)rup(H, 256);
    return f;
}

namespace {

// The folded stages run as CTA-pair GEMMs with 256-row tiles (every padded extent is a multiple
// of 256); the two-set stages (3 and 4) use N = 256 per operand set (two accumulators fill the
// tensor memory), the width the fused kernel's accumulator buffers assume.
constexpr int kPairDualN = 256;

// Even / odd basis halves of one side length n (hi and lo parts), padded to hp = rup(n/2, 256).
struct FoldSide {
    int n = 0, hp = 0;
    int f16 = 0;   // float16 bases (one part) instead of bf16 hi / lo
    void *Pe[2], *Po[2], *PeT[2], *PoT[2];
    float* lamP;
};

// One image's folded operands and intermediates (hi and lo parts).
struct FoldImage {
    FoldDims dim{};
    void *Re[2], *Ro[2];   // H x hMp
    void* T1[4][2];        // (x, sign) = (e+, e-, o+, o-), hMp x hNp
    void* T3[2][2];        // x = e, o: Hp x hMp
    void* P4[2];           // float16 form: stage 4's scaled basis halves (even, odd), hMp x hMp
    void* T2[4][2];        // (x, y) = ee, eo, oe, oo: hMp x hNp
};

size_t fold_side_bytes(int n) {
    const size_t hp = rup((n + 1) / 2, 256);
    return 2 * 4 * rup(hp * hp * 2, 1024) + rup(2 * hp * 4, 1024);
}

size_t fold_image_bytes(int H, int W) {
    const FoldDims fd = fold_dims(H, W);
    const size_t hNp = fd.hNp, hMp = fd.hMp;
    return 2 * (2 * rup((size_t)H * hMp * 2, 1024) + 4 * rup(hMp * hNp * 2, 1024) +
                4 * rup(hMp * hNp * 2, 1024) + 2 * rup((size_t)fd.Hp * hMp * 2, 1024)) +
           2 * rup(hMp * hMp * 2, 1024);
}

template <typename Take>
void carve_fold_side(FoldSide& sd, int n, Take take, int f16 = 0) {
    sd.n = n;
    sd.f16 = f16;
    sd.hp = (int)rup((n + 1) / 2, 256);
    const size_t e = (size_t)sd.hp * sd.hp * 2;
    for (int q = 0; q < 2; ++q) {
        sd.Pe[q] = take(e); sd.Po[q] = take(e); sd.PeT[q] = take(e); sd.PoT[q] = take(e);
    }
    sd.lamP = static_cast<float*>(take(2 * (size_t)sd.hp * 4));
}

void build_fold_side(const FoldSide& sd) {
    using B = __nv_bfloat16;
    auto bf = [](void* x) { return static_cast<B*>(x); };
    k_build_fold16<<<1024, 256>>>(bf(sd.Pe[0]), bf(sd.Po[0]), bf(sd.PeT[0]), bf(sd.PoT[0]),
                                  bf(sd.Pe[1]), bf(sd.Po[1]), bf(sd.PeT[1]), bf(sd.PoT[1]),
                                  sd.lamP, sd.n, sd.hp, sd.f16);
}

template <typename Take>
void carve_fold_image(FoldImage& im, int H, int W, Take take) {
    const FoldDims fd = fold_dims(H, W);
    im.dim = fd;
    const size_t hNp = fd.hNp, hMp = fd.hMp;
    for (int q = 0; q < 2; ++q) {
        im.Re[q] = take((size_t)H * hMp * 2);
        im.Ro[q] = take((size_t)H * hMp * 2);
    }
    for (int q = 0; q < 2; ++q)
        for (int b = 0; b < 4; ++b) im.T1[b][q] = take(hMp * hNp * 2);
    for (int q = 0; q < 2; ++q)
        for (int b = 0; b < 4; ++b) im.T2[b][q] = take(hMp * hNp * 2);
    // T3 rows H .. Hp-1 are read as A rows of stage 4 (masked there) and never written: zero
    for (int q = 0; q < 2; ++q)
        for (int x = 0; x < 2; ++x) im.T3[x][q] = take((size_t)fd.Hp * hMp * 2);
    for (int x = 0; x < 2; ++x) im.P4[x] = take(hMp * hMp * 2);
}

// Appends one image's nine problems (2, 4, 2 and 1 per stage) to the stage tables.
bool append_fold_problems(std::vector<GemmTile> (&tab)[4], const FoldImage& im,
                          const FoldSide& sN, const FoldSide& sM, int H, int W, const float* rU,
                          float* zU, int ld, DevState* st, double* partials, int flexible,
                          int skip, float tau, int f16 = 0, bool encode = true) {
    const FoldDims fd = im.dim;
    const int hN = fd.hN, hM = fd.hM, hNp = fd.hNp, hMp = fd.hMp;
    // the bases' padded sides are the operands' (every tensor map below assumes it)
    if (sN.hp != hNp || sM.hp != hMp || sN.n != H || sM.n != W) return false;
    bool ok = true;
    UEpiArgs base{};
    base.st = st;
    base.partials = partials;
    base.flexible = flexible;
    base.skip_if_done = skip;
    base.f16 = f16;
    {
        const double sn = std::sin(3.14159265358979323846 / (2.0 * H));
        base.lam1 = (float)(4.0 * sn * sn);   // the smallest nonzero eigenvalue of side H
        base.inv_sqrt_n = (float)(1.0 / std::sqrt((double)H * (double)W));
    }
    int bbox = 128;
    bool halves = false;   // two-set stages: also B maps with 64-row boxes (half-width tiles)
    // tensor maps (skipped when only the schedule is wanted: no driver call)
    auto mm = [&](CUtensorMap* m, const void* ptr, int rows, int cols, int box_rows) {
        return encode ? make_map(m, ptr, rows, cols, box_rows) : true;
    };
    auto set0 = [&](GemmTile& g, void* const* A, int ar, int ac, void* const* Bm, int br, int bc) {
        ok &= mm(&g.a0, A[0], ar, ac, UBM);
        ok &= mm(&g.a1, A[1], ar, ac, UBM);
        ok &= mm(&g.b0, Bm[0], br, bc, bbox);
        ok &= mm(&g.b1, Bm[1], br, bc, bbox);
        g.a2 = g.a0; g.a3 = g.a1; g.b2 = g.b0; g.b3 = g.b1;
        if (halves) {
            ok &= mm(&g.bh0, Bm[0], br, bc, 64);
            ok &= mm(&g.bh1, Bm[1], br, bc, 64);
        } else {
            g.bh0 = g.b0; g.bh1 = g.b1;
        }
        g.bh2 = g.bh0; g.bh3 = g.bh1;
    };
    auto set1 = [&](GemmTile& g, void* const* A, int ar, int ac, void* const* Bm, int br, int bc) {
        ok &= mm(&g.a2, A[0], ar, ac, UBM);
        ok &= mm(&g.a3, A[1], ar, ac, UBM);
        ok &= mm(&g.b2, Bm[0], br, bc, bbox);
        ok &= mm(&g.b3, Bm[1], br, bc, bbox);
        if (halves) {
            ok &= mm(&g.bh2, Bm[0], br, bc, 64);
            ok &= mm(&g.bh3, Bm[1], br, bc, 64);
        }
    };
    // Every operand is stored padded (extents hNp, hMp, Hp, multiples of 256); padding rows and
    // columns of the bases are zero, and the epilogues mask what lies beyond the half sides.
    // stage 1 (x = e, o): T1x+-[l'][i'] = Y(i') +- Y(H-1-i') with Y(i) = sum_j' PxT_M[l'][j'] Rx[i][j'];
    // the second operand set reads the B rows mirrored (a negative start row reads zeros)
    for (int x = 0; x < 2; ++x) {
        GemmTile g{};
        set0(g, x ? sM.PoT : sM.PeT, hMp, hMp, x ? im.Ro : im.Re, H, hMp);
        g.mirror_b1 = 1;
        g.nb_rows = H;
        g.M = hMp; g.N = hNp; g.K = hMp;
        g.ep = base;
        g.ep.C = im.T1[2 * x][0]; g.ep.C_lo = im.T1[2 * x][1];
        g.ep.C2 = im.T1[2 * x + 1][0]; g.ep.C2_lo = im.T1[2 * x + 1][1];
        g.ep.ldc = hNp;
        g.ep.vn = hN;
        g.ep.mid = (H % 2 == 1) ? H / 2 : -1;
        tab[0].push_back(g);
    }
    // stage 2 (x, y): T2xy[l'][k'] = tau sum_i' T1x(+ for y = e, - for y = o)[l'][i'] PyT_N[k'][i']
    // divided by the eigenvalue sum at frequencies (2k' + y, 2l' + x); r^T z from the spectral
    // coefficients, numbered by the image's own 256 x 256 tiles (tiles2 per problem)
    const int tiles2 = (hMp / 256) * (hNp / 256);
    for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) {
            GemmTile g{};
            set0(g, im.T1[2 * x + y], hMp, hNp, y ? sN.PoT : sN.PeT, hNp, hNp);
            g.M = hMp; g.N = hNp; g.K = hNp;
            g.ep = base;
            g.ep.C = im.T2[2 * x + y][0]; g.ep.C_lo = im.T2[2 * x + y][1]; g.ep.ldc = hNp;
            // valid frequencies of each parity: (n + 1) / 2 even, n / 2 odd
            g.ep.vm = x ? W / 2 : hM;
            g.ep.vn = y ? H / 2 : hN;
            g.ep.lam_m = sM.lamP + x * hMp;
            g.ep.lam_n = sN.lamP + y * hNp;
            g.ep.scale = tau;
            g.ep.keep_origin = (x == 0 && y == 0) ? 0 : 1;
            g.ep.rho_base = (2 * x + y) * tiles2;
            g.ep.rho_count = 4 * tiles2;
            tab[1].push_back(g);
        }
    bbox = kPairDualN / 2;
    halves = true;
    // stage 3 (x): with E from the even and O from the odd frequencies along i,
    // T3x[i'][l'] = E + O and T3x[H-1-i'][l'] = E - O (i' < hN)
    for (int x = 0; x < 2; ++x) {
        GemmTile g{};
        set0(g, sN.Pe, hNp, hNp, im.T2[2 * x], hMp, hNp);
        set1(g, sN.Po, hNp, hNp, im.T2[2 * x + 1], hMp, hNp);
        g.M = hNp; g.N = hMp; g.K = hNp;
        g.ep = base;
        g.ep.C = im.T3[x][0]; g.ep.C_lo = im.T3[x][1]; g.ep.ldc = hMp; g.ep.mrows = H;
        g.ep.vm = hN;
        tab[2].push_back(g);
    }
    // stage 4: Z[i][j'] = E + O, Z[i][W-1-j'] = E - O (i < H, j' < hM), E from T3e, O from T3o;
    // the float16 form's B is the basis scaled per frequency (the inverse of stage 2's row scale)
    {
        GemmTile g{};
        void* const p4e[2] = {im.P4[0], im.P4[0]};
        void* const p4o[2] = {im.P4[1], im.P4[1]};
        set0(g, im.T3[0], fd.Hp, hMp, f16 ? p4e : sM.Pe, hMp, hMp);
        set1(g, im.T3[1], fd.Hp, hMp, f16 ? p4o : sM.Po, hMp, hMp);
        g.M = fd.Hp; g.N = hMp; g.K = hMp;
        g.ep = base;
        g.ep.C = zU; g.ep.ldc = ld; g.ep.mcols = W; g.ep.rU = rU;
        g.ep.vm = H; g.ep.vn = hM;
        tab[3].push_back(g);
    }
    return ok;
}

// Tile grid of every problem (256 rows x 128 columns for the mirrored stage 1, 256 x kPairDualN
// for the two-set stages, 256 x 256 for stage 2) and each problem's first tile in its launch.
bool number_fold_tiles(std::vector<GemmTile> (&tab)[4], int (&tiles)[4]) {
    for (int k = 0; k < 4; ++k) {
        int n = 0;
        for (auto& g : tab[k]) {
            const int tn = k == 0 ? 128 : (k == 1 ? 256 : kPairDualN);
            if (g.M % 256 != 0 || g.N % tn != 0) return false;
            g.gx = g.N / tn;
            g.blk0 = n;
            n += (g.M / 256) * g.gx;
        }
        tiles[k] = n;
    }
    // stage 2 numbers an image's r^T z slots by its own tiles: its four problems are consecutive,
    // problem q starts at tile rho_base = q * tiles2 of the image, rho_count = 4 * tiles2
    if (tab[1].size() % 4 != 0) return false;
    for (size_t i = 0; i < tab[1].size(); i += 4) {
        const int a = tab[1][i].blk0;
        for (int q = 0; q < 4; ++q) {
            const GemmTile& g = tab[1][i + q];
            const int nt = (g.M / 256) * g.gx;
            if (g.ep.rho_base != q * nt || g.ep.rho_count != 4 * nt || g.blk0 != a + q * nt ||
                g.ep.st != tab[1][i].ep.st)
                return false;
        }
    }
    return true;
}

// ---- fused launch: problem table, work list with panel dependencies ----------------------
struct FusedDev {
    GemmTile* probs = nullptr;
    FoldItem* items = nullptr;
    unsigned* ctr = nullptr;     // n_ctr panel counters and the exit counter
    DevState** sts = nullptr;    // the images' states
    int n_probs = 0, n_items = 0, cap_items = 0, n_ctr = 0, n_st = 0, pairs = 0, honour_stop = 1;
    int f16 = 0;                 // float16 operands (one MMA per K step)
};

// Items and panel counters of one image's four stages.
void fused_counts(int H, int W, int& items, int& ctrs) {
    const FoldDims d = fold_dims(H, W);
    const int mb = d.hMp / 256, nb = d.hNp / 256;
    items = 2 * mb * (d.hNp / 128) + 4 * mb * nb + 2 * nb * mb + (d.Hp / 256) * mb;
    ctrs = 2 * mb + 4 * mb + 2 * nb;
}

// Work-list capacity: the tiles plus up to kMaxSplit two-set tiles split into halves.
constexpr int kMaxSplit = 1024;

size_t fused_bytes(int n_img, int items, int ctrs) {
    return rup((size_t)9 * n_img * sizeof(GemmTile), 1024) +
           rup((size_t)(items + kMaxSplit) * sizeof(FoldItem), 1024) +
           rup((size_t)(ctrs + 1) * 4, 1024) +
           rup((size_t)n_img * sizeof(DevState*), 1024);
}

template <typename Take>
void carve_fused(FusedDev& fd, int n_img, int items, int ctrs, Take take) {
    items += kMaxSplit;
    fd.probs = static_cast<GemmTile*>(take((size_t)9 * n_img * sizeof(GemmTile)));
    fd.items = static_cast<FoldItem*>(take((size_t)items * sizeof(FoldItem)));
    fd.ctr = static_cast<unsigned*>(take((size_t)(ctrs + 1) * 4));
    fd.sts = static_cast<DevState**>(take((size_t)n_img * sizeof(DevState*)));
    fd.n_st = n_img;
    fd.n_probs = 9 * n_img;
    fd.n_items = items;
    fd.cap_items = items;
    fd.n_ctr = ctrs;
}

// From the per-stage tables (every image's problems in image order, tiles numbered): one problem
// table and the work list, stage after stage.  Stage-2 tiles of an image stay consecutive (its
// r^T z run flags assume that); stage-4 tiles of an image are ordered by the last stage-3 panel
// they read.  `pairs` is the launch's pair count (the static item -> pair assignment).
// `stall` (a test hook): every stage-2 tile waits for one count more than its panel reaches, so
// that the bounded wait runs out and the launch ends with the timeout status.
bool build_fused(const std::vector<GemmTile> (&tab)[4], const std::vector<int>& Hs,
                 int pairs, int reduce_rho, std::vector<GemmTile>& probs,
                 std::vector<FoldItem>& items, int& n_ctr, int stall = 0) {
    const int n_img = (int)Hs.size();
    if ((int)tab[0].size() != 2 * n_img || (int)tab[1].size() != 4 * n_img ||
        (int)tab[2].size() != 2 * n_img || (int)tab[3].size() != n_img)
        return false;
    probs.clear();
    items.clear();
    int off[4];
    for (int k = 0; k < 4; ++k) {
        off[k] = (int)probs.size();
        for (GemmTile g : tab[k]) {
            g.epi = k == 0 ? UE_FOLD16
                           : k == 1 ? (reduce_rho ? UE_EIG16_RHO : UE_EIG16)
                                    : k == 2 ? UE_UNFOLD16 : UE_UNFOLDZ;
            g.dual = k >= 2 ? 1 : 0;
            probs.push_back(g);
        }
    }
    // counters: per image, stage-1 panels (x, l'-block), stage-2 panels (xy, l'-block), stage-3
    // panels (x, i'-block)
    std::vector<int> c1(n_img), c2(n_img), c3(n_img), mbs(n_img), nbs(n_img);
    int n = 0;
    for (int i = 0; i < n_img; ++i) {
        mbs[i] = tab[1][4 * i].M / 256;
        nbs[i] = tab[2][2 * i].M / 256;
        c1[i] = n; n += 2 * mbs[i];
        c2[i] = n; n += 4 * mbs[i];
        c3[i] = n; n += 2 * nbs[i];
    }
    n_ctr = n;
    auto ntiles = [](const GemmTile& g) { return (g.M / 256) * g.gx; };
    // stage 1: no dependencies (the folded residual comes from the previous launch)
    for (int i = 0; i < n_img; ++i)
        for (int x = 0; x < 2; ++x) {
            const GemmTile& g = tab[0][2 * i + x];
            for (int l = 0; l < ntiles(g); ++l) {
                FoldItem f{};
                f.prob = off[0] + 2 * i + x;
                f.local = l;
                f.sig = c1[i] + x * mbs[i] + l / g.gx;
                items.push_back(f);
            }
        }
    // stage 2 (x, y): the stage-1 panel of T1x at the same l'-block
    std::vector<int> r2a(n_img), r2b(n_img);
    for (int i = 0; i < n_img; ++i) {
        r2a[i] = (int)items.size();
        for (int q = 0; q < 4; ++q) {
            const GemmTile& g = tab[1][4 * i + q];
            const int x = q >> 1;
            const int need = 2 * tab[0][2 * i + x].gx;
            for (int l = 0; l < ntiles(g); ++l) {
                FoldItem f{};
                f.prob = off[1] + 4 * i + q;
                f.local = l;
                f.sig = c2[i] + q * mbs[i] + l / g.gx;
                f.ndep = 1;
                f.dep[0] = c1[i] + x * mbs[i] + l / g.gx;
                f.need[0] = need + (stall ? 1 : 0);
                items.push_back(f);
            }
        }
        r2b[i] = (int)items.size();
    }
    // stage 3 (x): B rows = the l'-block of T2(x, e) and T2(x, o)
    for (int i = 0; i < n_img; ++i)
        for (int x = 0; x < 2; ++x) {
            const GemmTile& g = tab[2][2 * i + x];
            const int need = 2 * tab[1][4 * i].gx;
            for (int l = 0; l < ntiles(g); ++l) {
                const int m = l / g.gx, nn = l % g.gx;
                FoldItem f{};
                f.prob = off[2] + 2 * i + x;
                f.local = l;
                f.sig = c3[i] + x * nbs[i] + m;
                f.ndep = 2;
                f.dep[0] = c2[i] + (2 * x) * mbs[i] + nn;
                f.dep[1] = c2[i] + (2 * x + 1) * mbs[i] + nn;
                f.need[0] = f.need[1] = need;
                items.push_back(f);
            }
        }
    // stage 4: A rows r of T3e and T3o come from i' = r (r < hN) or i' = H - 1 - r (r >= hN)
    for (int i = 0; i < n_img; ++i) {
        const GemmTile& g = tab[3][i];
        const int H = Hs[i], hN = (H + 1) / 2;
        const int need = 2 * tab[2][2 * i].gx;
        std::vector<std::pair<int, FoldItem>> st4;
        for (int l = 0; l < ntiles(g); ++l) {
            const int m = l / g.gx;
            const int lo = 256 * m, hi = std::min(256 * m + 256, H);   // rows [lo, hi)
            std::vector<int> m3;
            auto add = [&](int ip) {
                const int b = ip / 256;
                if (std::find(m3.begin(), m3.end(), b) == m3.end()) m3.push_back(b);
            };
            for (int r = lo; r < hi; r += 1) {
                if (r < hN) add(r);
                else add(H - 1 - r);
            }
            FoldItem f{};
            f.prob = off[3] + i;
            f.local = l;
            f.sig = -1;
            int key = -1;
            for (int x = 0; x < 2; ++x)
                for (int b : m3) {
                    if (f.ndep >= kMaxDeps) return false;
                    f.dep[f.ndep] = c3[i] + x * nbs[i] + b;
                    f.need[f.ndep] = need;
                    ++f.ndep;
                    key = std::max(key, b);
                }
            st4.push_back({key, f});
        }
        std::stable_sort(st4.begin(), st4.end(),
                         [](const std::pair<int, FoldItem>& a, const std::pair<int, FoldItem>& b) {
                             return a.first < b.first;
                         });
        for (auto& e : st4) items.push_back(e.second);
    }
    // tile coordinates and the stop flag, so that the kernel's producer and issuer need only the
    // item record
    for (FoldItem& f : items) {
        const GemmTile& g = probs[f.prob];
        const int tn = g.dual ? 256 : (g.mirror_b1 ? 128 : 256);
        f.st = g.ep.st;
        f.skip = g.ep.skip_if_done;
        f.m0 = (f.local / g.gx) * 256;
        f.n0 = (f.local % g.gx) * tn;
        f.nb1 = g.mirror_b1 ? g.nb_rows - f.n0 - 128 : f.n0 + 128;
        f.nkb = g.K / UBK;
        f.dual = g.dual;
        f.epi = g.epi;
    }
    // Half-width tail: the last two-set tiles (stage 4, no consumers) may be split into two
    // N = 128 halves each, so that the last wave fills the pairs that would otherwise idle.  The
    // count is chosen by the makespan of the static assignment (item t on pair t mod pairs),
    // counting a tile's k-blocks per operand set, a half tile at 1/0.77 of its size (N = 128 MMAs
    // ran at ~77 % of the N = 256 rate).  The arithmetic of every output element is unchanged.
    {
        int n_tail = 0;   // trailing stage-4 tiles
        for (int t = (int)items.size() - 1; t >= 0 && items[t].epi == UE_UNFOLDZ; --t) ++n_tail;
        const int max_split = std::min({n_tail, pairs, kMaxSplit});
        auto dur = [](const FoldItem& f) { return (double)f.nkb * (f.dual ? 2 : 1); };
        const int n = (int)items.size();
        std::vector<double> base(pairs, 0.0);
        int best_x = 0;
        double best = 0.0;
        for (int x = 0; x <= max_split; ++x) {
            std::fill(base.begin(), base.end(), 0.0);
            int t = 0;
            for (int i = 0; i < n - x; ++i, ++t) base[t % pairs] += dur(items[i]);
            for (int i = n - x; i < n; ++i)
                for (int h = 0; h < 2; ++h, ++t) base[t % pairs] += items[i].nkb / 0.77;
            const double mk = *std::max_element(base.begin(), base.end());
            if (x == 0 || mk < best - 1e-9) {
                best = mk;
                best_x = x;
            }
        }
        if (best_x > 0) {
            std::vector<FoldItem> tail(items.end() - best_x, items.end());
            items.resize(items.size() - best_x);
            for (const FoldItem& f : tail)
                for (int h = 0; h < 2; ++h) {
                    FoldItem g = f;
                    g.half = 1;
                    g.n0 = f.n0 + 128 * h;
                    g.nb1 = g.n0 + 64;
                    items.push_back(g);
                }
        }
    }
    // r^T z run flags of stage 2 (item t runs on pair t mod pairs)
    for (int i = 0; i < n_img; ++i) {
        const int a = r2a[i], b = r2b[i];
        for (int t = a; t < b; ++t) {
            items[t].rho_end = t + pairs >= b ? 1 : 0;
            items[t].rho_nslot = 2 * std::min(pairs, b - a);
        }
    }
    return true;
}

// Copies the tables; the images' states are the stage-4 problems' (one per image).
cudaError_t upload_fused(FusedDev& fd, const std::vector<GemmTile>& probs,
                         const std::vector<FoldItem>& items, int n_ctr, cudaStream_t s) {
    if ((int)probs.size() != fd.n_probs || (int)items.size() > fd.cap_items || n_ctr != fd.n_ctr)
        return cudaErrorInvalidValue;
    fd.n_items = (int)items.size();
    std::vector<DevState*> sts;
    fd.honour_stop = 1;
    for (const GemmTile& g : probs) {
        if (g.epi == UE_UNFOLDZ) sts.push_back(g.ep.st);
        if (!g.ep.skip_if_done) fd.honour_stop = 0;
    }
    if ((int)sts.size() != fd.n_st) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemcpyAsync(fd.probs, probs.data(), probs.size() * sizeof(GemmTile),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(fd.sts, sts.data(), sts.size() * sizeof(DevState*),
                        cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(fd.items, items.data(), items.size() * sizeof(FoldItem),
                           cudaMemcpyHostToDevice, s);
}

// Pairs of the fused launch: every pair must be resident at once (tiles wait on other pairs).
int fused_pairs(int n_sm) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_sm);
    cfg.blockDim = dim3(k2Threads);
    cfg.dynamicSmemBytes = Q2Cfg<0>::kSmem;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k2_fold_fused, &cfg) != cudaSuccess || nc < 1) {
        cudaGetLastError();
        return 0;
    }
    return std::min(n_sm / 2, nc);
}

cudaError_t launch_fused(const FusedDev& fd, cudaStream_t s) {
    k2_fold_fused<<<2 * fd.pairs, k2Threads, Q2Cfg<0>::kSmem, s>>>(
        fd.probs, fd.items, fd.n_items, fd.ctr, fd.n_ctr, fd.sts, fd.n_st, fd.honour_stop, fd.f16);
    return cudaGetLastError();
}

cudaError_t set_fold_attrs() {
    static bool done = false;
    if (done) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(
        k2_fold_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, Q2Cfg<0>::kSmem);
    if (e != cudaSuccess) return e;
    done = true;
    return cudaSuccess;
}

int device_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

FoldRRec fold_r_rec(const FoldImage& im, const float* rU, int ld, int H, int W,
                    const DevState* st, int f16 = 0) {
    using B = __nv_bfloat16;
    FoldRRec r{};
    r.rU = rU; r.ld = ld; r.H = H; r.W = W; r.ldo = im.dim.hMp;
    r.Re = static_cast<B*>(im.Re[0]); r.Relo = static_cast<B*>(im.Re[1]);
    r.Ro = static_cast<B*>(im.Ro[0]); r.Rolo = static_cast<B*>(im.Ro[1]);
    r.st = st;
    r.f16 = f16;
    r.inv_sqrt_n = (float)(1.0 / std::sqrt((double)H * (double)W));
    return r;
}

// Host-side record of a single-image plan's folded form and of the arguments its device tables
// were last built for (the tables bake in the planes, the CG state and the epilogue flags).
struct FoldBufs {
    FoldSide sN, sM;
    FoldImage img;
    FoldDims dim{};
    std::vector<GemmTile> tab[4];
    bool bound = false;
    const float* rU = nullptr;
    float* zU = nullptr;
    int ld = 0, flexible = 0, skip = 0;
    DevState* st = nullptr;
    double* partials = nullptr;
    float tau = 0.f;
    int rho = -1;                  // r^T z formed in stage 2 (the tables' stage-2 epilogue)
    int stall = 0;                 // test hook: stage-2 waits that run out (see build_fused)
    int n_sm = 0;                  // SMs of the device
    FusedDev fused;
};

size_t fold_bytes(int H, int W) {
    size_t b = fold_side_bytes(H) + fold_image_bytes(H, W);
    if (H != W) b += fold_side_bytes(W);
    int items = 0, ctrs = 0;
    fused_counts(H, W, items, ctrs);
    return b + fused_bytes(1, items, ctrs) + 64 * 1024;
}

cudaError_t fold_setup(DctPlan& d, char* p) {
    const int H = d.H, W = d.W;
    char* const p_begin = p;
    auto take = [&](size_t bytes) {
        void* r = p;
        p += rup(bytes, 1024);
        return r;
    };
    FoldBufs* fp = new FoldBufs();
    FoldBufs& f = *fp;
    d.fold_host = fp;
    const int f16 = d.prec == IRLS_PREC_FP16 ? 1 : 0;
    carve_fold_side(f.sN, H, take, f16);
    if (H != W) carve_fold_side(f.sM, W, take, f16);
    else f.sM = f.sN;
    carve_fold_image(f.img, H, W, take);
    f.dim = f.img.dim;
    f.fused.f16 = f16;
    {
        int items = 0, ctrs = 0;
        fused_counts(H, W, items, ctrs);
        carve_fused(f.fused, 1, items, ctrs, take);
    }
    // padding (columns hM.. of the folded residual, which nothing else writes) stays zero
    cudaError_t e = cudaMemset(p_begin, 0, (size_t)(p - p_begin));
    if (e != cudaSuccess) return e;
    d.Re = f.img.Re[0]; d.Relo = f.img.Re[1]; d.Ro = f.img.Ro[0]; d.Rolo = f.img.Ro[1];
    build_fold_side(f.sN);
    if (H != W) build_fold_side(f.sM);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = set_fold_attrs()) != cudaSuccess) return e;
    f.n_sm = device_sms();
    f.fused.pairs = fused_pairs(f.n_sm);
    return f.n_sm > 1 && f.fused.pairs > 0 ? cudaSuccess : cudaErrorInvalidDevice;
}

// (Re)builds the fused launch's problem table and work list for the given planes, state and
// flags and copies them in stream order (a launch still reading the previous tables finishes
// first).
cudaError_t fold_bind(const DctPlan& d, FoldBufs& f, const float* rU, float* zU, int ld,
                      DevState* st, double* partials, int flexible, int skip, int rho,
                      cudaStream_t s) {
    for (auto& t : f.tab) t.clear();
    if (!append_fold_problems(f.tab, f.img, f.sN, f.sM, d.H, d.W, rU, zU, ld, st, partials,
                              flexible, skip, d.tau, f.fused.f16))
        return cudaErrorNotSupported;
    if (f.fused.f16) {
        // stage 4's basis, scaled per frequency by tau / (mu + lambda_1): depends on tau
        const double sn = std::sin(3.14159265358979323846 / (2.0 * d.H));
        k_build_fold_stage4_f16<<<1024, 256, 0, s>>>(static_cast<__half*>(f.img.P4[0]),
                                                     static_cast<__half*>(f.img.P4[1]), d.W,
                                                     f.dim.hMp, 4.0 * sn * sn, (double)d.tau);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    int tiles[4];
    if (!number_fold_tiles(f.tab, tiles)) return cudaErrorInvalidValue;
    std::vector<GemmTile> probs;
    std::vector<FoldItem> items;
    int n_ctr = 0;
    if (!build_fused(f.tab, std::vector<int>{d.H}, f.fused.pairs, rho, probs, items, n_ctr,
                     f.stall))
        return cudaErrorInvalidValue;
    cudaError_t e = upload_fused(f.fused, probs, items, n_ctr, s);
    if (e != cudaSuccess) return e;
    f.bound = true;
    f.rU = rU; f.zU = zU; f.ld = ld; f.st = st; f.partials = partials;
    f.flexible = flexible; f.skip = skip; f.tau = d.tau; f.rho = rho;
    return cudaSuccess;
}

cudaError_t fold_apply(const DctPlan& d, const float* rU, float* zU, int ld, DevState* st,
                       int reduce_rho, int flexible, double* partials, int skip_if_done,
                       cudaStream_t s) {
    FoldBufs& f = *static_cast<FoldBufs*>(d.fold_host);
    if (!f.bound || f.rU != rU || f.zU != zU || f.ld != ld || f.st != st ||
        f.partials != partials || f.flexible != flexible || f.skip != skip_if_done ||
        f.tau != d.tau || f.rho != reduce_rho) {
        cudaError_t e =
            fold_bind(d, f, rU, zU, ld, st, partials, flexible, skip_if_done, reduce_rho, s);
        if (e != cudaSuccess) return e;
    }
    k_fold_r<<<fold_r_blocks(d.H, d.W, f.fused.f16), 256, 0, s>>>(
        fold_r_rec(f.img, rU, ld, d.H, d.W, st, f.fused.f16), skip_if_done);
    return launch_fused(f.fused, s);
}

}  // namespace

// Zeroes the fused launch's counters (each launch leaves them zero; this recovers from a launch
// that stopped on a timeout).
cudaError_t umma_dct_reset(const DctPlan& d, cudaStream_t s) {
    if (!d.fold_host) return cudaSuccess;
    const FusedDev& fd = static_cast<const FoldBufs*>(d.fold_host)->fused;
    return cudaMemsetAsync(fd.ctr, 0, (size_t)(fd.n_ctr + 1) * 4, s);
}

// Test hook: the folded launch's stage-2 waits run out (on) or not (off); false without a
// folded form.
bool umma_dct_stall(DctPlan& d, int on) {
    if (!d.fold_host || !d.fold) return false;
    FoldBufs& f = *static_cast<FoldBufs*>(d.fold_host);
    f.stall = on ? 1 : 0;
    f.bound = false;   // the tables are rebuilt on the next application
    return true;
}

void umma_dct_release(DctPlan& d) {
    delete static_cast<FoldBufs*>(d.fold_host);
    d.fold_host = nullptr;
    d.fold = d.fold_ready = 0;
}

// The fused folded launch's work list for images H[t] x W[t] run by `pairs` CTA pairs, built on
// the host exactly as the launch's set-up builds it, but with no tensor maps and no device
// memory (operand pointers are null).  Per item, kFoldSchedInts ints: stage (0-3), image, tile
// within its problem, first row, first column, columns, k-blocks per operand set, two operand
// sets, half width, counter completed (-1: none), dependency count, 8 counters waited for, 8
// counts waited for, r^T z run end, r^T z slot count, the problem's M, N and K, the problem
// among its stage's problems.  Also the counter count and the launch's item capacity.  False
// on a side below 256 (the folded form's minimum) or above 32768, or on a table the builders
// reject.
bool fold_schedule(const int* H, const int* W, int T, int pairs, int& n_items, int& n_ctr,
                   int& cap_items, std::vector<int>& rec) {
    if (T < 1 || pairs < 1) return false;
    std::vector<GemmTile> tab[4];
    std::vector<std::vector<float>> lam(2 * T);
    int est_items = 0, est_ctrs = 0;
    for (int t = 0; t < T; ++t) {
        if (H[t] < 256 || W[t] < 256 || H[t] > 32768 || W[t] > 32768) return false;
        FoldImage im{};
        im.dim = fold_dims(H[t], W[t]);
        FoldSide sN{}, sM{};
        sN.n = H[t];
        sN.hp = im.dim.hNp;
        sM.n = W[t];
        sM.hp = im.dim.hMp;
        lam[2 * t].assign(2 * (size_t)sN.hp, 0.f);
        lam[2 * t + 1].assign(2 * (size_t)sM.hp, 0.f);
        sN.lamP = lam[2 * t].data();
        sM.lamP = lam[2 * t + 1].data();
        if (!append_fold_problems(tab, im, sN, sM, H[t], W[t], nullptr, nullptr, W[t], nullptr,
                                  nullptr, 0, 1, 1e-2f, 0, false))
            return false;
        int it = 0, ct = 0;
        fused_counts(H[t], W[t], it, ct);
        est_items += it;
        est_ctrs += ct;
    }
    int tiles[4];
    if (!number_fold_tiles(tab, tiles)) return false;
    std::vector<GemmTile> probs;
    std::vector<FoldItem> items;
    if (!build_fused(tab, std::vector<int>(H, H + T), pairs, 1, probs, items, n_ctr)) return false;
    if (n_ctr != est_ctrs) return false;
    n_items = (int)items.size();
    cap_items = est_items + kMaxSplit;
    const int off[4] = {0, 2 * T, 6 * T, 8 * T}, per[4] = {2, 4, 2, 1};
    rec.assign((size_t)n_items * kFoldSchedInts, 0);
    for (int i = 0; i < n_items; ++i) {
        const FoldItem& f = items[i];
        const GemmTile& g = probs[f.prob];
        const int k = f.epi == UE_FOLD16 ? 0 : f.epi == UE_UNFOLD16 ? 2 : f.epi == UE_UNFOLDZ ? 3 : 1;
        int* r = rec.data() + (size_t)i * kFoldSchedInts;
        r[0] = k;
        r[1] = (f.prob - off[k]) / per[k];
        r[2] = f.local;
        r[3] = f.m0;
        r[4] = f.n0;
        r[5] = (f.half || k == 0) ? 128 : 256;
        r[6] = f.nkb;
        r[7] = f.dual;
        r[8] = f.half;
        r[9] = f.sig;
        r[10] = f.ndep;
        for (int d = 0; d < kMaxDeps; ++d) {
            r[11 + d] = d < f.ndep ? f.dep[d] : -1;
            r[19 + d] = d < f.ndep ? f.need[d] : 0;
        }
        r[27] = f.rho_end;
        r[28] = f.rho_nslot;
        r[29] = g.M;
        r[30] = g.N;
        r[31] = g.K;
        r[32] = f.prob - off[k];
    }
    return true;
}

size_t umma_dct_bytes(int H, int W, int prec) {
    const bool split = prec == IRLS_PREC_BF16X3;
    const size_t Hp = rup(H, 128), Wp = rup(W, 128);
    size_t n = 2 * Hp * Hp + 3 * Hp * Wp;
    if (H != W) n += 2 * Wp * Wp;
    if (split) n *= 2;
    size_t bytes = n * 2 + 32 * 1024;
    if (foldable(H, W, split || prec == IRLS_PREC_FP16)) bytes += fold_bytes(H, W);
    return bytes;
}

cudaError_t umma_dct_setup(DctPlan& d, char* mem) {
    const size_t Hp = d.Hp, Wp = d.Wp;
    const bool split = d.prec == IRLS_PREC_BF16X3;
    // every operand of every stage split: measured at 4096 x 4096, leaving any one operand of
    // any stage in a single bf16 pass raises the CG count from ~330 to 600-3000+ per outer step
    d.split = split ? 0xFF : 0;
    char* p = mem;
    auto take = [&](size_t elems) {
        void* r = p;
        p += rup(elems * 2, 1024);
        return r;
    };
    auto take2 = [&](size_t elems, void*& hi, void*& lo) {
        hi = take(elems);
        lo = split ? take(elems) : nullptr;
    };
    take2(Hp * Hp, d.PN16, d.PN16lo);
    take2(Hp * Hp, d.PNT16, d.PNT16lo);
    if (d.H != d.W) {
        take2(Wp * Wp, d.PM16, d.PM16lo);
        take2(Wp * Wp, d.PMT16, d.PMT16lo);
    } else {
        d.PM16 = d.PN16; d.PM16lo = d.PN16lo;
        d.PMT16 = d.PNT16; d.PMT16lo = d.PNT16lo;
    }
    take2(Hp * Wp, d.R16, d.R16lo);
    take2(Hp * Wp, d.S16a, d.S16alo);
    take2(Hp * Wp, d.S16b, d.S16blo);
    umma_dct_release(d);
    if (foldable(d.H, d.W, split || d.prec == IRLS_PREC_FP16)) {
        cudaError_t ef = fold_setup(d, p);
        if (ef != cudaSuccess) return ef;
        d.fold = d.fold_ready = 1;
    }
    using B = __nv_bfloat16;
    k_build_basis16<<<1024, 256>>>(static_cast<B*>(d.PN16), static_cast<B*>(d.PNT16),
                                   static_cast<B*>(d.PN16lo), static_cast<B*>(d.PNT16lo), d.H, d.Hp);
    if (d.H != d.W)
        k_build_basis16<<<1024, 256>>>(static_cast<B*>(d.PM16), static_cast<B*>(d.PMT16),
                                       static_cast<B*>(d.PM16lo), static_cast<B*>(d.PMT16lo), d.W,
                                       d.Wp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    TmapSet ts;
    std::memset(&ts, 0, sizeof(ts));
    const int H_ = d.Hp, W_ = d.Wp;
    bool ok = true;
    // (rows, cols) of A and B per stage, and the output width N that fixes the B box height
    const int mask = d.split;
    auto stage = [&](int si, void* a, void* al, int ar, int ac, void* b, void* bl, int br, int bc,
                     int N) {
        StageMaps& m = ts.st[si];
        const bool sa = split_a(mask, si), sb = split_b(mask, si);
        const int bn = pick_bn(N, sa || sb);
        ok &= make_map(&m.a0, a, ar, ac, UBM);
        ok &= make_map(&m.a1, sa ? al : a, ar, ac, UBM);
        ok &= make_map(&m.b0, b, br, bc, bn);
        ok &= make_map(&m.b1, sb ? bl : b, br, bc, bn);
    };
    // stage 1: A = PMT (Wp x Wp), B = R (Hp x Wp), N = Hp
    stage(0, d.PMT16, d.PMT16lo, W_, W_, d.R16, d.R16lo, H_, W_, H_);
    // stage 2: A = T1 (Wp x Hp), B = PNT (Hp x Hp), N = Hp
    stage(1, d.S16a, d.S16alo, W_, H_, d.PNT16, d.PNT16lo, H_, H_, H_);
    // stage 3: A = PN (Hp x Hp), B = T2 (Wp x Hp), N = Wp
    stage(2, d.PN16, d.PN16lo, H_, H_, d.S16b, d.S16blo, W_, H_, W_);
    // stage 4: A = T3 (Hp x Wp), B = PM (Wp x Wp), N = Wp
    stage(3, d.S16a, d.S16alo, H_, W_, d.PM16, d.PM16lo, W_, W_, W_);
    if (!ok) return cudaErrorNotSupported;
    if ((e = set_attrs<256, 1, 1>()) != cudaSuccess) return e;
    if ((e = set_attrs<128, 1, 1>()) != cudaSuccess) return e;
    if ((e = set_attrs<128, 2, 2>()) != cudaSuccess) return e;
    if ((e = set_attrs<128, 2, 1>()) != cudaSuccess) return e;
    if ((e = set_attrs<128, 1, 2>()) != cudaSuccess) return e;
    std::memcpy(d.tmap_storage, &ts, sizeof(ts));
    d.umma_ok = 1;
    return cudaSuccess;
}

cudaError_t umma_dct_apply(const DctPlan& d, const float* rU, float* zU, int ld, DevState* st,
                           int reduce_rho, const StencilArgs& a, double* partials,
                           int skip_if_done, cudaStream_t s) {
    if (!d.umma_ok) return cudaErrorNotSupported;
    if (d.fold) return fold_apply(d, rU, zU, ld, st, reduce_rho, a.flexible, partials, skip_if_done, s);
    const TmapSet& ts = *reinterpret_cast<const TmapSet*>(d.tmap_storage);
    const int Hp = d.Hp, Wp = d.Wp;
    const int mk = d.split;
    UEpiArgs ep{};
    ep.st = st;
    ep.partials = partials;
    ep.flexible = a.flexible;
    ep.skip_if_done = skip_if_done;
    cudaError_t e;
    // stage 1: T1 (Wp x Hp) = PMT . R^T; lo part kept if stage 2 splits its A operand
    ep.C = d.S16a; ep.C_lo = split_a(mk, 1) ? d.S16alo : nullptr; ep.ldc = Hp;
    e = launch_stage<UE_STORE16>(ts.st[0], Wp, Hp, Wp, split_a(mk, 0), split_b(mk, 0), ep, s);
    if (e != cudaSuccess) return e;
    // stage 2: T2 (Wp x Hp) = tau (T1 . PNT^T) / eig, zero frequency and padding -> 0
    ep.C = d.S16b; ep.C_lo = split_b(mk, 2) ? d.S16blo : nullptr; ep.ldc = Hp; ep.vm = d.W;
    ep.vn = d.H; ep.lam_m = d.lamM; ep.lam_n = d.lamN; ep.scale = d.tau;
    e = launch_stage<UE_EIG16>(ts.st[1], Wp, Hp, Hp, split_a(mk, 1), split_b(mk, 1), ep, s);
    if (e != cudaSuccess) return e;
    // stage 3: T3 (Hp x Wp) = PN . T2^T
    ep.C = d.S16a; ep.C_lo = split_a(mk, 3) ? d.S16alo : nullptr; ep.ldc = Wp;
    e = launch_stage<UE_STORE16>(ts.st[2], Hp, Wp, Hp, split_a(mk, 2), split_b(mk, 2), ep, s);
    if (e != cudaSuccess) return e;
    // stage 4: Z (H x W, pitch ld) = T3 . PM^T, and rho / beta
    ep.C = zU; ep.C_lo = nullptr; ep.ldc = ld; ep.vm = d.H; ep.vn = d.W; ep.rU = rU;
    if (reduce_rho)
        return launch_stage<UE_ZU_RHO>(ts.st[3], Hp, Wp, Wp, split_a(mk, 3), split_b(mk, 3), ep, s);
    return launch_stage<UE_ZU>(ts.st[3], Hp, Wp, Wp, split_a(mk, 3), split_b(mk, 3), ep, s);
}


// ------------------------------------------------------------------------------------------
// batched (grouped) form
// ------------------------------------------------------------------------------------------
namespace {

__global__ void k_build_lambda16(float* lam, int N, int Np) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < Np; k += gridDim.x * blockDim.x) {
        double v = 0.0;
        if (k < N) {
            const double sn = sinpi((double)k / (2.0 * N));
            v = 4.0 * sn * sn;
        }
        lam[k] = (float)v;
    }
}

struct SideBasis {
    int n, np;
    void *P, *PT, *Plo, *PTlo;
    float* lam;
};

struct BatchLayout {
    std::vector<int> sides;        // distinct side lengths
    size_t side_bytes = 0, image_bytes = 0, tiles_bytes = 0, total = 0;
};

BatchLayout batch_layout(const int* H, const int* W, int T, int prec, int fold) {
    BatchLayout L;
    if (fold) {
        for (int t = 0; t < T; ++t)
            for (int n : {H[t], W[t]})
                if (std::find(L.sides.begin(), L.sides.end(), n) == L.sides.end())
                    L.sides.push_back(n);
        for (int n : L.sides) L.side_bytes += fold_side_bytes(n);
        for (int t = 0; t < T; ++t) L.image_bytes += fold_image_bytes(H[t], W[t]);
        // the fold records and the fused launch's tables
        int items = 0, ctrs = 0;
        for (int t = 0; t < T; ++t) {
            int it = 0, ct = 0;
            fused_counts(H[t], W[t], it, ct);
            items += it;
            ctrs += ct;
        }
        L.tiles_bytes = rup((size_t)T * sizeof(FoldRRec), 1024) + fused_bytes(T, items, ctrs);
        L.total = L.side_bytes + L.image_bytes + L.tiles_bytes + 4096;
        return L;
    }
    const size_t mult = prec == IRLS_PREC_BF16X3 ? 2 : 1;
    for (int t = 0; t < T; ++t)
        for (int n : {H[t], W[t]})
            if (std::find(L.sides.begin(), L.sides.end(), n) == L.sides.end()) L.sides.push_back(n);
    for (int n : L.sides) {
        const size_t np = rup(n, 128);
        L.side_bytes += mult * 2 * rup(np * np * 2, 1024) + rup(np * 4, 1024);
    }
    for (int t = 0; t < T; ++t)
        L.image_bytes += mult * 3 * rup((size_t)rup(H[t], 128) * rup(W[t], 128) * 2, 1024);
    L.tiles_bytes = 4 * rup((size_t)T * sizeof(GemmTile), 1024);
    L.total = L.side_bytes + L.image_bytes + L.tiles_bytes + 4096;
    return L;
}

}  // namespace

// Per-tile r^T z slots of the folded form's stage 2: 16 per 256 x 256 tile (two CTAs x eight
// epilogue warps), four quarter problems of rup(H/2, 256) x rup(W/2, 256)
size_t dct_rho_slots(int H, int W) {
    return (size_t)(rup((H + 1) / 2, 256) / 256) * (rup((W + 1) / 2, 256) / 256) * 4 * 2 *
           k2EpiWarps;
}

size_t batch_dct_bytes(const int* H, const int* W, int T, int prec, int fold) {
    return batch_layout(H, W, T, prec, fold).total;
}

namespace {

// Folded form of a batch: bases per distinct side, each image's operands, and the four stage
// tables holding every image's problems in image order (an image's problems are consecutive,
// as its per-tile r^T z slots need).  The workspace arrives zeroed (padding stays zero).
cudaError_t batch_fold_setup(BatchDctPlan& bd, const int* H, const int* W, int T,
                             const BatchLayout& L, char* p, float tau, int flexible,
                             const float* const* rU, float* const* zU, const int* ld,
                             DevState* states, double* const* partials) {
    auto take = [&](size_t bytes) {
        void* r = p;
        p += rup(bytes, 1024);
        return r;
    };
    std::vector<FoldSide> sides(L.sides.size());
    for (size_t i = 0; i < L.sides.size(); ++i) {
        carve_fold_side(sides[i], L.sides[i], take);
        build_fold_side(sides[i]);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto side = [&](int n) -> const FoldSide& {
        for (const auto& sd : sides)
            if (sd.n == n) return sd;
        return sides[0];
    };
    std::vector<GemmTile> tab[4];
    std::vector<FoldRRec> recs(T);
    int blk = 0;
    for (int t = 0; t < T; ++t) {
        FoldImage im;
        carve_fold_image(im, H[t], W[t], take);
        if (!append_fold_problems(tab, im, side(H[t]), side(W[t]), H[t], W[t], rU[t], zU[t], ld[t],
                                  states + t, partials[t], flexible, 1, tau))
            return cudaErrorNotSupported;
        recs[t] = fold_r_rec(im, rU[t], ld[t], H[t], W[t], states + t);
        recs[t].blk0 = blk;
        recs[t].nblk = fold_r_blocks(H[t], W[t]);
        blk += recs[t].nblk;
    }
    int tiles[4];
    if (!number_fold_tiles(tab, tiles)) return cudaErrorInvalidValue;
    if ((e = set_fold_attrs()) != cudaSuccess) return e;
    bd.n_sm = device_sms();
    FusedDev fd;
    fd.pairs = fused_pairs(bd.n_sm);
    if (bd.n_sm < 2 || fd.pairs < 1) return cudaErrorInvalidDevice;
    {
        int items = 0, ctrs = 0;
        for (int t = 0; t < T; ++t) {
            int it = 0, ct = 0;
            fused_counts(H[t], W[t], it, ct);
            items += it;
            ctrs += ct;
        }
        carve_fused(fd, T, items, ctrs, take);
        std::vector<GemmTile> probs;
        std::vector<FoldItem> fitems;
        int n_ctr = 0;
        if (!build_fused(tab, std::vector<int>(H, H + T), fd.pairs, 1, probs, fitems, n_ctr))
            return cudaErrorInvalidValue;
        if ((e = upload_fused(fd, probs, fitems, n_ctr, 0)) != cudaSuccess) return e;
        if ((e = cudaMemset(fd.ctr, 0, (size_t)(fd.n_ctr + 1) * 4)) != cudaSuccess) return e;
    }
    bd.d_probs = fd.probs; bd.d_items = fd.items; bd.d_ctr = fd.ctr; bd.d_sts = fd.sts;
    bd.n_probs = fd.n_probs; bd.n_items = fd.n_items; bd.n_ctr = fd.n_ctr; bd.pairs = fd.pairs;
    bd.n_st = fd.n_st; bd.honour_stop = fd.honour_stop;
    bd.d_frec = take((size_t)T * sizeof(FoldRRec));
    bd.frec_blocks = blk;
    e = cudaMemcpy(bd.d_frec, recs.data(), (size_t)T * sizeof(FoldRRec), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    return cudaDeviceSynchronize();
}

}  // namespace

cudaError_t batch_dct_setup(BatchDctPlan& bd, const int* H, const int* W, int T, int prec,
                            int fold, float tau, int flexible, char* mem, const float* const* rU,
                            float* const* zU, const int* ld, DevState* states,
                            double* const* partials) {
    const bool split = prec == IRLS_PREC_BF16X3;
    bd.T = T; bd.prec = prec; bd.split = split ? 1 : 0; bd.tau = tau; bd.fold = fold ? 1 : 0;
    BatchLayout L = batch_layout(H, W, T, prec, fold);
    char* p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(mem) + 1023) & ~uintptr_t(1023));
    if (fold) {
        for (int t = 0; t < T; ++t)
            if (!foldable(H[t], W[t], split)) return cudaErrorInvalidValue;
        return batch_fold_setup(bd, H, W, T, L, p, tau, flexible, rU, zU, ld, states, partials);
    }
    auto take = [&](size_t bytes) {
        void* r = p;
        p += rup(bytes, 1024);
        return r;
    };
    using B = __nv_bfloat16;
    std::vector<SideBasis> basis;
    for (int n : L.sides) {
        SideBasis sb{};
        sb.n = n;
        sb.np = (int)rup(n, 128);
        const size_t e = (size_t)sb.np * sb.np * 2;
        sb.P = take(e); sb.PT = take(e);
        sb.Plo = split ? take(e) : nullptr;
        sb.PTlo = split ? take(e) : nullptr;
        sb.lam = static_cast<float*>(take((size_t)sb.np * 4));
        k_build_basis16<<<1024, 256>>>(static_cast<B*>(sb.P), static_cast<B*>(sb.PT),
                                       static_cast<B*>(sb.Plo), static_cast<B*>(sb.PTlo), n, sb.np);
        k_build_lambda16<<<4, 256>>>(sb.lam, n, sb.np);
        basis.push_back(sb);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto side = [&](int n) -> const SideBasis& {
        for (const auto& b : basis)
            if (b.n == n) return b;
        return basis[0];
    };
    std::vector<GemmTile> host[4];
    for (auto& h : host) h.resize(T);
    int cta[4] = {0, 0, 0, 0};
    bd.r16.resize(T); bd.r16lo.resize(T); bd.ld16.resize(T);
    bool ok = true;
    for (int t = 0; t < T; ++t) {
        const int Hp = (int)rup(H[t], 128), Wp = (int)rup(W[t], 128);
        const size_t e16 = (size_t)Hp * Wp * 2;
        void* R = take(e16); void* Rlo = split ? take(e16) : nullptr;
        void* Sa = take(e16); void* Salo = split ? take(e16) : nullptr;
        void* Sb = take(e16); void* Sblo = split ? take(e16) : nullptr;
        bd.r16[t] = R; bd.r16lo[t] = Rlo; bd.ld16[t] = Wp;
        const SideBasis& bn = side(H[t]);
        const SideBasis& bm = side(W[t]);
        auto maps = [&](GemmTile& g, void* a, void* al, int ar, int ac, void* b, void* bl, int br,
                        int bc) {
            ok &= make_map(&g.a0, a, ar, ac, UBM);
            ok &= make_map(&g.a1, split ? al : a, ar, ac, UBM);
            ok &= make_map(&g.b0, b, br, bc, 128);
            ok &= make_map(&g.b1, split ? bl : b, br, bc, 128);
        };
        UEpiArgs ep{};
        ep.st = states + t;
        ep.partials = partials[t];
        ep.flexible = flexible;
        ep.skip_if_done = 1;
        // stage 1: T1 (Wp x Hp) = PMT . R^T
        GemmTile& g0 = host[0][t];
        maps(g0, bm.PT, bm.PTlo, Wp, Wp, R, Rlo, Hp, Wp);
        g0.ep = ep; g0.ep.C = Sa; g0.ep.C_lo = split ? Salo : nullptr; g0.ep.ldc = Hp;
        g0.M = Wp; g0.N = Hp; g0.K = Wp;
        // stage 2: T2 (Wp x Hp) = tau (T1 . PNT^T) / eig
        GemmTile& g1 = host[1][t];
        maps(g1, Sa, Salo, Wp, Hp, bn.PT, bn.PTlo, Hp, Hp);
        g1.ep = ep; g1.ep.C = Sb; g1.ep.C_lo = split ? Sblo : nullptr; g1.ep.ldc = Hp;
        g1.ep.vm = W[t]; g1.ep.vn = H[t]; g1.ep.lam_m = bm.lam; g1.ep.lam_n = bn.lam;
        g1.ep.scale = tau;
        g1.M = Wp; g1.N = Hp; g1.K = Hp;
        // stage 3: T3 (Hp x Wp) = PN . T2^T
        GemmTile& g2 = host[2][t];
        maps(g2, bn.P, bn.Plo, Hp, Hp, Sb, Sblo, Wp, Hp);
        g2.ep = ep; g2.ep.C = Sa; g2.ep.C_lo = split ? Salo : nullptr; g2.ep.ldc = Wp;
        g2.M = Hp; g2.N = Wp; g2.K = Hp;
        // stage 4: Z (H x W, pitch ld) = T3 . PM^T, and rho / beta
        GemmTile& g3 = host[3][t];
        maps(g3, Sa, Salo, Hp, Wp, bm.P, bm.Plo, Wp, Wp);
        g3.ep = ep; g3.ep.C = zU[t]; g3.ep.C_lo = nullptr; g3.ep.ldc = ld[t];
        g3.ep.vm = H[t]; g3.ep.vn = W[t]; g3.ep.rU = rU[t];
        g3.M = Hp; g3.N = Wp; g3.K = Wp;
        for (int s = 0; s < 4; ++s) {
            GemmTile& g = host[s][t];
            g.gx = g.N / 128;
            g.blk0 = cta[s];
            cta[s] += (g.M / UBM) * g.gx;
        }
    }
    if (!ok) return cudaErrorNotSupported;
    for (int s = 0; s < 4; ++s) {
        bd.d_tiles[s] = take((size_t)T * sizeof(GemmTile));
        bd.total_ctas[s] = cta[s];
        e = cudaMemcpy(bd.d_tiles[s], host[s].data(), (size_t)T * sizeof(GemmTile),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return e;
    }
    using C22 = UCfg<128, 2, 2>;
    using C11 = UCfg<128, 1, 1>;
    const int sm = split ? C22::kSmem : C11::kSmem;
    for (auto f : {kb_umma_gemm<UE_STORE16, 2, 2>, kb_umma_gemm<UE_EIG16, 2, 2>,
                   kb_umma_gemm<UE_ZU_RHO, 2, 2>, kb_umma_gemm<UE_STORE16, 1, 1>,
                   kb_umma_gemm<UE_EIG16, 1, 1>, kb_umma_gemm<UE_ZU_RHO, 1, 1>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 split ? C22::kSmem : C11::kSmem);
        if (e != cudaSuccess) return e;
    }
    (void)sm;
    return cudaSuccess;
}

cudaError_t batch_dct_reset(const BatchDctPlan& bd, cudaStream_t s) {
    if (!bd.fold) return cudaSuccess;
    return cudaMemsetAsync(bd.d_ctr, 0, (size_t)(bd.n_ctr + 1) * 4, s);
}

cudaError_t batch_dct_apply(const BatchDctPlan& bd, cudaStream_t s) {
    using C22 = UCfg<128, 2, 2>;
    using C11 = UCfg<128, 1, 1>;
    const int T = bd.T;
    if (bd.fold) {
        k_fold_r_batched<<<bd.frec_blocks, 256, 0, s>>>(static_cast<const FoldRRec*>(bd.d_frec), T);
        FusedDev fd;
        fd.probs = static_cast<GemmTile*>(bd.d_probs);
        fd.items = static_cast<FoldItem*>(bd.d_items);
        fd.ctr = static_cast<unsigned*>(bd.d_ctr);
        fd.sts = static_cast<DevState**>(bd.d_sts);
        fd.n_probs = bd.n_probs; fd.n_items = bd.n_items; fd.n_ctr = bd.n_ctr; fd.pairs = bd.pairs;
        fd.n_st = bd.n_st; fd.honour_stop = bd.honour_stop;
        return launch_fused(fd, s);
    }
    auto tiles = [&](int k) { return static_cast<const GemmTile*>(bd.d_tiles[k]); };
    if (bd.split) {
        kb_umma_gemm<UE_STORE16, 2, 2><<<bd.total_ctas[0], kUThreads, C22::kSmem, s>>>(tiles(0), T);
        kb_umma_gemm<UE_EIG16, 2, 2><<<bd.total_ctas[1], kUThreads, C22::kSmem, s>>>(tiles(1), T);
        kb_umma_gemm<UE_STORE16, 2, 2><<<bd.total_ctas[2], kUThreads, C22::kSmem, s>>>(tiles(2), T);
        kb_umma_gemm<UE_ZU_RHO, 2, 2><<<bd.total_ctas[3], kUThreads, C22::kSmem, s>>>(tiles(3), T);
    } else {
        kb_umma_gemm<UE_STORE16, 1, 1><<<bd.total_ctas[0], kUThreads, C11::kSmem, s>>>(tiles(0), T);
        kb_umma_gemm<UE_EIG16, 1, 1><<<bd.total_ctas[1], kUThreads, C11::kSmem, s>>>(tiles(1), T);
        kb_umma_gemm<UE_STORE16, 1, 1><<<bd.total_ctas[2], kUThreads, C11::kSmem, s>>>(tiles(2), T);
        kb_umma_gemm<UE_ZU_RHO, 1, 1><<<bd.total_ctas[3], kUThreads, C11::kSmem, s>>>(tiles(3), T);
    }
    return cudaGetLastError();
}

}  // namespace irls
