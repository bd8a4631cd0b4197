// Laplacian-block preconditioner of Sec. 3.3 by fast transforms: the same map as the dense
// products, z_U = P_N [ (P_N^T (tau r_U) P_M) / (l_i + m_j) ] P_M^T with the (0,0) entry set to
// zero, with every orthonormal DCT-II (P^T x) and DCT-III (P y) evaluated through a complex FFT
// of the same length (Makhoul's even/odd reordering) in float32 on the CUDA cores.
//
// Three launches per application, each one pass over a float32 plane:
//   rows_fwd  T[i][l]   = tau * DCT-II along the row i of r_U
//   cols      T[.][l]   = DCT-III( DCT-II(T[.][l]) / (l_k + m_l) ) per column l, in place;
//             rho_U     = sum_kl S_kl^2 / (tau (l_k + m_l)) = r_U^T z_U (Parseval), folded into
//                         the CG scalars by the last block
//   rows_inv  z_U[i][.] = DCT-III along the row i of T
// Two real sequences share one complex transform (the first as the real part, the second as the
// imaginary part); their spectra separate by the conjugate symmetry of a real sequence's DFT.
// The complex FFT is a Stockham auto-sort of radix-16 stages (then one radix-8, 4 or 2 stage) in
// shared memory; a block has one thread per radix-16 butterfly, which holds its sixteen values
// in registers between the stage's two barriers.  Row blocks load their two rows with 16-byte
// loads and store every element straight to its slot of the even/odd reordering; column blocks
// copy their strip in by 16-byte asynchronous copies in its natural order and fold the
// reordering into the first stage's reads.  Lengths: powers of two, and 2000, 4000, 8000, 16000
// (radix-5 stages after the radix-2^k ones).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "irls_internal.cuh"
#include "reduce.cuh"

namespace irls {

namespace {

constexpr int kFftMinN = 64;
constexpr int kFftMaxRowN = 16384;   // row transforms
constexpr int kFftMaxColN = 8192;    // column transforms

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// 16-byte asynchronous global -> shared copy; with `fill` false the 16 bytes are zeros.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool fill) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = fill ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---- in-register DFTs (forward sign: X_q = sum_r v_r exp(-2 pi i r q / R)) --------------------
template <int R>
__device__ __forceinline__ void dft(float2* v);

template <>
__device__ __forceinline__ void dft<2>(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void dft<4>(float2* v) {
    const float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = make_float2(d02.x + d13.y, d02.y - d13.x);   // d02 - i d13
    v[3] = make_float2(d02.x - d13.y, d02.y + d13.x);   // d02 + i d13
}

constexpr float kR2 = 0.70710678118654752f;    // cos(pi/4)
constexpr float kC8 = 0.92387953251128674f;    // cos(pi/8)
constexpr float kS8 = 0.38268343236508977f;    // sin(pi/8)

template <>
__device__ __forceinline__ void dft<8>(float2* v) {
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft<4>(e);
    dft<4>(o);
    o[1] = make_float2((o[1].x + o[1].y) * kR2, (o[1].y - o[1].x) * kR2);   // * exp(-i pi/4)
    o[2] = make_float2(o[2].y, -o[2].x);                                    // * -i
    o[3] = make_float2((o[3].y - o[3].x) * kR2, -(o[3].x + o[3].y) * kR2);  // * exp(-3 i pi/4)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 4] = csub(e[k], o[k]);
    }
}

// Length 16 as 4 x 4: DFT4 over n2 of v[n1 + 4 n2] for each n1, twiddle exp(-2 pi i n1 k2 / 16),
// DFT4 over n1; output k2 + 4 k1.
template <>
__device__ __forceinline__ void dft<16>(float2* v) {
    float2 y[4][4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) {
        float2 c[4] = {v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]};
        dft<4>(c);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) y[n1][k2] = c[k2];
    }
    // exp(-2 pi i e / 16) for e = n1 k2 in {1, 2, 3, 4, 6, 9}
    y[1][1] = cmul(y[1][1], make_float2(kC8, -kS8));
    y[1][2] = cmul(y[1][2], make_float2(kR2, -kR2));
    y[1][3] = cmul(y[1][3], make_float2(kS8, -kC8));
    y[2][1] = cmul(y[2][1], make_float2(kR2, -kR2));
    y[2][2] = make_float2(y[2][2].y, -y[2][2].x);
    y[2][3] = cmul(y[2][3], make_float2(-kR2, -kR2));
    y[3][1] = cmul(y[3][1], make_float2(kS8, -kC8));
    y[3][2] = cmul(y[3][2], make_float2(-kR2, -kR2));
    y[3][3] = cmul(y[3][3], make_float2(-kC8, kS8));
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        float2 c[4] = {y[0][k2], y[1][k2], y[2][k2], y[3][k2]};
        dft<4>(c);
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = c[k1];
    }
}

// Length 5: X_0 = v_0 + t1 + t2, X_{1,4} = a1 -/+ i b1, X_{2,3} = a2 -/+ i b2 with
// t1 = v1 + v4, t2 = v2 + v3, a1 = v0 + c1 t1 + c2 t2, a2 = v0 + c2 t1 + c1 t2,
// b1 = s1 (v1 - v4) + s2 (v2 - v3), b2 = s2 (v1 - v4) - s1 (v2 - v3), c_k + i s_k = exp(2 pi i k / 5).
constexpr float kC51 = 0.30901699437494745f, kC52 = -0.80901699437494734f;
constexpr float kS51 = 0.95105651629515353f, kS52 = 0.58778525229247325f;
template <>
__device__ __forceinline__ void dft<5>(float2* v) {
    const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    const float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    const float2 a1 = make_float2(v[0].x + kC51 * t1.x + kC52 * t2.x, v[0].y + kC51 * t1.y + kC52 * t2.y);
    const float2 a2 = make_float2(v[0].x + kC52 * t1.x + kC51 * t2.x, v[0].y + kC52 * t1.y + kC51 * t2.y);
    const float2 b1 = make_float2(kS51 * t3.x + kS52 * t4.x, kS51 * t3.y + kS52 * t4.y);
    const float2 b2 = make_float2(kS52 * t3.x - kS51 * t4.x, kS52 * t3.y - kS51 * t4.y);
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = make_float2(a1.x + b1.y, a1.y - b1.x);   // a1 - i b1
    v[4] = make_float2(a1.x - b1.y, a1.y + b1.x);   // a1 + i b1
    v[2] = make_float2(a2.x + b2.y, a2.y - b2.x);
    v[3] = make_float2(a2.x - b2.y, a2.y + b2.x);
}

// ---- shared-memory layouts of NF complex sequences of length N ------------------------------
// Pair: element m of transform f as one float2 (row 2f, row 2f + 1), one float2 of padding
// every 16 (the stages' strided accesses and the reordered stores of the load fall on distinct
// banks).  Row transforms.
template <int N, int NF>
struct PairL {
    static constexpr int P2 = N + N / 16;
    static constexpr int FLOATS = NF * 2 * P2;
    __device__ static __forceinline__ int off(int f, int m) { return 2 * (f * P2 + m + (m >> 4)); }
    __device__ static __forceinline__ float2 ld(const float* s, int f, int m) {
        return *reinterpret_cast<const float2*>(s + off(f, m));
    }
    __device__ static __forceinline__ void st(float* s, int f, int m, float2 v) {
        *reinterpret_cast<float2*>(s + off(f, m)) = v;
    }
};
// Strip: element m of all NF transforms in one row of 2 NF floats (transform f at 2f, 2f + 1),
// 4 floats of padding every 8 rows.  Column transforms: row m holds the 2 NF columns of image
// row m, copied in as they lie in memory.
template <int N, int NF>
struct StripL {
    static_assert(NF > 2, "two transforms a row: the swizzled layout below");
    static constexpr int FLOATS = N * 2 * NF + 4 * (N / 8);
    __device__ static __forceinline__ int off(int f, int m) { return m * 2 * NF + 2 * f + 4 * (m >> 3); }
    __device__ static __forceinline__ float2 ld(const float* s, int f, int m) {
        return *reinterpret_cast<const float2*>(s + off(f, m));
    }
    __device__ static __forceinline__ void st(float* s, int f, int m, float2 v) {
        *reinterpret_cast<float2*>(s + off(f, m)) = v;
    }
};

// Two transforms (four columns) a row: the 16-byte rows are swizzled instead of padded, row m
// at slot m ^ h(m / 8) with h(g) = (g / 2 + g % 2) % 8, so that the eight rows a half-warp
// touches lie in eight different 16-byte bank groups for consecutive rows, rows two apart (the
// first stage's reordered reads) and rows sixteen apart (its writes).
template <int N>
struct StripL<N, 2> {
    static constexpr int FLOATS = N * 4;
    __device__ static __forceinline__ int row(int m) {
        const int g = m >> 3;
        return m ^ (((g >> 1) + (g & 1)) & 7);
    }
    __device__ static __forceinline__ int off(int f, int m) { return 4 * row(m) + 2 * f; }
    __device__ static __forceinline__ float2 ld(const float* s, int f, int m) {
        return *reinterpret_cast<const float2*>(s + off(f, m));
    }
    __device__ static __forceinline__ void st(float* s, int f, int m, float2 v) {
        *reinterpret_cast<float2*>(s + off(f, m)) = v;
    }
};

// Element of the even/odd reordered sequence v_m of a length-N DCT: v_m = x_{2m} (m < N/2),
// x_{2N-1-2m} (m >= N/2); and where x_i goes.
template <int N>
__device__ __forceinline__ int reorder_src(int m) { return m < N / 2 ? 2 * m : 2 * N - 1 - 2 * m; }
template <int N>
__device__ __forceinline__ int reorder_pos(int i) { return (i & 1) ? N - 1 - (i >> 1) : (i >> 1); }

// exp(-2 pi i e / N) from the two-level table in shared memory: lo[e % 64] * hi[e / 64].
template <int N>
__device__ __forceinline__ float2 twiddle(const float2* tws, int e) {
    return cmul(tws[e & 63], tws[64 + (e >> 6)]);
}

// Entries of the two-level twiddle table of length N: 64 low and ceil(N / 64) high.
template <int N>
struct TwN {
    static constexpr int V = 64 + (N + 63) / 64;
    static constexpr int PADDED = (V + 1) & ~1;   // a 16-byte multiple
};

// Copies the two-level twiddle table of length N into shared memory.
template <int N, int T>
__device__ __forceinline__ void load_twiddles(float2* tws, const float2* __restrict__ tw) {
    for (int e = threadIdx.x; e < TwN<N>::V; e += T)
        tws[e] = e < 64 ? __ldg(&tw[e]) : __ldg(&tw[(e - 64) * 64]);
}

// Stockham stages of NF forward complex FFTs of length N in shared memory (layout L), from the
// stage whose sub-transforms have length NS; tws is the two-level table of exp(-2 pi i m / N).
// Thread t takes butterflies t, t + T, ... (the transform index varies fastest).  With REORD
// the first stage reads its inputs through the even/odd reordering.  Every stage reads, waits
// at a barrier, then writes over its inputs.
template <class L, int N, int NF, int T, int NS, bool REORD>
__device__ __forceinline__ void fft_stages(float* s, const float2* tws) {
    if constexpr (NS < N) {
        constexpr int REM = N / NS;
        constexpr int R = (REM % 16 == 0) ? 16 : (REM % 8 == 0) ? 8 : (REM % 4 == 0) ? 4
                        : (REM % 2 == 0) ? 2 : 5;
        static_assert(REM % R == 0, "lengths of the form 2^a 5^b");
        constexpr int NJ = N / R;                 // butterflies per transform
        constexpr int NB = NJ * NF;               // butterflies per stage
        constexpr int PER = (NB + T - 1) / T;     // butterflies per thread
        float2 v[PER][R];
#pragma unroll
        for (int b = 0; b < PER; ++b) {
            const int idx = threadIdx.x + b * T;
            if (NB % T == 0 || idx < NB) {
                const int f = idx % NF, j = idx / NF;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int m = j + r * NJ;
                    v[b][r] = L::ld(s, f, REORD ? reorder_src<N>(m) : m);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < PER; ++b) {
            const int idx = threadIdx.x + b * T;
            if (NB % T == 0 || idx < NB) {
                const int f = idx % NF, j = idx / NF;
                const int k = j % NS;
                if constexpr (NS > 1) {
                    // odd powers from the table, even ones as squares of lower powers
                    float2 w[R];
#pragma unroll
                    for (int r = 1; r < R; ++r)
                        w[r] = (r & 1) ? twiddle<N>(tws, k * r * (N / (NS * R))) : cmul(w[r / 2], w[r / 2]);
#pragma unroll
                    for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
                }
                dft<R>(v[b]);
                const int base = (j / NS) * NS * R + k;
#pragma unroll
                for (int r = 0; r < R; ++r) L::st(s, f, base + r * NS, v[b][r]);
            }
        }
        __syncthreads();
        fft_stages<L, N, NF, T, NS * R, false>(s, tws);
    }
}

// c_k of the orthonormal DCT basis, P[i][k] = c_k cos(pi k (2i+1) / 2N).
template <int N>
__device__ __forceinline__ float dct_c(int k) {
    return k == 0 ? __fsqrt_rn(1.f / (float)N) : __fsqrt_rn(2.f / (float)N);
}

// DCT-II coefficients X_k of the two real sequences packed in the transform Z (a: real part,
// b: imaginary part), from Z_k and Z_{N-k}; t = exp(-i pi k / 2N), c = c_k (times any scale).
__device__ __forceinline__ void dct2_coeffs(float2 Z, float2 Zc, float2 t, float c, float& xa,
                                            float& xb) {
    const float var = 0.5f * (Z.x + Zc.x), vai = 0.5f * (Z.y - Zc.y);   // spectrum of a
    const float vbr = 0.5f * (Z.y + Zc.y), vbi = -0.5f * (Z.x - Zc.x);  // spectrum of b
    xa = c * (t.x * var - t.y * vai);
    xb = c * (t.x * vbr - t.y * vbi);
}

// Spectrum V_k of the reordered sequence whose DCT-III has coefficients Y (already multiplied by
// c_k): V_k = exp(i pi k / 2N) (Y_k - i Y_{N-k}) sk, sk = 1 at k = 0 (Y_N = 0) and 1/2 else.
__device__ __forceinline__ float2 dct3_spec(float yk, float yp, float2 t, float sk) {
    return make_float2((t.x * yk - t.y * yp) * sk, (-t.x * yp - t.y * yk) * sk);
}

// conj(Va + i Vb): the packed spectrum of two real sequences, conjugated so that a forward FFT
// followed by a conjugation evaluates the inverse sum without a 1/N factor.
__device__ __forceinline__ float2 pack_conj(float2 va, float2 vb) {
    return make_float2(va.x - vb.y, -(va.y + vb.x));
}

// Writes transform f's conjugated packed spectra at slots k and N-k (0 <= k <= N/2) from the
// DCT-III coefficients (times c) of both sequences at k and at N-k; t = exp(-i pi k / 2N).
// The spectrum of a real sequence is Hermitian, so slot N-k takes the conjugates of slot k's
// two spectra: one complex product per sequence serves both slots.
template <class L, int N>
__device__ __forceinline__ void inv_pair(float* s, int f, int k, float ya_k, float yb_k, float ya_p,
                                         float yb_p, float2 t) {
    if (k == 0) {   // V_0 = Y_0 (Y_N = 0)
        L::st(s, f, 0, make_float2(ya_k, -yb_k));
        return;
    }
    const float2 pa = dct3_spec(ya_k, ya_p, t, 0.5f), pb = dct3_spec(yb_k, yb_p, t, 0.5f);
    L::st(s, f, k, pack_conj(pa, pb));
    if (k != N - k) L::st(s, f, N - k, make_float2(pa.x + pb.y, pa.y - pb.x));
}

// DCT-II coefficients of both sequences at k and at N-k from Z_k and Z_{N-k}: with
// w = t_k V_k (t_k = exp(-i pi k / 2N), V_k a sequence's spectrum), X_k = c_k Re w and
// X_{N-k} = -c_{N-k} Im w, since t_{N-k} V_{N-k} = -i conj(w).
__device__ __forceinline__ void dct2_pair(float2 Z, float2 Zc, float2 t, float ck, float cc,
                                          float& xa_k, float& xb_k, float& xa_c, float& xb_c) {
    const float2 va = make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y - Zc.y));
    const float2 vb = make_float2(0.5f * (Z.y + Zc.y), -0.5f * (Z.x - Zc.x));
    const float2 wa = cmul(t, va), wb = cmul(t, vb);
    xa_k = ck * wa.x;
    xb_k = ck * wb.x;
    xa_c = -cc * wa.y;
    xb_c = -cc * wb.y;
}

// Launch shapes: one thread per radix-16 butterfly of the block's NF transforms.  Rows: the
// pairs of rows of up to 4096 elements a block; columns: strips of 4 to 32 columns.
template <int N>
struct RowCfg {
    static constexpr int NF = (4096 / N) < 1 ? 1 : ((4096 / N) > 16 ? 16 : 4096 / N);
    static constexpr int T = (N * NF / 16 + 31) / 32 * 32;   // whole warps
    using L = PairL<N, NF>;
    static constexpr size_t SMEM = (size_t)L::FLOATS * sizeof(float) + TwN<N>::PADDED * sizeof(float2);
    static constexpr int WANT = 4;          // blocks per SM the carve-out is sized for
};
template <int N>
struct ColCfg {
    static constexpr int NF = (2048 / N) < 2 ? 2 : ((2048 / N) > 16 ? 16 : 2048 / N);
    static constexpr int T = (N * NF / 16 + 31) / 32 * 32;   // whole warps
    using L = StripL<N, NF>;
    static constexpr int TWN = TwN<N>::PADDED;             // twiddle table, 16-byte multiple
    static constexpr int TTN = N / 2 + 2;                  // exp(-i pi k / 2N), k <= N/2
    static constexpr size_t SMEM = (size_t)L::FLOATS * sizeof(float) +
                                   (size_t)(TWN + TTN) * sizeof(float2) + (size_t)N * sizeof(float);
    static constexpr int MINB = 1024 / T;   // at most 64 registers a thread
    static constexpr int WANT = MINB;
};

// ---- rows, forward: T[i][k] = tau * sum_j r_U[i][j] P_M[j][k] ---------------------------------
template <int N>
__global__ void __launch_bounds__(RowCfg<N>::T, 1024 / RowCfg<N>::T)
k_fftdct_rows_fwd(const float* __restrict__ R, float* __restrict__ Tout, int H, int ld, float tau,
                  const float2* __restrict__ tw, const float2* __restrict__ tt, const DevState* st,
                  int skip_if_done) {
    using C = RowCfg<N>;
    using L = typename C::L;
    constexpr int NF = C::NF, T = C::T, Q = N / 4;
    if (skip_if_done && st->done) return;
    extern __shared__ __align__(16) float sm[];
    float2* tws = reinterpret_cast<float2*>(sm + L::FLOATS);
    load_twiddles<N, T>(tws, tw);
    const int row0 = blockIdx.x * 2 * NF;
    // up to four 16-byte pieces of each of the two rows a thread (all loads first), every element
    // stored straight to its slot of the even/odd reordering
    static_assert(NF * Q <= 4 * T, "four pieces per thread at most");
    float4 va[4], vb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int it = threadIdx.x + u * T;
        const int f = it / Q, n = (it % Q) * 4;
        const int ra = row0 + 2 * f, rb = ra + 1;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool in = it < NF * Q;
        va[u] = in && ra < H ? __ldg(reinterpret_cast<const float4*>(R + (size_t)ra * ld + n)) : z4;
        vb[u] = in && rb < H ? __ldg(reinterpret_cast<const float4*>(R + (size_t)rb * ld + n)) : z4;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int it = threadIdx.x + u * T;
        if (NF * Q < 4 * T && it >= NF * Q) continue;
        const int f = it / Q, n = (it % Q) * 4;
        L::st(sm, f, reorder_pos<N>(n), make_float2(va[u].x, vb[u].x));
        L::st(sm, f, reorder_pos<N>(n + 1), make_float2(va[u].y, vb[u].y));
        L::st(sm, f, reorder_pos<N>(n + 2), make_float2(va[u].z, vb[u].z));
        L::st(sm, f, reorder_pos<N>(n + 3), make_float2(va[u].w, vb[u].w));
    }
    __syncthreads();
    fft_stages<L, N, NF, T, 1, false>(sm, tws);
    for (int it = threadIdx.x; it < NF * Q; it += T) {
        const int f = it / Q, k0 = (it % Q) * 4;
        const int ra = row0 + 2 * f, rb = ra + 1;
        float xa[4], xb[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int k = k0 + c;
            dct2_coeffs(L::ld(sm, f, k), L::ld(sm, f, (k == 0 ? 0 : N - k)), __ldg(&tt[k]),
                        dct_c<N>(k) * tau, xa[c], xb[c]);
        }
        if (ra < H)
            *reinterpret_cast<float4*>(Tout + (size_t)ra * ld + k0) = make_float4(xa[0], xa[1], xa[2], xa[3]);
        if (rb < H)
            *reinterpret_cast<float4*>(Tout + (size_t)rb * ld + k0) = make_float4(xb[0], xb[1], xb[2], xb[3]);
    }
}

// ---- columns: forward DCT, division by the eigenvalues, inverse DCT (in place) ---------------
// Block b owns the 2 NF columns 2 NF b ... (transform f: columns 2f and 2f + 1 of that range).
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::T, ColCfg<N>::MINB)
k_fftdct_cols(float* __restrict__ Tio, int W, int ld, float tau, const float* __restrict__ lamN,
              const float* __restrict__ lamM, const float2* __restrict__ tw,
              const float2* __restrict__ tt, DevState* st, double* partials, int reduce_rho,
              int skip_if_done, int flexible) {
    using C = ColCfg<N>;
    using L = typename C::L;
    constexpr int NF = C::NF, T = C::T, QC = NF / 2;   // 16-byte chunks per row
    if (skip_if_done && st->done) return;
    extern __shared__ __align__(16) float sm[];
    float2* tws = reinterpret_cast<float2*>(sm + L::FLOATS);
    // the middle step's tables (t_k for k <= N/2 and the eigenvalues l_k) come in with the strip
    float2* stt = tws + C::TWN;
    float* slam = reinterpret_cast<float*>(stt + C::TTN);
    load_twiddles<N, T>(tws, tw);
    const int j0 = blockIdx.x * 2 * NF;
    for (int c = threadIdx.x; c < N * QC; c += T) {
        const int i = c / QC, q = c % QC;
        const int col = j0 + 4 * q;
        const bool ok = col < W;
        cp_async16(sm + L::off(2 * q, i), Tio + (size_t)i * ld + (ok ? col : 0), ok);
    }
    for (int c = threadIdx.x; c < C::TTN / 2; c += T) cp_async16(stt + 2 * c, tt + 2 * c, true);
    for (int c = threadIdx.x; c < N / 4; c += T) cp_async16(slam + 4 * c, lamN + 4 * c, true);
    cp_async_wait_all();
    __syncthreads();
    fft_stages<L, N, NF, T, 1, true>(sm, tws);
    CSum part;
    constexpr int NK = N / 2 + 1;
    for (int it = threadIdx.x; it < NF * NK; it += T) {
        const int f = it % NF, k = it / NF;
        const int kc = (k == 0 ? 0 : N - k);
        const int ja = j0 + 2 * f, jb = ja + 1;
        const float2 t = stt[k];
        const float ck = dct_c<N>(k), cc = dct_c<N>(kc);
        float xa_k, xb_k, xa_c, xb_c;
        dct2_pair(L::ld(sm, f, k), L::ld(sm, f, kc), t, ck, cc, xa_k, xb_k, xa_c, xb_c);
        const float lk = slam[k], lc = slam[kc];
        const float ma = ja < W ? __ldg(&lamM[ja]) : 0.f, mb = jb < W ? __ldg(&lamM[jb]) : 0.f;
        // S / (l + m); the (0,0) entry (the constant, the Laplacian's null space) and the
        // columns past W are zero
        // (the denominators lie in (0, 8]: the fast division is within 2 ulp)
        const float sa_k = (ja < W && (k | ja) != 0) ? __fdividef(xa_k, lk + ma) : 0.f;
        const float sb_k = jb < W ? __fdividef(xb_k, lk + mb) : 0.f;
        const float sa_c = (ja < W && (kc | ja) != 0) ? __fdividef(xa_c, lc + ma) : 0.f;
        const float sb_c = jb < W ? __fdividef(xb_c, lc + mb) : 0.f;
        const float pk = xa_k * sa_k + xb_k * sb_k;
        part.add(kc != k ? pk + (xa_c * sa_c + xb_c * sb_c) : pk);
        inv_pair<L, N>(sm, f, k, ck * sa_k, ck * sb_k, cc * sa_c, cc * sb_c, t);
    }
    __syncthreads();
    fft_stages<L, N, NF, T, 1, false>(sm, tws);
    for (int c = threadIdx.x; c < N * QC; c += T) {
        const int i = c / QC, q = c % QC;
        const int col = j0 + 4 * q;
        if (col >= W) continue;
        const float4 v = *reinterpret_cast<const float4*>(sm + L::off(2 * q, reorder_pos<N>(i)));
        *reinterpret_cast<float4*>(Tio + (size_t)i * ld + col) = make_float4(v.x, -v.y, v.z, -v.w);
    }
    if (!reduce_rho) return;
    // r_U^T z_U = sum S^2 / (tau (l + m)) (the basis is orthonormal)
    double vv[1] = {part.value() / (double)tau}, tot[1];
    const Blk blk = single_blk();
    if (grid_reduce<1>(vv, partials, &st->counter, tot, blk.nblk, blk.bid) && threadIdx.x == 0) {
        const double rho_new = tot[0] + st->rz_v;
        if (!(rho_new > 0.0) || !isfinite(rho_new)) {
            // rho <= 0 is a breakdown unless the residual is already at the accuracy rounding
            // allows (relative 1e-3 and below)
            if (st->rel > 1e-3 || !isfinite(rho_new)) st->status |= ST_BREAKDOWN;
            st->done = 1;
        } else if (st->p_fresh) {
            st->rho = rho_new;
            st->beta = 0.0;
        } else {
            const double num = flexible ? rho_new - st->rz_old : rho_new;
            st->beta = num / st->rho;
            st->rho = rho_new;
        }
    }
}

// ---- rows, inverse: z_U[i][j] = sum_k T[i][k] P_M[j][k] --------------------------------------
template <int N>
__global__ void __launch_bounds__(RowCfg<N>::T, 1024 / RowCfg<N>::T)
k_fftdct_rows_inv(const float* __restrict__ Tin, float* __restrict__ Z, int H, int ld,
                  const float2* __restrict__ tw, const float2* __restrict__ tt, const DevState* st,
                  int skip_if_done) {
    using C = RowCfg<N>;
    using L = typename C::L;
    constexpr int NF = C::NF, T = C::T, Q = N / 4;
    if (skip_if_done && st->done) return;
    extern __shared__ __align__(16) float sm[];
    float2* tws = reinterpret_cast<float2*>(sm + L::FLOATS);
    load_twiddles<N, T>(tws, tw);
    const int row0 = blockIdx.x * 2 * NF;
    static_assert(NF * Q <= 4 * T, "four pieces per thread at most");
    float4 va[4], vb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int it = threadIdx.x + u * T;
        const int f = it / Q, k = (it % Q) * 4;
        const int ra = row0 + 2 * f, rb = ra + 1;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool in = it < NF * Q;
        va[u] = in && ra < H ? *reinterpret_cast<const float4*>(Tin + (size_t)ra * ld + k) : z4;
        vb[u] = in && rb < H ? *reinterpret_cast<const float4*>(Tin + (size_t)rb * ld + k) : z4;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int it = threadIdx.x + u * T;
        if (NF * Q < 4 * T && it >= NF * Q) continue;
        const int f = it / Q, k = (it % Q) * 4;
        L::st(sm, f, k, make_float2(va[u].x, vb[u].x));
        L::st(sm, f, k + 1, make_float2(va[u].y, vb[u].y));
        L::st(sm, f, k + 2, make_float2(va[u].z, vb[u].z));
        L::st(sm, f, k + 3, make_float2(va[u].w, vb[u].w));
    }
    __syncthreads();
    constexpr int NK = N / 2 + 1;
    for (int it = threadIdx.x; it < NF * NK; it += T) {
        const int f = it % NF, k = it / NF;
        const int kc = (k == 0 ? 0 : N - k);
        const float2 xk = L::ld(sm, f, k), xc = L::ld(sm, f, kc);
        const float ck = dct_c<N>(k), cc = dct_c<N>(kc);
        inv_pair<L, N>(sm, f, k, ck * xk.x, ck * xk.y, cc * xc.x, cc * xc.y, __ldg(&tt[k]));
    }
    __syncthreads();
    fft_stages<L, N, NF, T, 1, false>(sm, tws);
    for (int it = threadIdx.x; it < NF * Q; it += T) {
        const int f = it / Q, n = (it % Q) * 4;
        const int ra = row0 + 2 * f, rb = ra + 1;
        const float2 v0 = L::ld(sm, f, reorder_pos<N>(n)), v1 = L::ld(sm, f, reorder_pos<N>(n + 1));
        const float2 v2 = L::ld(sm, f, reorder_pos<N>(n + 2)), v3 = L::ld(sm, f, reorder_pos<N>(n + 3));
        if (ra < H)
            *reinterpret_cast<float4*>(Z + (size_t)ra * ld + n) = make_float4(v0.x, v1.x, v2.x, v3.x);
        if (rb < H)
            *reinterpret_cast<float4*>(Z + (size_t)rb * ld + n) = make_float4(-v0.y, -v1.y, -v2.y, -v3.y);
    }
}

// Twiddles of one transform length: tw[m] = exp(-2 pi i m / N), tt[k] = exp(-i pi k / 2N),
// from FP64 cospi / sinpi.
__global__ void k_build_fft_tables(float2* tw, float2* tt, int N) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < N; k += gridDim.x * blockDim.x) {
        const double a = 2.0 * (double)k / (double)N, b = (double)k / (2.0 * (double)N);
        tw[k] = make_float2((float)cospi(a), (float)-sinpi(a));
        tt[k] = make_float2((float)cospi(b), (float)-sinpi(b));
    }
}

bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

// Lengths compiled in besides the powers of two: 2^a 5^3 (radix-5 stages after the radix-2^k
// ones), the sides of the 4000 x M images of the paper's size study.
bool row_len_ok(int n) {
    return pow2_in(n, kFftMinN, kFftMaxRowN) || n == 2000 || n == 4000 || n == 8000 || n == 16000;
}
bool col_len_ok(int n) {
    return pow2_in(n, kFftMinN, kFftMaxColN) || n == 2000 || n == 4000 || n == 8000;
}

// Dynamic shared memory of a launch, and a carve-out that holds `want` blocks per SM (the rest
// of the SM's 256 KB stays L1).  Set before every launch: a host call of about a microsecond,
// and still right after the device's state was reset.
template <class K>
cudaError_t prepare(K k, size_t smem, int want) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const size_t per_block = smem + 1024;   // with the per-block reservation
    const int pct = (int)std::min<size_t>(100, (per_block * want * 100 + 228 * 1024 - 1) / (228 * 1024));
    return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

template <int N>
cudaError_t rows_fwd(const float* R, float* Tout, int H, int ld, float tau, const float2* tw,
                     const float2* tt, const DevState* st, int skip, cudaStream_t s) {
    using C = RowCfg<N>;
    cudaError_t e = prepare(k_fftdct_rows_fwd<N>, C::SMEM, C::WANT);
    if (e != cudaSuccess) return e;
    const int blocks = (H + 2 * C::NF - 1) / (2 * C::NF);
    k_fftdct_rows_fwd<N><<<blocks, C::T, C::SMEM, s>>>(R, Tout, H, ld, tau, tw, tt, st, skip);
    return cudaGetLastError();
}

template <int N>
cudaError_t rows_inv(const float* Tin, float* Z, int H, int ld, const float2* tw, const float2* tt,
                     const DevState* st, int skip, cudaStream_t s) {
    using C = RowCfg<N>;
    cudaError_t e = prepare(k_fftdct_rows_inv<N>, C::SMEM, C::WANT);
    if (e != cudaSuccess) return e;
    const int blocks = (H + 2 * C::NF - 1) / (2 * C::NF);
    k_fftdct_rows_inv<N><<<blocks, C::T, C::SMEM, s>>>(Tin, Z, H, ld, tw, tt, st, skip);
    return cudaGetLastError();
}

template <int N>
cudaError_t cols(float* Tio, int W, int ld, float tau, const float* lamN, const float* lamM,
                 const float2* tw, const float2* tt, DevState* st, double* partials, int reduce_rho,
                 int skip, int flexible, cudaStream_t s) {
    using C = ColCfg<N>;
    cudaError_t e = prepare(k_fftdct_cols<N>, C::SMEM, C::WANT);
    if (e != cudaSuccess) return e;
    const int blocks = (W + 2 * C::NF - 1) / (2 * C::NF);
    k_fftdct_cols<N><<<blocks, C::T, C::SMEM, s>>>(Tio, W, ld, tau, lamN, lamM, tw, tt, st,
                                                   partials, reduce_rho, skip, flexible);
    return cudaGetLastError();
}

int col_nf(int H) { return std::max(2, std::min(16, 2048 / H)); }

}  // namespace

bool fft_dct_supported(int H, int W) {
    return col_len_ok(H) && row_len_ok(W);
}

size_t fft_dct_bytes(int H, int W) {
    if (!fft_dct_supported(H, W)) return 0;
    return 2 * ((size_t)H + (size_t)W) * sizeof(float2) + 1024;
}

int fft_dct_max_blocks(int H, int W) {
    if (!fft_dct_supported(H, W)) return 0;
    return (W + 2 * col_nf(H) - 1) / (2 * col_nf(H));
}

cudaError_t fft_dct_setup(DctPlan& d, char* mem) {
    d.fft_ready = 0;
    if (!fft_dct_supported(d.H, d.W)) return cudaSuccess;
    float2* f = reinterpret_cast<float2*>(mem);
    d.fftTwN = f; f += d.H;
    d.fftTtN = f; f += d.H;
    d.fftTwM = f; f += d.W;
    d.fftTtM = f; f += d.W;
    k_build_fft_tables<<<(d.H + 255) / 256, 256>>>(d.fftTwN, d.fftTtN, d.H);
    k_build_fft_tables<<<(d.W + 255) / 256, 256>>>(d.fftTwM, d.fftTtM, d.W);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) d.fft_ready = 1;
    return e;
}

cudaError_t fft_dct_apply(const DctPlan& d, const float* rU, float* zU, int ld, DevState* st,
                          int reduce_rho, const StencilArgs& a, double* partials, int skip_if_done,
                          cudaStream_t s) {
    if (!d.fft_ready) return cudaErrorInvalidValue;
    const int H = d.H, W = d.W;
    float* T = d.T1;
    cudaError_t e = cudaErrorInvalidValue;
    switch (W) {
#define IRLS_FFT_ROWS(n) \
    case n: e = rows_fwd<n>(rU, T, H, ld, d.tau, d.fftTwM, d.fftTtM, st, skip_if_done, s); break;
        IRLS_FFT_ROWS(64) IRLS_FFT_ROWS(128) IRLS_FFT_ROWS(256) IRLS_FFT_ROWS(512)
        IRLS_FFT_ROWS(1024) IRLS_FFT_ROWS(2048) IRLS_FFT_ROWS(4096) IRLS_FFT_ROWS(8192)
        IRLS_FFT_ROWS(16384) IRLS_FFT_ROWS(2000) IRLS_FFT_ROWS(4000) IRLS_FFT_ROWS(8000)
        IRLS_FFT_ROWS(16000)
#undef IRLS_FFT_ROWS
        default: break;
    }
    if (e != cudaSuccess) return e;
    e = cudaErrorInvalidValue;
    switch (H) {
#define IRLS_FFT_COLS(n)                                                                        \
    case n:                                                                                     \
        e = cols<n>(T, W, ld, d.tau, d.lamN, d.lamM, d.fftTwN, d.fftTtN, st, partials,          \
                    reduce_rho, skip_if_done, a.flexible, s);                                   \
        break;
        IRLS_FFT_COLS(64) IRLS_FFT_COLS(128) IRLS_FFT_COLS(256) IRLS_FFT_COLS(512)
        IRLS_FFT_COLS(1024) IRLS_FFT_COLS(2048) IRLS_FFT_COLS(4096) IRLS_FFT_COLS(8192)
        IRLS_FFT_COLS(2000) IRLS_FFT_COLS(4000) IRLS_FFT_COLS(8000)
#undef IRLS_FFT_COLS
        default: break;
    }
    if (e != cudaSuccess) return e;
    e = cudaErrorInvalidValue;
    switch (W) {
#define IRLS_FFT_ROWS(n) \
    case n: e = rows_inv<n>(T, zU, H, ld, d.fftTwM, d.fftTtM, st, skip_if_done, s); break;
        IRLS_FFT_ROWS(64) IRLS_FFT_ROWS(128) IRLS_FFT_ROWS(256) IRLS_FFT_ROWS(512)
        IRLS_FFT_ROWS(1024) IRLS_FFT_ROWS(2048) IRLS_FFT_ROWS(4096) IRLS_FFT_ROWS(8192)
        IRLS_FFT_ROWS(16384) IRLS_FFT_ROWS(2000) IRLS_FFT_ROWS(4000) IRLS_FFT_ROWS(8000)
        IRLS_FFT_ROWS(16000)
#undef IRLS_FFT_ROWS
        default: break;
    }
    return e;
}

}  // namespace irls
