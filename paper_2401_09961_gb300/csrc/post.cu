// Post-processing of an unwrapped image (Sec. 4.5): the "rounded IRLS" output, 2pi-congruent to
// the input, and the best-shift error against a reference unwrapping.  FP64 grid reductions
// (deterministic last-block sums); the per-pixel integer decisions in float32, one correctly
// rounded operation at a time.
#include "irls_internal.cuh"
#include "reduce.cuh"

namespace irls {

namespace {

constexpr int kPostThreads = 256;
constexpr float kTwoPiF = 6.28318530717958647692f;   // 2pi rounded to float32

// sum cos(U - X), sum sin(U - X) in FP64; the last block stores the circular mean offset
// c = atan2(S, C) in st->aux[0]
__global__ void __launch_bounds__(kPostThreads)
k_circ_offset(const float* __restrict__ U, const float* __restrict__ X, size_t n, DevState* st,
              double* partials) {
    double c = 0.0, s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        double sn, cs;
        sincos((double)U[i] - (double)X[i], &sn, &cs);
        c += cs;
        s += sn;
    }
    double v[2] = {c, s}, tot[2];
    if (grid_reduce<2>(v, partials, &st->counter, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0)
        st->aux[0] = atan2(tot[1], tot[0]);
}

// K = rint(((U - c) - X) / 2pi), U_round = X + 2pi K
__global__ void __launch_bounds__(kPostThreads)
k_round_congruent(const float* __restrict__ U, const float* __restrict__ X, size_t n,
                  const DevState* st, float* __restrict__ Ur, int* __restrict__ K) {
    const float c = (float)st->aux[0];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float x = X[i];
        const float t = __fsub_rn(__fsub_rn(U[i], c), x);
        const float k = rintf(__fdiv_rn(t, kTwoPiF));
        if (Ur) Ur[i] = __fadd_rn(x, __fmul_rn(kTwoPiF, k));
        if (K) K[i] = (int)k;
    }
}

// alpha = mean(Xu - U) (FP64) into st->aux[1]
__global__ void __launch_bounds__(kPostThreads)
k_shift_mean(const float* __restrict__ U, const float* __restrict__ Xu, size_t n, DevState* st,
             double* partials) {
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        s += (double)Xu[i] - (double)U[i];
    double v[1] = {s}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0)
        st->aux[1] = tot[0] / (double)n;
}

// E = (Xu - U) - alpha (float32), sum E^2 (FP64) into st->aux[2]
__global__ void __launch_bounds__(kPostThreads)
k_shift_error(const float* __restrict__ U, const float* __restrict__ Xu, size_t n, DevState* st,
              double* partials, float* __restrict__ E) {
    const double alpha = st->aux[1];
    const float a32 = (float)alpha;
    double s2 = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float e = __fsub_rn(__fsub_rn(Xu[i], U[i]), a32);
        if (E) E[i] = e;
        const double ed = ((double)Xu[i] - (double)U[i]) - alpha;
        s2 += ed * ed;
    }
    double v[1] = {s2}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0)
        st->aux[2] = tot[0];
}

int post_blocks(size_t n, int max_blocks) {
    size_t b = (n + kPostThreads - 1) / kPostThreads;
    if (b > 1024) b = 1024;
    if (b > (size_t)max_blocks) b = (size_t)max_blocks;
    return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t launch_round_congruent(const float* U, const float* X, size_t n, DevState* st,
                                   double* partials, int max_blocks, float* Ur, int* K,
                                   cudaStream_t s) {
    const int nb = post_blocks(n, max_blocks);
    k_circ_offset<<<nb, kPostThreads, 0, s>>>(U, X, n, st, partials);
    k_round_congruent<<<nb, kPostThreads, 0, s>>>(U, X, n, st, Ur, K);
    return cudaGetLastError();
}

cudaError_t launch_best_shift(const float* U, const float* Xu, size_t n, DevState* st,
                              double* partials, int max_blocks, float* E, cudaStream_t s) {
    const int nb = post_blocks(n, max_blocks);
    k_shift_mean<<<nb, kPostThreads, 0, s>>>(U, Xu, n, st, partials);
    k_shift_error<<<nb, kPostThreads, 0, s>>>(U, Xu, n, st, partials, E);
    return cudaGetLastError();
}

}  // namespace irls
