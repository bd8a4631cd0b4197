// Deterministic grid-wide FP64 reductions finished by the last block of a launch.
#pragma once

#include <cuda_runtime.h>

namespace irls {

// Compensated float32 sum (Knuth's two-sum): hi + lo carries the running sum of the added terms
// with an error that does not grow with their number, at seven float32 operations per added
// term.  The per-thread partials of every inner product of the CG iteration are accumulated in
// one (each added term is a single value or a partial of at most four values of one image row),
// then carried into the FP64 warp, block and grid sums as (double)hi + (double)lo.  The
// intrinsics keep the compiler from contracting or reordering the error terms.
struct CSum {
    float hi, lo;
    __device__ __forceinline__ CSum() : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ void add(float x) {
        const float s = __fadd_rn(hi, x);
        const float bp = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Error-free transformations in float32: a + b = s + e and a * b = p + e exactly (Knuth's
// two-sum; the product's error from one fused multiply-add).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// The terms of A x that cancel (Sec. 3.2, the vectorised A), carried as hi + lo pairs so that
// the difference keeps the accuracy of its float32 operands:
//   s * (y0 + y1 + y2 + y3)        (the U row: s = 1/tau times a sum of four edge terms)
//   d * v - s * y                   (a V row: D V minus the penalty term)
__device__ __forceinline__ void sum4_scaled(float s, float y0, float y1, float y2, float y3,
                                            float& hi, float& lo) {
    float t, e1, e2, e3;
    two_sum(y0, y1, t, e1);
    two_sum(t, y2, t, e2);
    two_sum(t, y3, t, e3);
    two_prod(s, t, hi, lo);
    lo = __fmaf_rn(s, __fadd_rn(__fadd_rn(e1, e2), e3), lo);
}
__device__ __forceinline__ void diff_prod(float d, float v, float s, float y, float& hi,
                                          float& lo) {
    float p1, e1, p2, e2, e3;
    two_prod(d, v, p1, e1);
    two_prod(s, y, p2, e2);
    two_sum(p1, -p2, hi, e3);
    lo = __fadd_rn(e3, __fsub_rn(e1, e2));
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block coordinates of one problem's launch grid: the launch's own grid for a single image, or
// the problem's share of a batched launch (several images in one grid).
struct Blk {
    int bx, by;
    unsigned nblk, bid;
};

__device__ __forceinline__ Blk single_blk() {
    Blk b;
    b.bx = blockIdx.x;
    b.by = blockIdx.y;
    b.nblk = gridDim.x * gridDim.y;
    b.bid = blockIdx.x + gridDim.x * blockIdx.y;
    return b;
}

// Sums NV per-thread values over the problem's blocks (nblk of them, this one is bid).  Every
// block writes its partial to partials[k * nblk + bid]; the block that takes the last ticket
// adds the partials in a fixed order (so a re-run is bit-identical) and returns true with `tot`
// valid in all of its threads.  Other blocks return false.  The ticket counter is reset by the last block, so the
// next launch on the same stream can reuse it.  There is no waiting: a block that is not last
// simply leaves.
template <int NV>
__device__ bool grid_reduce(const double (&v)[NV], double* partials, unsigned int* counter,
                            double (&tot)[NV], unsigned nblk, unsigned bid) {
    __shared__ double sw[NV][32];
    __shared__ int s_last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5, nwarp = (nthr + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double t = warp_sum(v[k]);
        if (lane == 0) sw[k][warp] = t;
    }
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int w = 0; w < nwarp; ++w) s += sw[k][w];
            partials[(size_t)k * nblk + bid] = s;
        }
        __threadfence();
        unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == nblk - 1u);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (unsigned b = tid; b < nblk; b += nthr) s += __ldcg(&partials[(size_t)k * nblk + b]);
        s = warp_sum(s);
        if (lane == 0) sw[k][warp] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (int w = 0; w < nwarp; ++w) s += sw[k][w];
        tot[k] = s;
    }
    if (tid == 0) *counter = 0u;
    return true;
}

}  // namespace irls
