// Deterministic grid-wide FP64 reductions finished by the last block of a launch.
#pragma once

#include <cuda_runtime.h>

namespace irls {

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
