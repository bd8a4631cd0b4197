// Tiled unwrapping of one large image (see irls_tiled_create in include/irls.h).
//
// The paper leaves very large images to future work (Sec. 5) after its 4000 x M study
// (Sec. 4.5).  Here an image is cut into overlapping tiles of one size, the tiles are solved
// together as one batch (Alg. 1 with Alg. 2 on each, one launch per phase for all of them), and
// each tile's free constant is fixed by its agreement with its neighbours on their overlaps:
//   1. gather: the tiles' X and coherence are copied out of the image (one launch);
//   2. the batched solve;
//   3. for each pair of neighbouring tiles, the mean of U_t - U_s over their overlap, then the
//      mean again over the pixels within pi of the first (two launches, one block per pair,
//      FP64 sums in a fixed order);
//   4. on the host, the constants c minimising sum n_ts (c_s - c_t - d_ts)^2 with c_0 = 0 (the
//      graph Laplacian of the tile grid, a few hundred unknowns: conjugate gradients in FP64);
//   5. scatter: every pixel takes U_t + c_t from the tile whose core holds it (consecutive
//      tiles split their overlap at (start of the next + end of this) // 2), and the image's
//      sum is reduced in the same launch; then U -= mean(U).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "irls_internal.cuh"
#include "reduce.cuh"

namespace irls {
void set_last_cuda_error(int code);
}

using namespace irls;

namespace {

struct Fail {};

inline void ck(cudaError_t e) {
    if (e != cudaSuccess) {
        set_last_cuda_error((int)e);
        throw Fail{};
    }
}

constexpr int kThr = 256;
constexpr float kPi = 3.14159265358979323846f;

// One pair of neighbouring tiles and their overlap rectangle (image coordinates).
struct PairRec {
    int t, s;            // tile indices (t left of / above s)
    int r0, c0, r1, c1;  // overlap [r0, r1) x [c0, c1)
};

struct TiledDev {
    int H, W, th, tw, T, nr, nc;
    const int* rs;       // tile row starts (nr)
    const int* cs;       // tile column starts (nc)
    const int* rcore;    // core row bounds (nr + 1)
    const int* ccore;    // core column bounds (nc + 1)
    float* const* Ut;    // tile solutions (T pointers, th x tw each, contiguous)
};

}  // namespace

struct irls_tiled_s {
    int H = 0, W = 0, tile = 0, overlap = 0, th = 0, tw = 0, T = 0;
    std::vector<int> rs, cs, rcore, ccore;
    std::vector<PairRec> pairs;
    irls_batch batch = nullptr;
    char* mem = nullptr;          // one device allocation, carved below
    float* tX = nullptr;          // T tiles of X
    float* tC = nullptr;          // T tiles of coherence
    float* tU = nullptr;          // T tile solutions
    int* d_idx = nullptr;         // rs, cs, rcore, ccore
    float** d_Ut = nullptr;       // T pointers
    PairRec* d_pairs = nullptr;
    double* d_off = nullptr;      // per pair: (sum, count) of pass 1, then of pass 2
    float* d_c = nullptr;         // per tile: constant as hi, lo floats
    DevState* st = nullptr;
    double* partials = nullptr;
    int scatter_blocks = 0;
    std::vector<const float*> pX, pC;
    std::vector<float*> pU;
};

namespace {

// Tile starts along a side of n pixels: 0, t - o, 2 (t - o), ... while the tile ends before n,
// then one tile ending flush at n; one tile of n when n <= t.
std::vector<int> tile_starts(int n, int t, int o) {
    std::vector<int> out;
    if (n <= t) {
        out.push_back(0);
        return out;
    }
    for (int a = 0; a + t < n; a += t - o) out.push_back(a);
    out.push_back(n - t);
    return out;
}

std::vector<int> core_bounds(const std::vector<int>& st, int t, int n) {
    t = std::min(t, n);
    std::vector<int> b(st.size() + 1);
    b[0] = 0;
    for (size_t a = 0; a + 1 < st.size(); ++a) b[a + 1] = (st[a + 1] + st[a] + t) / 2;
    b[st.size()] = n;
    return b;
}

// X (and coherence) of every tile, copied out of the image: block = (tile, row), threads over
// the tile's columns.
__global__ void k_tile_gather(const float* __restrict__ X, const float* __restrict__ coh,
                              TiledDev d, float* __restrict__ tX, float* __restrict__ tC) {
    const int row = blockIdx.x % d.th, t = blockIdx.x / d.th;
    const int a = t / d.nc, b = t % d.nc;
    const size_t src = (size_t)(d.rs[a] + row) * d.W + d.cs[b];
    const size_t dst = ((size_t)t * d.th + row) * d.tw;
    for (int j = threadIdx.x; j < d.tw; j += blockDim.x) {
        tX[dst + j] = X[src + j];
        if (coh != nullptr) tC[dst + j] = coh[src + j];
    }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    __syncthreads();
    return s;
}

// Pass 1 (pass2 = 0): sum and count of U_t - U_s over the pair's overlap.  Pass 2: the same over
// the pixels within pi of pass 1's mean.  One block per pair, fixed order: deterministic.
__global__ void k_pair_offsets(TiledDev d, const PairRec* __restrict__ pairs,
                               double* __restrict__ off, int pass2) {
    __shared__ double sh[kThr / 32];
    const PairRec p = pairs[blockIdx.x];
    const int at = p.t / d.nc, bt = p.t % d.nc, as = p.s / d.nc, bs = p.s % d.nc;
    const float* Ut = d.Ut[p.t];
    const float* Us = d.Ut[p.s];
    const int w = p.c1 - p.c0;
    const size_t n = (size_t)(p.r1 - p.r0) * w;
    float m0 = 0.f;
    if (pass2) {
        const double c = off[4 * blockIdx.x + 1];
        m0 = c > 0.0 ? (float)(off[4 * blockIdx.x] / c) : 0.f;
    }
    CSum sum;
    double cnt = 0.0;
    for (size_t q = threadIdx.x; q < n; q += blockDim.x) {
        const int i = p.r0 + (int)(q / w), j = p.c0 + (int)(q % w);
        const float dv = Ut[(size_t)(i - d.rs[at]) * d.tw + (j - d.cs[bt])] -
                         Us[(size_t)(i - d.rs[as]) * d.tw + (j - d.cs[bs])];
        if (!pass2 || fabsf(dv - m0) < kPi) {
            sum.add(dv);
            cnt += 1.0;
        }
    }
    const double s = block_sum(sum.value(), sh);
    const double c = block_sum(cnt, sh);
    if (threadIdx.x == 0) {
        off[4 * blockIdx.x + 2 * pass2] = s;
        off[4 * blockIdx.x + 2 * pass2 + 1] = c;
    }
}

__device__ __forceinline__ int find_core(const int* bounds, int n, int x) {
    int lo = 0, hi = n - 1;   // bounds[0..n] with bounds[0] = 0, bounds[n] = size
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bounds[mid] <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Every pixel from the tile whose core holds it, plus that tile's constant; the image's sum
// into st->mean_u (divided by H W) by the launch's last block.
__global__ void k_tile_scatter(TiledDev d, const float* __restrict__ cst, float* __restrict__ U,
                               DevState* st, double* partials) {
    const size_t n = (size_t)d.H * d.W;
    CSum acc;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(q / d.W), j = (int)(q % d.W);
        const int a = find_core(d.rcore, d.nr, i), b = find_core(d.ccore, d.nc, j);
        const int t = a * d.nc + b;
        const float u = d.Ut[t][(size_t)(i - d.rs[a]) * d.tw + (j - d.cs[b])];
        const float v = __fadd_rn(__fadd_rn(u, cst[2 * t]), cst[2 * t + 1]);
        U[q] = v;
        acc.add(v);
    }
    double v[1] = {acc.value()}, tot[1];
    if (grid_reduce<1>(v, partials, &st->counter, tot, gridDim.x, blockIdx.x) && threadIdx.x == 0)
        st->mean_u = tot[0] / ((double)d.H * (double)d.W);
}

__global__ void k_sub_mean(float* __restrict__ U, size_t n, const DevState* st) {
    const float m = (float)st->mean_u;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
         q += (size_t)gridDim.x * blockDim.x)
        U[q] -= m;
}

// min over c (c_0 = 0) of sum n (c_s - c_t - d)^2: the normal equations L c = g of the weighted
// tile-grid Laplacian, reduced by c_0 = 0, solved by conjugate gradients in FP64 (symmetric
// positive definite on a connected grid).
void solve_constants(int T, const std::vector<PairRec>& pairs, const std::vector<double>& d,
                     const std::vector<double>& w, std::vector<double>& c) {
    c.assign(T, 0.0);
    if (T <= 1) return;
    std::vector<double> g(T, 0.0);
    for (size_t k = 0; k < pairs.size(); ++k) {
        g[pairs[k].s] += w[k] * d[k];
        g[pairs[k].t] -= w[k] * d[k];
    }
    auto apply = [&](const std::vector<double>& x, std::vector<double>& y) {
        std::fill(y.begin(), y.end(), 0.0);
        for (size_t k = 0; k < pairs.size(); ++k) {
            const int t = pairs[k].t, s = pairs[k].s;
            const double f = w[k] * (x[s] - x[t]);
            y[s] += f;
            y[t] -= f;
        }
        y[0] = 0.0;   // c_0 is fixed
    };
    std::vector<double> r = g, p, q(T);
    r[0] = 0.0;
    p = r;
    double rr = 0.0, r0 = 0.0;
    for (double x : r) rr += x * x;
    r0 = rr;
    for (int it = 0; it < 10 * T + 100 && rr > 1e-30 * r0 && rr > 0.0; ++it) {
        apply(p, q);
        double pq = 0.0;
        for (int k = 0; k < T; ++k) pq += p[k] * q[k];
        if (!(pq > 0.0)) break;
        const double al = rr / pq;
        double rn = 0.0;
        for (int k = 0; k < T; ++k) {
            c[k] += al * p[k];
            r[k] -= al * q[k];
            rn += r[k] * r[k];
        }
        const double be = rn / rr;
        rr = rn;
        for (int k = 0; k < T; ++k) p[k] = r[k] + be * p[k];
    }
}

size_t au(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" {

int irls_tiled_create(int H, int W, int tile, int overlap, const irls_opts* opts,
                      irls_tiled* out) {
    if (!out) return IRLS_ERR_ARG;
    *out = nullptr;
    if (H < 1 || W < 1 || tile < 2 || overlap < 1 || overlap >= tile) return IRLS_ERR_ARG;
    if ((long long)H * W > (1LL << 31)) return IRLS_ERR_SHAPE;
    irls_tiled_s* g = new (std::nothrow) irls_tiled_s;
    if (!g) return IRLS_ERR_OOM;
    g->H = H; g->W = W; g->tile = tile; g->overlap = overlap;
    g->th = std::min(tile, H);
    g->tw = std::min(tile, W);
    g->rs = tile_starts(H, tile, overlap);
    g->cs = tile_starts(W, tile, overlap);
    g->rcore = core_bounds(g->rs, tile, H);
    g->ccore = core_bounds(g->cs, tile, W);
    const int nr = (int)g->rs.size(), nc = (int)g->cs.size();
    g->T = nr * nc;
    for (int a = 0; a < nr; ++a)
        for (int b = 0; b < nc; ++b) {
            const int t = a * nc + b;
            if (b + 1 < nc) {
                PairRec p{t, t + 1, g->rs[a], g->cs[b + 1], g->rs[a] + g->th, g->cs[b] + g->tw};
                if (p.c1 > p.c0) g->pairs.push_back(p);
            }
            if (a + 1 < nr) {
                PairRec p{t, t + nc, g->rs[a + 1], g->cs[b], g->rs[a] + g->th, g->cs[b] + g->tw};
                if (p.r1 > p.r0) g->pairs.push_back(p);
            }
        }
    std::vector<int> Hs(g->T, g->th), Ws(g->T, g->tw);
    int rc = irls_batch_create(g->T, Hs.data(), Ws.data(), opts, &g->batch);
    if (rc != IRLS_OK) {
        delete g;
        return rc;
    }
    try {
        const size_t plane = (size_t)g->th * g->tw;
        const size_t nidx = g->rs.size() + g->cs.size() + g->rcore.size() + g->ccore.size();
        const size_t P = std::max<size_t>(g->pairs.size(), 1);
        g->scatter_blocks = (int)std::min<size_t>(((size_t)H * W + kThr - 1) / kThr, 4096);
        size_t off = 0;
        const size_t oX = off; off = au(off + 3 * (size_t)g->T * plane * sizeof(float));
        const size_t oI = off; off = au(off + nidx * sizeof(int));
        const size_t oP = off; off = au(off + (size_t)g->T * sizeof(float*));
        const size_t oR = off; off = au(off + P * sizeof(PairRec));
        const size_t oO = off; off = au(off + 4 * P * sizeof(double));
        const size_t oC = off; off = au(off + 2 * (size_t)g->T * sizeof(float));
        const size_t oS = off; off = au(off + sizeof(DevState));
        const size_t oQ = off; off = au(off + 8 * (size_t)g->scatter_blocks * sizeof(double));
        cudaError_t e = cudaMalloc(&g->mem, off);
        if (e != cudaSuccess) {
            set_last_cuda_error((int)e);
            irls_batch_destroy(g->batch);
            delete g;
            return IRLS_ERR_OOM;
        }
        g->tX = reinterpret_cast<float*>(g->mem + oX);
        g->tC = g->tX + (size_t)g->T * plane;
        g->tU = g->tC + (size_t)g->T * plane;
        g->d_idx = reinterpret_cast<int*>(g->mem + oI);
        g->d_Ut = reinterpret_cast<float**>(g->mem + oP);
        g->d_pairs = reinterpret_cast<PairRec*>(g->mem + oR);
        g->d_off = reinterpret_cast<double*>(g->mem + oO);
        g->d_c = reinterpret_cast<float*>(g->mem + oC);
        g->st = reinterpret_cast<DevState*>(g->mem + oS);
        g->partials = reinterpret_cast<double*>(g->mem + oQ);
        std::vector<int> idx;
        for (auto* v : {&g->rs, &g->cs, &g->rcore, &g->ccore}) idx.insert(idx.end(), v->begin(), v->end());
        ck(cudaMemcpy(g->d_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
        std::vector<float*> ut(g->T);
        for (int t = 0; t < g->T; ++t) {
            ut[t] = g->tU + (size_t)t * plane;
            g->pX.push_back(g->tX + (size_t)t * plane);
            g->pC.push_back(g->tC + (size_t)t * plane);
            g->pU.push_back(ut[t]);
        }
        ck(cudaMemcpy(g->d_Ut, ut.data(), ut.size() * sizeof(float*), cudaMemcpyHostToDevice));
        if (!g->pairs.empty())
            ck(cudaMemcpy(g->d_pairs, g->pairs.data(), g->pairs.size() * sizeof(PairRec),
                          cudaMemcpyHostToDevice));
        ck(cudaMemset(g->st, 0, sizeof(DevState)));
    } catch (Fail&) {
        if (g->mem) cudaFree(g->mem);
        irls_batch_destroy(g->batch);
        delete g;
        return IRLS_ERR_CUDA;
    }
    *out = g;
    return IRLS_OK;
}

int irls_tiled_destroy(irls_tiled g) {
    if (!g) return IRLS_OK;
    cudaDeviceSynchronize();
    if (g->mem) cudaFree(g->mem);
    irls_batch_destroy(g->batch);
    delete g;
    return IRLS_OK;
}

int irls_tiled_info(irls_tiled g, int* n_tiles, int* tile_h, int* tile_w, int* n_pairs) {
    if (!g || !n_tiles || !tile_h || !tile_w || !n_pairs) return IRLS_ERR_ARG;
    *n_tiles = g->T;
    *tile_h = g->th;
    *tile_w = g->tw;
    *n_pairs = (int)g->pairs.size();
    return IRLS_OK;
}

int irls_tiled_batch(irls_tiled g, irls_batch* batch) {
    if (!g || !batch) return IRLS_ERR_ARG;
    *batch = g->batch;
    return IRLS_OK;
}

int irls_unwrap_tiled(irls_tiled g, const float* d_X, const float* d_coherence, float* d_U,
                      irls_stats* per_tile, double* h_constants, void* stream) {
    if (!g || !d_X || !d_U) return IRLS_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int T = g->T, nr = (int)g->rs.size(), nc = (int)g->cs.size();
    TiledDev d;
    d.H = g->H; d.W = g->W; d.th = g->th; d.tw = g->tw; d.T = T; d.nr = nr; d.nc = nc;
    d.rs = g->d_idx;
    d.cs = d.rs + nr;
    d.rcore = d.cs + nc;
    d.ccore = d.rcore + nr + 1;
    d.Ut = g->d_Ut;
    int rc = IRLS_OK;
    try {
        TraceRange r_all("irls_unwrap_tiled");
        k_tile_gather<<<T * g->th, kThr, 0, s>>>(d_X, d_coherence, d, g->tX, g->tC);
        ck(cudaGetLastError());
        rc = irls_unwrap_batched_ex(g->batch, g->pX.data(),
                                    d_coherence ? g->pC.data() : nullptr, g->pU.data(),
                                    per_tile, stream);
        if (rc < 0) return rc;
        const int P = (int)g->pairs.size();
        std::vector<double> c;
        if (P > 0) {
            k_pair_offsets<<<P, kThr, 0, s>>>(d, g->d_pairs, g->d_off, 0);
            ck(cudaGetLastError());
            k_pair_offsets<<<P, kThr, 0, s>>>(d, g->d_pairs, g->d_off, 1);
            ck(cudaGetLastError());
            std::vector<double> off(4 * (size_t)P);
            ck(cudaMemcpyAsync(off.data(), g->d_off, off.size() * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
            ck(cudaStreamSynchronize(s));
            std::vector<double> dd(P), w(P);
            for (int k = 0; k < P; ++k) {
                // the second mean when it kept any pixel, else the first
                const bool two = off[4 * k + 3] > 0.0;
                w[k] = two ? off[4 * k + 3] : off[4 * k + 1];
                dd[k] = two ? off[4 * k + 2] / off[4 * k + 3]
                            : (off[4 * k + 1] > 0.0 ? off[4 * k] / off[4 * k + 1] : 0.0);
            }
            solve_constants(T, g->pairs, dd, w, c);
        } else {
            c.assign(T, 0.0);
        }
        std::vector<float> cf(2 * (size_t)T);
        for (int t = 0; t < T; ++t) {
            cf[2 * t] = (float)c[t];
            cf[2 * t + 1] = (float)(c[t] - (double)cf[2 * t]);
            if (h_constants) h_constants[t] = c[t];
        }
        ck(cudaMemcpyAsync(g->d_c, cf.data(), cf.size() * sizeof(float), cudaMemcpyHostToDevice,
                           s));
        k_tile_scatter<<<g->scatter_blocks, kThr, 0, s>>>(d, g->d_c, d_U, g->st, g->partials);
        ck(cudaGetLastError());
        k_sub_mean<<<g->scatter_blocks, kThr, 0, s>>>(d_U, (size_t)g->H * g->W, g->st);
        ck(cudaGetLastError());
        // cf is a host vector: the copy above must finish before it goes out of scope
        ck(cudaStreamSynchronize(s));
    } catch (Fail&) {
        return IRLS_ERR_CUDA;
    }
    return rc;
}

}  // extern "C"
