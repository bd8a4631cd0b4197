// Allocation-free form of the Laplacian preconditioner (see irls_precond_laplacian_noalloc in
// include/irls.h).  Some callers cannot allocate device memory: plug-ins whose host framework
// owns every device byte through its own allocator, and latency-critical code that must never
// meet cudaMalloc's implicit device synchronisation or an out-of-memory failure from
// fragmentation after start-up.  For them the DCT bases and intermediates of a float32
// preconditioner application live in one fixed buffer compiled into this library, sized for
// images of up to IRLS_NOALLOC_MAX_SIDE x IRLS_NOALLOC_MAX_SIDE pixels.
#include <cmath>
#include <mutex>

#include "irls_internal.cuh"

namespace irls {
size_t dct_scratch_floats(int H, int W);
cudaError_t dct_apply_fp32_scratch(const float* R, float* Z, int H, int W, float tau, float* work,
                                   cudaStream_t s);
void set_last_cuda_error(int code);
}  // namespace irls

namespace {

constexpr int kMaxSide = IRLS_NOALLOC_MAX_SIDE;
// bases P_N, P_N^T, P_M, P_M^T, two intermediates and the pitched input: seven planes of
// kMaxSide^2 floats, plus two eigenvalue vectors (1.84 MB for kMaxSide = 256)
constexpr size_t kScratchFloats = 7u * kMaxSide * kMaxSide + 2u * kMaxSide;

// The scratch itself.  Every device that loads the library holds it until the process exits.
// In host code this name is only a host-side stand-in: kernels get its device address, looked
// up below with cudaGetSymbolAddress.
static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_addr[kMaxDevices] = {};

}  // namespace

extern "C" int irls_precond_laplacian_noalloc(const float* d_R, float* d_Z, int H, int W,
                                              float tau, void* stream) {
    using namespace irls;
    if (!d_R || !d_Z) return IRLS_ERR_ARG;
    if (!(tau > 0.f) || !std::isfinite(tau)) return IRLS_ERR_ARG;
    if (H < 1 || W < 1 || H > kMaxSide || W > kMaxSide) return IRLS_ERR_SHAPE;
    if (dct_scratch_floats(H, W) > kScratchFloats) return IRLS_ERR_SHAPE;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_last_cuda_error((int)e);
        return IRLS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return IRLS_ERR_UNSUPPORTED;
    float* scratch = nullptr;
    {
        // set-up, once per device, with that device current: the device address of the buffer
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_addr[dev] == nullptr) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                set_last_cuda_error((int)e);
                return IRLS_ERR_CUDA;
            }
            g_addr[dev] = static_cast<float*>(p);
        }
        scratch = g_addr[dev];
    }
    e = dct_apply_fp32_scratch(d_R, d_Z, H, W, tau, scratch, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_last_cuda_error((int)e);
        return IRLS_ERR_CUDA;
    }
    return IRLS_OK;
}
