// Tensor-core (tcgen05) form of the DCT preconditioner: placeholder until the kernel lands.
#include "irls_internal.cuh"

namespace irls {

size_t umma_dct_bytes(int, int) { return 0; }
cudaError_t umma_dct_setup(DctPlan&, char*) { return cudaErrorNotSupported; }
cudaError_t umma_dct_apply(const DctPlan&, float*, int, DevState*, const StencilArgs&, double*, int,
                           cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace irls
