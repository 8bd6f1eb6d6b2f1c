// Tensor-core (tcgen05) complex GEMM step: placeholder until the kernel lands.
#include "kernels.cuh"

namespace tnk {

bool gemm_tc_supports(const StepDesc &) { return false; }

cudaError_t launch_step_gemm_tc(const StepDesc &, int, int32_t *, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace tnk
