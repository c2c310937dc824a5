// Instantiates the CUDA-core kernels for __nv_bfloat16 storage, 3-D operands.
#include "kron_fiber.cuh"

namespace kron {
kron_status launch_fiber_bf16_d3(const KronDesc& d, cudaStream_t s) {
    return launch_fiber_d<float, __nv_bfloat16, 3>(d, s);
}
}  // namespace kron
