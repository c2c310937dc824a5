// Instantiates the CUDA-core kernels for __half storage, 3-D operands.
#include "kron_fiber.cuh"

namespace kron {
kron_status launch_fiber_f16_d3(const KronDesc& d, cudaStream_t s) {
    return launch_fiber_d<float, __half, 3>(d, s);
}
}  // namespace kron
