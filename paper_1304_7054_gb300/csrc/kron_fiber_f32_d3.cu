// Instantiates the CUDA-core kernels for float storage, 3-D operands.
#include "kron_fiber.cuh"

namespace kron {
kron_status launch_fiber_f32_d3(const KronDesc& d, cudaStream_t s) {
    return launch_fiber_d<float, float, 3>(d, s);
}
}  // namespace kron
