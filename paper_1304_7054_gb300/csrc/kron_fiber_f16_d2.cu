// Instantiates the CUDA-core kernels for __half storage, 2-D operands.
#include "kron_fiber.cuh"

namespace kron {
kron_status launch_fiber_f16_d2(const KronDesc& d, cudaStream_t s) {
    return launch_fiber_d<float, __half, 2>(d, s);
}
}  // namespace kron
