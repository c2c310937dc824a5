// Instantiates the CUDA-core kernels for cf32 (interleaved complex) storage, 2-D operands.
#include "kron_fiber.cuh"

namespace kron {
kron_status launch_fiber_c32_d2(const KronDesc& d, cudaStream_t s) {
    return launch_fiber_d<cf32, cf32, 2>(d, s);
}
}  // namespace kron
