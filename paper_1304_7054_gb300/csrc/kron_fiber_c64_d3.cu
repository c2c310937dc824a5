// Instantiates the CUDA-core kernels for cf64 (interleaved complex) storage, 3-D operands.
#include "kron_fiber.cuh"

namespace kron {
kron_status launch_fiber_c64_d3(const KronDesc& d, cudaStream_t s) {
    return launch_fiber_d<cf64, cf64, 3>(d, s);
}
}  // namespace kron
