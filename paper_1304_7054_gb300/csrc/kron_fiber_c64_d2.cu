// Instantiates the CUDA-core kernels for cf64 (interleaved complex) storage, 2-D operands.
#include "kron_fiber.cuh"

namespace kron {
kron_status launch_fiber_c64_d2(const KronDesc& d, cudaStream_t s) {
    return launch_fiber_d<cf64, cf64, 2>(d, s);
}
}  // namespace kron
