// Instantiates the CUDA-core kernels for double storage, 2-D operands.
#include "kron_fiber.cuh"

namespace kron {
kron_status launch_fiber_f64_d2(const KronDesc& d, cudaStream_t s) {
    return launch_fiber_d<double, double, 2>(d, s);
}
}  // namespace kron
