// Launchers of the 3-D split tensor bodies (one warp, or several warps, per
// instance), instantiated apart from the 2-D ones so that the two halves compile
// in parallel.  The kernels and their launch logic are in kron_tc.cuh.
#include "kron_tc.cuh"

namespace kron {

kron_status launch_tc3_any(const KronDesc& d, cudaStream_t st) {
    switch (d.io) {
        case KRON_R32F: return launch_tc3<float>(d, st);
        case KRON_R16BF: return launch_tc3<__nv_bfloat16>(d, st);
        case KRON_R16F: return launch_tc3<__half>(d, st);
        default: return KRON_ERR_NOT_SUPPORTED;
    }
}

}  // namespace kron
