// Host-side declarations shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kron.h"

namespace kron {

constexpr int kMaxN = 16;
constexpr int kFiberThreads = 256;   // threads per CTA of the CUDA-core kernels

// One call, after validation: components already have op() applied and are
// zero-padded to N x N (column-major); N = the largest dimension of the call.
// Mode naming: M1 acts on mode 1 (the fastest index of X), M2 on mode 2, M3 on
// mode 3.  2-D: M1 = op(B), M2 = op(A).  3-D: M1 = op(C), M2 = op(B), M3 = op(A).
struct KronDesc {
    int D = 2;          // 2 or 3
    int N = 1;          // padded size, 1..16
    double m1[kMaxN * kMaxN];
    double m2[kMaxN * kMaxN];
    double m3[kMaxN * kMaxN];
    // imaginary parts (complex storage; zero otherwise)
    double m1i[kMaxN * kMaxN] = {};
    double m2i[kMaxN * kMaxN] = {};
    double m3i[kMaxN * kMaxN] = {};
    const void* X = nullptr;
    void* Y = nullptr;
    int64_t batch = 0, ldxp = 0, ldyp = 0;
    int ldx = 0, ldx2 = 0, ldy = 0, ldy2 = 0;
    int xe[3] = {1, 1, 1};   // extents of op(X) per mode
    int ye[3] = {1, 1, 1};   // extents of Y per mode
    int transx = 0;
    int conjx = 0;      // complex: op(X) is the Hermitian transpose
    double alpha = 1.0, beta = 0.0;
    double alpha_im = 0.0, beta_im = 0.0;
    kron_dtype io = KRON_R32F;
    kron_compute comp = KRON_COMPUTE_NATIVE;
    // derived by the dispatcher
    int contiguous = 0;  // square, minimal leading dims, 16-B aligned X: bulk-copy tiles
    int ycontig = 0;     // square, minimal leading dims, 16-B aligned Y
    int yvec = 0;        // Y fiber store chunk in bytes (0 = element stores)
    // launch configuration (0 = choose automatically)
    int P = 0;           // instances per tile
    int nstage = -1;     // bulk-copy pipeline depth; 0 = generic loads; -1 = auto
    int grid = 0;        // CTAs; 0 = persistent (all resident CTAs)
    int variant = 0;     // kernel body (kron_variant); 0 = built-in choice
    int fps = 0;         // fibers per step of the last contraction; 0 = default
    int warps = 0;       // compute warps per CTA (bodies that take it); 0 = default
};

size_t elem_size(kron_dtype t);
bool is_complex(kron_dtype t);
// KRON_OK when [p, p + bytes) lies inside one device or managed allocation.
kron_status device_range(const void* p, size_t bytes);

// Fills d.P / d.nstage from the tile-configuration table, if it has an entry.
void apply_tile_config(KronDesc& d);
// Appends one entry to the tuning cache file (KRON_TUNE_CACHE), if set.
void tune_cache_append(int kind, int n, kron_dtype io, kron_compute comp, int P, int nstage);
// Compute-mode key under which the mixed-size path stores its per-class tile sizes.
constexpr int kVarlenTag = 7;
// Size of the fixed device array used by kron_varlen_execute_noalloc (32 bytes
// of tables per instance: up to 262,144 instances).
constexpr size_t kVarlenNoallocScratchBytes = (size_t)8 << 20;

// Device status word of the current device (device pointer).
unsigned* device_error_word();
// Limit of the first operand wait set by kron_set_first_wait_limit_ns (0 = off).
unsigned long long first_wait_limit_ns();

// CUDA-core (fiber) kernels, one entry per storage type and kind (one
// translation unit each, so they compile in parallel).
kron_status launch_fiber_f32_d2(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_f32_d3(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_f64_d2(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_f64_d3(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_bf16_d2(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_bf16_d3(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_f16_d2(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_f16_d3(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_c32_d2(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_c32_d3(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_c64_d2(const KronDesc& d, cudaStream_t s);
kron_status launch_fiber_c64_d3(const KronDesc& d, cudaStream_t s);

// Packed-pair FP32 kernels (even N, contiguous X and Y); KRON_ERR_NOT_SUPPORTED
// for shapes they do not handle.
kron_status launch_pair_f32_d2(const KronDesc& d, cudaStream_t s);
kron_status launch_pair_f32_d3(const KronDesc& d, cudaStream_t s);
kron_status launch_pair_bf16_d2(const KronDesc& d, cudaStream_t s);
kron_status launch_pair_bf16_d3(const KronDesc& d, cudaStream_t s);
kron_status launch_pair_f16_d2(const KronDesc& d, cudaStream_t s);
kron_status launch_pair_f16_d3(const KronDesc& d, cudaStream_t s);

// 2-D n = 16 FP32 pair kernel with the exchange in place in the operand tile
// (contiguous X and Y, 16 instances per tile); KRON_ERR_NOT_SUPPORTED otherwise.
kron_status launch_pair16(const KronDesc& d, cudaStream_t s);
// FP32 2-D n = 16 tensor-copy body: default tile, most compute warps, deepest ring.
constexpr int kPair16TDefaultP = 16;
constexpr int kPair16TMaxWarps = 16;
constexpr int kPair16TMaxRing = 12;
// 2-D n = 10, 14 FP32 pair kernels with the exchange in place (tiles of a
// multiple of 8 instances); KRON_ERR_NOT_SUPPORTED otherwise.
kron_status launch_pair2ip(const KronDesc& d, cudaStream_t s);
// 3-D FP32 pair kernels with all contractions in place (n = 16: one instance
// per tile; n = 10, 14: four); KRON_ERR_NOT_SUPPORTED otherwise.
kron_status launch_pair3ip(const KronDesc& d, cudaStream_t s);

// Batched GEMM with a varying first factor (TGEMM_A), after validation; the 1-D
// product (TKRON1) is the case m = 1.
struct GemmADesc {
    int m = 1, n = 1, k = 1;
    double b[16 * 16];       // op(B): b[l * 16 + j], l < k, j < n
    const void* A = nullptr;
    void* C = nullptr;
    int lda = 1, ldc = 1;
    int transa = 0;          // op(A^p)(i, l) at i + lda l (0) or l + lda i (1)
    int64_t lda2 = 0, ldc2 = 0, batch = 0;
    double alpha = 1.0, beta = 0.0;
    kron_dtype io = KRON_R32F;
    int grid = 0;            // CTAs; 0 = one persistent wave
};
kron_status launch_gemm_a(const GemmADesc& g, cudaStream_t s);
// TKRON1 given as that descriptor with m = 1 (FP32 / 16-bit storage);
// KRON_ERR_NOT_SUPPORTED otherwise.
kron_status launch_kron1(const GemmADesc& g, cudaStream_t s);

// Odd-n FP32 kernels (2-D and 3-D) with all contractions in place (tiles of a
// multiple of 4 instances); KRON_ERR_NOT_SUPPORTED otherwise.
kron_status launch_fiberip(const KronDesc& d, cudaStream_t s);

// Tensor-core split-precision kernels (R32F or R16BF storage).
kron_status launch_tc(const KronDesc& d, cudaStream_t s);

// SM count and per-SM shared memory of the current device (cached).
struct DeviceInfo {
    int device = -1;
    int sms = 0;
    size_t smem_per_block_optin = 0;
    size_t smem_per_sm = 0;
};
const DeviceInfo& device_info();

// Raises the dynamic shared-memory limit of kernel `fn` on the current device to
// at least `bytes` (remembered per kernel and device).  False on a CUDA error.
bool ensure_smem_optin(const void* fn, size_t bytes);

}  // namespace kron
