// C ABI entry points: argument validation, component preparation (op() applied
// once on the host, paper Sec. 2.2), choice of kernel, and the device status word.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "kron_device.cuh"
#include "kron_internal.h"

namespace kron {

// Device status word (bit kDevErrTimeout = a bounded device-side wait expired).
__device__ unsigned g_kron_device_error;

size_t elem_size(kron_dtype t) {
    switch (t) {
        case KRON_R32F: return 4;
        case KRON_R64F: return 8;
        case KRON_R16BF:
        case KRON_R16F: return 2;
        case KRON_C32F: return 8;
        case KRON_C64F: return 16;
    }
    return 0;
}

bool is_complex(kron_dtype t) { return t == KRON_C32F || t == KRON_C64F; }

constexpr int kMaxDevices = 64;

const DeviceInfo& device_info() {
    static DeviceInfo info[kMaxDevices];
    static std::mutex mu;
    static DeviceInfo none;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return none;
    std::lock_guard<std::mutex> lock(mu);
    DeviceInfo& d = info[dev];
    if (d.device != dev) {
        int sms = 0, optin = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
            return none;
        d.sms = sms;
        d.smem_per_block_optin = (size_t)optin;
        d.smem_per_sm = (size_t)per_sm;
        d.device = dev;
    }
    return d;
}

bool ensure_smem_optin(const void* fn, size_t bytes) {
    static std::map<std::pair<const void*, int>, size_t> done;
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lock(mu);
    size_t& cur = done[std::make_pair(fn, dev)];
    if (bytes <= cur) return true;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return false;
    cur = bytes;
    return true;
}

unsigned* device_error_word() {
    static unsigned* ptr[kMaxDevices] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_kron_device_error) != cudaSuccess) return nullptr;
        ptr[dev] = static_cast<unsigned*>(p);
    }
    return ptr[dev];
}

static std::atomic<unsigned long long> g_first_wait_ns{0};

unsigned long long first_wait_limit_ns() { return g_first_wait_ns.load(std::memory_order_relaxed); }

static bool trans_flag(char t, int* is_t) {
    switch (t) {
        case 'N': case 'n': *is_t = 0; return true;
        case 'T': case 't': case 'C': case 'c': *is_t = 1; return true;
        default: return false;
    }
}

// 'C' / 'c' (Hermitian transpose) conjugates complex data.
static int conj_flag(char t, kron_dtype io) { return is_complex(io) && (t == 'C' || t == 'c'); }

static bool dim_ok(int v) { return v >= 1 && v <= kMaxN; }

// op(M) (rows x cols) from the stored matrix (leading dimension ld), zero-padded
// into an N x N column-major block.
static void op_pad(double* out, int N, const void* M, int ld, int is_t, int rows, int cols, bool dbl) {
    for (int e = 0; e < N * N; ++e) out[e] = 0.0;
    for (int c = 0; c < cols; ++c)
        for (int r = 0; r < rows; ++r) {
            const size_t idx = is_t ? (size_t)c + (size_t)ld * r : (size_t)r + (size_t)ld * c;
            out[r + N * c] = dbl ? static_cast<const double*>(M)[idx] : (double)static_cast<const float*>(M)[idx];
        }
}

// Complex op(M) (rows x cols), conjugated for 'C', zero-padded into N x N
// real and imaginary parts.  M holds interleaved (re, im) pairs.
static void op_pad_complex(double* re, double* im, int N, const void* M, int ld, int is_t, int conj, int rows,
                           int cols, bool dbl) {
    for (int e = 0; e < N * N; ++e) re[e] = im[e] = 0.0;
    for (int c = 0; c < cols; ++c)
        for (int r = 0; r < rows; ++r) {
            const size_t idx = is_t ? (size_t)c + (size_t)ld * r : (size_t)r + (size_t)ld * c;
            const double vr = dbl ? static_cast<const double*>(M)[2 * idx] : (double)static_cast<const float*>(M)[2 * idx];
            const double vi =
                dbl ? static_cast<const double*>(M)[2 * idx + 1] : (double)static_cast<const float*>(M)[2 * idx + 1];
            re[r + N * c] = vr;
            im[r + N * c] = conj ? -vi : vi;
        }
}

// A host scalar of the compute type of io: (re, im) for complex storage.
static void scalar_of(const void* v, kron_dtype io, double* re, double* im) {
    *im = 0.0;
    switch (io) {
        case KRON_R64F: *re = *static_cast<const double*>(v); break;
        case KRON_C64F: *re = static_cast<const double*>(v)[0]; *im = static_cast<const double*>(v)[1]; break;
        case KRON_C32F: *re = static_cast<const float*>(v)[0]; *im = static_cast<const float*>(v)[1]; break;
        default: *re = (double)*static_cast<const float*>(v); break;
    }
}

static bool ranges_overlap(const void* a, size_t abytes, const void* b, size_t bbytes) {
    const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
    return a0 < b0 + bbytes && b0 < a0 + abytes;
}

}  // namespace kron

// Whether address p is device-accessible memory: a device allocation of the
// current GPU or a managed allocation.
static kron_status device_pointer(const void* p) {
    cudaPointerAttributes at;
    const cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorInvalidValue ? KRON_ERR_INVALID_VALUE : KRON_ERR_CUDA;
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return KRON_ERR_INVALID_VALUE;
    if (at.type == cudaMemoryTypeDevice) {   // memory of another GPU: the launch runs on the current one
        int cur = -1;
        if (cudaGetDevice(&cur) != cudaSuccess) return KRON_ERR_CUDA;
        if (at.device != cur) return KRON_ERR_INVALID_VALUE;
    }
    return KRON_OK;
}

// Whether [p, p + bytes) is device-accessible memory of the current GPU (device
// or managed), mapped without a hole.  A host pointer or an extent beyond the
// mapping would make a kernel fault, so the calls reject both before any launch.
// The driver reports one mapped range per query; allocators that map memory in
// chunks (virtual memory management, e.g. expandable segments) give one range
// per chunk, so the check walks adjacent ranges, each of which must itself be
// device memory of this GPU.  KRON_ERR_CUDA when the runtime cannot answer (no
// device).
kron_status kron::device_range(const void* p, size_t bytes) {
    kron_status st = device_pointer(p);
    if (st != KRON_OK) return st;
    // The allocation's extent, from the driver (resolved once).
    typedef int (*GetRange)(unsigned long long*, size_t*, unsigned long long);
    static GetRange get_range = [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        cudaGetLastError();
        return reinterpret_cast<GetRange>(fn);
    }();
    if (!get_range) return KRON_OK;   // type check only
    const unsigned long long end = (unsigned long long)(uintptr_t)p + bytes;
    unsigned long long cur = (unsigned long long)(uintptr_t)p;
    for (int seg = 0; seg < 65536; ++seg) {
        unsigned long long base = 0;
        size_t size = 0;
        if (get_range(&base, &size, cur) != 0 || size == 0 || base + size <= cur) return KRON_ERR_INVALID_VALUE;
        if (end <= base + size) return KRON_OK;
        cur = base + size;   // first byte after this range: mapped device memory of this GPU, or the end
        if ((st = device_pointer((const void*)(uintptr_t)cur)) != KRON_OK) return st;
    }
    return KRON_ERR_INVALID_VALUE;
}

namespace kron {

static void choose_yvec(KronDesc& d) {
    const size_t s = elem_size(d.io);
    d.yvec = 0;
    if (d.ye[0] != d.N) return;
    for (int vb = 16; vb >= 4; vb /= 2) {
        if ((size_t)vb < s) break;
        const bool ok = (d.N * s) % vb == 0 && ((uintptr_t)d.Y) % vb == 0 && ((size_t)d.ldy * s) % vb == 0 &&
                        (d.D == 2 || ((size_t)d.ldy2 * s) % vb == 0) && ((size_t)d.ldyp * s) % vb == 0;
        if (ok) { d.yvec = vb; return; }
    }
}

static kron_status dispatch(KronDesc& d, cudaStream_t st) {
    apply_tile_config(d);
    if (d.io == KRON_C32F) return d.D == 2 ? launch_fiber_c32_d2(d, st) : launch_fiber_c32_d3(d, st);
    if (d.io == KRON_C64F) return d.D == 2 ? launch_fiber_c64_d2(d, st) : launch_fiber_c64_d3(d, st);
    if (d.comp == KRON_COMPUTE_32F_BF16X3) return launch_tc(d, st);
    // An explicit kernel body (kron_set_kernel_config) for contiguous batches.
    if (d.contiguous && d.ycontig && d.variant != KRON_VARIANT_AUTO) {
        kron_status r = KRON_ERR_NOT_SUPPORTED;
        if (d.variant == KRON_VARIANT_IN_PLACE) {
            if (d.D == 2 && d.N == 16) r = launch_pair16(d, st);
            else if (d.io == KRON_R32F && d.D == 2 && (d.N == 10 || d.N == 14)) r = launch_pair2ip(d, st);
            else if (d.io == KRON_R32F && d.D == 3 && (d.N == 10 || d.N == 14 || d.N == 16)) r = launch_pair3ip(d, st);
            else if (d.io == KRON_R32F && (d.N & 1) && d.N >= 3) r = launch_fiberip(d, st);
        } else if (d.variant == KRON_VARIANT_EXCHANGE && d.N % 2 == 0) {
            switch (d.io) {
                case KRON_R32F: r = d.D == 2 ? launch_pair_f32_d2(d, st) : launch_pair_f32_d3(d, st); break;
                case KRON_R16BF: r = d.D == 2 ? launch_pair_bf16_d2(d, st) : launch_pair_bf16_d3(d, st); break;
                case KRON_R16F: r = d.D == 2 ? launch_pair_f16_d2(d, st) : launch_pair_f16_d3(d, st); break;
                default: break;
            }
        }
        if (r != KRON_ERR_NOT_SUPPORTED) return r;   // otherwise the scalar body below
    } else if (d.contiguous && d.ycontig && d.N % 2 == 0 && d.io != KRON_R64F) {
        kron_status r = KRON_ERR_NOT_SUPPORTED;
        // In-place kernels where they beat the generic one (n = 16 in 2-D for every storage type).
        if (d.D == 2 && d.N == 16 && d.comp == KRON_COMPUTE_NATIVE) r = launch_pair16(d, st);
        else if (d.io == KRON_R32F) {
            if (d.D == 2 && (d.N == 10 || d.N == 14)) r = launch_pair2ip(d, st);
            else if (d.D == 3 && (d.N == 16 || d.N == 10 || d.N == 14)) r = launch_pair3ip(d, st);
        }
        if (r != KRON_ERR_NOT_SUPPORTED) return r;
        switch (d.io) {
            case KRON_R32F: r = d.D == 2 ? launch_pair_f32_d2(d, st) : launch_pair_f32_d3(d, st); break;
            case KRON_R16BF: r = d.D == 2 ? launch_pair_bf16_d2(d, st) : launch_pair_bf16_d3(d, st); break;
            case KRON_R16F: r = d.D == 2 ? launch_pair_f16_d2(d, st) : launch_pair_f16_d3(d, st); break;
            default: break;
        }
        if (r != KRON_ERR_NOT_SUPPORTED) return r;
    }
    if ((d.N & 1) && d.N >= 3 && d.io == KRON_R32F && d.contiguous && d.ycontig && d.variant == KRON_VARIANT_AUTO) {
        const kron_status r = launch_fiberip(d, st);   // odd n, all contractions in place
        if (r != KRON_ERR_NOT_SUPPORTED) return r;
    }
    switch (d.io) {
        case KRON_R32F: return d.D == 2 ? launch_fiber_f32_d2(d, st) : launch_fiber_f32_d3(d, st);
        case KRON_R64F: return d.D == 2 ? launch_fiber_f64_d2(d, st) : launch_fiber_f64_d3(d, st);
        case KRON_R16BF: return d.D == 2 ? launch_fiber_bf16_d2(d, st) : launch_fiber_bf16_d3(d, st);
        case KRON_R16F: return d.D == 2 ? launch_fiber_f16_d2(d, st) : launch_fiber_f16_d3(d, st);
    }
    return KRON_ERR_INVALID_VALUE;
}

static kron_status check_modes(kron_dtype io, kron_compute comp) {
    if (io != KRON_R32F && io != KRON_R64F && io != KRON_R16BF && io != KRON_R16F && !is_complex(io))
        return KRON_ERR_INVALID_VALUE;
    if (comp == KRON_COMPUTE_NATIVE) return KRON_OK;
    if (is_complex(io)) return comp == KRON_COMPUTE_32F_BF16X3 ? KRON_ERR_NOT_SUPPORTED : KRON_ERR_INVALID_VALUE;
    if (comp == KRON_COMPUTE_32F_BF16X3)
        return (io == KRON_R32F || io == KRON_R16BF || io == KRON_R16F) ? KRON_OK : KRON_ERR_NOT_SUPPORTED;
    return KRON_ERR_INVALID_VALUE;
}

}  // namespace kron

using namespace kron;

extern "C" {

KRON_API const char* kron_status_string(kron_status s) {
    switch (s) {
        case KRON_OK: return "KRON_OK";
        case KRON_ERR_INVALID_VALUE: return "KRON_ERR_INVALID_VALUE";
        case KRON_ERR_NOT_SUPPORTED: return "KRON_ERR_NOT_SUPPORTED";
        case KRON_ERR_ALIAS: return "KRON_ERR_ALIAS";
        case KRON_ERR_WORKSPACE: return "KRON_ERR_WORKSPACE";
        case KRON_ERR_CUDA: return "KRON_ERR_CUDA";
        case KRON_ERR_DEVICE_TIMEOUT: return "KRON_ERR_DEVICE_TIMEOUT";
    }
    return "KRON_ERR_UNKNOWN";
}

KRON_API int kron_version(void) { return 10000; }

KRON_API kron_status kron_check_device_buffer(const void* p, size_t bytes) {
    if (!p) return KRON_ERR_INVALID_VALUE;
    return device_range(p, bytes);
}

KRON_API kron_status kron2_batched(kron_stream_t stream, char transa, char transb, char transx, int ma, int na,
                                   int mb, int nb, int64_t batch_count, const void* alpha, const void* A, int lda,
                                   const void* B, int ldb, const void* X, int ldx, int64_t ldxp, const void* beta,
                                   void* Y, int ldy, int64_t ldyp, kron_dtype io, kron_compute comp) {
    int ta, tb, tx;
    if (!trans_flag(transa, &ta) || !trans_flag(transb, &tb) || !trans_flag(transx, &tx))
        return KRON_ERR_INVALID_VALUE;
    if (!dim_ok(ma) || !dim_ok(na) || !dim_ok(mb) || !dim_ok(nb)) return KRON_ERR_INVALID_VALUE;
    if (batch_count < 0 || ldxp < 0) return KRON_ERR_INVALID_VALUE;
    kron_status st = check_modes(io, comp);
    if (st != KRON_OK) return st;
    if (lda < (ta ? na : ma) || ldb < (tb ? nb : mb)) return KRON_ERR_INVALID_VALUE;
    const int xrows = tx ? na : nb, xcols = tx ? nb : na;
    if (ldx < xrows || ldy < mb) return KRON_ERR_INVALID_VALUE;
    if (ldyp < (int64_t)ldy * (ma - 1) + mb) return KRON_ERR_INVALID_VALUE;
    if (!alpha || !beta) return KRON_ERR_INVALID_VALUE;
    if (batch_count == 0) return KRON_OK;
    if (!A || !B || !X || !Y) return KRON_ERR_INVALID_VALUE;
    const size_t es = elem_size(io);
    if (((uintptr_t)X) % es || ((uintptr_t)Y) % es) return KRON_ERR_INVALID_VALUE;
    const size_t xbytes = ((size_t)(batch_count - 1) * ldxp + (size_t)ldx * (xcols - 1) + xrows) * es;
    const size_t ybytes = ((size_t)(batch_count - 1) * ldyp + (size_t)ldy * (ma - 1) + mb) * es;
    if (ranges_overlap(X, xbytes, Y, ybytes)) return KRON_ERR_ALIAS;
    if ((st = device_range(X, xbytes)) != KRON_OK || (st = device_range(Y, ybytes)) != KRON_OK) return st;

    static thread_local KronDesc d;
    d = KronDesc();
    const bool dbl = io == KRON_R64F || io == KRON_C64F;
    d.D = 2;
    d.N = std::max(std::max(ma, na), std::max(mb, nb));
    if (is_complex(io)) {
        op_pad_complex(d.m1, d.m1i, d.N, B, ldb, tb, conj_flag(transb, io), mb, nb, dbl);
        op_pad_complex(d.m2, d.m2i, d.N, A, lda, ta, conj_flag(transa, io), ma, na, dbl);
    } else {
        op_pad(d.m1, d.N, B, ldb, tb, mb, nb, dbl);
        op_pad(d.m2, d.N, A, lda, ta, ma, na, dbl);
    }
    memset(d.m3, 0, sizeof(d.m3));
    d.X = X;
    d.Y = Y;
    d.batch = batch_count;
    d.ldx = ldx;
    d.ldxp = ldxp;
    d.ldy = ldy;
    d.ldyp = ldyp;
    d.ldx2 = 0;
    d.ldy2 = 0;
    d.transx = tx;
    d.conjx = conj_flag(transx, io);
    d.xe[0] = nb; d.xe[1] = na; d.xe[2] = 1;
    d.ye[0] = mb; d.ye[1] = ma; d.ye[2] = 1;
    scalar_of(alpha, io, &d.alpha, &d.alpha_im);
    scalar_of(beta, io, &d.beta, &d.beta_im);
    d.io = io;
    d.comp = comp;
    const int N = d.N;
    d.contiguous = ma == N && na == N && mb == N && nb == N && !tx && !d.conjx && ldx == N && ldxp == (int64_t)N * N &&
                   ((uintptr_t)X) % 16 == 0;
    d.ycontig = d.contiguous && ldy == N && ldyp == (int64_t)N * N && ((uintptr_t)Y) % 16 == 0;
    choose_yvec(d);
    return dispatch(d, (cudaStream_t)stream);
}

static double host_scalar(const void* v, kron_dtype io) {
    return io == KRON_R64F ? *static_cast<const double*>(v) : (double)*static_cast<const float*>(v);
}

static double host_elem(const void* M, size_t idx, kron_dtype io) {
    return io == KRON_R64F ? static_cast<const double*>(M)[idx] : (double)static_cast<const float*>(M)[idx];
}

KRON_API kron_status kron_gemm_a_batched(kron_stream_t stream, char transa, char transb, int m, int n, int k,
                                         const void* alpha, const void* A, int lda, int64_t lda2, const void* B,
                                         int ldb, const void* beta, void* C, int ldc, int64_t ldc2,
                                         int64_t batch_count, int grid_size, kron_dtype io, kron_compute comp) {
    int ta, tb;
    if (!trans_flag(transa, &ta) || !trans_flag(transb, &tb)) return KRON_ERR_INVALID_VALUE;
    if (m < 1 || m > (1 << 24) || !dim_ok(n) || !dim_ok(k)) return KRON_ERR_INVALID_VALUE;
    if (batch_count < 0 || grid_size < 0 || lda2 < 0 || ldc2 < 0) return KRON_ERR_INVALID_VALUE;
    kron_status st = check_modes(io, comp);
    if (st != KRON_OK) return st;
    if (comp != KRON_COMPUTE_NATIVE || is_complex(io)) return KRON_ERR_NOT_SUPPORTED;
    if (lda < (ta ? k : m) || ldb < (tb ? n : k) || ldc < m) return KRON_ERR_INVALID_VALUE;
    const int64_t cext = (int64_t)ldc * (n - 1) + m;   // elements spanned by one C^p
    if (batch_count > 1 && ldc2 < cext) return KRON_ERR_INVALID_VALUE;   // instances of C may not overlap
    if (!alpha || !beta) return KRON_ERR_INVALID_VALUE;
    if (batch_count == 0) return KRON_OK;
    if (!A || !B || !C) return KRON_ERR_INVALID_VALUE;
    const size_t es = elem_size(io);
    if (((uintptr_t)A) % es || ((uintptr_t)C) % es) return KRON_ERR_INVALID_VALUE;
    const int64_t aext = ta ? (int64_t)lda * (m - 1) + k : (int64_t)lda * (k - 1) + m;
    const size_t abytes = ((size_t)(batch_count - 1) * lda2 + aext) * es;
    const size_t cbytes = ((size_t)(batch_count - 1) * ldc2 + cext) * es;
    if (ranges_overlap(A, abytes, C, cbytes)) return KRON_ERR_ALIAS;
    if ((st = device_range(A, abytes)) != KRON_OK || (st = device_range(C, cbytes)) != KRON_OK) return st;
    static thread_local GemmADesc g;
    g = GemmADesc();
    g.m = m;
    g.n = n;
    g.k = k;
    for (int l = 0; l < k; ++l)
        for (int j = 0; j < n; ++j)
            g.b[l * 16 + j] = host_elem(B, tb ? (size_t)j + (size_t)ldb * l : (size_t)l + (size_t)ldb * j, io);
    g.A = A;
    g.C = C;
    g.lda = lda;
    g.ldc = ldc;
    g.transa = ta;
    g.lda2 = lda2;
    g.ldc2 = ldc2;
    g.batch = batch_count;
    g.alpha = host_scalar(alpha, io);
    g.beta = host_scalar(beta, io);
    g.io = io;
    g.grid = grid_size;
    return launch_gemm_a(g, (cudaStream_t)stream);
}

KRON_API kron_status kron1_batched(kron_stream_t stream, char transa, int ma, int na, int64_t batch_count,
                                   const void* alpha, const void* A, int lda, const void* X, int64_t ldxp,
                                   const void* beta, void* Y, int64_t ldyp, kron_dtype io, kron_compute comp) {
    int ta;
    if (!trans_flag(transa, &ta)) return KRON_ERR_INVALID_VALUE;
    if (!dim_ok(ma) || !dim_ok(na)) return KRON_ERR_INVALID_VALUE;
    if (batch_count < 0 || ldxp < 0 || ldyp < 0) return KRON_ERR_INVALID_VALUE;
    kron_status st = check_modes(io, comp);
    if (st != KRON_OK) return st;
    if (comp != KRON_COMPUTE_NATIVE || is_complex(io)) return KRON_ERR_NOT_SUPPORTED;
    if (lda < (ta ? na : ma)) return KRON_ERR_INVALID_VALUE;
    if (batch_count > 1 && ldyp < ma) return KRON_ERR_INVALID_VALUE;   // outputs may not overlap
    if (!alpha || !beta) return KRON_ERR_INVALID_VALUE;
    if (batch_count == 0) return KRON_OK;
    if (!A || !X || !Y) return KRON_ERR_INVALID_VALUE;
    const size_t es = elem_size(io);
    if (((uintptr_t)X) % es || ((uintptr_t)Y) % es) return KRON_ERR_INVALID_VALUE;
    const size_t xbytes = ((size_t)(batch_count - 1) * ldxp + na) * es;
    const size_t ybytes = ((size_t)(batch_count - 1) * ldyp + ma) * es;
    if (ranges_overlap(X, xbytes, Y, ybytes)) return KRON_ERR_ALIAS;
    if ((st = device_range(X, xbytes)) != KRON_OK || (st = device_range(Y, ybytes)) != KRON_OK) return st;
    // y^p (1 x ma) = x^p (1 x na) op(A)^T: TGEMM_A with m = 1, x^p as the one row
    // of A^p (column stride 1, instance stride ldxp) and the shared factor op(A)^T.
    static thread_local GemmADesc g;
    g = GemmADesc();
    g.m = 1;
    g.n = ma;
    g.k = na;
    for (int l = 0; l < na; ++l)
        for (int j = 0; j < ma; ++j)
            g.b[l * 16 + j] = host_elem(A, ta ? (size_t)l + (size_t)lda * j : (size_t)j + (size_t)lda * l, io);
    g.A = X;
    g.lda = 1;
    g.lda2 = ldxp;
    g.transa = 0;
    g.C = Y;
    g.ldc = 1;
    g.ldc2 = ldyp;
    g.batch = batch_count;
    g.alpha = host_scalar(alpha, io);
    g.beta = host_scalar(beta, io);
    g.io = io;
    const kron_status r = launch_kron1(g, (cudaStream_t)stream);
    return r == KRON_ERR_NOT_SUPPORTED ? launch_gemm_a(g, (cudaStream_t)stream) : r;
}

KRON_API kron_status kron3_batched(kron_stream_t stream, char transa, char transb, char transc, int ma, int na,
                                   int mb, int nb, int mc, int nc, int64_t batch_count, const void* alpha,
                                   const void* A, int lda, const void* B, int ldb, const void* C, int ldc,
                                   const void* X, int ldx, int ldx2, int64_t ldxp, const void* beta, void* Y,
                                   int ldy, int ldy2, int64_t ldyp, kron_dtype io, kron_compute comp) {
    int ta, tb, tc;
    if (!trans_flag(transa, &ta) || !trans_flag(transb, &tb) || !trans_flag(transc, &tc))
        return KRON_ERR_INVALID_VALUE;
    if (!dim_ok(ma) || !dim_ok(na) || !dim_ok(mb) || !dim_ok(nb) || !dim_ok(mc) || !dim_ok(nc))
        return KRON_ERR_INVALID_VALUE;
    if (batch_count < 0 || ldxp < 0) return KRON_ERR_INVALID_VALUE;
    kron_status st = check_modes(io, comp);
    if (st != KRON_OK) return st;
    if (lda < (ta ? na : ma) || ldb < (tb ? nb : mb) || ldc < (tc ? nc : mc)) return KRON_ERR_INVALID_VALUE;
    if (ldx < nc || (int64_t)ldx2 < (int64_t)ldx * nb) return KRON_ERR_INVALID_VALUE;
    if (ldy < mc || (int64_t)ldy2 < (int64_t)ldy * mb) return KRON_ERR_INVALID_VALUE;
    if (ldyp < (int64_t)ldy2 * (ma - 1) + (int64_t)ldy * (mb - 1) + mc) return KRON_ERR_INVALID_VALUE;
    if (!alpha || !beta) return KRON_ERR_INVALID_VALUE;
    if (batch_count == 0) return KRON_OK;
    if (!A || !B || !C || !X || !Y) return KRON_ERR_INVALID_VALUE;
    const size_t es = elem_size(io);
    if (((uintptr_t)X) % es || ((uintptr_t)Y) % es) return KRON_ERR_INVALID_VALUE;
    const size_t xbytes =
        ((size_t)(batch_count - 1) * ldxp + (size_t)ldx2 * (na - 1) + (size_t)ldx * (nb - 1) + nc) * es;
    const size_t ybytes =
        ((size_t)(batch_count - 1) * ldyp + (size_t)ldy2 * (ma - 1) + (size_t)ldy * (mb - 1) + mc) * es;
    if (ranges_overlap(X, xbytes, Y, ybytes)) return KRON_ERR_ALIAS;
    if ((st = device_range(X, xbytes)) != KRON_OK || (st = device_range(Y, ybytes)) != KRON_OK) return st;

    static thread_local KronDesc d;
    d = KronDesc();
    const bool dbl = io == KRON_R64F || io == KRON_C64F;
    d.D = 3;
    d.N = std::max(std::max(std::max(ma, na), std::max(mb, nb)), std::max(mc, nc));
    if (is_complex(io)) {
        op_pad_complex(d.m1, d.m1i, d.N, C, ldc, tc, conj_flag(transc, io), mc, nc, dbl);
        op_pad_complex(d.m2, d.m2i, d.N, B, ldb, tb, conj_flag(transb, io), mb, nb, dbl);
        op_pad_complex(d.m3, d.m3i, d.N, A, lda, ta, conj_flag(transa, io), ma, na, dbl);
    } else {
        op_pad(d.m1, d.N, C, ldc, tc, mc, nc, dbl);
        op_pad(d.m2, d.N, B, ldb, tb, mb, nb, dbl);
        op_pad(d.m3, d.N, A, lda, ta, ma, na, dbl);
    }
    d.X = X;
    d.Y = Y;
    d.batch = batch_count;
    d.ldx = ldx;
    d.ldx2 = ldx2;
    d.ldxp = ldxp;
    d.ldy = ldy;
    d.ldy2 = ldy2;
    d.ldyp = ldyp;
    d.transx = 0;
    d.xe[0] = nc; d.xe[1] = nb; d.xe[2] = na;
    d.ye[0] = mc; d.ye[1] = mb; d.ye[2] = ma;
    scalar_of(alpha, io, &d.alpha, &d.alpha_im);
    scalar_of(beta, io, &d.beta, &d.beta_im);
    d.io = io;
    d.comp = comp;
    const int N = d.N;
    d.contiguous = ma == N && na == N && mb == N && nb == N && mc == N && nc == N && ldx == N &&
                   ldx2 == N * N && ldxp == (int64_t)N * N * N && ((uintptr_t)X) % 16 == 0;
    d.ycontig = d.contiguous && ldy == N && ldy2 == N * N && ldyp == (int64_t)N * N * N && ((uintptr_t)Y) % 16 == 0;
    choose_yvec(d);
    return dispatch(d, (cudaStream_t)stream);
}

KRON_API kron_status kron_set_first_wait_limit_ns(unsigned long long ns) {
    if (ns > kWaitLimitNs) return KRON_ERR_INVALID_VALUE;
    g_first_wait_ns.store(ns, std::memory_order_relaxed);
    return KRON_OK;
}

KRON_API kron_status kron_device_status(kron_stream_t stream) {
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return KRON_ERR_CUDA;
    unsigned v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_kron_device_error, sizeof(v)) != cudaSuccess) return KRON_ERR_CUDA;
    if (v && cudaMemcpyToSymbol(g_kron_device_error, &zero, sizeof(zero)) != cudaSuccess) return KRON_ERR_CUDA;
    return (v & kDevErrTimeout) ? KRON_ERR_DEVICE_TIMEOUT : KRON_OK;
}

}  // extern "C"
