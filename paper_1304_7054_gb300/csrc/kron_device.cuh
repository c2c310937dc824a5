// Device-side building blocks shared by the kernels: bulk-copy (TMA) helpers,
// bounded mbarrier waits, storage-type conversions and vector stores.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kron {

// Packed float pairs for fma.rn.f32x2 (two FP32 FMAs per instruction).
typedef unsigned long long f2;   // two packed floats, low word = first element

__device__ __forceinline__ f2 f2_pack(float lo, float hi) {
    return (f2)__float_as_uint(lo) | ((f2)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float f2_lo(f2 v) { return __uint_as_float((unsigned)v); }
__device__ __forceinline__ float f2_hi(f2 v) { return __uint_as_float((unsigned)(v >> 32)); }

__device__ __forceinline__ f2 ffma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 fmul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// A float pair rounded (RNE) to two packed 16-bit storage values.
template <typename S> __device__ __forceinline__ unsigned pack16(f2 v);
template <> __device__ __forceinline__ unsigned pack16<__nv_bfloat16>(f2 v) {
    unsigned r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(f2_hi(v)), "f"(f2_lo(v)));
    return r;
}
template <> __device__ __forceinline__ unsigned pack16<__half>(f2 v) {
    unsigned r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(f2_hi(v)), "f"(f2_lo(v)));
    return r;
}

// Bits of the device status word (see kron_device_status in kron.h).
constexpr unsigned kDevErrTimeout = 1u;
// A bounded wait gives up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Smallest s >= lo with s == r (mod 32): strides of the on-chip exchange
// buffers, chosen so that the two access patterns of a transposition hit
// distinct shared-memory banks.
__host__ __device__ constexpr int stride_mod32(int lo, int r) {
    return lo + ((r - lo) % 32 + 32) % 32;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Longest time one try_wait may keep the thread suspended; it resumes as soon as
// the phase completes.  Without the hint the wait returns after a short
// system-defined time, and the retries cost issue slots and shared-memory
// bandwidth that the compute warps of the same SM need.
constexpr unsigned kWaitSuspendNs = 1000000u;

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kWaitSuspendNs)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of `bar` to complete, for at most kWaitLimitNs (plus
// at most 8 suspensions of kWaitSuspendNs).  On expiry it records
// kDevErrTimeout in *err and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    for (;;) {
#pragma unroll 1
        for (int i = 0; i < 8; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > kWaitLimitNs) {
            atomicOr(err, kDevErrTimeout);
            return false;
        }
    }
}

// Non-blocking test of phase `parity` of `bar`.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of `bar` by polling (no suspension), for at most
// limit_ns of %globaltimer.  On expiry it records kDevErrTimeout in *err and
// returns false.  Used with a short limit to make a real wait run out (the
// failure-path test of kron_set_first_wait_limit_ns).
__device__ __forceinline__ bool mbar_wait_polled(uint64_t* bar, unsigned parity, unsigned* err,
                                                 unsigned long long limit_ns) {
    const unsigned long long t0 = global_timer_ns();
    for (;;) {
        if (mbar_test(bar, parity)) return true;
        if (global_timer_ns() - t0 >= limit_ns) {
            atomicOr(err, kDevErrTimeout);
            return false;
        }
    }
}

// L2 policy for data read exactly once (the operand stream).
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 1-D bulk copy (TMA) global -> shared, completion signalled on `bar` as
// transaction bytes.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 1-D bulk copy (TMA) shared -> global in the thread's current bulk group.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
// As bulk_s2g, with an L2 cache policy for the written lines.
__device__ __forceinline__ void bulk_s2g_hint(void* dst, const void* src, unsigned bytes, uint64_t policy) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes), "l"(policy)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// The shared-memory sources of this thread's bulk stores have been read.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// All but the most recent of this thread's bulk-store groups have been read.
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// This thread's bulk stores are complete.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Named barrier 1 over the first 128 threads of the CTA (the compute warps of a
// kernel with a producer warp); returns the OR of v over them.
__device__ __forceinline__ bool compute_sync_or(bool v) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, 1, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((unsigned)v)
        : "memory");
    return r != 0;
}

// ---------------------------------------------------------------------------
// Storage <-> compute conversions (round to nearest even on the way down).
// ---------------------------------------------------------------------------
template <typename T, typename S> __device__ __forceinline__ T load_cvt(S v);
template <> __device__ __forceinline__ float load_cvt<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double load_cvt<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float load_cvt<float, __nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}
template <> __device__ __forceinline__ float load_cvt<float, __half>(__half v) { return __half2float(v); }

template <typename S, typename T> __device__ __forceinline__ S store_cvt(T v);
template <> __device__ __forceinline__ float store_cvt<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double store_cvt<double, double>(double v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 store_cvt<__nv_bfloat16, float>(float v) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half store_cvt<__half, float>(float v) { return __float2half_rn(v); }

template <typename S> __device__ __forceinline__ uint32_t bits_of(S v);
template <> __device__ __forceinline__ uint32_t bits_of<float>(float v) { return __float_as_uint(v); }
template <> __device__ __forceinline__ uint32_t bits_of<__nv_bfloat16>(__nv_bfloat16 v) {
    return static_cast<uint32_t>(__bfloat16_as_ushort(v));
}
template <> __device__ __forceinline__ uint32_t bits_of<__half>(__half v) {
    return static_cast<uint32_t>(__half_as_ushort(v));
}

template <typename S> __device__ __forceinline__ S from_bits(uint32_t b);
template <> __device__ __forceinline__ float from_bits<float>(uint32_t b) { return __uint_as_float(b); }
template <> __device__ __forceinline__ __nv_bfloat16 from_bits<__nv_bfloat16>(uint32_t b) {
    return __ushort_as_bfloat16(static_cast<unsigned short>(b));
}
template <> __device__ __forceinline__ __half from_bits<__half>(uint32_t b) {
    return __ushort_as_half(static_cast<unsigned short>(b));
}

// Packs storage values o[base .. base + 32/bits-per-element) into one 32-bit word.
template <typename S, int N>
__device__ __forceinline__ uint32_t pack_word(const S (&o)[N], int base) {
    if constexpr (sizeof(S) == 4) {
        return bits_of<S>(o[base]);
    } else {
        return bits_of<S>(o[base]) | (bits_of<S>(o[base + 1]) << 16);
    }
}

// Writes the N contiguous storage elements o[] to dst in chunks of VB bytes
// (VB in {16, 8, 4}); requires N*sizeof(S) % VB == 0 and dst VB-aligned.
// Streaming stores: results are not re-read by this kernel.
template <int VB, typename S, int N>
__device__ __forceinline__ void store_chunks(S* dst, const S (&o)[N]) {
    constexpr int E = VB / (int)sizeof(S);   // elements per chunk
    constexpr int WPE = (int)(4 / sizeof(S)); // elements per 32-bit word
    static_assert((N * (int)sizeof(S)) % VB == 0, "chunking");
#pragma unroll
    for (int c = 0; c < N / E; ++c) {
        if constexpr (VB == 16) {
            uint4 v;
            v.x = pack_word<S, N>(o, c * E + 0 * WPE);
            v.y = pack_word<S, N>(o, c * E + 1 * WPE);
            v.z = pack_word<S, N>(o, c * E + 2 * WPE);
            v.w = pack_word<S, N>(o, c * E + 3 * WPE);
            __stcs(reinterpret_cast<uint4*>(dst + c * E), v);
        } else if constexpr (VB == 8) {
            uint2 v;
            v.x = pack_word<S, N>(o, c * E + 0 * WPE);
            v.y = pack_word<S, N>(o, c * E + 1 * WPE);
            __stcs(reinterpret_cast<uint2*>(dst + c * E), v);
        } else {
            static_assert(VB == 4, "chunk size");
            __stcs(reinterpret_cast<unsigned int*>(dst + c * E), pack_word<S, N>(o, c * E));
        }
    }
}

}  // namespace kron
