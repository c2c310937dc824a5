// Mixed-size batches: one persistent launch over instances of different sizes
// and kinds, captured in a CUDA graph.
//
// The paper's interfaces take one size and one uniform instance stride per call
// (Sec. 3); a finite-element mesh with mixed polynomial degrees needs many such
// calls.  Here a plan groups the instances by class (kind, n), cuts each class
// into tiles of P_c instances, and one kernel walks the tile list.  Every class
// has a compile-time body -- the same sum factorisation as the fixed-size
// CUDA-core kernels (paper Sec. 2.1, Algorithm 1's modes with the intermediates
// on chip) -- and its components sit at a fixed slot of the parameter bank, so
// each FMA reads its coefficients as a constant operand.  Every contraction is
// done in packed pairs of output rows (fma.rn.f32x2 with the coefficient pair
// (M[i,l], M[i+1,l]) and the operand duplicated), so each stage writes its
// outputs as adjacent pairs; rows are padded to an even count.
//
// Data flow per CTA: two operand buffers and one exchange buffer.  While one
// tile is contracted, the next one arrives in the other operand buffer by bulk
// copies, one per instance: an instance starts anywhere (4-byte alignment for
// FP32), so each copy takes the 16-byte-aligned span around it and the instance
// sits at its alignment phase inside a 16-byte-aligned slot.  In 3-D the second
// contraction writes over the dead operands and the last one into the exchange
// buffer; in 2-D the last one writes over the dead operands.  Either way each
// instance's results are contiguous, at the phase of its place in Y: the
// 16-byte-aligned middle leaves by one bulk copy and the at most three elements
// on either side by plain stores.  Global memory is thus read and written in
// whole aligned granules, with no per-element address work.  Before the next
// tile writes a buffer that outgoing copies still read, warp 0 waits for them.
//
// Workspace (caller-owned device memory, written on the first execute with a
// given pointer): tile table (int4: class key, first sorted index, count, 0),
// then the sorted instance offsets (int64 X offsets, then int64 Y offsets).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "kron_device.cuh"
#include "kron_fiber.cuh"
#include "kron_internal.h"
#include "kron_pair.cuh"

namespace kron {

constexpr int kVlThreads = 256;
constexpr int kVlBufBytes = 22528;                     // default budget of one buffer
constexpr int kVlMaxBufBytes = 49152;                  // largest buffer a tuned tile may take
constexpr int kVlKeys = 32;                            // class key = 16 (kind - 2) + n - 1

__host__ __device__ constexpr int sq_sum(int n) { return (n - 1) * n * (2 * n - 1) / 6; }   // sum k^2, k < n
// Rows of a component padded to an even count, and the sum over k < n of
// pad(k) * k (the odd k < n add k each: (n/2)^2 in total).
__host__ __device__ constexpr int vl_rows(int n) { return n + (n & 1); }
__host__ __device__ constexpr int vl_psum(int n) { return sq_sum(n) + (n / 2) * (n / 2); }
// Parameter-bank slot (floats) of class (kind, n): 2-D classes hold M1, M2, 3-D
// classes M1, M2, M3, each vl_rows(n) x n column-major with zero padding rows.
__host__ __device__ constexpr int vl_slot(int kind, int n) {
    return kind == 2 ? 2 * vl_psum(n) : 2 * vl_psum(17) + 3 * vl_psum(n);
}
constexpr int kVlCoef = 2 * vl_psum(17) + 3 * vl_psum(17);   // 7800 floats
// Padded row length of the exchange buffers: even (64-bit pair stores) and
// 2 mod 4, so that lanes a row apart hit distinct banks.
__host__ __device__ constexpr int vl_kp(int n) {
    return vl_rows(n) + ((vl_rows(n) % 4 == 2) ? 0 : 2);
}

struct VlClass {
    int P;              // instances per tile (0 = class absent)
    unsigned inv;       // ceil(2^32 / n^kind): exact quotient e / n^kind for e < 4096
};

struct __align__(8) VarlenArgs {
    float coef[kVlCoef];      // 8-byte aligned: read as coefficient pairs
    VlClass cls[kVlKeys];
    const int4* tiles;
    const int64_t* xoff;
    const int64_t* yoff;
    const void* X;
    void* Y;
    int ntiles;
    int alpha_one, beta_zero;  // Y = alpha (K x) + beta Y (beta = 0: Y is not read)
    float alpha, beta;
    unsigned* err;
};

static_assert(sizeof(VarlenArgs) <= 32764, "kernel parameter space");

__device__ __forceinline__ int vl_nx(int key) {
    const int n = (key & 15) + 1;
    return key < 16 ? n * n : n * n * n;
}

// Slot of one instance in an operand buffer: its elements plus up to 15 bytes
// of alignment phase, rounded to 16 bytes.
__host__ __device__ constexpr int vl_slot_bytes(int nx, int es) { return (nx * es + 15 + 15) / 16 * 16; }
__host__ __device__ constexpr int vl_max(int a, int b) { return a > b ? a : b; }
// Exchange elements of one instance (FP32): KP x N (2-D) or KP x N x N (3-D).
__host__ __device__ constexpr int vl_exq(int kind, int n) { return vl_kp(n) * (kind == 2 ? n : n * n); }
// Per-instance stride of the operand buffers (bytes).  In 3-D the second
// contraction writes its FP32 exchange layout over the dead operands, so the
// slot holds either.
__host__ __device__ constexpr int vl_xs_bytes(int kind, int n, int es) {
    return kind == 2 ? vl_slot_bytes(n * n, es)
                     : (vl_max(vl_slot_bytes(n * n * n, es), 4 * vl_exq(3, n)) + 15) / 16 * 16;
}
// Per-instance stride of the exchange buffer (floats).  In 3-D the last
// contraction writes the results there (contiguous, at their phase in Y), so a
// slot is 16-byte aligned and holds either.
__host__ __device__ constexpr int vl_e1_floats(int kind, int n, int es) {
    return kind == 2 ? vl_exq(2, n) : (vl_max(vl_exq(3, n), vl_slot_bytes(n * n * n, es) / 4) + 3) / 4 * 4;
}

// Alignment phase (in elements) of element offset `off` of an array at `base`.
template <typename S>
__device__ __forceinline__ int vl_phase(const void* base, int off) {
    return (int)((((unsigned)(uintptr_t)base) + (unsigned)off * (unsigned)sizeof(S)) & 15u) / (int)sizeof(S);
}

// Issued by warp 0: one bulk copy per instance of tile `td` (X offsets xo[]) into
// the slots of buffer `xt`, completing on `bar`.  Each copy covers the aligned
// 16-byte granules that hold the instance.
template <typename S>
__device__ __forceinline__ void vl_issue_loads(const VarlenArgs& a, int4 td, const int* xo, unsigned char* xt,
                                               uint64_t* bar, uint64_t pol) {
    const int lane = threadIdx.x & 31;
    const int nx = vl_nx(td.x);
    const int slot = vl_xs_bytes(td.x < 16 ? 2 : 3, (td.x & 15) + 1, (int)sizeof(S));
    unsigned bytes = 0;
    for (int q = lane; q < td.z; q += 32) {
        const unsigned ph = (((unsigned)(uintptr_t)a.X) + (unsigned)xo[q] * (unsigned)sizeof(S)) & 15u;
        bytes += (ph + (unsigned)nx * (unsigned)sizeof(S) + 15u) & ~15u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    fence_proxy_async_smem();
    if (lane == 0) mbar_arrive_expect_tx(bar, bytes);
    __syncwarp();
    for (int q = lane; q < td.z; q += 32) {
        const uintptr_t src = (uintptr_t)(static_cast<const S*>(a.X) + xo[q]);
        const unsigned ph = (unsigned)(src & 15u);
        bulk_g2s(xt + q * slot, (const void*)(src - ph), (ph + (unsigned)nx * (unsigned)sizeof(S) + 15u) & ~15u, bar,
                 pol);
    }
}

// Issued by warp 0 after the last contraction: per instance, the aligned middle
// of its run in Y by one bulk copy, the partial granules at both ends by plain
// stores.  Instance q's results start at xt + q * slot plus their phase in Y, so
// slot and Y agree modulo 16 bytes.
template <typename S>
__device__ __forceinline__ void vl_issue_stores(const VarlenArgs& a, int4 td, const int* yo, const unsigned char* xt,
                                                int slot) {
    const int lane = threadIdx.x & 31;
    const int nx = vl_nx(td.x);
    const uint64_t pol = l2_evict_first_policy();
    for (int q = lane; q < td.z; q += 32) {
        S* dst = static_cast<S*>(a.Y) + yo[q];
        const unsigned ph = (unsigned)((uintptr_t)dst & 15u);
        const S* src = reinterpret_cast<const S*>(xt + q * slot + ph);
        const unsigned total = (unsigned)nx * (unsigned)sizeof(S);
        const unsigned head = ph ? 16u - ph : 0u;
        if (head >= total) {   // the whole instance inside one granule
            for (int e = 0; e < nx; ++e) dst[e] = src[e];
            continue;
        }
        const unsigned mid = (total - head) & ~15u;
        for (unsigned e = 0; e < head / sizeof(S); ++e) dst[e] = src[e];
        if (mid)
            bulk_s2g_hint(reinterpret_cast<unsigned char*>(dst) + head, reinterpret_cast<const unsigned char*>(src) + head,
                          mid, pol);
        for (unsigned e = (head + mid) / sizeof(S); e < (unsigned)nx; ++e) dst[e] = src[e];
    }
    bulk_commit();
}

// Packed-pair contraction of one fiber: (y[2r], y[2r+1]) = M[2r:2r+2, :] x, with
// M stored as vl_rows(N) x N (column-major, read as coefficient pairs).
template <int N>
__device__ __forceinline__ void vl_contract(const float* M, const float (&x)[N], f2 (&y)[vl_rows(N) / 2]) {
    constexpr int R = vl_rows(N) / 2;
    const f2* Mp = reinterpret_cast<const f2*>(M);
    const f2 x0 = f2_pack(x[0], x[0]);
#pragma unroll
    for (int r = 0; r < R; ++r) y[r] = fmul2(Mp[r], x0);
#pragma unroll
    for (int l = 1; l < N; ++l) {
        const f2 xl = f2_pack(x[l], x[l]);
#pragma unroll
        for (int r = 0; r < R; ++r) y[r] = ffma2(Mp[r + R * l], xl, y[r]);
    }
}

// Stores output pairs (rows 2r, 2r+1) at dst[2r] (float, 8-byte aligned).
template <int N>
__device__ __forceinline__ void vl_store_pairs(float* dst, const f2 (&y)[vl_rows(N) / 2]) {
#pragma unroll
    for (int r = 0; r < vl_rows(N) / 2; ++r) *reinterpret_cast<f2*>(dst + 2 * r) = y[r];
}

// Output fiber of N elements at dst[0..N) (contiguous): pairs (rows 2r, 2r+1)
// rounded to the storage type and stored as one word where dst is aligned for
// it, else element by element (the padding row of an odd N is dropped).
template <typename S, int N>
__device__ __forceinline__ void vl_stage_out(S* dst, const f2 (&y)[vl_rows(N) / 2]) {
    const bool paired = ((uintptr_t)dst & (2 * sizeof(S) - 1)) == 0;
    if (paired) {
#pragma unroll
        for (int r = 0; r < N / 2; ++r) {
            if constexpr (sizeof(S) == 4)
                *reinterpret_cast<f2*>(dst + 2 * r) = y[r];
            else
                *reinterpret_cast<unsigned*>(dst + 2 * r) = pack16<S>(y[r]);
        }
    } else {
#pragma unroll
        for (int r = 0; r < N / 2; ++r) {
            dst[2 * r] = store_cvt<S, float>(f2_lo(y[r]));
            dst[2 * r + 1] = store_cvt<S, float>(f2_hi(y[r]));
        }
    }
    if constexpr (N & 1) dst[N - 1] = store_cvt<S, float>(f2_lo(y[N / 2]));
}

// One tile of class (D, N) in operand buffer xt: instance q's operands at slot q,
// phase vl_phase(X, xo[q]).  Its results, contiguous and column-major at phase
// vl_phase(Y, yo[q]), go to operand slot q (2-D) or exchange slot q (3-D).
// Exchange layouts put each stage's output pairs next to each other:
//   2-D   W(l, j)    at j + KP l            in ex1  (stage 1 writes pairs along j)
//   3-D   T(i, j, k) at k + KP i + KP N j   in ex1  (stage A: pairs along k)
//         U(i, j, k) at j + KP k + KP N i   in xt   (stage B: pairs along j)
// and the last stage writes pairs along i.
template <typename S, int N, int D>
__device__ __forceinline__ void vl_tile(const VarlenArgs& a, int4 td, unsigned char* xt, float* ex1, const int* xo,
                                        const int* yo) {
    constexpr int KP = vl_kp(N);
    constexpr int R = vl_rows(N) / 2;
    constexpr int EXQ = vl_e1_floats(D, N, (int)sizeof(S));   // exchange stride per instance (floats)
    constexpr int SLOT = vl_xs_bytes(D, N, (int)sizeof(S));   // operand stride per instance (bytes)
    const float* m1 = a.coef + vl_slot(D, N);
    const float* m2 = m1 + vl_rows(N) * N;
    const float* m3 = m2 + vl_rows(N) * N;
    const int cnt = td.z;
    const int tid = threadIdx.x;
    const void* X = a.X;
    const void* Y = a.Y;
    if constexpr (D == 2) {
        const int F = cnt * N;
        for (int f = tid; f < F; f += kVlThreads) {   // stage 1: mode 2, fibers (l, q)
            const int q = f / N, l = f - q * N;
            const S* xr = reinterpret_cast<const S*>(xt + q * SLOT) + vl_phase<S>(X, xo[q]) + l;
            float x[N];
#pragma unroll
            for (int m = 0; m < N; ++m) x[m] = load_cvt<float, S>(xr[N * m]);
            f2 w[R];
            vl_contract<N>(m2, x, w);
            vl_store_pairs<N>(ex1 + q * EXQ + KP * l, w);
        }
        __syncthreads();
        for (int f = tid; f < F; f += kVlThreads) {   // stage 2: mode 1, fibers (j, q)
            const int q = f / N, j = f - q * N;
            const float* wr = ex1 + q * EXQ + j;
            float w[N];
#pragma unroll
            for (int l = 0; l < N; ++l) w[l] = wr[KP * l];
            f2 y[R];
            vl_contract<N>(m1, w, y);
            vl_stage_out<S, N>(reinterpret_cast<S*>(xt + q * SLOT) + vl_phase<S>(Y, yo[q]) + N * j, y);
        }
    } else {
        const int F = cnt * N * N;
        for (int f = tid; f < F; f += kVlThreads) {   // stage A: mode 3, fibers (i, j)
            const int q = f / (N * N), r = f - q * (N * N);
            const int i = r % N, j = r / N;
            const S* xr = reinterpret_cast<const S*>(xt + q * SLOT) + vl_phase<S>(X, xo[q]) + i + N * j;
            float x[N];
#pragma unroll
            for (int p = 0; p < N; ++p) x[p] = load_cvt<float, S>(xr[N * N * p]);
            f2 t[R];
            vl_contract<N>(m3, x, t);
            vl_store_pairs<N>(ex1 + q * EXQ + KP * i + KP * N * j, t);
        }
        __syncthreads();
        for (int f = tid; f < F; f += kVlThreads) {   // stage B: mode 2, fibers (i, k)
            const int q = f / (N * N), r = f - q * (N * N);
            const int k = r % N, i = r / N;
            const float* tr = ex1 + q * EXQ + k + KP * i;
            float t[N];
#pragma unroll
            for (int m = 0; m < N; ++m) t[m] = tr[KP * N * m];
            f2 u[R];
            vl_contract<N>(m2, t, u);
            vl_store_pairs<N>(reinterpret_cast<float*>(xt + q * SLOT) + KP * k + KP * N * i, u);
        }
        __syncthreads();
        for (int f = tid; f < F; f += kVlThreads) {   // stage C: mode 1, fibers (j, k)
            const int q = f / (N * N), r = f - q * (N * N);
            const int j = r % N, k = r / N;
            const float* ur = reinterpret_cast<const float*>(xt + q * SLOT) + j + KP * k;
            float u[N];
#pragma unroll
            for (int l = 0; l < N; ++l) u[l] = ur[KP * N * l];
            f2 y[R];
            vl_contract<N>(m1, u, y);
            vl_stage_out<S, N>(reinterpret_cast<S*>(ex1 + q * EXQ) + vl_phase<S>(Y, yo[q]) + N * (j + N * k), y);
        }
    }
}

template <typename S, int D>
__device__ __forceinline__ void vl_dispatch_n(const VarlenArgs& a, int4 td, unsigned char* xt, float* ex1,
                                              const int* xo, const int* yo) {
    switch ((td.x & 15) + 1) {
        case 1: vl_tile<S, 1, D>(a, td, xt, ex1, xo, yo); break;
        case 2: vl_tile<S, 2, D>(a, td, xt, ex1, xo, yo); break;
        case 3: vl_tile<S, 3, D>(a, td, xt, ex1, xo, yo); break;
        case 4: vl_tile<S, 4, D>(a, td, xt, ex1, xo, yo); break;
        case 5: vl_tile<S, 5, D>(a, td, xt, ex1, xo, yo); break;
        case 6: vl_tile<S, 6, D>(a, td, xt, ex1, xo, yo); break;
        case 7: vl_tile<S, 7, D>(a, td, xt, ex1, xo, yo); break;
        case 8: vl_tile<S, 8, D>(a, td, xt, ex1, xo, yo); break;
        case 9: vl_tile<S, 9, D>(a, td, xt, ex1, xo, yo); break;
        case 10: vl_tile<S, 10, D>(a, td, xt, ex1, xo, yo); break;
        case 11: vl_tile<S, 11, D>(a, td, xt, ex1, xo, yo); break;
        case 12: vl_tile<S, 12, D>(a, td, xt, ex1, xo, yo); break;
        case 13: vl_tile<S, 13, D>(a, td, xt, ex1, xo, yo); break;
        case 14: vl_tile<S, 14, D>(a, td, xt, ex1, xo, yo); break;
        case 15: vl_tile<S, 15, D>(a, td, xt, ex1, xo, yo); break;
        case 16: vl_tile<S, 16, D>(a, td, xt, ex1, xo, yo); break;
    }
}

template <typename S>
__global__ void __launch_bounds__(kVlThreads, 3) varlen_kernel(const __grid_constant__ VarlenArgs a, int xbuf_bytes) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);   // one barrier per operand buffer
    // Offsets of the instances of three consecutive tiles of this CTA (a ring):
    // X offsets then Y offsets, kVlThreads each (a tile has at most that many).
    int* ring = reinterpret_cast<int*>(smem + 128);
    unsigned char* xbuf = smem + 128 + 6 * kVlThreads * sizeof(int);
    float* ex1 = reinterpret_cast<float*>(xbuf + 2 * xbuf_bytes);
    const int G = gridDim.x;
    const int tid = threadIdx.x;
    const int t0 = blockIdx.x;
    if (t0 >= a.ntiles) return;
    const int4 none = make_int4(0, 0, 0, 0);
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_barrier_init();
    }
    // Pipeline: descriptors are read two tiles ahead, instance offsets one tile
    // ahead (through the ring), operands one tile ahead (the other buffer).
    int4 d0 = a.tiles[t0];
    int4 d1 = t0 + G < a.ntiles ? a.tiles[t0 + G] : none;
    int4 d2 = t0 + 2 * G < a.ntiles ? a.tiles[t0 + 2 * G] : none;
    if (tid < d0.z) {
        ring[tid] = (int)a.xoff[d0.y + tid];
        ring[kVlThreads + tid] = (int)a.yoff[d0.y + tid];
    }
    if (tid < d1.z) {
        ring[2 * kVlThreads + tid] = (int)a.xoff[d1.y + tid];
        ring[3 * kVlThreads + tid] = (int)a.yoff[d1.y + tid];
    }
    __syncthreads();
    const uint64_t pol = l2_evict_first_policy();
    int it = 0;
    for (int tile = t0; tile < a.ntiles; ++it, tile += G) {
        const int b = it & 1;
        const int s0 = it % 3, s1 = (it + 1) % 3, s2 = (it + 2) % 3;
        // offsets of tile + 2G, stored at the end of this tile
        int xo2 = 0, yo2 = 0;
        if (tid < d2.z) {
            xo2 = (int)a.xoff[d2.y + tid];
            yo2 = (int)a.yoff[d2.y + tid];
        }
        const int4 d3 = tile + 3 * G < a.ntiles ? a.tiles[tile + 3 * G] : none;
        if (tid < 32) {
            // The previous tile's results have left shared memory (the other operand
            // buffer or the exchange buffer) before either is written again; then the
            // operands of this tile (first iteration only) and of the next one.
            bulk_wait_read();
            __syncwarp();
            for (int u = it == 0 ? 0 : 1; u < 2; ++u) {
                const int4 du = u ? d1 : d0;
                if (!du.z) break;
                vl_issue_loads<S>(a, du, ring + 2 * kVlThreads * (u ? s1 : s0), xbuf + (b ^ u) * xbuf_bytes,
                                  &full[b ^ u], pol);
            }
        }
        const bool ok = mbar_wait_bounded(&full[b], (unsigned)(it >> 1) & 1u, a.err);
        if (__syncthreads_or(!ok)) {
            // wait (bounded) for copies still in flight into this CTA's buffers
            if (tid == 0) {
                mbar_wait_bounded(&full[b], (unsigned)(it >> 1) & 1u, a.err);
                if (d1.z) mbar_wait_bounded(&full[b ^ 1], (unsigned)((it + 1) >> 1) & 1u, a.err);
            }
            if (tid < 32) bulk_wait_all();
            return;
        }
        const int key = d0.x;
        const int n = (key & 15) + 1;
        unsigned char* xt = xbuf + b * xbuf_bytes;
        const int* xo = ring + 2 * kVlThreads * s0;
        const int* yo = xo + kVlThreads;
        if (key < 16)
            vl_dispatch_n<S, 2>(a, d0, xt, ex1, xo, yo);
        else
            vl_dispatch_n<S, 3>(a, d0, xt, ex1, xo, yo);
        if (!a.alpha_one || !a.beta_zero) {
            // Epilogue Y = alpha (K x) + beta Y on the staged results (a separate pass,
            // so the contraction bodies stay as small as without it).  The values are
            // the storage-rounded results: for 16-bit storage this rounds twice.
            __syncthreads();
            const int nx = vl_nx(key);
            const int slot = key < 16 ? vl_xs_bytes(2, n, (int)sizeof(S)) : 4 * vl_e1_floats(3, n, (int)sizeof(S));
            unsigned char* base = key < 16 ? xt : reinterpret_cast<unsigned char*>(ex1);
            const S* Yg = static_cast<const S*>(a.Y);
            for (int e = tid; e < d0.z * nx; e += kVlThreads) {
                const int q = e / nx, r = e - q * nx;
                S* v = reinterpret_cast<S*>(base + q * slot) + vl_phase<S>(a.Y, yo[q]) + r;
                float o = load_cvt<float, S>(*v);
                if (!a.alpha_one) o *= a.alpha;
                if (!a.beta_zero) o = __fmaf_rn(a.beta, load_cvt<float, S>(Yg[yo[q] + r]), o);
                *v = store_cvt<S, float>(o);
            }
        }
        fence_proxy_async_smem();   // results visible to the bulk copies
        __syncthreads();
        if (tid < 32) {
            if (key < 16)
                vl_issue_stores<S>(a, d0, yo, xt, vl_xs_bytes(2, n, (int)sizeof(S)));
            else
                vl_issue_stores<S>(a, d0, yo, reinterpret_cast<const unsigned char*>(ex1),
                                   4 * vl_e1_floats(3, n, (int)sizeof(S)));
        }
        if (tid < d2.z) {
            ring[2 * kVlThreads * s2 + tid] = xo2;
            ring[2 * kVlThreads * s2 + kVlThreads + tid] = yo2;
        }
        __syncthreads();
        d0 = d1;
        d1 = d2;
        d2 = d3;
    }
    if (tid < 32) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Largest tile of class (kind, n) whose operand and exchange buffers stay within
// `budget` bytes each.
static int vl_max_P(int kind, int n, size_t es, int budget) {
    const int xs = vl_xs_bytes(kind, n, (int)es), ex = 4 * vl_e1_floats(kind, n, (int)es);
    return std::max(1, std::min(kVlThreads, budget / std::max(xs, ex)));
}

// Default tile, within the default buffer budget: as many instances as one
// round of fibers (one per thread) covers in 2-D, two rounds in 3-D (the
// tuner's choice on the mixed batch for most 3-D sizes: a second round halves
// the share of the barrier waits).
static int vl_default_P(int kind, int n, size_t es) {
    const int fibers = kind == 2 ? kVlThreads / n : 2 * kVlThreads / (n * n);
    return std::max(1, std::min(fibers, vl_max_P(kind, n, es, kVlBufBytes)));
}

}  // namespace kron

struct kron_varlen_plan {
    kron_dtype io;
    int64_t batch;
    int64_t x_total, y_total;                  // elements spanned by X / Y (bounds + aliasing)
    int present[kron::kVlKeys];
    int P[kron::kVlKeys];
    std::vector<int32_t> cls_of;               // per instance: class key
    std::vector<int64_t> xoff, yoff;           // per instance, draw order
    // derived
    std::vector<int64_t> order;                // instances sorted by class
    std::vector<int4> tiles;
    size_t ws_bytes = 0;
    size_t smem = 0;
    int xbuf_bytes = 0;                        // one operand buffer (two per CTA)
    int grid = 0;
    kron::VarlenArgs* args = nullptr;          // heap: ~30 KB
    // graph state
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t node = nullptr;
    const void* g_X = nullptr;
    void* g_Y = nullptr;
    void* g_ws = nullptr;
    void* uploaded_ws = nullptr;               // workspace that holds this plan's tables
    int uploaded_version = -1;
    int version = 0;                           // bumped whenever the tables change
    int graph_version = -1;                    // tables the instantiated graph was built for
    int device = -1;
    double alpha = 1.0, beta = 0.0;            // kron_varlen_plan_set_scaling
};

namespace kron {

static void* vl_kernel_ptr(kron_dtype io) {
    switch (io) {
        case KRON_R32F: return (void*)varlen_kernel<float>;
        case KRON_R16BF: return (void*)varlen_kernel<__nv_bfloat16>;
        case KRON_R16F: return (void*)varlen_kernel<__half>;
        default: return nullptr;
    }
}

// Sort by class, cut tiles, order them largest work first, size the workspace and smem.
static kron_status vl_build(kron_varlen_plan* p) {
    const size_t es = elem_size(p->io);
    std::vector<std::vector<int64_t>> by(kVlKeys);
    for (int64_t i = 0; i < p->batch; ++i) by[p->cls_of[i]].push_back(i);
    p->order.clear();
    p->tiles.clear();
    struct T { int64_t work; int4 td; };
    std::vector<T> tl;
    size_t max_x = 0, max_smem_rest = 0;
    for (int key = 0; key < kVlKeys; ++key) {
        if (by[key].empty()) continue;
        const int kind = key < 16 ? 2 : 3, n = (key & 15) + 1;
        const int P = p->P[key];
        const int64_t start = (int64_t)p->order.size();
        for (int64_t i : by[key]) p->order.push_back(i);
        const int64_t cnt = (int64_t)by[key].size();
        const int64_t flops = kind == 2 ? 4LL * n * n * n : 6LL * n * n * n * n;
        for (int64_t s = 0; s < cnt; s += P) {
            const int c = (int)std::min<int64_t>(P, cnt - s);
            tl.push_back(T{flops * c, make_int4(key, (int)(start + s), c, 0)});
        }
        max_x = std::max(max_x, (size_t)P * vl_xs_bytes(kind, n, (int)es));
        max_smem_rest = std::max(max_smem_rest, (size_t)P * vl_e1_floats(kind, n, (int)es) * sizeof(float));
    }
    if (p->order.size() > (size_t)INT32_MAX) return KRON_ERR_NOT_SUPPORTED;
    std::stable_sort(tl.begin(), tl.end(), [](const T& a, const T& b) { return a.work > b.work; });
    for (const T& t : tl) p->tiles.push_back(t.td);
    p->xbuf_bytes = (int)round_up(max_x, 128);
    p->smem = 128 + 6 * kVlThreads * sizeof(int) + 2 * (size_t)p->xbuf_bytes + max_smem_rest;
    // Sized for one tile per instance (the most any tile size can give), so that
    // re-tuning never outgrows a workspace sized before it.
    p->ws_bytes = round_up(p->order.size() * sizeof(int4), 256) + 2 * round_up(p->order.size() * 8, 256);
    p->version++;
    return KRON_OK;
}

static kron_status vl_fill_args(kron_varlen_plan* p, const void* X, void* Y, void* ws) {
    VarlenArgs& a = *p->args;
    for (int key = 0; key < kVlKeys; ++key) {
        const int kind = key < 16 ? 2 : 3, n = (key & 15) + 1;
        const unsigned nx = kind == 2 ? n * n : n * n * n;
        a.cls[key].P = p->present[key] ? p->P[key] : 0;
        a.cls[key].inv = nx == 1 ? 0u : (unsigned)((0x100000000ull + nx - 1) / nx);
    }
    char* w = static_cast<char*>(ws);
    a.tiles = reinterpret_cast<const int4*>(w);
    a.xoff = reinterpret_cast<const int64_t*>(w + round_up(p->order.size() * sizeof(int4), 256));
    a.yoff = a.xoff + round_up(p->order.size() * 8, 256) / 8;
    a.X = X;
    a.Y = Y;
    a.ntiles = (int)p->tiles.size();
    a.alpha = (float)p->alpha;
    a.beta = (float)p->beta;
    a.alpha_one = p->alpha == 1.0;
    a.beta_zero = p->beta == 0.0;
    a.err = device_error_word();
    return a.err ? KRON_OK : KRON_ERR_CUDA;
}

static kron_status vl_upload(kron_varlen_plan* p, void* ws, cudaStream_t st) {
    const size_t tb = round_up(p->order.size() * sizeof(int4), 256);
    const size_t ob = round_up(p->order.size() * 8, 256);
    std::vector<char> host(p->ws_bytes, 0);
    memcpy(host.data(), p->tiles.data(), p->tiles.size() * sizeof(int4));
    int64_t* xo = reinterpret_cast<int64_t*>(host.data() + tb);
    int64_t* yo = reinterpret_cast<int64_t*>(host.data() + tb + ob);
    for (size_t s = 0; s < p->order.size(); ++s) {
        xo[s] = p->xoff[p->order[s]];
        yo[s] = p->yoff[p->order[s]];
    }
    if (cudaMemcpyAsync(ws, host.data(), p->ws_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return KRON_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return KRON_ERR_CUDA;   // host buffer is a temporary
    p->uploaded_ws = ws;
    p->uploaded_version = p->version;
    return KRON_OK;
}

static void vl_drop_graph(kron_varlen_plan* p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    p->node = nullptr;
}

static kron_status vl_launch(kron_varlen_plan* p, const void* X, void* Y, void* ws, cudaStream_t st) {
    if (p->tiles.empty()) return KRON_OK;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    if (p->smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    void* fn = vl_kernel_ptr(p->io);
    if (!ensure_smem_optin(fn, p->smem)) return KRON_ERR_CUDA;
    if (p->uploaded_ws != ws || p->uploaded_version != p->version) {
        kron_status r = vl_upload(p, ws, st);
        if (r != KRON_OK) return r;
    }
    kron_status r = vl_fill_args(p, X, Y, ws);
    if (r != KRON_OK) return r;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kVlThreads, p->smem) != cudaSuccess)
        return KRON_ERR_CUDA;
    int grid = std::max(1, per_sm) * dev.sms;
    grid = (int)std::min<size_t>((size_t)grid, p->tiles.size());
    int xbe = p->xbuf_bytes;
    void* kargs[2] = {p->args, &xbe};
    cudaKernelNodeParams kp = {};
    kp.func = fn;
    kp.gridDim = dim3((unsigned)grid);
    kp.blockDim = dim3(kVlThreads);
    kp.sharedMemBytes = (unsigned)p->smem;
    kp.kernelParams = kargs;
    if (p->exec && p->graph_version == p->version && p->grid == grid) {
        // same tables and launch shape: only the pointers may differ
        if (cudaGraphExecKernelNodeSetParams(p->exec, p->node, &kp) != cudaSuccess) vl_drop_graph(p);
    } else {
        vl_drop_graph(p);
    }
    if (!p->exec) {
        if (cudaGraphCreate(&p->graph, 0) != cudaSuccess) return KRON_ERR_CUDA;
        if (cudaGraphAddKernelNode(&p->node, p->graph, nullptr, 0, &kp) != cudaSuccess ||
            cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) {
            vl_drop_graph(p);
            return KRON_ERR_CUDA;
        }
        p->graph_version = p->version;
    }
    p->grid = grid;
    p->g_X = X;
    p->g_Y = Y;
    p->g_ws = ws;
    return cudaGraphLaunch(p->exec, st) == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

}  // namespace kron

using namespace kron;

extern "C" {

KRON_API kron_status kron_varlen_plan_create(kron_varlen_plan** plan, int num_classes, const kron_class_desc* classes,
                                             int64_t batch_count, const int32_t* h_class_of, const int64_t* h_x_off,
                                             const int64_t* h_y_off, kron_dtype io, kron_compute comp) {
    if (!plan) return KRON_ERR_INVALID_VALUE;
    *plan = nullptr;
    if (num_classes < 0 || num_classes > kVlKeys || batch_count < 0) return KRON_ERR_INVALID_VALUE;
    if (num_classes > 0 && !classes) return KRON_ERR_INVALID_VALUE;
    if (batch_count > 0 && (!h_class_of || !h_x_off || !h_y_off)) return KRON_ERR_INVALID_VALUE;
    if (io != KRON_R32F && io != KRON_R16BF && io != KRON_R16F) {
        return (io == KRON_R64F || is_complex(io)) ? KRON_ERR_NOT_SUPPORTED : KRON_ERR_INVALID_VALUE;
    }
    if (comp != KRON_COMPUTE_NATIVE) return comp == KRON_COMPUTE_32F_BF16X3 ? KRON_ERR_NOT_SUPPORTED
                                                                            : KRON_ERR_INVALID_VALUE;
    if (batch_count >= INT32_MAX) return KRON_ERR_NOT_SUPPORTED;
    kron_varlen_plan* p = new (std::nothrow) kron_varlen_plan();
    if (!p) return KRON_ERR_INVALID_VALUE;
    p->args = new (std::nothrow) VarlenArgs();
    if (!p->args) { delete p; return KRON_ERR_INVALID_VALUE; }
    memset(p->args, 0, sizeof(VarlenArgs));
    p->io = io;
    p->batch = batch_count;
    std::fill(p->present, p->present + kVlKeys, 0);
    std::vector<int> key_of_class(num_classes);
    for (int c = 0; c < num_classes; ++c) {
        const kron_class_desc& d = classes[c];
        if ((d.kind != 2 && d.kind != 3) || d.n < 1 || d.n > kMaxN || !d.A || !d.B || (d.kind == 3 && !d.C)) {
            kron_varlen_plan_destroy(p);
            return KRON_ERR_INVALID_VALUE;
        }
        const int key = 16 * (d.kind - 2) + d.n - 1;
        if (p->present[key]) {   // one component set per (kind, n)
            kron_varlen_plan_destroy(p);
            return KRON_ERR_INVALID_VALUE;
        }
        p->present[key] = 1;
        key_of_class[c] = key;
        const int n = d.n;
        const int rows = vl_rows(n);
        float* slot = p->args->coef + vl_slot(d.kind, n);
        // mode 1 first: 2-D (Y = B X A^T) B, A; 3-D C, B, A
        const void* mats[3] = {d.kind == 2 ? d.B : d.C, d.kind == 2 ? d.A : d.B, d.A};
        for (int c = 0; c < d.kind; ++c) {
            const float* M = static_cast<const float*>(mats[c]);
            float* dst = slot + c * rows * n;
            for (int col = 0; col < n; ++col)
                for (int r = 0; r < rows; ++r) dst[r + rows * col] = r < n ? M[r + n * col] : 0.0f;
        }
        int tp = 0, td = 0;
        kron_get_tile_config(d.kind, n, io, (kron_compute)kVarlenTag, &tp, &td);
        p->P[key] = (tp > 0 && tp <= vl_max_P(d.kind, n, elem_size(io), kVlMaxBufBytes)) ? tp
                                                                                     : vl_default_P(d.kind, n, elem_size(io));
    }
    p->cls_of.resize(batch_count);
    p->xoff.assign(h_x_off, h_x_off + batch_count);
    p->yoff.assign(h_y_off, h_y_off + batch_count);
    int64_t xt = 0, yt = 0;
    for (int64_t i = 0; i < batch_count; ++i) {
        const int c = h_class_of[i];
        if (c < 0 || c >= num_classes || h_x_off[i] < 0 || h_y_off[i] < 0) {
            kron_varlen_plan_destroy(p);
            return KRON_ERR_INVALID_VALUE;
        }
        const int key = key_of_class[c];
        p->cls_of[i] = key;
        const int n = (key & 15) + 1;
        const int64_t nx = key < 16 ? (int64_t)n * n : (int64_t)n * n * n;
        xt = std::max(xt, h_x_off[i] + nx);
        yt = std::max(yt, h_y_off[i] + nx);
    }
    // Instances of Y must not overlap (each output element written once).
    {
        std::vector<std::pair<int64_t, int64_t>> r(batch_count);
        for (int64_t i = 0; i < batch_count; ++i) {
            const int n = (p->cls_of[i] & 15) + 1;
            const int64_t nx = p->cls_of[i] < 16 ? (int64_t)n * n : (int64_t)n * n * n;
            r[i] = {h_y_off[i], h_y_off[i] + nx};
        }
        std::sort(r.begin(), r.end());
        for (int64_t i = 1; i < batch_count; ++i)
            if (r[i].first < r[i - 1].second) {
                kron_varlen_plan_destroy(p);
                return KRON_ERR_INVALID_VALUE;
            }
    }
    if (xt >= INT32_MAX || yt >= INT32_MAX) {   // the kernel keeps element offsets in 32 bits
        kron_varlen_plan_destroy(p);
        return KRON_ERR_NOT_SUPPORTED;
    }
    p->x_total = xt;
    p->y_total = yt;
    kron_status st = vl_build(p);
    if (st != KRON_OK) {
        kron_varlen_plan_destroy(p);
        return st;
    }
    *plan = p;
    return KRON_OK;
}

KRON_API kron_status kron_varlen_workspace_size(const kron_varlen_plan* plan, size_t* bytes) {
    if (!plan || !bytes) return KRON_ERR_INVALID_VALUE;
    *bytes = plan->ws_bytes;
    return KRON_OK;
}

static kron_status vl_check_exec(kron_varlen_plan* plan, const void* X, void* Y, void* workspace,
                                 size_t workspace_bytes) {
    if (!plan) return KRON_ERR_INVALID_VALUE;
    if (plan->batch == 0) return KRON_OK;
    if (!X || !Y) return KRON_ERR_INVALID_VALUE;
    if (!workspace || workspace_bytes < plan->ws_bytes || ((uintptr_t)workspace) % 256) return KRON_ERR_WORKSPACE;
    const size_t es = elem_size(plan->io);
    if (((uintptr_t)X) % es || ((uintptr_t)Y) % es) return KRON_ERR_INVALID_VALUE;
    const uintptr_t x0 = (uintptr_t)X, x1 = x0 + plan->x_total * es;
    const uintptr_t y0 = (uintptr_t)Y, y1 = y0 + plan->y_total * es;
    const uintptr_t w0 = (uintptr_t)workspace, w1 = w0 + plan->ws_bytes;
    if (x0 < y1 && y0 < x1) return KRON_ERR_ALIAS;
    if ((w0 < y1 && y0 < w1) || (w0 < x1 && x0 < w1)) return KRON_ERR_WORKSPACE;
    kron_status st;
    if ((st = device_range(X, plan->x_total * es)) != KRON_OK || (st = device_range(Y, plan->y_total * es)) != KRON_OK)
        return st;
    if ((st = device_range(workspace, plan->ws_bytes)) != KRON_OK) return st == KRON_ERR_CUDA ? st : KRON_ERR_WORKSPACE;
    return KRON_OK;
}

KRON_API kron_status kron_varlen_execute(kron_varlen_plan* plan, const void* X, void* Y, void* workspace,
                                         size_t workspace_bytes, kron_stream_t stream) {
    kron_status st = vl_check_exec(plan, X, Y, workspace, workspace_bytes);
    if (st != KRON_OK || plan->batch == 0) return st;
    return vl_launch(plan, X, Y, workspace, (cudaStream_t)stream);
}

KRON_API kron_status kron_varlen_tune(kron_varlen_plan* plan, const void* X, void* Y, void* workspace,
                                      size_t workspace_bytes, kron_stream_t stream) {
    kron_status st = vl_check_exec(plan, X, Y, workspace, workspace_bytes);
    if (st != KRON_OK || plan->batch == 0) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return KRON_ERR_CUDA;
    auto time_it = [&](float* ms) -> kron_status {
        kron_status r = KRON_OK;
        for (int w = 0; w < 2 && r == KRON_OK; ++w) r = vl_launch(plan, X, Y, workspace, s);
        if (r != KRON_OK) return r;
        cudaEventRecord(e0, s);
        for (int w = 0; w < 5 && r == KRON_OK; ++w) r = vl_launch(plan, X, Y, workspace, s);
        cudaEventRecord(e1, s);
        if (r != KRON_OK || cudaEventSynchronize(e1) != cudaSuccess) return KRON_ERR_CUDA;
        cudaEventElapsedTime(ms, e0, e1);
        return KRON_OK;
    };
    // Coordinate descent over the classes, largest work first: for each class try
    // tile sizes around its current one and keep the fastest whole-batch time.
    std::vector<std::pair<int64_t, int>> work;
    std::vector<int64_t> count(kVlKeys, 0);
    for (int64_t i = 0; i < plan->batch; ++i) count[plan->cls_of[i]]++;
    for (int key = 0; key < kVlKeys; ++key)
        if (count[key]) {
            const int n = (key & 15) + 1;
            work.push_back({count[key] * (key < 16 ? 4LL * n * n * n : 6LL * n * n * n * n), key});
        }
    std::sort(work.rbegin(), work.rend());
    float best = 0;
    st = time_it(&best);
    for (size_t w = 0; w < work.size() && st == KRON_OK; ++w) {
        const int key = work[w].second;
        const int kind = key < 16 ? 2 : 3, n = (key & 15) + 1;
        const int pmax = vl_max_P(kind, n, elem_size(plan->io), kVlMaxBufBytes);
        const int cur = plan->P[key];
        int best_P = cur;
        // Besides the neighbours of the current tile: the tile whose fibers per stage
        // fill the CTA's threads most evenly (P n^(kind-1) against whole rounds of
        // kVlThreads), the smallest such when several tie.
        const int fib = kind == 2 ? n : n * n;
        int even_P = 1;
        double even_eff = 0.0;
        for (int q = 1; q <= pmax; ++q) {
            const int rounds = (q * fib + kVlThreads - 1) / kVlThreads;
            const double eff = (double)(q * fib) / ((double)rounds * kVlThreads);
            if (eff > even_eff + 1e-9) { even_eff = eff; even_P = q; }
        }
        for (int cand : {cur / 2, cur * 2, cur * 4, cur / 4, cur + cur / 2, even_P}) {
            if (cand < 1 || cand > pmax || cand == cur) continue;
            plan->P[key] = cand;
            vl_build(plan);
            float ms = 0;
            st = time_it(&ms);
            if (st != KRON_OK) break;
            if (ms < best) { best = ms; best_P = cand; }
        }
        plan->P[key] = best_P;
        vl_build(plan);
        kron_set_tile_config(kind, n, plan->io, (kron_compute)kVarlenTag, best_P, 0);
        tune_cache_append(kind, n, plan->io, (kron_compute)kVarlenTag, best_P, 0);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// ---------------------------------------------------------------------------
// Allocation-free execute.  The tables go into a fixed file-scope device array
// instead of a caller workspace.  Its device address is looked up once per
// device (with that device current) by the first call on that device.  Every
// call rewrites the tables it needs before its launch, so no state is carried
// over; concurrent calls on the same device share the array and would race.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_varlen_noalloc_scratch[kron::kVarlenNoallocScratchBytes];

static void* noalloc_scratch() {
    static void* ptr[64] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_varlen_noalloc_scratch) != cudaSuccess) return nullptr;
        ptr[dev] = p;
    }
    return ptr[dev];
}

KRON_API kron_status kron_varlen_execute_noalloc(kron_varlen_plan* plan, const void* X, void* Y,
                                                 kron_stream_t stream) {
    if (!plan) return KRON_ERR_INVALID_VALUE;
    if (plan->batch == 0) return KRON_OK;
    if (plan->ws_bytes > kVarlenNoallocScratchBytes) return KRON_ERR_WORKSPACE;   // batch above the maximum
    if (!X || !Y) return KRON_ERR_INVALID_VALUE;
    const size_t es = elem_size(plan->io);
    if (((uintptr_t)X) % es || ((uintptr_t)Y) % es) return KRON_ERR_INVALID_VALUE;
    const uintptr_t x0 = (uintptr_t)X, x1 = x0 + plan->x_total * es;
    const uintptr_t y0 = (uintptr_t)Y, y1 = y0 + plan->y_total * es;
    if (x0 < y1 && y0 < x1) return KRON_ERR_ALIAS;
    if (plan->tiles.empty()) return KRON_OK;
    kron_status rs;
    if ((rs = device_range(X, plan->x_total * es)) != KRON_OK || (rs = device_range(Y, plan->y_total * es)) != KRON_OK)
        return rs;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    if (plan->smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    void* ws = noalloc_scratch();
    if (!ws) return KRON_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    kron_status r = vl_upload(plan, ws, st);   // the shared array may hold another call's tables
    if (r != KRON_OK) return r;
    r = vl_fill_args(plan, X, Y, ws);
    if (r != KRON_OK) return r;
    void* fn = vl_kernel_ptr(plan->io);
    if (!ensure_smem_optin(fn, plan->smem)) return KRON_ERR_CUDA;   // the attribute only ever grows
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kVlThreads, plan->smem) != cudaSuccess)
        return KRON_ERR_CUDA;
    int grid = std::max(1, per_sm) * dev.sms;
    grid = (int)std::min<size_t>((size_t)grid, plan->tiles.size());
    int xbe = plan->xbuf_bytes;
    void* kargs[2] = {plan->args, &xbe};
    if (cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kVlThreads), kargs, plan->smem, st) != cudaSuccess)
        return KRON_ERR_CUDA;
    return KRON_OK;
}

KRON_API kron_status kron_varlen_plan_set_scaling(kron_varlen_plan* plan, double alpha, double beta) {
    if (!plan || !std::isfinite(alpha) || !std::isfinite(beta)) return KRON_ERR_INVALID_VALUE;
    plan->alpha = alpha;   // read by the next execute (the kernel node's parameters are set on every call)
    plan->beta = beta;
    return KRON_OK;
}

KRON_API kron_status kron_varlen_plan_destroy(kron_varlen_plan* plan) {
    if (!plan) return KRON_OK;
    vl_drop_graph(plan);
    delete plan->args;
    delete plan;
    return KRON_OK;
}

}  // extern "C"
