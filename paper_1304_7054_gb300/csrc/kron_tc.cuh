#pragma once
// Tensor-core split-precision kernels (KRON_COMPUTE_32F_BF16X3).
//
// Each FP32 value v is split into two bfloat16 values, hi = bf16(v) and
// lo = bf16(v - hi) (round to nearest even; v - hi is exact), and every product
// a*b of a contraction is evaluated as a_hi*b_hi + a_hi*b_lo + a_lo*b_hi with
// FP32 accumulation on the tensor cores (mma.sync m16n8k16, bf16 inputs, f32
// accumulators).  The dropped a_lo*b_lo term and the residual of the split are
// below 2^-16 relative, which gives FP32-level accuracy.  For bf16 storage the
// operand is exact (lo = 0) and its products with the split components need two
// MMAs instead of three.
//
// 2-D (Y = M1 X M2^T, paper Sec. 2 vec identity), one warp per 16 x 16 tile:
// one instance for n > 8 (zero-padded), two for 4 < n <= 8 and four for n <= 4
// on the tile's diagonal:
//   stage 1  W = M1 X       A = M1 (constant fragments), B = X (from the tile)
//   stage 2  Y = W M2^T     A = W taken straight from the stage-1 accumulators
//                           (the m16n8 accumulator layout of two n-tiles is the
//                           m16k16 A-fragment layout), B = M2^T (constant)
// Operand tiles of P instances stream into shared memory with 1-D bulk copies
// (TMA) in an mbarrier pipeline, as in the CUDA-core kernels.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "kron_device.cuh"
#include "kron_fiber.cuh"
#include "kron_internal.h"

namespace kron {

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// The same shape on f16 operands (f16 storage: the stored operand enters as it is).
__device__ __forceinline__ void mma_f16_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// mma.sync.aligned and ldmatrix.sync.aligned need the whole warp converged on the
// same instruction; the groups of them that follow bounds tests or tail stores
// (which may leave the lanes diverged) start with a warp synchronisation.
__device__ __forceinline__ void converge() { __syncwarp(); }

// (x0, x1) -> packed bf16 pairs hi = (bf16(x0), bf16(x1)), lo = (bf16(x0 - hi0), bf16(x1 - hi1)).
__device__ __forceinline__ void split_pair(float x0, float x1, unsigned& hi, unsigned& lo) {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
    const float r0 = x0 - __uint_as_float(hi << 16);
    const float r1 = x1 - __uint_as_float(hi & 0xffff0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(r1), "f"(r0));
}

template <int N>
struct TcArgs2 {
    // Row-major 16 x 16 components as packed bf16 pairs along the row:
    // word r*8 + c/2 holds (M[r][c], M[r][c+1]); hi and lo parts of the split.
    unsigned m1h[128], m1l[128];
    unsigned m2h[128], m2l[128];
    // f16 storage: M1 * 2^s as an f16 split (the first product then takes the
    // stored f16 operand as it is, two MMAs instead of three); M2 above is then
    // scaled by 2^-s.  f16a = 0: not used (bf16 split of the operand instead).
    unsigned f1h[128], f1l[128];
    int f16a;
    const void* X;
    void* Y;
    int64_t batch;
    int P;
    int nstage;
    int beta_zero, alpha_one;
    int ypair;                  // Y aligned to two elements: the stacked body stores pairs
    float alpha, beta;
    unsigned* err;
};

// Two elements (X[l][m], X[l+1][m]) of an instance in the tile (zero outside n x n).
template <typename S, int N>
__device__ __forceinline__ void x_pair(const S* xq, int l, int m, float& v0, float& v1) {
    v0 = (l < N && m < N) ? load_cvt<float, S>(xq[l + N * m]) : 0.f;
    v1 = (l + 1 < N && m < N) ? load_cvt<float, S>(xq[l + 1 + N * m]) : 0.f;
}

// The same pair of a 16-bit operand as its raw bits (two packed values).
template <int N, typename S>
__device__ __forceinline__ unsigned x_pair_bf16(const S* xq, int l, int m) {
    const unsigned short* xs = reinterpret_cast<const unsigned short*>(xq);
    if constexpr (N % 2 == 0) {
        return (l < N && m < N) ? *reinterpret_cast<const unsigned*>(xs + l + N * m) : 0u;
    } else {
        const unsigned a = (l < N && m < N) ? (unsigned)xs[l + N * m] : 0u;
        const unsigned b = (l + 1 < N && m < N) ? (unsigned)xs[l + 1 + N * m] : 0u;
        return a | (b << 16);
    }
}

// Small instances share one 16 x 16 tile: 16 / B instances of size n <= B sit
// on its diagonal in B x B blocks, with blockdiag(M, ..., M) as the component.
// Off-diagonal blocks stay zero through both products, so one tile computes
// all of them with the MMAs of one instance.
__host__ __device__ constexpr int tc2_block(int n) { return n <= 4 ? 4 : (n <= 8 ? 8 : 16); }

// Element pair (l, l+1) x column m of the block-diagonal operand tile.
template <typename S, int N, int B>
__device__ __forceinline__ void x_pair_blk(const S* const (&xq)[16 / B], int l, int m, float& v0, float& v1) {
    const int b = l / B;
    if (b == m / B && xq[b]) {
        x_pair<S, N>(xq[b], l % B, m % B, v0, v1);
    } else {
        v0 = 0.f;
        v1 = 0.f;
    }
}

template <int N, int B, typename S>
__device__ __forceinline__ unsigned x_pair_bf16_blk(const S* const (&xq)[16 / B], int l, int m) {
    const int b = l / B;
    return (b == m / B && xq[b]) ? x_pair_bf16<N>(xq[b], l % B, m % B) : 0u;
}

// One 16 x 16 tile: 16 / B instances (xq[b] / yq[b], null when absent).
template <typename S, int N, int B>
__device__ __forceinline__ void tc2_instance(const TcArgs2<N>& a, const S* const (&xq)[16 / B],
                                             S* const (&yq)[16 / B], const unsigned (&m1h)[4],
                                             const unsigned (&m1l)[4], const unsigned (&m2h)[2][2],
                                             const unsigned (&m2l)[2][2], const unsigned (&f1h)[4],
                                             const unsigned (&f1l)[4]) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    if constexpr (sizeof(S) == 4) {
        // FP32 storage: one n-tile after the other (measured faster than the
        // step-by-step order below, which pays off for 16-bit storage).
        // ---- stage 1: W = M1 X -----------------------------------------------------------
        float w[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int m = 8 * nt + g;
#pragma unroll
            for (int e = 0; e < 4; ++e) w[nt][e] = 0.f;
            float x0, x1, x2, x3;
            if constexpr (N == 16) {
                const float2 p0 = *reinterpret_cast<const float2*>(xq[0] + 2 * t + 16 * m);
                const float2 p1 = *reinterpret_cast<const float2*>(xq[0] + 2 * t + 8 + 16 * m);
                x0 = p0.x; x1 = p0.y; x2 = p1.x; x3 = p1.y;
            } else {
                x_pair_blk<S, N, B>(xq, 2 * t, m, x0, x1);
                x_pair_blk<S, N, B>(xq, 2 * t + 8, m, x2, x3);
            }
            unsigned bh0, bl0, bh1, bl1;
            split_pair(x0, x1, bh0, bl0);
            split_pair(x2, x3, bh1, bl1);
            converge();
            mma_bf16_16816(w[nt], m1l, bh0, bh1);
            mma_bf16_16816(w[nt], m1h, bl0, bl1);
            mma_bf16_16816(w[nt], m1h, bh0, bh1);
        }
        // ---- stage 2: Y = W M2^T, W from the accumulators --------------------------------
        unsigned wh[4], wl[4];
        split_pair(w[0][0], w[0][1], wh[0], wl[0]);
        split_pair(w[0][2], w[0][3], wh[1], wl[1]);
        split_pair(w[1][0], w[1][1], wh[2], wl[2]);
        split_pair(w[1][2], w[1][3], wh[3], wl[3]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            float y[4] = {0.f, 0.f, 0.f, 0.f};
            converge();
            mma_bf16_16816(y, wl, m2h[nt][0], m2h[nt][1]);
            mma_bf16_16816(y, wh, m2l[nt][0], m2l[nt][1]);
            mma_bf16_16816(y, wh, m2h[nt][0], m2h[nt][1]);
            const int j = 8 * nt + 2 * t;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = g + 8 * (e >> 1), jj = j + (e & 1);
                const int b = i / B, il = i % B, jl = jj % B;
                if (b == jj / B && yq[b] && il < N && jl < N) {
                    S* dst = yq[b] + il + N * jl;
                    float v = a.alpha_one ? y[e] : a.alpha * y[e];
                    if (!a.beta_zero) v = fmaf(a.beta, load_cvt<float, S>(*dst), v);
                    __stcs(reinterpret_cast<float*>(dst), v);
                }
            }
        }
    } else {
        // ---- stage 1: W = M1 X ---------------------------------------------------------------
        // The MMAs go step by step across the two n-tiles (the first products of both,
        // then the second ...): one n-tile's dependent products are separated by the other's.
        float w[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) w[nt][e] = 0.f;
        if constexpr (std::is_same<S, __nv_bfloat16>::value) {
            unsigned b0[2], b1[2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                b0[nt] = x_pair_bf16_blk<N, B>(xq, 2 * t, 8 * nt + g);
                b1[nt] = x_pair_bf16_blk<N, B>(xq, 2 * t + 8, 8 * nt + g);
            }
            converge();
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_bf16_16816(w[nt], m1l, b0[nt], b1[nt]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_bf16_16816(w[nt], m1h, b0[nt], b1[nt]);
        } else if (std::is_same<S, __half>::value && a.f16a) {
            unsigned b0[2], b1[2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                b0[nt] = x_pair_bf16_blk<N, B>(xq, 2 * t, 8 * nt + g);
                b1[nt] = x_pair_bf16_blk<N, B>(xq, 2 * t + 8, 8 * nt + g);
            }
            converge();
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_f16_16816(w[nt], f1l, b0[nt], b1[nt]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_f16_16816(w[nt], f1h, b0[nt], b1[nt]);
        } else {
            unsigned bh0[2], bl0[2], bh1[2], bl1[2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int m = 8 * nt + g;   // f16 storage without the scaled f16 split
                float x0, x1, x2, x3;
                x_pair_blk<S, N, B>(xq, 2 * t, m, x0, x1);
                x_pair_blk<S, N, B>(xq, 2 * t + 8, m, x2, x3);
                split_pair(x0, x1, bh0[nt], bl0[nt]);
                split_pair(x2, x3, bh1[nt], bl1[nt]);
            }
            converge();
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_bf16_16816(w[nt], m1l, bh0[nt], bh1[nt]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_bf16_16816(w[nt], m1h, bl0[nt], bl1[nt]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) mma_bf16_16816(w[nt], m1h, bh0[nt], bh1[nt]);
        }
        // ---- stage 2: Y = W M2^T, W from the accumulators ------------------------------------
        unsigned wh[4], wl[4];
        split_pair(w[0][0], w[0][1], wh[0], wl[0]);
        split_pair(w[0][2], w[0][3], wh[1], wl[1]);
        split_pair(w[1][0], w[1][1], wh[2], wl[2]);
        split_pair(w[1][2], w[1][3], wh[3], wl[3]);
        float y[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) y[nt][e] = 0.f;
        converge();
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_bf16_16816(y[nt], wl, m2h[nt][0], m2h[nt][1]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_bf16_16816(y[nt], wh, m2l[nt][0], m2l[nt][1]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma_bf16_16816(y[nt], wh, m2h[nt][0], m2h[nt][1]);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int j = 8 * nt + 2 * t;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int i = g + 8 * (e >> 1), jj = j + (e & 1);
                const int b = i / B, il = i % B, jl = jj % B;
                if (b == jj / B && yq[b] && il < N && jl < N) {
                    S* dst = yq[b] + il + N * jl;
                    float v = a.alpha_one ? y[nt][e] : a.alpha * y[nt][e];
                    if (!a.beta_zero) v = fmaf(a.beta, load_cvt<float, S>(*dst), v);
                    *dst = store_cvt<S, float>(v);
                }
            }
        }
    }
}

constexpr int kTcThreads = 128;

template <typename S, int N>
__global__ void __launch_bounds__(kTcThreads) tc2_kernel(const __grid_constant__ TcArgs2<N> a) {
    constexpr int NX = N * N;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    const int P = a.P;
    const size_t xstage = round_up((size_t)P * NX * sizeof(S), 128);
    unsigned char* xbase = smem + 128;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t ntiles = (a.batch + P - 1) / P;
    const int64_t grid = gridDim.x;

    // Constant fragments: A of M1 (rows g, g+8; pair columns t, t+4) and B of
    // M2^T for both n-tiles (column j = 8 nt + g of M2^T is row j of M2).
    unsigned m1h[4], m1l[4], m2h[2][2], m2l[2][2], f1h[4] = {0u, 0u, 0u, 0u}, f1l[4] = {0u, 0u, 0u, 0u};
    if (std::is_same<S, __half>::value && a.f16a) {
        f1h[0] = a.f1h[g * 8 + t];           f1l[0] = a.f1l[g * 8 + t];
        f1h[1] = a.f1h[(g + 8) * 8 + t];     f1l[1] = a.f1l[(g + 8) * 8 + t];
        f1h[2] = a.f1h[g * 8 + t + 4];       f1l[2] = a.f1l[g * 8 + t + 4];
        f1h[3] = a.f1h[(g + 8) * 8 + t + 4]; f1l[3] = a.f1l[(g + 8) * 8 + t + 4];
    }
    m1h[0] = a.m1h[g * 8 + t];       m1l[0] = a.m1l[g * 8 + t];
    m1h[1] = a.m1h[(g + 8) * 8 + t]; m1l[1] = a.m1l[(g + 8) * 8 + t];
    m1h[2] = a.m1h[g * 8 + t + 4];   m1l[2] = a.m1l[g * 8 + t + 4];
    m1h[3] = a.m1h[(g + 8) * 8 + t + 4]; m1l[3] = a.m1l[(g + 8) * 8 + t + 4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int j = 8 * nt + g;
        m2h[nt][0] = a.m2h[j * 8 + t];     m2l[nt][0] = a.m2l[j * 8 + t];
        m2h[nt][1] = a.m2h[j * 8 + t + 4]; m2l[nt][1] = a.m2l[j * 8 + t + 4];
    }

    uint64_t pol = 0;
    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        pol = l2_evict_first_policy();
        for (int s = 0; s < a.nstage; ++s) {
            const int64_t tl = blockIdx.x + s * grid;
            if (tl < ntiles) {
                const int64_t i0 = tl * P;
                const int cnt = (int)min((int64_t)P, a.batch - i0);
                const unsigned bytes = ((unsigned)cnt * NX * (unsigned)sizeof(S)) & ~15u;
                mbar_arrive_expect_tx(&bars[s], bytes);
                if (bytes) bulk_g2s(xbase + s * xstage, static_cast<const S*>(a.X) + i0 * NX, bytes, &bars[s], pol);
            }
        }
    }
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
        const int s = it % a.nstage;
        S* xt = reinterpret_cast<S*>(xbase + s * xstage);
        const int64_t inst0 = tile * P;
        const int cnt = (int)min((int64_t)P, a.batch - inst0);
        bool ok = mbar_wait_bounded(&bars[s], (unsigned)(it / a.nstage) & 1u, a.err);
        const unsigned bytes = (unsigned)cnt * NX * (unsigned)sizeof(S);
        const unsigned b16 = bytes & ~15u;
        if (bytes != b16) {
            const S* src = static_cast<const S*>(a.X) + inst0 * NX;
            for (int e = b16 / sizeof(S) + tid; e < cnt * NX; e += kTcThreads) xt[e] = src[e];
            __syncthreads();
        }
        if (ok) {
            constexpr int B = tc2_block(N), PK = 16 / B;
            for (int q0 = warp * PK; q0 < cnt; q0 += PK * (kTcThreads / 32)) {
                const S* xq[PK];
                S* yq[PK];
#pragma unroll
                for (int b = 0; b < PK; ++b) {
                    const bool live = q0 + b < cnt;
                    xq[b] = live ? xt + (q0 + b) * NX : nullptr;
                    yq[b] = live ? static_cast<S*>(a.Y) + (inst0 + q0 + b) * NX : nullptr;
                }
                tc2_instance<S, N, B>(a, xq, yq, m1h, m1l, m2h, m2l, f1h, f1l);
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                for (int j = it; j < it + a.nstage; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&bars[j % a.nstage], (unsigned)(j / a.nstage) & 1u, a.err);
            }
            return;
        }
        if (tid == 0) {
            const int64_t next = tile + a.nstage * grid;
            if (next < ntiles) {
                const int64_t i0 = next * P;
                const int c2 = (int)min((int64_t)P, a.batch - i0);
                const unsigned nb = ((unsigned)c2 * NX * (unsigned)sizeof(S)) & ~15u;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[s], nb);
                if (nb) bulk_g2s(xt, static_cast<const S*>(a.X) + i0 * NX, nb, &bars[s], pol);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 3-D: one warp per instance, three tensor-core contractions.
//
//   per plane p (modes 1 and 2), two planes at a time for instruction-level
//   parallelism:
//     stage 1  W' = M2 X_p^T      A = M2 (constant), B = X_p^T read from the
//                                 FP32 instance in shared memory and split
//     stage 2  T_p^T = W' M1^T    A = W' from the accumulators, B = M1^T (constant)
//              T_p^T is split and stored as row p of the matrix T[p][r],
//              r = i + 16 j (hi half and lo half, 512 bytes each); for n = 16
//              row p overwrites the FP32 plane p it was computed from
//   stage 3 (mode 3), per 16 rows r:  Y[r][k] = sum_p T[p][r] M3[k][p]
//              A via ldmatrix.trans of T, B = M3^T (constant); rows r = i + 16 j
//              make consecutive lanes write consecutive elements of Y.
// The intermediates never leave shared memory; each warp owns its buffers and
// its bulk-copy barrier, so the warps of a CTA never wait for each other.
// ---------------------------------------------------------------------------
// One warp per CTA: the per-CTA shared-memory reservation then lets 13 (n = 16)
// instead of 12 warps reside per SM (measured 1% faster at n = 16, 7% at n = 10).
constexpr int kTc3Warps = 1;

template <int N>
struct TcArgs3 {
    unsigned m1h[128], m1l[128];   // row-major packed bf16 pairs, as TcArgs2
    unsigned m2h[128], m2l[128];
    unsigned m3h[128], m3l[128];
    unsigned f2h[128], f2l[128];   // f16 storage: M2 * 2^s as an f16 split (M1 scaled by 2^-s)
    int f16a;                      // 0: not used
    const void* X;
    void* Y;
    int64_t batch;
    int beta_zero, alpha_one;
    int ypair;                     // Y 4-byte aligned: 16-bit results leave as pairs
    float alpha, beta;
    unsigned* err;
};

// n < 16 or 16-bit storage: T has its own 16 KB buffer, so the operand buffer is
// free after modes 1 and 2 and the next instance is fetched while mode 3 runs.
// n = 16 with FP32 storage: T rows overwrite the operand planes (a separate T
// buffer halves the resident warps and measured 1.32x slower), so the next fetch
// waits for mode 3.
template <typename S, int N>
struct Tc3Layout {
    // the instance, at its alignment phase when n^3 elements are not a whole
    // number of 16-byte units (odd n): the copy takes the aligned span around it
    static constexpr bool ALIGNED = (N * N * N * sizeof(S)) % 16 == 0;
    static constexpr uint32_t XB = (uint32_t)round_up((size_t)N * N * N * sizeof(S) + (ALIGNED ? 0 : 32), 128);
    static constexpr bool INPLACE = (N == 16 && sizeof(S) == 4);   // T rows overwrite the operand planes
    static constexpr uint32_t TB = INPLACE ? 0u : 16384u;
    static constexpr uint32_t PER_WARP = XB + TB;
};

__device__ __forceinline__ void ldsm_x4_trans(unsigned (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr)
                 : "memory");
}

// Byte offset of 16-byte chunk c (8 elements) of row p of T, hi half; the lo half
// follows 512 bytes later.  Rows are 1 KB apart; the chunk index is XOR-ed with
// the row so that the eight rows read by one ldmatrix matrix, and the eight
// chunks written by one store instruction, fall in distinct banks.
__device__ __forceinline__ uint32_t trow_off(int p, int c) {
    return (uint32_t)(p * 1024 + 16 * ((c ^ (p & 7) ^ ((c >> 3) & 1)) & 31));
}

template <typename S, int N>
__device__ __forceinline__ float xval(const S* xs, int l, int m, int p) {
    if constexpr (N == 16) return load_cvt<float, S>(xs[l + 16 * m + 256 * p]);
    else return (l < N && m < N) ? load_cvt<float, S>(xs[l + N * m + N * N * p]) : 0.f;
}

// Modes 1 and 2 of plane p: writes row p of T (hi and lo halves).
// f16a (f16 storage): bh receives the raw f16 pairs, for f16 MMAs.
template <typename S, int N>
__device__ __forceinline__ void tc3_plane_load(const S* xs, int p, int g, int t, unsigned (&bh)[4],
                                               unsigned (&bl)[4], bool f16a) {
    if constexpr (N == 16 && sizeof(S) == 2) {
        // 16-bit planes: the four 8 x 8 blocks of X_p^T by one ldmatrix.trans.
        // Matrix mi = 2 nt + h holds rows m = 8 h + r (16 contiguous bytes: l =
        // 8 nt .. 8 nt + 7), so lane (g, t) receives X_p[8 nt + g][8 h + 2t, +1].
        const int lane = 4 * g + t, mi = lane >> 3, r = lane & 7;
        unsigned v[4];
        converge();
        ldsm_x4_trans(v, smem_u32(xs + 8 * (mi >> 1) + 16 * (8 * (mi & 1) + r) + 256 * p));
        if constexpr (std::is_same<S, __nv_bfloat16>::value) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                bh[e] = v[e];   // bfloat16 operands are their own hi part
                bl[e] = 0u;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (f16a) {
                    bh[e] = v[e];
                    bl[e] = 0u;
                } else {
                    const float2 x = __half22float2(*reinterpret_cast<const __half2*>(&v[e]));
                    split_pair(x.x, x.y, bh[e], bl[e]);
                }
            }
        }
        return;
    }
    if (std::is_same<S, __half>::value && f16a) {
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int l = 8 * nt + g;
            // B pairs run along m (stride N in the plane): two raw 16-bit values each
            const unsigned short* xp = reinterpret_cast<const unsigned short*>(xs) + N * N * p;
            auto raw = [&](int ll, int m) -> unsigned { return (ll < N && m < N) ? (unsigned)xp[ll + N * m] : 0u; };
            bh[2 * nt] = raw(l, 2 * t) | (raw(l, 2 * t + 1) << 16);
            bh[2 * nt + 1] = raw(l, 2 * t + 8) | (raw(l, 2 * t + 9) << 16);
            bl[2 * nt] = bl[2 * nt + 1] = 0u;
        }
        return;
    }
    // B fragment of X_p^T for n-tiles nt = 0, 1: column n = l = 8 nt + g,
    // rows k = m = 2t, 2t+1 and 2t+8, 2t+9
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int l = 8 * nt + g;
        split_pair(xval<S, N>(xs, l, 2 * t, p), xval<S, N>(xs, l, 2 * t + 1, p), bh[2 * nt], bl[2 * nt]);
        split_pair(xval<S, N>(xs, l, 2 * t + 8, p), xval<S, N>(xs, l, 2 * t + 9, p), bh[2 * nt + 1],
                   bl[2 * nt + 1]);
    }
}

// XEXACT: the operand is a bfloat16 value (bf16 storage), so its lo part is zero
// and the product with it is skipped.
// f16a: the operand pairs are raw f16 values and the first product runs as f16
// MMAs with the f16 split of M2 (f2h, f2l).
template <bool XEXACT>
__device__ __forceinline__ void tc3_plane_compute(const unsigned (&bh)[4], const unsigned (&bl)[4],
                                                  const unsigned (&m2h)[4], const unsigned (&m2l)[4],
                                                  const unsigned (&m1h)[2][2], const unsigned (&m1l)[2][2],
                                                  float (&z)[2][4], bool f16a, const unsigned (&f2h)[4],
                                                  const unsigned (&f2l)[4]) {
    float w[2][4];
    converge();
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) w[nt][e] = 0.f;
        if (f16a) {
            mma_f16_16816(w[nt], f2l, bh[2 * nt], bh[2 * nt + 1]);
            mma_f16_16816(w[nt], f2h, bh[2 * nt], bh[2 * nt + 1]);
            continue;
        }
        mma_bf16_16816(w[nt], m2l, bh[2 * nt], bh[2 * nt + 1]);
        if constexpr (!XEXACT) mma_bf16_16816(w[nt], m2h, bl[2 * nt], bl[2 * nt + 1]);
        mma_bf16_16816(w[nt], m2h, bh[2 * nt], bh[2 * nt + 1]);
    }
    unsigned wh[4], wl[4];
    split_pair(w[0][0], w[0][1], wh[0], wl[0]);
    split_pair(w[0][2], w[0][3], wh[1], wl[1]);
    split_pair(w[1][0], w[1][1], wh[2], wl[2]);
    split_pair(w[1][2], w[1][3], wh[3], wl[3]);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) z[nt][e] = 0.f;
        mma_bf16_16816(z[nt], wl, m1h[nt][0], m1h[nt][1]);
        mma_bf16_16816(z[nt], wh, m1l[nt][0], m1l[nt][1]);
        mma_bf16_16816(z[nt], wh, m1h[nt][0], m1h[nt][1]);
    }
}

// Planes p and p + 1 at once: the same products in the same order per output as
// two tc3_plane_compute calls, issued step by step across the four (plane,
// n-tile) chains so that the dependent MMAs of one chain are separated by the
// independent ones of the other three.
template <bool XEXACT>
__device__ __forceinline__ void tc3_planes_compute2(const unsigned (&bh0)[4], const unsigned (&bl0)[4],
                                                    const unsigned (&bh1)[4], const unsigned (&bl1)[4],
                                                    const unsigned (&m2h)[4], const unsigned (&m2l)[4],
                                                    const unsigned (&m1h)[2][2], const unsigned (&m1l)[2][2],
                                                    float (&z0)[2][4], float (&z1)[2][4], bool f16a,
                                                    const unsigned (&f2h)[4], const unsigned (&f2l)[4]) {
    float w0[2][4], w1[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) w0[nt][e] = w1[nt][e] = 0.f;
    if (f16a) {   // f16 products plane by plane (step by step measured 2-6x slower with several warps)
        tc3_plane_compute<XEXACT>(bh0, bl0, m2h, m2l, m1h, m1l, z0, f16a, f2h, f2l);
        tc3_plane_compute<XEXACT>(bh1, bl1, m2h, m2l, m1h, m1l, z1, f16a, f2h, f2l);
        return;
    }
    converge();
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        mma_bf16_16816(w0[nt], m2l, bh0[2 * nt], bh0[2 * nt + 1]);
        mma_bf16_16816(w1[nt], m2l, bh1[2 * nt], bh1[2 * nt + 1]);
    }
    if constexpr (!XEXACT) {
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            mma_bf16_16816(w0[nt], m2h, bl0[2 * nt], bl0[2 * nt + 1]);
            mma_bf16_16816(w1[nt], m2h, bl1[2 * nt], bl1[2 * nt + 1]);
        }
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        mma_bf16_16816(w0[nt], m2h, bh0[2 * nt], bh0[2 * nt + 1]);
        mma_bf16_16816(w1[nt], m2h, bh1[2 * nt], bh1[2 * nt + 1]);
    }
    unsigned wh0[4], wl0[4], wh1[4], wl1[4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        split_pair(w0[nt][0], w0[nt][1], wh0[2 * nt], wl0[2 * nt]);
        split_pair(w0[nt][2], w0[nt][3], wh0[2 * nt + 1], wl0[2 * nt + 1]);
        split_pair(w1[nt][0], w1[nt][1], wh1[2 * nt], wl1[2 * nt]);
        split_pair(w1[nt][2], w1[nt][3], wh1[2 * nt + 1], wl1[2 * nt + 1]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) z0[nt][e] = z1[nt][e] = 0.f;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        mma_bf16_16816(z0[nt], wl0, m1h[nt][0], m1h[nt][1]);
        mma_bf16_16816(z1[nt], wl1, m1h[nt][0], m1h[nt][1]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        mma_bf16_16816(z0[nt], wh0, m1l[nt][0], m1l[nt][1]);
        mma_bf16_16816(z1[nt], wh1, m1l[nt][0], m1l[nt][1]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        mma_bf16_16816(z0[nt], wh0, m1h[nt][0], m1h[nt][1]);
        mma_bf16_16816(z1[nt], wh1, m1h[nt][0], m1h[nt][1]);
    }
}

// z[nt] = T^T[j' = g, g+8][i = 8 nt + 2t, +1] of plane p -> row p of T, r = i + 16 j'.
__device__ __forceinline__ void tc3_plane_store(unsigned char* tb, int p, int g, int t, const float (&z)[2][4]) {
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        unsigned h0, l0, h1, l1;
        split_pair(z[nt][0], z[nt][1], h0, l0);
        split_pair(z[nt][2], z[nt][3], h1, l1);
        const uint32_t o0 = trow_off(p, nt + 2 * g) + 4 * t;
        const uint32_t o1 = trow_off(p, nt + 2 * g + 16) + 4 * t;
        *reinterpret_cast<unsigned*>(tb + o0) = h0;
        *reinterpret_cast<unsigned*>(tb + o0 + 512) = l0;
        *reinterpret_cast<unsigned*>(tb + o1) = h1;
        *reinterpret_cast<unsigned*>(tb + o1 + 512) = l1;
    }
}

// Results y of row block mt, n-tile nt: Y[i][mt][k] for i = g, g + 8 and
// k = 8 nt + 2t, +1, with the epilogue.
template <typename S, int N>
__device__ __forceinline__ void tc3_store(const TcArgs3<N>& a, S* yq, int mt, int nt, int g, int t,
                                          const float (&y)[4]) {
    if constexpr (N == 16 && sizeof(S) == 2) {
        if (a.beta_zero && a.ypair) {
            // Pairs of adjacent rows i (lanes g, g ^ 1) as one 32-bit store:
            // the even lane stores column k = 2t, the odd lane k = 2t + 1.
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] = a.alpha_one ? y[e] : a.alpha * y[e];
            const bool odd = g & 1;
            const float s1 = __shfl_xor_sync(0xffffffffu, odd ? v[0] : v[1], 4);
            const float s3 = __shfl_xor_sync(0xffffffffu, odd ? v[2] : v[3], 4);
            const int i0 = g & ~1, k = 8 * nt + 2 * t + (odd ? 1 : 0);
            const f2 lo = odd ? f2_pack(s1, v[1]) : f2_pack(v[0], s1);
            const f2 hi = odd ? f2_pack(s3, v[3]) : f2_pack(v[2], s3);
            *reinterpret_cast<unsigned*>(yq + i0 + N * mt + N * N * k) = pack16<S>(lo);
            *reinterpret_cast<unsigned*>(yq + i0 + 8 + N * mt + N * N * k) = pack16<S>(hi);
            return;
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int i = g + 8 * (e >> 1), k = 8 * nt + 2 * t + (e & 1);
        if (i < N && k < N) {
            S* dst = yq + i + N * mt + N * N * k;
            float v = a.alpha_one ? y[e] : a.alpha * y[e];
            if (!a.beta_zero) v = fmaf(a.beta, load_cvt<float, S>(*dst), v);
            if constexpr (sizeof(S) == 4)
                __stcs(reinterpret_cast<float*>(dst), v);
            else
                *dst = store_cvt<S, float>(v);
        }
    }
}

template <typename S, int N>
__device__ __forceinline__ void tc3_rows(const TcArgs3<N>& a, S* yq, uint32_t tb_s, int mt, int lane,
                                         const unsigned (&m3h)[2][2], const unsigned (&m3l)[2][2]) {
    const int g = lane >> 2, t = lane & 3, mi = lane >> 3, rr = lane & 7;
    unsigned ah[4], al[4];
    const uint32_t to = trow_off(rr + 8 * (mi >> 1), 2 * mt + (mi & 1));
    converge();
    ldsm_x4_trans(ah, tb_s + to);
    ldsm_x4_trans(al, tb_s + to + 512);
    float y[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
        for (int e = 0; e < 4; ++e) y[nt][e] = 0.f;
        mma_bf16_16816(y[nt], al, m3h[nt][0], m3h[nt][1]);
        mma_bf16_16816(y[nt], ah, m3l[nt][0], m3l[nt][1]);
        mma_bf16_16816(y[nt], ah, m3h[nt][0], m3h[nt][1]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) tc3_store<S, N>(a, yq, mt, nt, g, t, y[nt]);
}

// Row blocks mt and mt + 1 at once, step by step across the four (row block,
// n-tile) chains (the same products in the same order per output).
template <typename S, int N>
__device__ __forceinline__ void tc3_rows2(const TcArgs3<N>& a, S* yq, uint32_t tb_s, int mt, int lane,
                                          const unsigned (&m3h)[2][2], const unsigned (&m3l)[2][2]) {
    const int g = lane >> 2, t = lane & 3, mi = lane >> 3, rr = lane & 7;
    unsigned ah0[4], al0[4], ah1[4], al1[4];
    const uint32_t to0 = trow_off(rr + 8 * (mi >> 1), 2 * mt + (mi & 1));
    const uint32_t to1 = trow_off(rr + 8 * (mi >> 1), 2 * (mt + 1) + (mi & 1));
    converge();
    ldsm_x4_trans(ah0, tb_s + to0);
    ldsm_x4_trans(al0, tb_s + to0 + 512);
    ldsm_x4_trans(ah1, tb_s + to1);
    ldsm_x4_trans(al1, tb_s + to1 + 512);
    float y0[2][4], y1[2][4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) y0[nt][e] = y1[nt][e] = 0.f;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        mma_bf16_16816(y0[nt], al0, m3h[nt][0], m3h[nt][1]);
        mma_bf16_16816(y1[nt], al1, m3h[nt][0], m3h[nt][1]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        mma_bf16_16816(y0[nt], ah0, m3l[nt][0], m3l[nt][1]);
        mma_bf16_16816(y1[nt], ah1, m3l[nt][0], m3l[nt][1]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        mma_bf16_16816(y0[nt], ah0, m3h[nt][0], m3h[nt][1]);
        mma_bf16_16816(y1[nt], ah1, m3h[nt][0], m3h[nt][1]);
    }
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) tc3_store<S, N>(a, yq, mt, nt, g, t, y0[nt]);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) tc3_store<S, N>(a, yq, mt + 1, nt, g, t, y1[nt]);
}

template <typename S, int N>
__global__ void __launch_bounds__(32 * kTc3Warps) tc3_kernel(const __grid_constant__ TcArgs3<N> a) {
    using L = Tc3Layout<S, N>;
    constexpr int NX = N * N * N;
    constexpr unsigned NXB = NX * (unsigned)sizeof(S);
    constexpr bool XEXACT = std::is_same<S, __nv_bfloat16>::value;
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem) + warp;
    unsigned char* wb = smem + 128 + (size_t)warp * L::PER_WARP;
    S* xs = reinterpret_cast<S*>(wb);                       // the instance (planes of N^2 values)
    unsigned char* tb = L::INPLACE ? wb : wb + L::XB;        // T rows, 1 KB each
    const uint32_t tb_s = smem_u32(tb);

    // Constant fragments.  A of M2 (rows j', columns m); B of M1^T and M3^T:
    // column n of M^T is row n of M, pairs along the row.
    unsigned m2h[4], m2l[4], m1h[2][2], m1l[2][2], m3h[2][2], m3l[2][2];
    const bool f16a = std::is_same<S, __half>::value && a.f16a;
    unsigned f2h[4] = {0u, 0u, 0u, 0u}, f2l[4] = {0u, 0u, 0u, 0u};
    if (f16a) {
        f2h[0] = a.f2h[g * 8 + t];           f2l[0] = a.f2l[g * 8 + t];
        f2h[1] = a.f2h[(g + 8) * 8 + t];     f2l[1] = a.f2l[(g + 8) * 8 + t];
        f2h[2] = a.f2h[g * 8 + t + 4];       f2l[2] = a.f2l[g * 8 + t + 4];
        f2h[3] = a.f2h[(g + 8) * 8 + t + 4]; f2l[3] = a.f2l[(g + 8) * 8 + t + 4];
    }
    m2h[0] = a.m2h[g * 8 + t];           m2l[0] = a.m2l[g * 8 + t];
    m2h[1] = a.m2h[(g + 8) * 8 + t];     m2l[1] = a.m2l[(g + 8) * 8 + t];
    m2h[2] = a.m2h[g * 8 + t + 4];       m2l[2] = a.m2l[g * 8 + t + 4];
    m2h[3] = a.m2h[(g + 8) * 8 + t + 4]; m2l[3] = a.m2l[(g + 8) * 8 + t + 4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int n = 8 * nt + g;
        m1h[nt][0] = a.m1h[n * 8 + t];     m1l[nt][0] = a.m1l[n * 8 + t];
        m1h[nt][1] = a.m1h[n * 8 + t + 4]; m1l[nt][1] = a.m1l[n * 8 + t + 4];
        m3h[nt][0] = a.m3h[n * 8 + t];     m3l[nt][0] = a.m3l[n * 8 + t];
        m3h[nt][1] = a.m3h[n * 8 + t + 4]; m3l[nt][1] = a.m3l[n * 8 + t + 4];
    }
    if constexpr (!L::INPLACE) {
        // rows p >= N of T stay zero for the whole kernel
        for (int e = lane; e < (16 - N) * 256; e += 32)
            reinterpret_cast<unsigned*>(tb + N * 1024)[e] = 0u;
    }

    const int64_t nwarps = (int64_t)gridDim.x * kTc3Warps;
    int64_t inst = (int64_t)blockIdx.x * kTc3Warps + warp;
    uint64_t pol = 0;
    // Instance q: its 16-byte-aligned span is copied, the instance starts `phase(q)`
    // elements into the buffer (0 whenever n^3 elements are whole 16-byte units).
    auto phase = [&](int64_t q) -> int {
        if constexpr (L::ALIGNED) return 0;
        else return (int)(((uintptr_t)(static_cast<const S*>(a.X) + q * NX) & 15u) / sizeof(S));
    };
    auto fetch = [&](int64_t q) {
        const int ph = phase(q);
        const unsigned bytes = (unsigned)(ph * sizeof(S) + NXB + 15u) & ~15u;
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(xs, static_cast<const S*>(a.X) + q * NX - ph, bytes, bar, pol);
    };
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
        pol = l2_evict_first_policy();
        if (inst < a.batch) fetch(inst);
    }
    __syncwarp();
    unsigned bphase = 0;
    for (; inst < a.batch; inst += nwarps, bphase ^= 1u) {
        if (!mbar_wait_bounded(bar, bphase, a.err)) return;   // nothing else in flight
        const S* xq = xs + phase(inst);

        // ---- modes 1 and 2, two planes per step ------------------------------------------
#pragma unroll 1
        for (int p = 0; p < N; p += 2) {
            const bool two = p + 1 < N;
            unsigned bh0[4], bl0[4], bh1[4], bl1[4];
            tc3_plane_load<S, N>(xq, p, g, t, bh0, bl0, f16a);
            if (two) tc3_plane_load<S, N>(xq, p + 1, g, t, bh1, bl1, f16a);
            float z0[2][4], z1[2][4];
            if constexpr (N % 2 == 0) {   // planes come in pairs: both at once
                tc3_planes_compute2<XEXACT>(bh0, bl0, bh1, bl1, m2h, m2l, m1h, m1l, z0, z1, f16a, f2h, f2l);
            } else {
                tc3_plane_compute<XEXACT>(bh0, bl0, m2h, m2l, m1h, m1l, z0, f16a, f2h, f2l);
                if (two) tc3_plane_compute<XEXACT>(bh1, bl1, m2h, m2l, m1h, m1l, z1, f16a, f2h, f2l);
            }
            __syncwarp();   // planes p, p+1 are read by every lane before they are overwritten
            tc3_plane_store(tb, p, g, t, z0);
            if (two) tc3_plane_store(tb, p + 1, g, t, z1);
        }
        __syncwarp();
        auto fetch_next = [&]() {
            if (lane == 0) {
                const int64_t next = inst + nwarps;
                if (next < a.batch) {
                    fence_proxy_async_smem();
                    fetch(next);
                }
            }
        };
        if constexpr (!L::INPLACE) fetch_next();   // the operand planes are no longer read

        // ---- mode 3, two row blocks per step ---------------------------------------------
        S* yq = static_cast<S*>(a.Y) + inst * NX;
#pragma unroll 1
        for (int mt = 0; mt < N; mt += 2) {
            if constexpr (N % 2 == 0) {   // row blocks come in pairs: both at once
                tc3_rows2<S, N>(a, yq, tb_s, mt, lane, m3h, m3l);
            } else {
                tc3_rows<S, N>(a, yq, tb_s, mt, lane, m3h, m3l);
                if (mt + 1 < N) tc3_rows<S, N>(a, yq, tb_s, mt + 1, lane, m3h, m3l);
            }
        }
        __syncwarp();   // T is free (in place: so are the operand planes)
        if constexpr (L::INPLACE) fetch_next();
    }
}

// 3-D, several warps per instance (tc3g_kernel): the CTA's W warps share one
// instance -- modes 1 and 2 split by plane pairs, mode 3 by row-block pairs,
// a CTA barrier between the two -- and the operand buffer is doubled, so the
// next instance lands while this one is contracted.  Per CTA: two operand
// buffers and (except FP32 n = 16, where T overwrites the operand planes) one
// T buffer: 32 KB at n = 16 against 16-24 KB per single-warp CTA, for 4-8
// times the warps per instance.
template <typename S, int N>
__global__ void __launch_bounds__(256) tc3g_kernel(const __grid_constant__ TcArgs3<N> a) {
    using L = Tc3Layout<S, N>;
    constexpr int NX = N * N * N;
    constexpr unsigned NXB = NX * (unsigned)sizeof(S);
    constexpr bool XEXACT = std::is_same<S, __nv_bfloat16>::value;
    extern __shared__ __align__(128) unsigned char smem[];
    const int W = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);   // one barrier per operand buffer
    unsigned char* xbuf = smem + 128;                     // operand buffers, L::XB bytes each
    unsigned char* tsep = xbuf + 2 * L::XB;               // T, unless in place

    unsigned m2h[4], m2l[4], m1h[2][2], m1l[2][2], m3h[2][2], m3l[2][2];
    const bool f16a = std::is_same<S, __half>::value && a.f16a;
    unsigned f2h[4] = {0u, 0u, 0u, 0u}, f2l[4] = {0u, 0u, 0u, 0u};
    if (f16a) {
        f2h[0] = a.f2h[g * 8 + t];           f2l[0] = a.f2l[g * 8 + t];
        f2h[1] = a.f2h[(g + 8) * 8 + t];     f2l[1] = a.f2l[(g + 8) * 8 + t];
        f2h[2] = a.f2h[g * 8 + t + 4];       f2l[2] = a.f2l[g * 8 + t + 4];
        f2h[3] = a.f2h[(g + 8) * 8 + t + 4]; f2l[3] = a.f2l[(g + 8) * 8 + t + 4];
    }
    m2h[0] = a.m2h[g * 8 + t];           m2l[0] = a.m2l[g * 8 + t];
    m2h[1] = a.m2h[(g + 8) * 8 + t];     m2l[1] = a.m2l[(g + 8) * 8 + t];
    m2h[2] = a.m2h[g * 8 + t + 4];       m2l[2] = a.m2l[g * 8 + t + 4];
    m2h[3] = a.m2h[(g + 8) * 8 + t + 4]; m2l[3] = a.m2l[(g + 8) * 8 + t + 4];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int n = 8 * nt + g;
        m1h[nt][0] = a.m1h[n * 8 + t];     m1l[nt][0] = a.m1l[n * 8 + t];
        m1h[nt][1] = a.m1h[n * 8 + t + 4]; m1l[nt][1] = a.m1l[n * 8 + t + 4];
        m3h[nt][0] = a.m3h[n * 8 + t];     m3l[nt][0] = a.m3l[n * 8 + t];
        m3h[nt][1] = a.m3h[n * 8 + t + 4]; m3l[nt][1] = a.m3l[n * 8 + t + 4];
    }
    if constexpr (!L::INPLACE) {
        for (int e = threadIdx.x; e < (16 - N) * 256; e += blockDim.x)
            reinterpret_cast<unsigned*>(tsep + N * 1024)[e] = 0u;
    }

    const int64_t G = gridDim.x;
    int64_t inst = blockIdx.x;
    uint64_t pol = 0;
    auto phase = [&](int64_t q) -> int {
        if constexpr (L::ALIGNED) return 0;
        else return (int)(((uintptr_t)(static_cast<const S*>(a.X) + q * NX) & 15u) / sizeof(S));
    };
    auto fetch = [&](int b, int64_t q) {
        const int ph = phase(q);
        const unsigned bytes = (unsigned)(ph * sizeof(S) + NXB + 15u) & ~15u;
        mbar_arrive_expect_tx(&full[b], bytes);
        bulk_g2s(xbuf + b * L::XB, static_cast<const S*>(a.X) + q * NX - ph, bytes, &full[b], pol);
    };
    if (threadIdx.x == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_barrier_init();
        pol = l2_evict_first_policy();
        if (inst < a.batch) fetch(0, inst);
        if (inst + G < a.batch) fetch(1, inst + G);
    }
    __syncthreads();
    for (int it = 0; inst < a.batch; inst += G, ++it) {
        const int b = it & 1;
        const bool ok = mbar_wait_bounded(&full[b], (unsigned)(it >> 1) & 1u, a.err);
        if (__syncthreads_or(!ok)) {
            // wait (bounded) for the copies that may still be in flight, then give up
            if (threadIdx.x == 0) {
                mbar_wait_bounded(&full[b], (unsigned)(it >> 1) & 1u, a.err);
                if (inst + G < a.batch) mbar_wait_bounded(&full[b ^ 1], (unsigned)((it + 1) >> 1) & 1u, a.err);
            }
            return;
        }
        const S* xq = reinterpret_cast<const S*>(xbuf + b * L::XB) + phase(inst);
        unsigned char* tb = L::INPLACE ? xbuf + b * L::XB : tsep;
        const uint32_t tb_s = smem_u32(tb);

        // ---- modes 1 and 2: plane pairs 2w, 2w + 2W, ... ---------------------------------
#pragma unroll 2
        for (int p = 2 * warp; p < N; p += 2 * W) {
            const bool two = p + 1 < N;
            unsigned bh0[4], bl0[4], bh1[4], bl1[4];
            tc3_plane_load<S, N>(xq, p, g, t, bh0, bl0, f16a);
            if (two) tc3_plane_load<S, N>(xq, p + 1, g, t, bh1, bl1, f16a);
            float z0[2][4], z1[2][4];
            if constexpr (N % 2 == 0) {   // planes come in pairs: both at once
                tc3_planes_compute2<XEXACT>(bh0, bl0, bh1, bl1, m2h, m2l, m1h, m1l, z0, z1, f16a, f2h, f2l);
            } else {
                tc3_plane_compute<XEXACT>(bh0, bl0, m2h, m2l, m1h, m1l, z0, f16a, f2h, f2l);
                if (two) tc3_plane_compute<XEXACT>(bh1, bl1, m2h, m2l, m1h, m1l, z1, f16a, f2h, f2l);
            }
            __syncwarp();   // planes p, p+1 are read by every lane before they are overwritten
            tc3_plane_store(tb, p, g, t, z0);
            if (two) tc3_plane_store(tb, p + 1, g, t, z1);
        }
        fence_proxy_async_smem();   // this thread's reads of the operand buffer precede a refill
        __syncthreads();            // T complete
        if (!L::INPLACE && threadIdx.x == 0 && inst + 2 * G < a.batch) fetch(b, inst + 2 * G);

        // ---- mode 3: row-block pairs 2w, 2w + 2W, ... -------------------------------------
        S* yq = static_cast<S*>(a.Y) + inst * NX;
#pragma unroll 2
        for (int mt = 2 * warp; mt < N; mt += 2 * W) {
            if constexpr (N % 2 == 0) {   // row blocks come in pairs: both at once
                tc3_rows2<S, N>(a, yq, tb_s, mt, lane, m3h, m3l);
            } else {
                tc3_rows<S, N>(a, yq, tb_s, mt, lane, m3h, m3l);
                if (mt + 1 < N) tc3_rows<S, N>(a, yq, tb_s, mt + 1, lane, m3h, m3l);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();            // T free (in place: so is the operand buffer)
        if (L::INPLACE && threadIdx.x == 0 && inst + 2 * G < a.batch) fetch(b, inst + 2 * G);
    }
}

// ---------------------------------------------------------------------------
// 2-D, 9 <= n <= 16: instances stacked along the MMA's N dimension (tc2s_kernel).
//
// The padded tile spends 16^3 of MMA work per product on an instance's n^3.
// Stacking G = 8 / gcd(n, 8) instances side by side makes G n a whole number of
// 8-wide n-tiles, so only the contracted dimension and the component's rows
// stay padded to 16 (bf16 storage at n = 12: 7.5 MMAs per instance instead of
// 10; n = 10: 6.25).
//   stage 1  W = M1 [X_1 ... X_G]   A = M1 (constant), B = the instances'
//            columns side by side: n-tile column 8 nt + g = q n + c is column c
//            of instance q.  W is split and written to the warp's exchange
//            buffer, row rho = q n + r holding W_q[r][0 .. n-1] (hi, then lo).
//   stage 2  Y_q^T = M2 W_q^T       A = M2 (constant), B = exchange rows read by
//            ldmatrix, stacked along N as rho.  Accumulator lane (g, t) holds
//            Y_q[r][j] and Y_q[r + 1][j] (rho = 8 nt + 2 t, j = g and g + 8):
//            adjacent in column-major Y, one paired store for even n.
// The exchange rows' columns n .. 15 stay zero (the padding of the stage-2
// contraction).  Rows are 80 bytes apart, so the eight rows of one ldmatrix
// matrix fall in eight distinct 16-byte bank groups.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int tc2s_group(int n) {
    return n % 8 == 0 ? 1 : (n % 4 == 0 ? 2 : (n % 2 == 0 ? 4 : 8));
}
constexpr int kTc2sRow = 80;   // exchange row: 16 hi + 16 lo 16-bit values, 16 bytes of padding

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr)
                 : "memory");
}

// A fragment (m16k16, row-major) of a 16 x 16 component stored as packed pairs.
__device__ __forceinline__ void a_frag(const unsigned* m, int g, int t, unsigned (&f)[4]) {
    f[0] = m[g * 8 + t];
    f[1] = m[(g + 8) * 8 + t];
    f[2] = m[g * 8 + t + 4];
    f[3] = m[(g + 8) * 8 + t + 4];
}

// W[r][cc], W[r][cc + 1] (stacked columns) into the exchange rows, split.
template <int N>
__device__ __forceinline__ void tc2s_put(unsigned char* ex, int cc, int r, float v0, float v1) {
    unsigned hi, lo;
    split_pair(v0, v1, hi, lo);
    const int q0 = cc / N, c0 = cc - q0 * N;
    unsigned char* p0 = ex + (q0 * N + r) * kTc2sRow + 2 * c0;
    if constexpr (N % 2 == 0) {   // c0 even: both columns in one instance, 4-byte aligned
        *reinterpret_cast<unsigned*>(p0) = hi;
        *reinterpret_cast<unsigned*>(p0 + 32) = lo;
    } else {                      // the second column may open the next instance
        const int q1 = (cc + 1) / N, c1 = cc + 1 - q1 * N;
        unsigned char* p1 = ex + (q1 * N + r) * kTc2sRow + 2 * c1;
        *reinterpret_cast<unsigned short*>(p0) = (unsigned short)hi;
        *reinterpret_cast<unsigned short*>(p0 + 32) = (unsigned short)lo;
        *reinterpret_cast<unsigned short*>(p1) = (unsigned short)(hi >> 16);
        *reinterpret_cast<unsigned short*>(p1 + 32) = (unsigned short)(lo >> 16);
    }
}

// One result element Y_q[r][j] (stacked row rho = q n + r) with the epilogue.
template <typename S, int N>
__device__ __forceinline__ void tc2s_out1(const TcArgs2<N>& a, S* yg, int live, int rho, int j, float v) {
    const int q = rho / N, r = rho - q * N;
    if (q >= live) return;
    S* dst = yg + q * N * N + r + N * j;
    if (!a.alpha_one) v *= a.alpha;
    if (!a.beta_zero) v = fmaf(a.beta, load_cvt<float, S>(*dst), v);
    if constexpr (sizeof(S) == 4)
        __stcs(reinterpret_cast<float*>(dst), v);
    else
        *dst = store_cvt<S, float>(v);
}

// Y_q[r][j], Y_q[r + 1][j] (rho = q n + r even).
template <typename S, int N>
__device__ __forceinline__ void tc2s_out(const TcArgs2<N>& a, S* yg, int live, int rho, int j, float v0, float v1) {
    if constexpr (N % 2 == 0) {
        const int q = rho / N, r = rho - q * N;
        if (q >= live) return;
        S* dst = yg + q * N * N + r + N * j;
        if (a.ypair) {
            if (!a.alpha_one) {
                v0 *= a.alpha;
                v1 *= a.alpha;
            }
            if (!a.beta_zero) {
                v0 = fmaf(a.beta, load_cvt<float, S>(dst[0]), v0);
                v1 = fmaf(a.beta, load_cvt<float, S>(dst[1]), v1);
            }
            if constexpr (sizeof(S) == 4)
                __stcs(reinterpret_cast<float2*>(dst), make_float2(v0, v1));
            else
                __stcs(reinterpret_cast<unsigned*>(dst), pack16<S>(f2_pack(v0, v1)));
            return;
        }
    }
    tc2s_out1<S, N>(a, yg, live, rho, j, v0);
    tc2s_out1<S, N>(a, yg, live, rho + 1, j, v1);
}

// Constant A fragments of the stacked body: M1 (stage 1; f16 storage: M1 2^s as
// an f16 split) and M2 (stage 2).
struct Tc2sFrags {
    unsigned m1h[4], m1l[4], f1h[4], f1l[4], m2h[4], m2l[4];
};

// One group of G instances, any n, any epilogue, any number of live instances.
template <typename S, int N>
__device__ __forceinline__ void tc2s_group_any(const TcArgs2<N>& a, const Tc2sFrags& f, const S* xg, S* yg, int live,
                                               unsigned char* ex, uint32_t ex_s) {
    constexpr int NX = N * N, G = tc2s_group(N), NT = G * N / 8;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // ---- stage 1: W = M1 [X_1 ... X_G] ---------------------------------------------------
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const int col = 8 * nt + g, q = col / N, c = col - q * N;
        const bool lq = q < live;
        const S* xq = xg + q * NX;
        float w[4] = {0.f, 0.f, 0.f, 0.f};
        if constexpr (std::is_same<S, __nv_bfloat16>::value) {
            const unsigned b0 = lq ? x_pair_bf16<N>(xq, 2 * t, c) : 0u;
            const unsigned b1 = lq ? x_pair_bf16<N>(xq, 2 * t + 8, c) : 0u;
            converge();
            mma_bf16_16816(w, f.m1l, b0, b1);
            mma_bf16_16816(w, f.m1h, b0, b1);
        } else if (std::is_same<S, __half>::value && a.f16a) {
            const unsigned b0 = lq ? x_pair_bf16<N>(xq, 2 * t, c) : 0u;
            const unsigned b1 = lq ? x_pair_bf16<N>(xq, 2 * t + 8, c) : 0u;
            converge();
            mma_f16_16816(w, f.f1l, b0, b1);
            mma_f16_16816(w, f.f1h, b0, b1);
        } else {
            float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
            if (lq) {
                x_pair<S, N>(xq, 2 * t, c, x0, x1);
                x_pair<S, N>(xq, 2 * t + 8, c, x2, x3);
            }
            unsigned bh0, bl0, bh1, bl1;
            split_pair(x0, x1, bh0, bl0);
            split_pair(x2, x3, bh1, bl1);
            converge();
            mma_bf16_16816(w, f.m1l, bh0, bh1);
            mma_bf16_16816(w, f.m1h, bl0, bl1);
            mma_bf16_16816(w, f.m1h, bh0, bh1);
        }
        // lane holds W[g][cc], W[g][cc + 1], W[g + 8][cc], W[g + 8][cc + 1]
        const int cc = 8 * nt + 2 * t;
        tc2s_put<N>(ex, cc, g, w[0], w[1]);
        if (g + 8 < N) tc2s_put<N>(ex, cc, g + 8, w[2], w[3]);
    }
    __syncwarp();
    // ---- stage 2: Y_q^T = M2 W_q^T, stacked --------------------------------------------------
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        unsigned b[4];   // hi (k 0-7, k 8-15), lo (k 0-7, k 8-15)
        converge();
        ldsm_x4(b, ex_s + (8 * nt + (lane & 7)) * kTc2sRow + (lane >> 3) * 16);
        float y[4] = {0.f, 0.f, 0.f, 0.f};   // products in the padded body's order
        mma_bf16_16816(y, f.m2h, b[2], b[3]);
        mma_bf16_16816(y, f.m2l, b[0], b[1]);
        mma_bf16_16816(y, f.m2h, b[0], b[1]);
        const int rho = 8 * nt + 2 * t;
        tc2s_out<S, N>(a, yg, live, rho, g, y[0], y[1]);
        if (g + 8 < N) tc2s_out<S, N>(a, yg, live, rho, g + 8, y[2], y[3]);
    }
    __syncwarp();
}

// The lane's offsets in the fast path (even n): per n-tile, the element offset of
// its X pair (column c of instance q, rows 2t, 2t + 1), the byte offset of its
// exchange store (row q n + g, columns 2t, 2t + 1 of the stacked W), the element
// offset of its Y pair (rows r, r + 1 of instance q', column g), and q' (the
// instance its stores belong to, for the last, partial group).
template <int N>
struct Tc2sLane {
    static constexpr int NT = tc2s_group(N) * N / 8;
    int xo[NT], eo[NT], yo[NT], qy[NT];
};

template <int N>
__device__ __forceinline__ void tc2s_lane_init(Tc2sLane<N>& L, int g, int t) {
#pragma unroll
    for (int nt = 0; nt < Tc2sLane<N>::NT; ++nt) {
        const int col = 8 * nt + g, q = col / N, c = col - q * N;
        L.xo[nt] = q * N * N + N * c + 2 * t;
        const int rho = 8 * nt + 2 * t, q2 = rho / N, r = rho - q2 * N;
        L.eo[nt] = (q2 * N + g) * kTc2sRow + 2 * r;
        L.yo[nt] = q2 * N * N + r + N * g;
        L.qy[nt] = q2;
    }
}

// K consecutive groups of an even n with the plain epilogue (alpha = 1, beta = 0,
// Y aligned to pairs): offsets from the lane's table (group k adds k G instances
// and k G n exchange rows), and the MMAs issued step by step across the K NT
// (group, n-tile) chains (every chain's first product, then every second, ...), so
// that the dependent products of one chain are separated by the independent ones
// of the others.  In the last, partial groups the operand slots of absent
// instances (q >= live) are read as they are -- stale values of the ring or the
// exchange rows after it, inside the CTA's shared memory (at most K G - 1
// instances past a tile) -- and only their stores are skipped: every column of W
// and every stacked row of the result depends on its own instance alone.
template <typename S, int N, int K>
__device__ __forceinline__ void tc2s_group_fast(const Tc2sFrags& f, const Tc2sLane<N>& L, const S* xg, S* yg,
                                                int live, unsigned char* ex, uint32_t ex_s) {
    constexpr int NT = Tc2sLane<N>::NT, CH = K * NT, G = tc2s_group(N);
    constexpr int XG = G * N * N, EG = G * N * kTc2sRow;   // per group: operand elements, exchange bytes
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const bool k8 = 2 * t + 8 < N;   // the lane's rows 2t + 8, 2t + 9 exist
    const bool r8 = g + 8 < N;       // the lane's W row / Y column g + 8 exists
    // ---- stage 1 ----------------------------------------------------------------------------
    float w[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) w[c][e] = 0.f;
    if constexpr (sizeof(S) == 2) {
        unsigned b0[CH], b1[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const unsigned* xp = reinterpret_cast<const unsigned*>(xg + (c / NT) * XG + L.xo[c % NT]);
            b0[c] = xp[0];
            b1[c] = k8 ? xp[4] : 0u;
        }
        if constexpr (std::is_same<S, __half>::value) {
#pragma unroll
            for (int c = 0; c < CH; ++c) mma_f16_16816(w[c], f.f1l, b0[c], b1[c]);
#pragma unroll
            for (int c = 0; c < CH; ++c) mma_f16_16816(w[c], f.f1h, b0[c], b1[c]);
        } else {
#pragma unroll
            for (int c = 0; c < CH; ++c) mma_bf16_16816(w[c], f.m1l, b0[c], b1[c]);
#pragma unroll
            for (int c = 0; c < CH; ++c) mma_bf16_16816(w[c], f.m1h, b0[c], b1[c]);
        }
    } else {
        unsigned bh0[CH], bl0[CH], bh1[CH], bl1[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const S* xp = xg + (c / NT) * XG + L.xo[c % NT];
            const float2 p0 = *reinterpret_cast<const float2*>(xp);
            const float2 p1 = k8 ? *reinterpret_cast<const float2*>(xp + 8) : make_float2(0.f, 0.f);
            split_pair(p0.x, p0.y, bh0[c], bl0[c]);
            split_pair(p1.x, p1.y, bh1[c], bl1[c]);
        }
#pragma unroll
        for (int c = 0; c < CH; ++c) mma_bf16_16816(w[c], f.m1l, bh0[c], bh1[c]);
#pragma unroll
        for (int c = 0; c < CH; ++c) mma_bf16_16816(w[c], f.m1h, bl0[c], bl1[c]);
#pragma unroll
        for (int c = 0; c < CH; ++c) mma_bf16_16816(w[c], f.m1h, bh0[c], bh1[c]);
    }
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        unsigned char* e0 = ex + (c / NT) * EG + L.eo[c % NT];
        unsigned hi, lo;
        split_pair(w[c][0], w[c][1], hi, lo);
        *reinterpret_cast<unsigned*>(e0) = hi;
        *reinterpret_cast<unsigned*>(e0 + 32) = lo;
        if (r8) {
            split_pair(w[c][2], w[c][3], hi, lo);
            *reinterpret_cast<unsigned*>(e0 + 8 * kTc2sRow) = hi;
            *reinterpret_cast<unsigned*>(e0 + 8 * kTc2sRow + 32) = lo;
        }
    }
    __syncwarp();
    // ---- stage 2 ----------------------------------------------------------------------------
    const uint32_t lrow = ex_s + (lane & 7) * kTc2sRow + (lane >> 3) * 16;
    unsigned b[CH][4];
    float y[CH][4];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        ldsm_x4(b[c], lrow + (c / NT) * EG + (c % NT) * 8 * kTc2sRow);
#pragma unroll
        for (int e = 0; e < 4; ++e) y[c][e] = 0.f;
    }
    __syncwarp();   // exchange rows read: the next groups may overwrite them
#pragma unroll
    for (int c = 0; c < CH; ++c) mma_bf16_16816(y[c], f.m2h, b[c][2], b[c][3]);
#pragma unroll
    for (int c = 0; c < CH; ++c) mma_bf16_16816(y[c], f.m2l, b[c][0], b[c][1]);
#pragma unroll
    for (int c = 0; c < CH; ++c) mma_bf16_16816(y[c], f.m2h, b[c][0], b[c][1]);
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        if ((c / NT) * G + L.qy[c % NT] >= live) continue;
        S* dst = yg + (c / NT) * XG + L.yo[c % NT];
        if constexpr (sizeof(S) == 4) {
            __stcs(reinterpret_cast<float2*>(dst), make_float2(y[c][0], y[c][1]));
            if (r8) __stcs(reinterpret_cast<float2*>(dst + 8 * N), make_float2(y[c][2], y[c][3]));
        } else {
            __stcs(reinterpret_cast<unsigned*>(dst), pack16<S>(f2_pack(y[c][0], y[c][1])));
            if (r8) __stcs(reinterpret_cast<unsigned*>(dst + 8 * N), pack16<S>(f2_pack(y[c][2], y[c][3])));
        }
    }
}

// FAST: every K groups by tc2s_group_fast (even n, plain epilogue, the stored
// operand entering the MMAs as it is or split from FP32); else every group by
// tc2s_group_any.  The two bodies are separate kernels: one kernel never chooses
// between them at run time.
template <typename S, int N, bool FAST, int K>
__global__ void __launch_bounds__(kTcThreads) tc2s_kernel(const __grid_constant__ TcArgs2<N> a) {
    constexpr int NX = N * N, G = tc2s_group(N);
    static_assert(N >= 9 && N <= 16 && (G * N) % 8 == 0, "stacked body: 9 <= n <= 16");
    static_assert(!FAST || N % 2 == 0, "the fast body takes even n");
    static_assert(K == 1 || (FAST && K == 2), "two groups per step in the fast body only");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    const int P = a.P;
    const size_t xstage = round_up((size_t)P * NX * sizeof(S), 128);
    unsigned char* xbase = smem + 128;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int64_t ntiles = (a.batch + P - 1) / P;
    const int64_t grid = gridDim.x;
    unsigned char* ex = xbase + a.nstage * xstage + warp * (K * G * N * kTc2sRow);
    const uint32_t ex_s = (uint32_t)__cvta_generic_to_shared(ex);
    for (int e = lane; e < K * G * N * kTc2sRow / 4; e += 32) reinterpret_cast<unsigned*>(ex)[e] = 0u;

    Tc2sFrags f;
    for (int e = 0; e < 4; ++e) f.f1h[e] = f.f1l[e] = 0u;
    if (std::is_same<S, __half>::value && a.f16a) {
        a_frag(a.f1h, g, t, f.f1h);
        a_frag(a.f1l, g, t, f.f1l);
    }
    a_frag(a.m1h, g, t, f.m1h);
    a_frag(a.m1l, g, t, f.m1l);
    a_frag(a.m2h, g, t, f.m2h);
    a_frag(a.m2l, g, t, f.m2l);
    Tc2sLane<N> L;
    if constexpr (FAST) tc2s_lane_init<N>(L, g, t);

    uint64_t pol = 0;
    if (tid == 0) {
        for (int s = 0; s < a.nstage; ++s) mbar_init(&bars[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
        pol = l2_evict_first_policy();
        for (int s = 0; s < a.nstage; ++s) {
            const int64_t tl = blockIdx.x + s * grid;
            if (tl < ntiles) {
                const int64_t i0 = tl * P;
                const int cnt = (int)min((int64_t)P, a.batch - i0);
                const unsigned bytes = ((unsigned)cnt * NX * (unsigned)sizeof(S)) & ~15u;
                mbar_arrive_expect_tx(&bars[s], bytes);
                if (bytes) bulk_g2s(xbase + s * xstage, static_cast<const S*>(a.X) + i0 * NX, bytes, &bars[s], pol);
            }
        }
    }
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
        const int s = it % a.nstage;
        S* xt = reinterpret_cast<S*>(xbase + s * xstage);
        const int64_t inst0 = tile * P;
        const int cnt = (int)min((int64_t)P, a.batch - inst0);
        bool ok = mbar_wait_bounded(&bars[s], (unsigned)(it / a.nstage) & 1u, a.err);
        const unsigned bytes = (unsigned)cnt * NX * (unsigned)sizeof(S);
        const unsigned b16 = bytes & ~15u;
        if (bytes != b16) {
            const S* src = static_cast<const S*>(a.X) + inst0 * NX;
            for (int e = b16 / sizeof(S) + tid; e < cnt * NX; e += kTcThreads) xt[e] = src[e];
            __syncthreads();
        }
        if (ok) {
            for (int q0 = warp * G * K; q0 < cnt; q0 += G * K * (kTcThreads / 32)) {
                const S* xg = xt + q0 * NX;
                S* yg = static_cast<S*>(a.Y) + (inst0 + q0) * NX;
                const int live = cnt - q0;   // instances q < live of this group exist
                if constexpr (FAST)
                    tc2s_group_fast<S, N, K>(f, L, xg, yg, live, ex, ex_s);
                else
                    tc2s_group_any<S, N>(a, f, xg, yg, live, ex, ex_s);
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                for (int j = it; j < it + a.nstage; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&bars[j % a.nstage], (unsigned)(j / a.nstage) & 1u, a.err);
            }
            return;
        }
        if (tid == 0) {
            const int64_t next = tile + a.nstage * grid;
            if (next < ntiles) {
                const int64_t i0 = next * P;
                const int c2 = (int)min((int64_t)P, a.batch - i0);
                const unsigned nb = ((unsigned)c2 * NX * (unsigned)sizeof(S)) & ~15u;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&bars[s], nb);
                if (nb) bulk_g2s(xt, static_cast<const S*>(a.X) + i0 * NX, nb, &bars[s], pol);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// float -> bfloat16 bits, round to nearest even (NaN kept quiet).
static inline unsigned short bf16_rne(float f) {
    unsigned u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x7fffffu)) return (unsigned short)((u >> 16) | 0x40);
    const unsigned lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    return (unsigned short)(u >> 16);
}
static inline float bf16_to_float(unsigned short h) {
    const unsigned u = (unsigned)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// Column-major N x N (double) -> row-major 16 x 16 packed bf16 pairs, split hi/lo.
// Row-major 16 x 16 split of blockdiag(M, ..., M) with B x B blocks (B = 16:
// M itself, zero-padded).
static inline void split_rowmajor(const double* m, int N, unsigned* hi, unsigned* lo, int B = 16, double scale = 1.0) {
    for (int r = 0; r < 16; ++r)
        for (int c2 = 0; c2 < 8; ++c2) {
            unsigned short h[2], l[2];
            for (int e = 0; e < 2; ++e) {
                const int c = 2 * c2 + e;
                const int rl = r % B, cl = c % B;
                const float v = (r / B == c / B && rl < N && cl < N) ? (float)(m[rl + N * cl] * scale) : 0.f;
                h[e] = bf16_rne(v);
                l[e] = bf16_rne(v - bf16_to_float(h[e]));
            }
            hi[r * 8 + c2] = (unsigned)h[0] | ((unsigned)h[1] << 16);
            lo[r * 8 + c2] = (unsigned)l[0] | ((unsigned)l[1] << 16);
        }
}

// Power-of-two scale 2^s that brings the largest |entry| of m into [2^14, 2^15),
// so that an f16 split of m * 2^s keeps 22 significant bits of the large
// entries and cannot overflow.  False (no f16 split) for a zero or non-finite
// matrix, or a scale whose inverse could underflow the other factor.
static inline bool f16_scale(const double* m, int N, int& s) {
    double mx = 0.0;
    for (int e = 0; e < N * N; ++e) {
        if (!std::isfinite(m[e])) return false;
        mx = std::max(mx, std::fabs(m[e]));
    }
    if (mx == 0.0) return false;
    int ex = 0;
    std::frexp(mx, &ex);   // mx in [2^(ex-1), 2^ex)
    s = 15 - ex;
    return s >= -40 && s <= 40;
}

// f16 hi / lo split of m * 2^s (round to nearest even), packed as split_rowmajor.
static inline void split_rowmajor_f16(const double* m, int N, int s, unsigned* hi, unsigned* lo, int B = 16) {
    for (int r = 0; r < 16; ++r)
        for (int c2 = 0; c2 < 8; ++c2) {
            unsigned short h[2], l[2];
            for (int e = 0; e < 2; ++e) {
                const int c = 2 * c2 + e;
                const int rl = r % B, cl = c % B;
                const float v = (r / B == c / B && rl < N && cl < N) ? (float)std::ldexp(m[rl + N * cl], s) : 0.f;
                const __half hv = __float2half_rn(v);
                const __half lv = __float2half_rn(v - __half2float(hv));
                h[e] = __half_as_ushort(hv);
                l[e] = __half_as_ushort(lv);
            }
            hi[r * 8 + c2] = (unsigned)h[0] | ((unsigned)h[1] << 16);
            lo[r * 8 + c2] = (unsigned)l[0] | ((unsigned)l[1] << 16);
        }
}

template <typename S, int N>
static kron_status launch_tc2_n(const KronDesc& d, cudaStream_t st) {
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    TcArgs2<N> a;
    split_rowmajor(d.m1, N, a.m1h, a.m1l, tc2_block(N));
    int s = 0;
    a.f16a = std::is_same<S, __half>::value && f16_scale(d.m1, N, s);
    if (a.f16a) {   // f16 storage: W = (M1 2^s) X in f16 MMAs, then W (M2 2^-s)^T
        split_rowmajor_f16(d.m1, N, s, a.f1h, a.f1l, tc2_block(N));
        split_rowmajor(d.m2, N, a.m2h, a.m2l, tc2_block(N), std::ldexp(1.0, -s));
    } else {
        memset(a.f1h, 0, sizeof(a.f1h));
        memset(a.f1l, 0, sizeof(a.f1l));
        split_rowmajor(d.m2, N, a.m2h, a.m2l, tc2_block(N));
    }
    a.X = d.X;
    a.Y = d.Y;
    a.batch = d.batch;
    a.alpha = (float)d.alpha;
    a.beta = (float)d.beta;
    a.beta_zero = d.beta == 0.0;
    a.alpha_one = d.alpha == 1.0;
    a.ypair = ((uintptr_t)d.Y % (2 * sizeof(S))) == 0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;
    // Body: the stacked one (KRON_VARIANT_EXCHANGE: intermediates through the
    // warp's exchange rows; 9 <= n <= 16) or the padded tile per instance
    // (KRON_VARIANT_IN_PLACE: the second product takes the first's accumulators).
    // Measured defaults (HBM fraction, stacked against padded): FP32 n = 10, 12, 14:
    // 0.80, 0.91, 0.87 against 0.48, 0.71, 0.81 -- stacked; 16-bit n = 10, 12: 0.55,
    // 0.67 against 0.30, 0.44 -- stacked; 16-bit n = 14, 16 with two groups per warp
    // step, 32-instance tiles, three in flight: 0.65, 0.93 against 0.60, 0.83-0.89 --
    // stacked; FP32 n = 16 (the padded tile wastes nothing; 1.0): padded; odd n
    // (eight instances per group, the slow general path): padded.
    constexpr bool kStackable = N >= 9 && N <= 16;
    if (d.variant == KRON_VARIANT_EXCHANGE && !kStackable) return KRON_ERR_NOT_SUPPORTED;
    constexpr bool kStackedDefault = kStackable && N % 2 == 0 && !(N == 16 && sizeof(S) == 4);
    constexpr bool kTwoGroups = sizeof(S) == 2 && N >= 14;   // default groups per warp step: 2
    const bool stacked = kStackable && (d.variant == KRON_VARIANT_EXCHANGE ||
                                        (d.variant == KRON_VARIANT_AUTO && kStackedDefault));
    // Measured defaults: at n = 16, 32 KB operand tiles (32 FP32 or 64 bf16
    // instances; three / two stages); below 16 instances of fewer bytes, 16 per tile
    // and three stages (more resident CTAs).
    int P = d.P > 0 ? d.P : (N == 16 ? (sizeof(S) == 4 ? 32 : 64) : 16);
    if (stacked && d.P <= 0) P = (sizeof(S) == 4 || kTwoGroups) ? 32 : 64;
    int mult = 1;
    while ((mult * N * N * sizeof(S)) % 16) ++mult;
    P = (P + mult - 1) / mult * mult;
    int nstage = d.nstage >= 1 ? d.nstage : ((N == 16 && sizeof(S) == 2) ? 2 : 3);
    if (stacked && d.nstage < 1) nstage = (sizeof(S) == 4 || kTwoGroups) ? 3 : 2;
    if (nstage > 8) nstage = 8;
    const bool fast = N % 2 == 0 && a.alpha_one && a.beta_zero && a.ypair &&
                      (!std::is_same<S, __half>::value || a.f16a);
    const int K = stacked && fast && (d.fps == 2 || (d.fps == 0 && kTwoGroups)) ? 2 : 1;   // groups per step
    const size_t exch = stacked ? (size_t)(kTcThreads / 32) * K * tc2s_group(N) * N * kTc2sRow : 0;
    auto smem_of = [&](int ns) { return 128 + ns * round_up((size_t)P * N * N * sizeof(S), 128) + exch; };
    size_t smem = smem_of(nstage);
    while (nstage > 1 && smem > dev.smem_per_block_optin) smem = smem_of(--nstage);
    if (smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    a.P = P;
    a.nstage = nstage;
    void (*kern)(const TcArgs2<N>) = tc2_kernel<S, N>;
    if constexpr (kStackable) {
        if (stacked) {
            kern = tc2s_kernel<S, N, false, 1>;
            if constexpr (N % 2 == 0) {
                if (fast) kern = K == 2 ? tc2s_kernel<S, N, true, 2> : tc2s_kernel<S, N, true, 1>;
            }
        }
    }
    if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
    const int64_t ntiles = (d.batch + P - 1) / P;
    int64_t grid = d.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTcThreads, smem) != cudaSuccess)
            return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kTcThreads, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

template <typename S, int N>
static kron_status launch_tc3_n(const KronDesc& d, cudaStream_t st) {
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    TcArgs3<N> a;
    split_rowmajor(d.m2, N, a.m2h, a.m2l);
    split_rowmajor(d.m3, N, a.m3h, a.m3l);
    int s = 0;
    a.f16a = std::is_same<S, __half>::value && f16_scale(d.m2, N, s);
    if (a.f16a) {   // f16 storage: W' = (M2 2^s) X_p^T in f16 MMAs, then W' (M1 2^-s)^T
        split_rowmajor_f16(d.m2, N, s, a.f2h, a.f2l);
        split_rowmajor(d.m1, N, a.m1h, a.m1l, 16, std::ldexp(1.0, -s));
    } else {
        memset(a.f2h, 0, sizeof(a.f2h));
        memset(a.f2l, 0, sizeof(a.f2l));
        split_rowmajor(d.m1, N, a.m1h, a.m1l);
    }
    a.X = d.X;
    a.Y = d.Y;
    a.ypair = ((uintptr_t)d.Y & 3u) == 0;
    a.batch = d.batch;
    a.alpha = (float)d.alpha;
    a.beta = (float)d.beta;
    a.beta_zero = d.beta == 0.0;
    a.alpha_one = d.alpha == 1.0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;
    using L = Tc3Layout<S, N>;
    // compute_warps 1: the single-warp kernel; else W warps share an instance.
    // Measured default: four warps at n = 14, 15, 16 (seven or eight plane pairs
    // to share) and for FP32 storage at n = 10, 12 (0.33 and 0.49 of HBM against
    // 0.30 and 0.35 with one warp); one warp for 16-bit storage below n = 14 (bf16:
    // the same speed; f16: several warps measured 2-6x slower at n = 10, 12 and odd
    // n, not understood) and for smaller n (too few plane pairs to share).
    const bool f16few = std::is_same<S, __half>::value && N != 16;
    const bool f32mid = sizeof(S) == 4 && N >= 10 && N % 2 == 0;
    const int W = d.warps > 0 ? d.warps : (((N >= 14 && !f16few) || f32mid) ? 4 : 1);
    if (W != 1) {
        const size_t smem = 128 + 2 * (size_t)L::XB + L::TB;
        if (W > 8 || smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
        auto kern = tc3g_kernel<S, N>;
        if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * W, smem) != cudaSuccess)
            return KRON_ERR_CUDA;
        int64_t grid = d.grid > 0 ? d.grid : (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
        if (grid > d.batch) grid = d.batch;
        if (grid < 1) grid = 1;
        kern<<<(unsigned)grid, 32 * W, smem, st>>>(a);
        return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
    }
    const size_t smem = 128 + kTc3Warps * (size_t)L::PER_WARP;
    if (smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    auto kern = tc3_kernel<S, N>;
    if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kTc3Warps, smem) != cudaSuccess)
        return KRON_ERR_CUDA;
    int64_t grid = d.grid > 0 ? d.grid : (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    const int64_t need = (d.batch + kTc3Warps - 1) / kTc3Warps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, 32 * kTc3Warps, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

template <typename S>
static kron_status launch_tc3(const KronDesc& d, cudaStream_t st) {
    switch (d.N) {
        case 1: return launch_tc3_n<S, 1>(d, st);
        case 2: return launch_tc3_n<S, 2>(d, st);
        case 3: return launch_tc3_n<S, 3>(d, st);
        case 4: return launch_tc3_n<S, 4>(d, st);
        case 5: return launch_tc3_n<S, 5>(d, st);
        case 6: return launch_tc3_n<S, 6>(d, st);
        case 7: return launch_tc3_n<S, 7>(d, st);
        case 8: return launch_tc3_n<S, 8>(d, st);
        case 9: return launch_tc3_n<S, 9>(d, st);
        case 10: return launch_tc3_n<S, 10>(d, st);
        case 11: return launch_tc3_n<S, 11>(d, st);
        case 12: return launch_tc3_n<S, 12>(d, st);
        case 13: return launch_tc3_n<S, 13>(d, st);
        case 14: return launch_tc3_n<S, 14>(d, st);
        case 15: return launch_tc3_n<S, 15>(d, st);
        case 16: return launch_tc3_n<S, 16>(d, st);
        default: return KRON_ERR_INVALID_VALUE;
    }
}

template <typename S>
static kron_status launch_tc2(const KronDesc& d, cudaStream_t st) {
    switch (d.N) {
        case 1: return launch_tc2_n<S, 1>(d, st);
        case 2: return launch_tc2_n<S, 2>(d, st);
        case 3: return launch_tc2_n<S, 3>(d, st);
        case 4: return launch_tc2_n<S, 4>(d, st);
        case 5: return launch_tc2_n<S, 5>(d, st);
        case 6: return launch_tc2_n<S, 6>(d, st);
        case 7: return launch_tc2_n<S, 7>(d, st);
        case 8: return launch_tc2_n<S, 8>(d, st);
        case 9: return launch_tc2_n<S, 9>(d, st);
        case 10: return launch_tc2_n<S, 10>(d, st);
        case 11: return launch_tc2_n<S, 11>(d, st);
        case 12: return launch_tc2_n<S, 12>(d, st);
        case 13: return launch_tc2_n<S, 13>(d, st);
        case 14: return launch_tc2_n<S, 14>(d, st);
        case 15: return launch_tc2_n<S, 15>(d, st);
        case 16: return launch_tc2_n<S, 16>(d, st);
        default: return KRON_ERR_INVALID_VALUE;
    }
}

}  // namespace kron
