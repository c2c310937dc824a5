// CUDA-core kernels for the batched Kronecker product action ("fiber" kernels).
//
// Sum factorisation (paper Sec. 2.1 and Algorithm 1): the action is applied one
// mode at a time.  A mode-k contraction maps every mode-k fiber x (N values) to
// y = M_k x; each thread owns one fiber per stage and computes its N x N
// products with the component entries taken straight from the kernel parameter
// (constant) bank -- the components are shared by the whole batch (Sec. 2.2,
// Sec. 4: stage the constant matrices once per block), so no instruction is
// spent loading them.
//
// One CTA processes a tile of P instances at a time and loops over tiles
// (persistent grid).  Operand tiles stream into shared memory with 1-D bulk
// copies (TMA, cp.async.bulk) in an `nstage`-deep mbarrier pipeline; the
// intermediates of the fused contractions stay in padded shared-memory buffers
// whose strides make both the writing and the reading pattern bank-conflict
// free; the last contraction writes mode-1 fibers of Y straight to global
// memory with vector stores.
//
//   2-D (Y = M1 X M2^T):   stage 1  W(l,:) = M2 X(l,:)     mode 2, per row l
//                          stage 2  Y(:,j) = M1 W(:,j)     mode 1, per column j
//   3-D:                   stage A  T(i,j,:) = M3 X(i,j,:) mode 3
//                          stage B  U(i,:,k) = M2 T(i,:,k) mode 2
//                          stage C  Y(:,j,k) = M1 U(:,j,k) mode 1
// The paper's Algorithm 1 writes its intermediate `tmp` to device memory
// (Sec. 5 attributes the 3-D slowdown to it); here it never leaves the SM.
#pragma once

#include <type_traits>

#include "kron_complex.cuh"
#include "kron_device.cuh"
#include "kron_internal.h"

namespace kron {

// Storage <-> compute for complex storage (the compute type is the same).
template <> __device__ __forceinline__ cf32 load_cvt<cf32, cf32>(cf32 v) { return v; }
template <> __device__ __forceinline__ cf64 load_cvt<cf64, cf64>(cf64 v) { return v; }
template <> __device__ __forceinline__ cf32 store_cvt<cf32, cf32>(cf32 v) { return v; }
template <> __device__ __forceinline__ cf64 store_cvt<cf64, cf64>(cf64 v) { return v; }

template <typename T, int N, int D>
struct FiberArgs {
    T m1[N * N];                  // mode-1 component, column-major, op() applied
    T m2[N * N];                  // mode-2 component
    T m3[D == 3 ? N * N : 1];     // mode-3 component (3-D)
    const void* X;
    void* Y;
    int64_t batch, ldxp, ldyp;
    int ldx, ldx2, ldy, ldy2;
    int xe1, xe2, xe3;            // extents of op(X); entries beyond are read as 0
    int ye1, ye2, ye3;            // extents of Y; entries beyond are not written
    int transx;
    int conjx;                    // complex storage: op(X) conjugates (transx = 'C')
    int P;                        // instances per tile
    int nstage;                   // bulk-copy pipeline depth (0: generic loads)
    int yvec;                     // Y store chunk bytes (16/8/4) or 0 (elements)
    int beta_zero, alpha_one;
    T alpha, beta;
    unsigned* err;
};

template <int N, int D>
struct FiberLayout {
    static constexpr int NX = ipow(N, D);         // elements per instance
    static constexpr int FPI = ipow(N, D - 1);    // fibers per instance and stage
    // 2-D W and 3-D U: element (i, j, k) of instance q at i + (N+1) j + S k + SQ q
    static constexpr int SU = stride_mod32(N * N + N - 1, N);
    static constexpr int SUQ = (D == 2) ? SU : SU * N;
    // 3-D T: element (i, j, k) of instance q at i + N j + ST k + STQ q
    static constexpr int ST = stride_mod32(N * N, N);
    static constexpr int STQ = ST * N;
    static constexpr int EX1 = (D == 2) ? SUQ : STQ;   // per-instance size, buffer 1
    static constexpr int EX2 = (D == 2) ? 0 : SUQ;     // per-instance size, buffer 2
};

__host__ __device__ constexpr size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

// y = M x for one fiber; M is an N x N column-major matrix in the parameter bank.
template <int N, typename T>
__device__ __forceinline__ void contract(const T* __restrict__ M, const T (&x)[N], T (&y)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = M[i] * x[0];
#pragma unroll
    for (int l = 1; l < N; ++l) {
#pragma unroll
        for (int i = 0; i < N; ++i) y[i] = madd(M[i + N * l], x[l], y[i]);
    }
}

// Complex FP32 y = M x on packed pairs.  An entry m = M[i, l] is read as the
// pair (Re m, Im m) -- its storage layout -- and x_l = (a, b) enters as the
// duplicated pairs (a, a) and (b, b).  Two accumulators per output,
//   P_i = sum_l (Re m * a, Im m * a),   Q_i = sum_l (Re m * b, Im m * b),
// give y_i = (P_i.re - Q_i.im, P_i.im + Q_i.re): the four real FMAs of each
// complex product in two fma.rn.f32x2, with the coefficients of one table.
template <int N>
__device__ __forceinline__ void contract_c32(const cf32* __restrict__ M, const cf32 (&x)[N], cf32 (&y)[N]) {
    const f2* Mp = reinterpret_cast<const f2*>(M);
    f2 P[N], Q[N];
    {
        const f2 a = f2_pack(x[0].re, x[0].re), b = f2_pack(x[0].im, x[0].im);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            P[i] = fmul2(Mp[i], a);
            Q[i] = fmul2(Mp[i], b);
        }
    }
#pragma unroll
    for (int l = 1; l < N; ++l) {
        const f2 a = f2_pack(x[l].re, x[l].re), b = f2_pack(x[l].im, x[l].im);
#pragma unroll
        for (int i = 0; i < N; ++i) {
            P[i] = ffma2(Mp[i + N * l], a, P[i]);
            Q[i] = ffma2(Mp[i + N * l], b, Q[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = cf32(f2_lo(P[i]) - f2_hi(Q[i]), f2_hi(P[i]) + f2_lo(Q[i]));
}

// Mode-K contraction of one fiber with the component of the kernel's arguments.
template <int K, typename T, int N, int D>
__device__ __forceinline__ void contract_mode(const FiberArgs<T, N, D>& a, const T (&x)[N], T (&y)[N]) {
    const T* M = K == 1 ? a.m1 : K == 2 ? a.m2 : a.m3;
    if constexpr (std::is_same<T, cf32>::value)
        contract_c32<N>(M, x, y);
    else
        contract<N, T>(M, x, y);
}

// Byte span of tile `tile` of a contiguous batch.  The bulk copy takes the
// 16-byte-aligned superset [a0, a1) of the tile's bytes [b0, b1), clipped to the
// last whole 16-byte unit of X; the tile's first element then sits `pre` bytes
// into the shared buffer, and the bytes [h0, b1) past the clip (end of the
// batch only) are copied by hand.
struct TileSpan {
    unsigned pre;     // b0 - a0
    unsigned copy;    // bytes moved by the bulk copy (multiple of 16)
    unsigned h0;      // first hand-copied byte, relative to a0
    unsigned end;     // b1 - a0
};

template <typename T, typename S, int N, int D>
__device__ __forceinline__ TileSpan tile_span(const FiberArgs<T, N, D>& a, int64_t tile) {
    constexpr int64_t NXB = (int64_t)ipow(N, D) * sizeof(S);
    const int64_t inst0 = tile * a.P;
    const int64_t cnt = min((int64_t)a.P, a.batch - inst0);
    const int64_t b0 = inst0 * NXB, b1 = b0 + cnt * NXB;
    const int64_t a0 = b0 & ~(int64_t)15;
    const int64_t lim = (a.batch * NXB) & ~(int64_t)15;
    const int64_t a1 = max(a0, min((b1 + 15) & ~(int64_t)15, lim));
    TileSpan sp;
    sp.pre = (unsigned)(b0 - a0);
    sp.copy = (unsigned)(a1 - a0);
    sp.h0 = (unsigned)max(a1 - a0, b0 - a0);
    sp.end = (unsigned)(b1 - a0);
    return sp;
}

template <typename T, typename S, int N, int D>
__device__ __forceinline__ void issue_tile(const FiberArgs<T, N, D>& a, void* dst, uint64_t* bar,
                                           int64_t tile, uint64_t pol) {
    constexpr int64_t NXB = (int64_t)ipow(N, D) * sizeof(S);
    const TileSpan sp = tile_span<T, S, N, D>(a, tile);
    const char* src = static_cast<const char*>(a.X) + ((tile * a.P * NXB) & ~(int64_t)15);
    mbar_arrive_expect_tx(bar, sp.copy);
    if (sp.copy) bulk_g2s(dst, src, sp.copy, bar, pol);
}

// Strided / transposed / rectangular operand tile, element by element.
template <typename T, typename S, int N, int D>
__device__ __forceinline__ void load_tile_generic(const FiberArgs<T, N, D>& a, S* xt, int64_t inst0, int cnt) {
    constexpr int NX = ipow(N, D);
    const S* X = static_cast<const S*>(a.X);
    const int E = cnt * NX;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int q = e / NX;
        const int r = e - q * NX;
        const int i1 = r % N;
        const int i2 = (r / N) % N;
        const int i3 = (D == 3) ? r / (N * N) : 0;
        S v = store_cvt<S, T>(T(0));
        if (i1 < a.xe1 && i2 < a.xe2 && i3 < a.xe3) {
            int64_t off = (inst0 + q) * a.ldxp;
            if constexpr (D == 2)
                off += a.transx ? (i2 + (int64_t)a.ldx * i1) : (i1 + (int64_t)a.ldx * i2);
            else
                off += i1 + (int64_t)a.ldx * i2 + (int64_t)a.ldx2 * i3;
            v = X[off];
            if constexpr (is_cplx<S>::value)
                if (a.conjx) v = conj_of(v);
        }
        xt[e] = v;
    }
}

// Epilogue + store of one mode-1 fiber of Y (N values, contiguous in Y).
template <typename T, typename S, int N, int D>
__device__ __forceinline__ void store_fiber(const FiberArgs<T, N, D>& a, S* dst, const T (&y)[N]) {
    S o[N];
    if (a.beta_zero) {
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] = store_cvt<S, T>(a.alpha_one ? y[i] : a.alpha * y[i]);
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const T old = (i < a.ye1) ? load_cvt<T, S>(dst[i]) : T(0);
            o[i] = store_cvt<S, T>(madd(a.alpha, y[i], a.beta * old));
        }
    }
    if constexpr (is_cplx<S>::value) {
        // 16-byte vector stores: one complex double, or two complex floats
        if (a.yvec == 16) {
            if constexpr (sizeof(S) == 16) {
#pragma unroll
                for (int i = 0; i < N; ++i) __stcs(reinterpret_cast<double2*>(dst) + i, make_double2(o[i].re, o[i].im));
                return;
            } else if constexpr (N % 2 == 0) {
#pragma unroll
                for (int c = 0; c < N / 2; ++c)
                    __stcs(reinterpret_cast<float4*>(dst) + c,
                           make_float4(o[2 * c].re, o[2 * c].im, o[2 * c + 1].re, o[2 * c + 1].im));
                return;
            }
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i < a.ye1) dst[i] = o[i];
        return;
    } else if constexpr (sizeof(S) == 8) {
        if (a.yvec == 16) {
#pragma unroll
            for (int c = 0; c < N / 2; ++c)
                __stcs(reinterpret_cast<double2*>(dst) + c, make_double2(o[2 * c], o[2 * c + 1]));
            if constexpr (N % 2) __stcs(dst + N - 1, o[N - 1]);
            return;
        }
    } else {
        if constexpr ((N * sizeof(S)) % 16 == 0) {
            if (a.yvec == 16) { store_chunks<16, S, N>(dst, o); return; }
        }
        if constexpr ((N * sizeof(S)) % 8 == 0) {
            if (a.yvec == 8) { store_chunks<8, S, N>(dst, o); return; }
        }
        if constexpr ((N * sizeof(S)) % 4 == 0) {
            if (a.yvec == 4) { store_chunks<4, S, N>(dst, o); return; }
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (i < a.ye1) dst[i] = o[i];
}

// Complex FP32 at 2-D holds two accumulators per output; three CTAs per SM
// (the shared-memory limit of the 2-D tiles) cap it at 85 registers.
template <typename T, int D>
constexpr int fiber_min_blocks() { return std::is_same<T, cf32>::value && D == 2 ? 3 : 1; }

template <typename T, typename S, int N, int D>
__global__ void __launch_bounds__(kFiberThreads, fiber_min_blocks<T, D>())
fiber_kernel(const __grid_constant__ FiberArgs<T, N, D> a) {
    using L = FiberLayout<N, D>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);   // up to 8 pipeline barriers
    const int P = a.P;
    const bool tma = a.nstage > 0;
    const int nbuf = tma ? a.nstage : 1;
    const size_t xstage = round_up((size_t)P * L::NX * sizeof(S) + 16, 128);
    unsigned char* xbase = smem + 128;
    T* ex1 = reinterpret_cast<T*>(xbase + nbuf * xstage);
    T* ex2 = ex1 + (size_t)P * L::EX1;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    const int64_t ntiles = (a.batch + P - 1) / P;
    const int64_t grid = gridDim.x;
    uint64_t pol = 0;

    if (tma) {
        if (tid == 0) {
            for (int s = 0; s < a.nstage; ++s) mbar_init(&bars[s], 1);
            fence_barrier_init();
        }
        __syncthreads();
        if (tid == 0) {
            pol = l2_evict_first_policy();
            for (int s = 0; s < a.nstage; ++s) {
                const int64_t t = blockIdx.x + s * grid;
                if (t < ntiles) issue_tile<T, S, N, D>(a, xbase + s * xstage, &bars[s], t, pol);
            }
        }
    }

    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
        const int s = tma ? it % a.nstage : 0;
        unsigned char* xraw = xbase + s * xstage;
        S* xt = reinterpret_cast<S*>(xraw);
        const int64_t inst0 = tile * P;
        const int cnt = (int)min((int64_t)P, a.batch - inst0);
        bool ok = true;
        if (tma) {
            ok = mbar_wait_bounded(&bars[s], (unsigned)(it / a.nstage) & 1u, a.err);
            const TileSpan sp = tile_span<T, S, N, D>(a, tile);
            xt = reinterpret_cast<S*>(xraw + sp.pre);
            if (sp.h0 < sp.end) {   // ragged end of the batch: the last bytes by hand
                const int64_t a0 = (inst0 * (int64_t)L::NX * (int64_t)sizeof(S)) & ~(int64_t)15;
                const S* src = reinterpret_cast<const S*>(static_cast<const char*>(a.X) + a0);
                S* dst = reinterpret_cast<S*>(xraw);
                for (unsigned e = sp.h0 / sizeof(S) + tid; e < sp.end / sizeof(S); e += nthr) dst[e] = src[e];
                __syncthreads();
            }
        } else {
            load_tile_generic<T, S, N, D>(a, xt, inst0, cnt);
            __syncthreads();
        }

        // ---- first contraction: reads the operand tile --------------------------------
        if constexpr (D == 2) {
            const int F = cnt * N;
            for (int f = tid; f < F; f += nthr) {
                const int q = f / N, l = f - q * N;
                const S* xr = xt + q * L::NX + l;
                T x[N], w[N];
#pragma unroll
                for (int m = 0; m < N; ++m) x[m] = load_cvt<T, S>(xr[N * m]);
                contract_mode<2>(a, x, w);
                T* wr = ex1 + q * L::SUQ + l;
#pragma unroll
                for (int j = 0; j < N; ++j) wr[(N + 1) * j] = w[j];
            }
        } else {
            const int F = cnt * N * N;
            for (int f = tid; f < F; f += nthr) {
                const int q = f / (N * N), r = f - q * (N * N);
                const int i = r % N, j = r / N;
                const S* xr = xt + q * L::NX + i + N * j;
                T x[N], t[N];
#pragma unroll
                for (int p = 0; p < N; ++p) x[p] = load_cvt<T, S>(xr[N * N * p]);
                contract_mode<3>(a, x, t);
                T* tr = ex1 + q * L::STQ + i + N * j;
#pragma unroll
                for (int k = 0; k < N; ++k) tr[L::ST * k] = t[k];
            }
        }
        // Everyone is done with the operand tile (and agrees on `ok`).
        if (__syncthreads_or(!ok)) {
            if (tid == 0 && tma) {   // let in-flight copies land before the CTA exits
                for (int j = it; j < it + a.nstage; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&bars[j % a.nstage], (unsigned)(j / a.nstage) & 1u, a.err);
            }
            return;
        }
        if (tma && tid == 0) {
            const int64_t next = tile + a.nstage * grid;
            if (next < ntiles) {
                fence_proxy_async_smem();
                issue_tile<T, S, N, D>(a, xraw, &bars[s], next, pol);
            }
        }

        // ---- remaining contractions ---------------------------------------------------
        S* Y = static_cast<S*>(a.Y);
        if constexpr (D == 2) {
            const int F = cnt * N;
            for (int f = tid; f < F; f += nthr) {
                const int q = f / N, j = f - q * N;
                const T* wr = ex1 + q * L::SUQ + (N + 1) * j;
                T w[N], y[N];
#pragma unroll
                for (int l = 0; l < N; ++l) w[l] = wr[l];
                contract_mode<1>(a, w, y);
                if (j < a.ye2) store_fiber<T, S, N, D>(a, Y + (inst0 + q) * a.ldyp + (int64_t)a.ldy * j, y);
            }
            __syncthreads();   // W is rewritten by the next tile's first stage
        } else {
            int F = cnt * N * N;
            for (int f = tid; f < F; f += nthr) {
                const int q = f / (N * N), r = f - q * (N * N);
                const int i = r % N, k = r / N;
                const T* tr = ex1 + q * L::STQ + i + L::ST * k;
                T t[N], u[N];
#pragma unroll
                for (int m = 0; m < N; ++m) t[m] = tr[N * m];
                contract_mode<2>(a, t, u);
                T* ur = ex2 + q * L::SUQ + i + L::SU * k;
#pragma unroll
                for (int j = 0; j < N; ++j) ur[(N + 1) * j] = u[j];
            }
            __syncthreads();
            for (int f = tid; f < F; f += nthr) {
                const int q = f / (N * N), r = f - q * (N * N);
                const int j = r % N, k = r / N;
                const T* ur = ex2 + q * L::SUQ + (N + 1) * j + L::SU * k;
                T u[N], y[N];
#pragma unroll
                for (int l = 0; l < N; ++l) u[l] = ur[l];
                contract_mode<1>(a, u, y);
                if (j < a.ye2 && k < a.ye3)
                    store_fiber<T, S, N, D>(
                        a, Y + (inst0 + q) * a.ldyp + (int64_t)a.ldy * j + (int64_t)a.ldy2 * k, y);
            }
            // U is rewritten only after the next tile's first barrier: no barrier here.
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <typename T, typename S, int N, int D>
size_t fiber_smem_bytes(int P, int nstage) {
    using L = FiberLayout<N, D>;
    const int nbuf = nstage > 0 ? nstage : 1;
    return 128 + nbuf * round_up((size_t)P * L::NX * sizeof(S) + 16, 128) +
           (size_t)P * (L::EX1 + L::EX2) * sizeof(T);
}

template <typename T, typename S, int N, int D>
kron_status launch_fiber_n(const KronDesc& d, cudaStream_t st) {
    using L = FiberLayout<N, D>;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    FiberArgs<T, N, D> a;
    auto elem = [](double re, double im) -> T {
        if constexpr (is_cplx<T>::value) {
            using R = decltype(T().re);
            return T(static_cast<R>(re), static_cast<R>(im));
        } else {
            return static_cast<T>(re);
        }
    };
    for (int e = 0; e < N * N; ++e) {
        a.m1[e] = elem(d.m1[e], d.m1i[e]);
        a.m2[e] = elem(d.m2[e], d.m2i[e]);
        if constexpr (D == 3) a.m3[e] = elem(d.m3[e], d.m3i[e]);
    }
    if constexpr (D == 2) a.m3[0] = T(0);
    a.X = d.X;
    a.Y = d.Y;
    a.batch = d.batch;
    a.ldxp = d.ldxp;
    a.ldyp = d.ldyp;
    a.ldx = d.ldx;
    a.ldx2 = d.ldx2;
    a.ldy = d.ldy;
    a.ldy2 = d.ldy2;
    a.xe1 = d.xe[0]; a.xe2 = d.xe[1]; a.xe3 = d.xe[2];
    a.ye1 = d.ye[0]; a.ye2 = d.ye[1]; a.ye3 = d.ye[2];
    a.transx = d.transx;
    a.conjx = d.conjx;
    a.yvec = d.yvec;
    a.alpha = elem(d.alpha, d.alpha_im);
    a.beta = elem(d.beta, d.beta_im);
    a.beta_zero = d.beta == 0.0 && d.beta_im == 0.0;
    a.alpha_one = d.alpha == 1.0 && d.alpha_im == 0.0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;

    // Instances per tile: about one fiber per thread and stage (tiles of any size
    // can be bulk-copied, see tile_span).  If the tile does not fit in shared
    // memory with a bulk-copy buffer, it is loaded element by element instead.
    const int P0 = d.P > 0 ? d.P : (kFiberThreads + L::FPI - 1) / L::FPI;
    int P = P0;
    int nstage = 0;
    if (d.contiguous) {
        nstage = d.nstage >= 1 ? d.nstage : 1;   // more resident CTAs beat a deeper pipeline (measured)
        if (nstage > 8) nstage = 8;
    }
    size_t smem = fiber_smem_bytes<T, S, N, D>(P, nstage);
    while (nstage > 1 && smem > dev.smem_per_block_optin) {
        --nstage;
        smem = fiber_smem_bytes<T, S, N, D>(P, nstage);
    }
    if (smem > dev.smem_per_block_optin && nstage > 0) {
        P = P0;
        nstage = 0;
        smem = fiber_smem_bytes<T, S, N, D>(P, nstage);
    }
    while (smem > dev.smem_per_block_optin && P > 1) smem = fiber_smem_bytes<T, S, N, D>(--P, nstage);
    if (smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    a.P = P;
    a.nstage = nstage;

    auto kern = fiber_kernel<T, S, N, D>;
    if (!ensure_smem_optin((const void*)kern, smem)) return KRON_ERR_CUDA;
    const int64_t ntiles = (d.batch + P - 1) / P;
    int64_t grid = d.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFiberThreads, smem) != cudaSuccess)
            return KRON_ERR_CUDA;
        if (per_sm < 1) per_sm = 1;
        grid = (int64_t)per_sm * dev.sms;
    }
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kFiberThreads, smem, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

template <typename T, typename S, int D>
kron_status launch_fiber_d(const KronDesc& d, cudaStream_t st) {
    switch (d.N) {
        case 1: return launch_fiber_n<T, S, 1, D>(d, st);
        case 2: return launch_fiber_n<T, S, 2, D>(d, st);
        case 3: return launch_fiber_n<T, S, 3, D>(d, st);
        case 4: return launch_fiber_n<T, S, 4, D>(d, st);
        case 5: return launch_fiber_n<T, S, 5, D>(d, st);
        case 6: return launch_fiber_n<T, S, 6, D>(d, st);
        case 7: return launch_fiber_n<T, S, 7, D>(d, st);
        case 8: return launch_fiber_n<T, S, 8, D>(d, st);
        case 9: return launch_fiber_n<T, S, 9, D>(d, st);
        case 10: return launch_fiber_n<T, S, 10, D>(d, st);
        case 11: return launch_fiber_n<T, S, 11, D>(d, st);
        case 12: return launch_fiber_n<T, S, 12, D>(d, st);
        case 13: return launch_fiber_n<T, S, 13, D>(d, st);
        case 14: return launch_fiber_n<T, S, 14, D>(d, st);
        case 15: return launch_fiber_n<T, S, 15, D>(d, st);
        case 16: return launch_fiber_n<T, S, 16, D>(d, st);
        default: return KRON_ERR_INVALID_VALUE;
    }
}

}  // namespace kron
