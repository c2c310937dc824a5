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
// Data flow per CTA: the operand elements of the next tile are loaded into
// registers (any alignment, coalesced) while the current tile is contracted in
// shared memory; the last contraction writes its fibers into the operand buffer
// (dead after the first contraction), from which consecutive threads copy the
// outputs to Y (coalesced); then the next tile is committed to that buffer.
//
// Workspace (caller-owned device memory, written on the first execute with a
// given pointer): tile table (int4: class key, first sorted index, count, 0),
// then the sorted instance offsets (int64 X offsets, then int64 Y offsets).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "kron_device.cuh"
#include "kron_fiber.cuh"
#include "kron_internal.h"
#include "kron_pair.cuh"

namespace kron {

constexpr int kVlThreads = 256;
constexpr int kVlRegs = 16;                            // prefetched elements per thread
constexpr int kVlMaxTile = kVlThreads * kVlRegs;       // elements per tile
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
    unsigned* err;
};

static_assert(sizeof(VarlenArgs) <= 32764, "kernel parameter space");

__device__ __forceinline__ int vl_nx(int key) {
    const int n = (key & 15) + 1;
    return key < 16 ? n * n : n * n * n;
}

// Loads the operand elements of tile `td` into registers (element e = tid +
// kVlThreads * r); xo[q] is the X offset of the tile's instance q (shared memory).
template <typename S>
__device__ __forceinline__ void vl_prefetch(const VarlenArgs& a, int4 td, const int* xo, S (&v)[kVlRegs]) {
    const int nx = vl_nx(td.x);
    const unsigned inv = a.cls[td.x].inv;
    const int total = td.z * nx;
    const S* X = static_cast<const S*>(a.X);
#pragma unroll
    for (int r = 0; r < kVlRegs; ++r) {
        const int e = threadIdx.x + kVlThreads * r;
        if (e < total) {
            const int q = nx == 1 ? e : (int)__umulhi((unsigned)e, inv);
            v[r] = X[(int64_t)xo[q] + (e - q * nx)];
        }
    }
}

template <typename S>
__device__ __forceinline__ void vl_commit(int4 td, const S (&v)[kVlRegs], S* xt) {
    const int total = td.z * vl_nx(td.x);
#pragma unroll
    for (int r = 0; r < kVlRegs; ++r) {
        const int e = threadIdx.x + kVlThreads * r;
        if (e < total) xt[e] = v[r];
    }
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

// Output pairs rounded to the storage type, staged at dst[2r].
template <typename S, int N>
__device__ __forceinline__ void vl_stage_out(S* dst, const f2 (&y)[vl_rows(N) / 2]) {
    if constexpr (sizeof(S) == 4) {
#pragma unroll
        for (int r = 0; r < vl_rows(N) / 2; ++r) *reinterpret_cast<f2*>(dst + 2 * r) = y[r];
    } else {
#pragma unroll
        for (int r = 0; r < vl_rows(N) / 2; ++r) *reinterpret_cast<unsigned*>(dst + 2 * r) = pack16<S>(y[r]);
    }
}

// One tile of class (D, N).  Operand tile xt: instance-major, column-major inside
// (linear).  Exchange layouts put each stage's output pairs next to each other:
//   2-D   W(l, j)    at j + KP l                 (stage 1 writes pairs along j)
//   3-D   T(i, j, k) at k + KP i + KP N j        (stage A: pairs along k)
//         U(i, j, k) at j + KP k + KP N i        (stage B: pairs along j)
//   out   Y(i, j, k) at i + KP (j + N k)         (last stage: pairs along i)
// The outputs are staged in the other operand buffer `ot` and copied to Y by
// consecutive threads.
template <typename S, int N, int D>
__device__ __forceinline__ void vl_tile(const VarlenArgs& a, int4 td, S* xt, S* ot, float* ex1, float* ex2,
                                        const int* yo) {
    constexpr int NX = ipow(N, D);
    constexpr int KP = vl_kp(N);
    constexpr int R = vl_rows(N) / 2;
    constexpr int EXQ = KP * ipow(N, D - 1);   // exchange / staging elements per instance
    const float* m1 = a.coef + vl_slot(D, N);
    const float* m2 = m1 + vl_rows(N) * N;
    const float* m3 = m2 + vl_rows(N) * N;
    const int cnt = td.z;
    const int tid = threadIdx.x;
    if constexpr (D == 2) {
        const int F = cnt * N;
        for (int f = tid; f < F; f += kVlThreads) {   // stage 1: mode 2, fibers (l, q)
            const int q = f / N, l = f - q * N;
            const S* xr = xt + q * NX + l;
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
            vl_stage_out<S, N>(ot + q * EXQ + KP * j, y);
        }
    } else {
        const int F = cnt * N * N;
        for (int f = tid; f < F; f += kVlThreads) {   // stage A: mode 3, fibers (i, j)
            const int q = f / (N * N), r = f - q * (N * N);
            const int i = r % N, j = r / N;
            const S* xr = xt + q * NX + i + N * j;
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
            vl_store_pairs<N>(ex2 + q * EXQ + KP * k + KP * N * i, u);
        }
        __syncthreads();
        for (int f = tid; f < F; f += kVlThreads) {   // stage C: mode 1, fibers (j, k)
            const int q = f / (N * N), r = f - q * (N * N);
            const int j = r % N, k = r / N;
            const float* ur = ex2 + q * EXQ + j + KP * k;
            float u[N];
#pragma unroll
            for (int l = 0; l < N; ++l) u[l] = ur[KP * N * l];
            f2 y[R];
            vl_contract<N>(m1, u, y);
            vl_stage_out<S, N>(ot + q * EXQ + KP * (j + N * k), y);
        }
    }
    __syncthreads();
    // coalesced copy of the finished instances to Y
    S* Y = static_cast<S*>(a.Y);
    const unsigned inv = a.cls[td.x].inv;
    for (int e = tid; e < cnt * NX; e += kVlThreads) {
        const int q = NX == 1 ? e : (int)__umulhi((unsigned)e, inv);
        const int r = e - q * NX;
        Y[(int64_t)yo[q] + r] = ot[q * EXQ + KP * (r / N) + r % N];
    }
}

template <typename S, int D>
__device__ __forceinline__ void vl_dispatch_n(const VarlenArgs& a, int4 td, S* xt, S* ot, float* ex1, float* ex2,
                                              const int* yo) {
    switch ((td.x & 15) + 1) {
        case 1: vl_tile<S, 1, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 2: vl_tile<S, 2, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 3: vl_tile<S, 3, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 4: vl_tile<S, 4, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 5: vl_tile<S, 5, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 6: vl_tile<S, 6, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 7: vl_tile<S, 7, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 8: vl_tile<S, 8, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 9: vl_tile<S, 9, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 10: vl_tile<S, 10, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 11: vl_tile<S, 11, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 12: vl_tile<S, 12, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 13: vl_tile<S, 13, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 14: vl_tile<S, 14, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 15: vl_tile<S, 15, D>(a, td, xt, ot, ex1, ex2, yo); break;
        case 16: vl_tile<S, 16, D>(a, td, xt, ot, ex1, ex2, yo); break;
    }
}

template <typename S>
__global__ void __launch_bounds__(kVlThreads) varlen_kernel(const __grid_constant__ VarlenArgs a, int xbuf_elems) {
    extern __shared__ __align__(128) unsigned char smem[];
    // Offsets of the instances of three consecutive tiles of this CTA (a ring):
    // X offsets then Y offsets, kVlThreads each (a tile has at most that many).
    int* ring = reinterpret_cast<int*>(smem);
    // One operand buffer: it is dead after the first contraction, so the last
    // contraction stages the outputs in it, and the next tile (held in registers
    // meanwhile) is committed into it after the copy-out.
    S* xb = reinterpret_cast<S*>(smem + 6 * kVlThreads * sizeof(int));
    float* ex1 = reinterpret_cast<float*>(
        smem + round_up(6 * kVlThreads * sizeof(int) + (size_t)xbuf_elems * sizeof(S), 128));
    const int G = gridDim.x;
    const int tid = threadIdx.x;
    const int t0 = blockIdx.x;
    if (t0 >= a.ntiles) return;
    const int4 none = make_int4(0, 0, 0, 0);
    // Pipeline: descriptors are read two tiles ahead, instance offsets one tile
    // ahead (through the ring), operand elements one tile ahead (registers), so no
    // global load is waited for at the start of a tile.
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
    S v[kVlRegs];
    vl_prefetch<S>(a, d0, ring, v);
    vl_commit<S>(d0, v, xb);
    __syncthreads();
    int it = 0;
    for (int tile = t0; tile < a.ntiles; ++it, tile += G) {
        const int s0 = it % 3, s1 = (it + 1) % 3, s2 = (it + 2) % 3;
        // offsets of tile + 2G, stored at the end of this tile
        int xo2 = 0, yo2 = 0;
        if (tid < d2.z) {
            xo2 = (int)a.xoff[d2.y + tid];
            yo2 = (int)a.yoff[d2.y + tid];
        }
        const int4 d3 = tile + 3 * G < a.ntiles ? a.tiles[tile + 3 * G] : none;
        if (d1.z) vl_prefetch<S>(a, d1, ring + 2 * kVlThreads * s1, v);
        const int key = d0.x;
        const int P = a.cls[key].P;
        const int n = (key & 15) + 1;
        // exchange buffer 2 starts after P * (per-instance size of buffer 1)
        float* ex2 = ex1 + (size_t)P * vl_kp(n) * (key < 16 ? n : n * n);
        const int* yo = ring + 2 * kVlThreads * s0 + kVlThreads;
        if (key < 16)
            vl_dispatch_n<S, 2>(a, d0, xb, xb, ex1, ex2, yo);
        else
            vl_dispatch_n<S, 3>(a, d0, xb, xb, ex1, ex2, yo);
        __syncthreads();   // outputs copied out before the next tile lands in xb
        if (d1.z) vl_commit<S>(d1, v, xb);
        if (tid < d2.z) {
            ring[2 * kVlThreads * s2 + tid] = xo2;
            ring[2 * kVlThreads * s2 + kVlThreads + tid] = yo2;
        }
        __syncthreads();
        d0 = d1;
        d1 = d2;
        d2 = d3;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static size_t vl_ex_floats(int kind, int n, int P) {
    const size_t exq = (size_t)vl_kp(n) * (kind == 2 ? n : n * n);
    return (size_t)P * exq * (kind == 2 ? 1 : 2);
}

static int vl_default_P(int kind, int n) {
    const int fpi = kind == 2 ? n : n * n;
    const int nx = kind == 2 ? n * n : n * n * n;
    int P = std::max(1, (kVlThreads + fpi - 1) / fpi);
    P = std::min(P, kVlMaxTile / nx);
    P = std::min(P, kVlThreads);
    return std::max(1, P);
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
    int xbuf_elems = 0;
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
        const int nx = kind == 2 ? n * n : n * n * n;
        const int P = p->P[key];
        const int64_t start = (int64_t)p->order.size();
        for (int64_t i : by[key]) p->order.push_back(i);
        const int64_t cnt = (int64_t)by[key].size();
        const int64_t flops = kind == 2 ? 4LL * n * n * n : 6LL * n * n * n * n;
        for (int64_t s = 0; s < cnt; s += P) {
            const int c = (int)std::min<int64_t>(P, cnt - s);
            tl.push_back(T{flops * c, make_int4(key, (int)(start + s), c, 0)});
        }
        max_x = std::max(max_x, (size_t)P * std::max(nx, (nx / n) * vl_kp(n)));   // operands / padded outputs
        max_smem_rest = std::max(max_smem_rest, vl_ex_floats(kind, n, P) * sizeof(float));
    }
    if (p->order.size() > (size_t)INT32_MAX) return KRON_ERR_NOT_SUPPORTED;
    std::stable_sort(tl.begin(), tl.end(), [](const T& a, const T& b) { return a.work > b.work; });
    for (const T& t : tl) p->tiles.push_back(t.td);
    p->xbuf_elems = (int)round_up(max_x, 64);
    p->smem = round_up(6 * kVlThreads * sizeof(int) + (size_t)p->xbuf_elems * es, 128) + max_smem_rest;
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
    int xbe = p->xbuf_elems;
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
        return (io == KRON_R64F) ? KRON_ERR_NOT_SUPPORTED : KRON_ERR_INVALID_VALUE;
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
        const int n = d.n, nn = n * n;
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
        const int nx = d.kind == 2 ? nn : nn * n;
        p->P[key] = (tp > 0 && tp * nx <= kVlMaxTile && tp <= kVlThreads) ? tp : vl_default_P(d.kind, n);
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
        const int nx = kind == 2 ? n * n : n * n * n;
        const int pmax = std::max(1, std::min(kVlThreads, kVlMaxTile / nx));
        const int cur = plan->P[key];
        int best_P = cur;
        for (int cand : {cur / 2, cur * 2, cur * 4, cur / 4, cur + cur / 2}) {
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
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan->smem) != cudaSuccess)
        return KRON_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kVlThreads, plan->smem) != cudaSuccess)
        return KRON_ERR_CUDA;
    int grid = std::max(1, per_sm) * dev.sms;
    grid = (int)std::min<size_t>((size_t)grid, plan->tiles.size());
    int xbe = plan->xbuf_elems;
    void* kargs[2] = {plan->args, &xbe};
    if (cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kVlThreads), kargs, plan->smem, st) != cudaSuccess)
        return KRON_ERR_CUDA;
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
