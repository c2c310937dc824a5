// 2-D pair kernels for n = 16 with the mode exchange done in place: FP32
// storage (pair16_kernel), and bf16 / f16 storage with FP32 arithmetic
// (pair16h_kernel, further below).
//
// The two contractions are those of the generic pair kernel (Sec. 2.1, the
// 2-D case of Algorithm 1: mode 2 with M2 = op(A) as pairs of fibers, then
// mode 1 with M1 = op(B) as pairs of rows), specialised to the paper's largest
// size in single precision:
//
//  * The intermediate W = X M2^T overwrites the operand tile: a thread reads
//    rows (l, l+1) of one instance into registers and writes rows (l, l+1) of
//    W to the same 32 words, and the second stage reads column j of W, whose
//    16 words no other thread touches.  The tile buffer is then the only
//    on-chip storage of a tile: 18 KB per tile, where the generic layout needs
//    54 KB for one tile and its exchange buffers.
//  * Instance q of a tile sits at word 288 q + r(q), with r(q) = 16 (q & 1) +
//    4 ((q >> 1) & 3).  The first stage (two instances per half-warp, 8-byte
//    accesses) and the second (eight instances per quarter-warp, 16-byte
//    accesses, one column each) then touch 32 distinct banks per access.
//  * The results overwrite W in place as well, and leave with one 1 KB bulk
//    copy (TMA) per instance, so L2 receives whole lines.
//  * One producer warp streams tiles in and results out through a ring of
//    buffers (full / empty mbarriers), one 1 KB bulk copy per instance each
//    way, both with an L2 evict-first policy (the data is streamed once); the
//    four compute warps never issue a global memory access (except the reads
//    of Y that beta != 0 needs).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "kron_pair.cuh"

namespace kron {

namespace {

constexpr int kN = 16, kNX = 256;
constexpr int kTileP = 16;                  // instances per tile
constexpr int kSlot = 288;                  // words between instance slots
constexpr int kTileWords = kTileP * kSlot;  // 18 KB per buffer
constexpr int kCompute = 128;               // compute threads (4 warps)
constexpr int kThreads = kCompute + 32;     // + one producer warp
constexpr int kMaxRing = 4;

__device__ __forceinline__ int slot_of(int q) { return kSlot * q + 16 * (q & 1) + 4 * ((q >> 1) & 3); }

__device__ __forceinline__ void load_col(const float* p, float (&w)[kN]) {
#pragma unroll
    for (int c = 0; c < kN / 4; ++c) {
        const float4 v = *reinterpret_cast<const float4*>(p + 4 * c);
        w[4 * c] = v.x;
        w[4 * c + 1] = v.y;
        w[4 * c + 2] = v.z;
        w[4 * c + 3] = v.w;
    }
}

__global__ void __launch_bounds__(kThreads, 6) pair16_kernel(const __grid_constant__ PairArgs<kN, 2> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxRing;
    float* ring = reinterpret_cast<float*>(smem + 128);
    const int NB = a.nstage;
    const int tid = threadIdx.x;
    const int64_t ntiles = (a.batch + kTileP - 1) / kTileP;
    const int64_t grid = gridDim.x;

    if (tid == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCompute);
        }
        fence_barrier_init();
    }
    __syncthreads();

    if (tid >= kCompute) {
        // Producer: tile `it` goes to buffer it % NB once the compute threads have
        // released that buffer's previous tile (it - NB), whose results they left
        // in the buffer: those are stored first, with one bulk copy per instance.
        const int lane = tid - kCompute;
        const uint64_t pol = l2_evict_first_policy();
        float* Y = static_cast<float*>(a.Y);
        auto store_tile = [&](int s, int64_t t) {
            const int64_t i0 = t * kTileP;
            const int c = (int)min((int64_t)kTileP, a.batch - i0);
            if (lane < c) {
                bulk_s2g_hint(Y + (i0 + lane) * kNX, ring + s * kTileWords + slot_of(lane), kNX * 4u, pol);
                bulk_commit();
            }
        };
        int it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
            const int s = it % NB;
            if (it >= NB) {
                if (!mbar_wait_bounded(&empty[s], (unsigned)(it / NB - 1) & 1u, a.err)) {
                    bulk_wait_all();
                    return;
                }
                store_tile(s, tile - (int64_t)NB * grid);
                bulk_wait_read();   // the results have left the buffer
            }
            const int64_t inst0 = tile * kTileP;
            const int cnt = (int)min((int64_t)kTileP, a.batch - inst0);
            float* buf = ring + s * kTileWords;
            // The compute threads' generic accesses to this buffer happen before their
            // arrival on empty[s]; order them before the bulk copies that overwrite it.
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(&full[s], (unsigned)cnt * kNX * 4u);
            __syncwarp();
            if (lane < cnt)
                bulk_g2s(buf + slot_of(lane), static_cast<const float*>(a.X) + (inst0 + lane) * kNX, kNX * 4u,
                         &full[s], pol);
        }
        for (int j = it > NB ? it - NB : 0; j < it; ++j) {   // the last tiles' results
            if (!mbar_wait_bounded(&empty[j % NB], (unsigned)(j / NB) & 1u, a.err)) break;
            store_tile(j % NB, blockIdx.x + (int64_t)j * grid);
        }
        bulk_wait_all();
        return;
    }

    const f2* m1p = reinterpret_cast<const f2*>(a.m1);
    const float* Y = static_cast<const float*>(a.Y);
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
        const int s = it % NB;
        float* buf = ring + s * kTileWords;
        const int64_t inst0 = tile * kTileP;
        const int cnt = (int)min((int64_t)kTileP, a.batch - inst0);
        const bool ok = (it == 0 && a.first_wait_ns)
                            ? mbar_wait_polled(&full[s], 0u, a.err, a.first_wait_ns)
                            : mbar_wait_bounded(&full[s], (unsigned)(it / NB) & 1u, a.err);

        // Stage 1: rows (l, l+1) of instance q times M2^T, written back in place.
        {
            const int q = tid >> 3, l = 2 * (tid & 7);
            if (q < cnt) {
                float* p = buf + slot_of(q) + l;
                f2 x[kN];
#pragma unroll
                for (int m = 0; m < kN; ++m) x[m] = *reinterpret_cast<const f2*>(p + kN * m);
                f2 w[kN];
                contract_dup<kN>(a.da, x, w);
#pragma unroll
                for (int j = 0; j < kN; ++j) *reinterpret_cast<f2*>(p + kN * j) = w[j];
            }
        }
        if (compute_sync_or(!ok)) {
            // A copy did not land in time: wait (bounded) for the ones that may still
            // be in flight into this CTA's buffers, then give up.  The producer cannot
            // issue beyond tile it + NB - 1, whose buffer this iteration still holds.
            if (tid == 0)
                for (int j = it; j < it + NB; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&full[j % NB], (unsigned)(j / NB) & 1u, a.err);
            return;
        }

        // Stage 2: column j of W of instance q times M1 (pairs of output rows); the
        // results overwrite the column.  Partial 16-byte stores from registers
        // would reach L2 as half sectors (1.7x the bytes of Y); the producer's
        // bulk copies write whole lines.
        const int q = tid & 15, j0 = tid >> 4;
        const bool live = q < cnt;
        float* wq = buf + slot_of(q);
        const float* yq = Y + (inst0 + q) * kNX;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + 8 * h;
            if (!live) continue;
            float w[kN];
            load_col(wq + kN * j, w);
            f2 y[kN / 2];
            contract_rows<kN>(m1p, w, y);
            if (!a.alpha_one) {
                const f2 al = f2_pack(a.alpha, a.alpha);
#pragma unroll
                for (int r = 0; r < kN / 2; ++r) y[r] = fmul2(y[r], al);
            }
            if (!a.beta_zero) {
                const f2 be = f2_pack(a.beta, a.beta);
#pragma unroll
                for (int r = 0; r < kN / 2; ++r) y[r] = ffma2(be, load_pair<float>(yq + kN * j + 2 * r), y[r]);
            }
#pragma unroll
            for (int c = 0; c < kN / 4; ++c)
                *reinterpret_cast<uint4*>(wq + kN * j + 4 * c) = make_uint4(
                    (unsigned)y[2 * c], (unsigned)(y[2 * c] >> 32), (unsigned)y[2 * c + 1], (unsigned)(y[2 * c + 1] >> 32));
        }
        fence_proxy_async_smem();   // results written: visible to the bulk stores
        mbar_arrive(&empty[s]);
    }
}

size_t pair16_smem_bytes(int nb) { return 128 + (size_t)nb * kTileWords * sizeof(float); }

// ---------------------------------------------------------------------------
// FP32, tiles moved by 3-D tensor copies (pair16t_kernel).  The same two
// contractions; a tile of P instances (P a multiple of 8) arrives and leaves
// by ONE tensor copy (cp.async.bulk.tensor) each way instead of one bulk copy
// per instance.  X and Y are described to the copy engine as 16 x 16 x batch
// arrays and the box is 20 x 17 x P: rows 16..19 and column 16 lie outside
// the array, so the loads fill them with zeros and the stores skip them, and
// in shared memory
//   element (i, j) of instance q sits at word i + 20 j + 340 q.
// A column stride of 20 words puts the 8 columns of a quarter-warp's 16-byte
// accesses on 8 distinct 4-bank groups (20 j mod 32 = 0, 20, 8, 28, 16, 4,
// 24, 12), and instances q and q + 4 lie 1360 = 16 (mod 32) words apart.  A
// warp owns the four instances {A, A+1, A+4, A+5} (A = 8 G + 2 u) through both
// stages, so the stages are separated by __syncwarp:
//   stage 1: lane (h, t) takes rows (2t, 2t+1) of instance A + (lane >> 4) +
//            4 h, h = (lane >> 3) & 1; a half-warp reads instances q and q + 4
//            with 8-byte accesses: 32 distinct banks.
//   stage 2: two passes, lanes 0-15 on instance A (then A + 4), lanes 16-31 on
//            A + 1 (A + 5), column j = lane & 15.
// Instances past the end of the batch are zero-filled by the load and skipped
// by the store, so the last tile needs no guard (except for beta's reads).
// ---------------------------------------------------------------------------
constexpr int kTRows = 20, kTCols = 17;
constexpr int kTInst = kTRows * kTCols;     // 340 words per instance
constexpr int kTMaxWarps = kPair16TMaxWarps;   // compute warps per CTA
constexpr int kTMaxRing = kPair16TMaxRing;

struct Pair16TArgs {   // 128-byte aligned (CUtensorMap)
    CUtensorMap tx, ty;                     // X, Y as 16 x 16 x batch FP32 arrays
    PairArgs<kN, 2> a;
    int groups;                             // compute groups of P / 4 warps; group g takes tiles it = g mod groups
};

__device__ __forceinline__ void tensor_load3(void* dst, const CUtensorMap* tm, int c2, uint64_t* bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"((unsigned long long)tm), "r"(0), "r"(0), "r"(c2), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void tensor_store3(const CUtensorMap* tm, int c2, const void* src, uint64_t pol) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2, %3}], [%4], %5;" ::
                     "l"((unsigned long long)tm), "r"(0), "r"(0), "r"(c2), "r"(smem_u32(src)), "l"(pol)
                 : "memory");
}

// bar.red.or over the `nthreads` threads that use named barrier `id`.
__device__ __forceinline__ bool sync_or_n(bool v, int id, int nthreads) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((unsigned)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(32 * (kTMaxWarps + 1), 1) pair16t_kernel(const __grid_constant__ Pair16TArgs ta) {
    const PairArgs<kN, 2>& a = ta.a;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kTMaxRing;
    float* ring = reinterpret_cast<float*>(smem + 256);
    const int NB = a.nstage;
    const int P = a.P;
    const int gwarps = P / 4;                  // warps of one compute group
    const int ncompute = 32 * gwarps * ta.groups;
    const int tileWords = P * kTInst;
    const unsigned tileBytes = (unsigned)tileWords * 4u;
    const int tid = threadIdx.x;
    const int ntiles = (int)((a.batch + P - 1) / P);
    const int grid = gridDim.x;

    if (tid == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 32 * gwarps);
        }
        fence_barrier_init();
    }
    __syncthreads();

    if (tid >= ncompute) {
        // Producer (one thread): tile `it` into buffer it % NB once the compute
        // warps released the buffer's previous tile, whose results leave first.
        if (tid != ncompute) return;
        const uint64_t pol = l2_evict_first_policy();
        int it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
            const int s = it % NB;
            float* buf = ring + s * tileWords;
            if (it >= NB) {
                if (!mbar_wait_bounded(&empty[s], (unsigned)(it / NB - 1) & 1u, a.err)) {
                    bulk_wait_all();
                    return;
                }
                tensor_store3(&ta.ty, (tile - NB * grid) * P, buf, pol);
                bulk_commit();
                bulk_wait_read();   // the results have left the buffer
            }
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&full[s], tileBytes);
            tensor_load3(buf, &ta.tx, tile * P, &full[s], pol);
        }
        for (int j = it > NB ? it - NB : 0; j < it; ++j) {   // the last tiles' results
            if (!mbar_wait_bounded(&empty[j % NB], (unsigned)(j / NB) & 1u, a.err)) break;
            tensor_store3(&ta.ty, (blockIdx.x + j * grid) * P, ring + (j % NB) * tileWords, pol);
            bulk_commit();
        }
        bulk_wait_all();
        return;
    }

    const f2* m1p = reinterpret_cast<const f2*>(a.m1);
    const float* Yg = static_cast<const float*>(a.Y);
    const int gidx = (tid >> 5) / gwarps;
    const int warp = (tid >> 5) - gidx * gwarps, lane = tid & 31;
    const int A = 8 * (warp >> 1) + 2 * (warp & 1);          // the warp's instances: A, A+1, A+4, A+5
    const int q1 = A + (lane >> 4) + 4 * ((lane >> 3) & 1);   // stage 1
    const int t1 = 2 * (lane & 7);
    const int j2 = lane & 15;                                 // stage 2
    const int G = ta.groups;
    for (int it = gidx, tile = blockIdx.x + gidx * grid; tile < ntiles; it += G, tile += G * grid) {
        const int s = it % NB;
        float* buf = ring + s * tileWords;
        const int64_t inst0 = (int64_t)tile * P;
        const int cnt = (int)min((int64_t)P, a.batch - inst0);
        const bool ok = (it < G && a.first_wait_ns)
                            ? mbar_wait_polled(&full[s], (unsigned)(it / NB) & 1u, a.err, a.first_wait_ns)
                            : mbar_wait_bounded(&full[s], (unsigned)(it / NB) & 1u, a.err);
        if (sync_or_n(!ok, 1 + gidx, 32 * gwarps)) {
            // A copy did not land in time: wait (bounded) for the ones that may still
            // be in flight into this CTA's buffers, then give up.
            if (warp == 0 && lane == 0)
                for (int j = it; j < it + NB; ++j)
                    if (blockIdx.x + j * grid < ntiles)
                        mbar_wait_bounded(&full[j % NB], (unsigned)(j / NB) & 1u, a.err);
            return;
        }
        // ---- stage 1: rows (t1, t1+1) of instance q1 times M2^T, in place ----
        {
            float* p = buf + q1 * kTInst + t1;
            f2 x[kN];
#pragma unroll
            for (int m = 0; m < kN; ++m) x[m] = *reinterpret_cast<const f2*>(p + kTRows * m);
            f2 w[kN];
            contract_dup<kN>(a.da, x, w);
#pragma unroll
            for (int j = 0; j < kN; ++j) *reinterpret_cast<f2*>(p + kTRows * j) = w[j];
        }
        __syncwarp();
        // ---- stage 2: column j2 of W times M1, in place; two instances per pass ----
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int q = A + (lane >> 4) + 4 * h;
            float* col = buf + q * kTInst + kTRows * j2;
            float w[kN];
            load_col(col, w);
            f2 y[kN / 2];
            contract_rows<kN>(m1p, w, y);
            if (!a.alpha_one) {
                const f2 al = f2_pack(a.alpha, a.alpha);
#pragma unroll
                for (int r = 0; r < kN / 2; ++r) y[r] = fmul2(y[r], al);
            }
            if (!a.beta_zero && q < cnt) {
                const f2 be = f2_pack(a.beta, a.beta);
                const float* yg = Yg + (inst0 + q) * kNX + kN * j2;
#pragma unroll
                for (int r = 0; r < kN / 2; ++r) y[r] = ffma2(be, load_pair<float>(yg + 2 * r), y[r]);
            }
#pragma unroll
            for (int c = 0; c < kN / 4; ++c)
                *reinterpret_cast<uint4*>(col + 4 * c) = make_uint4(
                    (unsigned)y[2 * c], (unsigned)(y[2 * c] >> 32), (unsigned)y[2 * c + 1], (unsigned)(y[2 * c + 1] >> 32));
        }
        fence_proxy_async_smem();   // results written: visible to the tensor store
        mbar_arrive(&empty[s]);
    }
}

size_t pair16t_smem_bytes(int P, int nb) { return 256 + (size_t)nb * P * kTInst * sizeof(float); }

// cuTensorMapEncodeTiled from the driver, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// X or Y as a 16 x 16 x batch FP32 array, copied in boxes of 20 x 17 x P.
bool encode_inst_map(CUtensorMap* m, const void* base, int64_t batch, int P) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {16, 16, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {16 * sizeof(float), 256 * sizeof(float)};
    const cuuint32_t box[3] = {kTRows, kTCols, (cuuint32_t)P};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// 16-bit storage (bf16, f16), FP32 arithmetic.  W (FP32) cannot overwrite a
// 16-bit operand, so it has its own buffer -- laid out as the FP32 kernel's
// tile, conflict-free -- while the results overwrite the dead operand slots
// and leave by bulk copy.  Operand slot q (two 16-bit elements per 32-bit
// word) starts at word 136 q + 4 ((q >> 2) & 1): the first stage's 32-bit
// reads (four instances per warp) and the second stage's 16-byte result
// writes (eight instances per quarter-warp) touch distinct banks.
// ---------------------------------------------------------------------------
constexpr int kHSlotWords = 136;
constexpr int kHTileBytes = 8704;                // 16 slots, rounded to 128 bytes
constexpr int kHWBytes = kTileWords * 4;         // W: the FP32 tile layout

__device__ __forceinline__ int hslot_words(int q) { return kHSlotWords * q + 4 * ((q >> 2) & 1); }

template <typename S>
__global__ void __launch_bounds__(kThreads) pair16h_kernel(const __grid_constant__ PairArgs<kN, 2> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + kMaxRing;
    const int NB = a.nstage;
    unsigned char* ring = smem + 128;
    float* W = reinterpret_cast<float*>(ring + NB * kHTileBytes);
    const int tid = threadIdx.x;
    const int64_t ntiles = (a.batch + kTileP - 1) / kTileP;
    const int64_t grid = gridDim.x;
    if (tid == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCompute);
        }
        fence_barrier_init();
    }
    __syncthreads();

    if (tid >= kCompute) {   // producer: 512-byte bulk copies, one per instance
        const int lane = tid - kCompute;
        const uint64_t pol = l2_evict_first_policy();
        S* Y = static_cast<S*>(a.Y);
        const S* X = static_cast<const S*>(a.X);
        auto slot = [&](int s, int q) { return reinterpret_cast<unsigned*>(ring + s * kHTileBytes) + hslot_words(q); };
        auto store_tile = [&](int s, int64_t t) {
            const int64_t i0 = t * kTileP;
            const int c = (int)min((int64_t)kTileP, a.batch - i0);
            if (lane < c) bulk_s2g_hint(Y + (i0 + lane) * kNX, slot(s, lane), kNX * 2u, pol);
            bulk_commit();
        };
        int it = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
            const int s = it % NB;
            if (it >= NB) {
                if (!mbar_wait_bounded(&empty[s], (unsigned)(it / NB - 1) & 1u, a.err)) {
                    bulk_wait_all();
                    return;
                }
                store_tile(s, tile - (int64_t)NB * grid);
                bulk_wait_read();
            }
            const int64_t inst0 = tile * kTileP;
            const int cnt = (int)min((int64_t)kTileP, a.batch - inst0);
            fence_proxy_async_smem();
            if (lane == 0) mbar_arrive_expect_tx(&full[s], (unsigned)cnt * kNX * 2u);
            __syncwarp();
            if (lane < cnt) bulk_g2s(slot(s, lane), X + (inst0 + lane) * kNX, kNX * 2u, &full[s], pol);
        }
        for (int j = it > NB ? it - NB : 0; j < it; ++j) {
            if (!mbar_wait_bounded(&empty[j % NB], (unsigned)(j / NB) & 1u, a.err)) break;
            store_tile(j % NB, blockIdx.x + (int64_t)j * grid);
        }
        bulk_wait_all();
        return;
    }

    const f2* m1p = reinterpret_cast<const f2*>(a.m1);
    const S* Yg = static_cast<const S*>(a.Y);
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += grid, ++it) {
        const int s = it % NB;
        unsigned* tw = reinterpret_cast<unsigned*>(ring + s * kHTileBytes);
        const int64_t inst0 = tile * kTileP;
        const int cnt = (int)min((int64_t)kTileP, a.batch - inst0);
        const bool ok = mbar_wait_bounded(&full[s], (unsigned)(it / NB) & 1u, a.err);
        compute_sync_or(false);   // the previous tile's second stage has read W
        // Stage 1: rows (l, l+1) of instance q (one 32-bit word per column) times M2^T.
        {
            const int q = tid >> 3, l = 2 * (tid & 7);
            if (q < cnt) {
                const S* xq = reinterpret_cast<const S*>(tw + hslot_words(q)) + l;
                f2 x[kN], w[kN];
#pragma unroll
                for (int m = 0; m < kN; ++m) x[m] = load_pair<S>(xq + kN * m);
                contract_dup<kN>(a.da, x, w);
                float* wq = W + slot_of(q) + l;
#pragma unroll
                for (int j = 0; j < kN; ++j) *reinterpret_cast<f2*>(wq + kN * j) = w[j];
            }
        }
        if (compute_sync_or(!ok)) {
            if (tid == 0)
                for (int j = it; j < it + NB; ++j)
                    if (blockIdx.x + (int64_t)j * grid < ntiles)
                        mbar_wait_bounded(&full[j % NB], (unsigned)(j / NB) & 1u, a.err);
            return;
        }
        // Stage 2: column j of W times M1; the 16-bit results go over the operand slot.
        const int q = tid & 15, j0 = tid >> 4;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + 8 * h;
            if (q >= cnt) continue;
            float w[kN];
            load_col(W + slot_of(q) + kN * j, w);
            f2 y[kN / 2];
            contract_rows<kN>(m1p, w, y);
            if (!a.alpha_one) {
                const f2 al = f2_pack(a.alpha, a.alpha);
#pragma unroll
                for (int r = 0; r < kN / 2; ++r) y[r] = fmul2(y[r], al);
            }
            if (!a.beta_zero) {
                const S* yg = Yg + (inst0 + q) * kNX + kN * j;
                const f2 be = f2_pack(a.beta, a.beta);
#pragma unroll
                for (int r = 0; r < kN / 2; ++r) y[r] = ffma2(be, load_pair<S>(yg + 2 * r), y[r]);
            }
            unsigned* yw = tw + hslot_words(q) + (kN / 2) * j;
#pragma unroll
            for (int c = 0; c < kN / 8; ++c)
                *reinterpret_cast<uint4*>(yw + 4 * c) = make_uint4(pack16<S>(y[4 * c]), pack16<S>(y[4 * c + 1]),
                                                                   pack16<S>(y[4 * c + 2]), pack16<S>(y[4 * c + 3]));
        }
        fence_proxy_async_smem();
        mbar_arrive(&empty[s]);
    }
}

size_t pair16h_smem_bytes(int nb) { return 128 + (size_t)nb * kHTileBytes + kHWBytes; }

}  // namespace

// 2-D, n = 16, FP32 arithmetic on FP32, bf16 or f16 storage, contiguous X and Y.
// Tile sizes other than 16 instances are left to the generic pair kernel.
kron_status launch_pair16(const KronDesc& d, cudaStream_t st) {
    if (d.D != 2 || d.N != kN || d.io == KRON_R64F || d.comp != KRON_COMPUTE_NATIVE || !d.contiguous ||
        !d.ycontig)
        return KRON_ERR_NOT_SUPPORTED;
    // FP32: the tensor-copy body (tiles of 8, 16, 24 or 32 instances); the slot
    // body below serves 16-bit storage, and FP32 where tensor maps cannot
    // describe the batch (2^31 instances or more) or are unavailable.
    const bool tens = d.io == KRON_R32F && d.batch < (1ll << 31) - 64 &&
                      (d.P <= 0 || (d.P % 8 == 0 && d.P <= 32));
    if (!tens && d.P > 0 && d.P != kTileP) return KRON_ERR_NOT_SUPPORTED;
    const DeviceInfo& dev = device_info();
    if (dev.sms <= 0) return KRON_ERR_CUDA;
    PairArgs<kN, 2> a;
    auto dup = [](double x) {
        const float v = (float)x;
        unsigned b;
        memcpy(&b, &v, sizeof(b));
        return ((f2)b << 32) | (f2)b;
    };
    for (int e = 0; e < kN * kN; ++e) {
        a.da[e] = dup(d.m2[e]);
        a.m1[e] = (float)d.m1[e];
    }
    a.db[0] = 0;
    a.X = d.X;
    a.Y = d.Y;
    a.batch = d.batch;
    a.alpha = (float)d.alpha;
    a.beta = (float)d.beta;
    a.beta_zero = d.beta == 0.0;
    a.alpha_one = d.alpha == 1.0;
    a.err = device_error_word();
    if (!a.err) return KRON_ERR_CUDA;
    a.first_wait_ns = d.io == KRON_R32F ? first_wait_limit_ns() : 0;
    if (tens) {
        Pair16TArgs ta;
        // Measured default: 16-instance tiles, an eight-deep ring and four groups
        // of four compute warps -- one CTA per SM holding 170 KB of tiles.
        const int P = d.P > 0 ? d.P : kPair16TDefaultP;
        if (encode_inst_map(&ta.tx, d.X, d.batch, P) && encode_inst_map(&ta.ty, d.Y, d.batch, P)) {
            const int warps = d.warps > 0 ? d.warps : kPair16TMaxWarps;
            const int groups = warps / (P / 4);
            if (groups < 1 || warps % (P / 4) || warps > kTMaxWarps) return KRON_ERR_NOT_SUPPORTED;
            ta.groups = groups;
            // The ring depth is a multiple of the number of groups: buffer it % NB
            // then always passes from a group to the same group (tile it - NB), so
            // a group starts its parity wait on a buffer only after its own
            // previous use of it has completed (a parity wait cannot tell phase u
            // from phase u - 2).
            int nb = d.nstage >= 1 ? d.nstage : 2 * groups;
            if (nb > kTMaxRing) nb = kTMaxRing;
            nb = nb < groups ? groups : nb / groups * groups;
            if (nb > kTMaxRing) return KRON_ERR_NOT_SUPPORTED;
            size_t smem = pair16t_smem_bytes(P, nb);
            while (nb > groups && smem > dev.smem_per_block_optin) smem = pair16t_smem_bytes(P, nb -= groups);
            if (smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
            a.P = P;
            a.nstage = nb;
            ta.a = a;
            const void* kern = (const void*)pair16t_kernel;
            if (!ensure_smem_optin(kern, smem)) return KRON_ERR_CUDA;
            const int threads = 32 * (groups * (P / 4) + 1);
            const int64_t ntiles = (d.batch + P - 1) / P;
            int64_t grid = d.grid;
            if (grid <= 0) {
                int per_sm = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess)
                    return KRON_ERR_CUDA;
                grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
            }
            if (grid > ntiles) grid = ntiles;
            if (grid < 1) grid = 1;
            void* args[] = {&ta};
            if (cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(threads), args, smem, st) != cudaSuccess)
                return KRON_ERR_CUDA;
            return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
        }
        if (d.P > 0 && d.P != kTileP) return KRON_ERR_NOT_SUPPORTED;
    }
    a.P = kTileP;
    // FP32: one buffer per CTA (measured best: the six to seven resident CTAs
    // per SM overlap one another's copies; a second buffer costs resident CTAs).
    // 16-bit: two (the tiles are half the size; measured 8 % faster than one).
    const bool h = d.io != KRON_R32F;
    int nb = d.nstage >= 1 ? d.nstage : (h ? 2 : 1);
    if (nb > kMaxRing) nb = kMaxRing;
    auto smem_of = [&](int n_b) { return h ? pair16h_smem_bytes(n_b) : pair16_smem_bytes(n_b); };
    size_t smem = smem_of(nb);
    while (nb > 1 && smem > dev.smem_per_block_optin) smem = smem_of(--nb);
    if (smem > dev.smem_per_block_optin) return KRON_ERR_NOT_SUPPORTED;
    a.nstage = nb;
    const void* kern = !h ? (const void*)pair16_kernel
                          : (d.io == KRON_R16BF ? (const void*)pair16h_kernel<__nv_bfloat16>
                                                : (const void*)pair16h_kernel<__half>);
    if (!ensure_smem_optin(kern, smem)) return KRON_ERR_CUDA;
    const int64_t ntiles = (d.batch + kTileP - 1) / kTileP;
    int64_t grid = d.grid;
    if (grid <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess)
            return KRON_ERR_CUDA;
        grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * dev.sms;
    }
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    void* args[] = {&a};
    if (cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(kThreads), args, smem, st) != cudaSuccess)
        return KRON_ERR_CUDA;
    return cudaPeekAtLastError() == cudaSuccess ? KRON_OK : KRON_ERR_CUDA;
}

}  // namespace kron
