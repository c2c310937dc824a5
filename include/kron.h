/*
 * kron.h -- C ABI of the GB300 batched Kronecker product library.
 *
 * Operation (paper Sec. 2.2, "Batched Kronecker products"): for p = 0..N-1
 *
 *   2-D:  vec(Y^p) <- alpha (op(A) (x) op(B)) vec(op(X^p)) + beta vec(Y^p)
 *         i.e.  Y^p = alpha op(B) op(X^p) op(A)^T + beta Y^p          (Sec. 2, vec identity)
 *   3-D:  vec(Y^p) <- alpha (op(A) (x) op(B) (x) op(C)) vec(X^p) + beta vec(Y^p)
 *         i.e.  Y^p[i,j,k] = alpha sum_{l,m,q} op(C)[i,l] op(B)[j,m] op(A)[k,q] X^p[l,m,q]
 *                            + beta Y^p[i,j,k]                          (Sec. 2.1, triple sum)
 *
 * The component matrices A, B (, C) are the same for the whole batch; the
 * operands X^p and results Y^p vary (Sec. 2.2).  Arrays are column-major
 * (Sec. 3).  The LAST Kronecker factor acts on the FASTEST (first) mode.
 *
 * Relation to the paper's TKRON2/TKRON3 (Sec. 3): the paper writes the 2-D
 * operator as B (x) A with Y = A X B^T and the 3-D one as C (x) B (x) A with A on
 * mode 1.  Hence   TKRON2(A, B, ...)    == kron2_batched(.., B, .., A, ..)
 * and              TKRON3(A, B, C, ...) == kron3_batched(.., C, .., B, .., A, ..)
 * (component arguments in reverse order; all other arguments keep their meaning).
 *
 * Conventions shared by every entry point
 *  - Status codes are returned, never thrown; all validation happens before any
 *    launch, so nothing is written when a call returns an error.
 *  - X, Y: DEVICE pointers owned by the caller.  X is read-only.  X and Y must
 *    not overlap (KRON_ERR_ALIAS); the operation is out of place.
 *  - A, B, C: HOST pointers to the components, read during the call and passed
 *    by value to the kernel (they are at most 3 x 16 x 16 values and constant
 *    over the batch; Sec. 2.2 notes that transposing them once up front costs
 *    little, which is what the library does).  After the call returns the host
 *    arrays may be reused.  Type: float for KRON_R32F / KRON_R16BF / KRON_R16F
 *    storage, double for KRON_R64F, interleaved complex float / double pairs
 *    for KRON_C32F / KRON_C64F (the complex field of Sec. 2).
 *  - alpha, beta: HOST pointers to scalars of the same type as the components.
 *    beta == 0 means Y is not read (NaN/Inf in Y are ignored, BLAS convention).
 *  - trans arguments: 'N' = op(M) = M, 'T' = M^T, 'C' = M^H, the Hermitian
 *    transpose (Sec. 2.2); for real storage 'C' is 'T'.
 *  - Leading dimensions are in elements (Sec. 3): ldx = column stride, ldx2 =
 *    plane stride (3-D), ldxp = offset between consecutive instances ("uniform
 *    offset from the previous entity").  ldxp may be 0 (one X for every p).
 *  - Sizes: every dimension in 1..16 (the paper's range, Sec. 1).
 *  - batch_count == 0 is a no-op returning KRON_OK.
 *  - The library never allocates device memory inside these calls (Sec. 4,
 *    work-array discussion): the fixed-size paths need no workspace and the
 *    mixed-size path takes a caller-owned workspace.
 *  - Calls are asynchronous on `stream` (NULL = legacy default stream).  A
 *    launch failure is reported as KRON_ERR_CUDA.  Device-side waits are
 *    bounded; an expired wait is recorded in a device status word read back by
 *    kron_device_status().
 */
#ifndef KRON_GB300_H
#define KRON_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KRON_API __attribute__((visibility("default")))

typedef struct CUstream_st* kron_stream_t; /* same type as cudaStream_t / CUstream */

typedef enum {
    KRON_OK = 0,
    KRON_ERR_INVALID_VALUE = 1,   /* a size, stride, flag or pointer argument is invalid */
    KRON_ERR_NOT_SUPPORTED = 2,   /* valid but not implemented (e.g. compute mode / dtype pair) */
    KRON_ERR_ALIAS = 3,           /* the X and Y address ranges overlap */
    KRON_ERR_WORKSPACE = 4,       /* workspace missing, too small or misaligned */
    KRON_ERR_CUDA = 5,            /* a CUDA runtime call failed (launch, graph, device query) */
    KRON_ERR_DEVICE_TIMEOUT = 6   /* a bounded device-side wait expired */
} kron_status;

/* Storage type of X and Y. */
typedef enum {
    KRON_R32F = 0,   /* float;  components/alpha/beta float  */
    KRON_R64F = 1,   /* double; components/alpha/beta double */
    KRON_R16BF = 2,  /* bfloat16 operands, FP32 accumulation; components float */
    KRON_R16F = 3,   /* float16 operands, FP32 accumulation; components float */
    KRON_C32F = 4,   /* complex float, interleaved (re, im); components/alpha/beta complex float */
    KRON_C64F = 5    /* complex double, interleaved (re, im); components/alpha/beta complex double */
} kron_dtype;

/* How the contractions are computed. */
typedef enum {
    /* CUDA cores: FP32 FMA for R32F/R16BF/R16F storage, FP64 FMA for R64F. */
    KRON_COMPUTE_NATIVE = 0,
    /* Tensor cores, split precision: each FP32 value v = hi + lo with hi, lo
       bfloat16 (round to nearest even); products hi*hi + hi*lo + lo*hi are
       accumulated in FP32.  Valid for R32F and R16BF storage. */
    KRON_COMPUTE_32F_BF16X3 = 1
} kron_compute;

KRON_API const char* kron_status_string(kron_status s);

/* Library version as 10000*major + 100*minor + patch. */
KRON_API int kron_version(void);

/*
 * kron_check_device_buffer -- the check every call makes on its X, Y (and
 * workspace) before launching: KRON_OK when [p, p + bytes) is device memory of
 * the current GPU or managed memory, mapped without a hole: one allocation, or
 * adjacent mapped ranges (allocators that map memory in chunks through the
 * virtual memory management API report one range per chunk).
 * KRON_ERR_INVALID_VALUE for a null, host or unregistered pointer, memory of
 * another GPU, or an extent past the end of the mapping (such a launch would
 * fault); KRON_ERR_CUDA when no device is usable.  Launches nothing.
 */
KRON_API kron_status kron_check_device_buffer(const void* p, size_t bytes);

/*
 * kron2_batched -- the paper's TKRON2 (Sec. 3) with the component order above.
 *
 *   op(A): ma x na, stored as A (lda >= rows of the stored matrix: ma if
 *          transa = 'N', na if 'T')
 *   op(B): mb x nb, stored as B (ldb likewise)
 *   op(X^p): nb x na; X^p is stored at X + p*ldxp with column stride ldx
 *          (ldx >= nb if transx = 'N', >= na if 'T')
 *   Y^p:   mb x ma at Y + p*ldyp, column stride ldy >= mb,
 *          ldyp >= ldy*(ma-1) + mb (instances of Y must not overlap)
 *   trans*: 'N'/'n' = no transpose, 'T'/'t' = transpose, 'C'/'c' = Hermitian
 *          transpose (= 'T' for real data); transx = 'C' conjugates X^p
 *
 * Complex storage (KRON_C32F, KRON_C64F) runs on the CUDA cores
 * (KRON_COMPUTE_NATIVE; the split tensor path is for real data).
 *
 * Errors: KRON_ERR_INVALID_VALUE (bad size, ld, trans, null pointer with
 * batch_count > 0, negative batch or stride), KRON_ERR_NOT_SUPPORTED (compute
 * mode not available for io), KRON_ERR_ALIAS (X and Y ranges overlap),
 * KRON_ERR_CUDA (launch failed).
 */
KRON_API kron_status kron2_batched(kron_stream_t stream, char transa, char transb, char transx,
                                   int ma, int na, int mb, int nb, int64_t batch_count,
                                   const void* alpha, const void* A, int lda, const void* B,
                                   int ldb, const void* X, int ldx, int64_t ldxp,
                                   const void* beta, void* Y, int ldy, int64_t ldyp,
                                   kron_dtype io, kron_compute comp);

/*
 * kron3_batched -- the paper's TKRON3 (Sec. 3) with the component order above;
 * like the paper, no transpose of X.
 *
 *   op(A): ma x na (mode 3), op(B): mb x nb (mode 2), op(C): mc x nc (mode 1)
 *   X^p: nc x nb x na at X + p*ldxp, element (l,m,q) at l + ldx*m + ldx2*q,
 *        ldx >= nc, ldx2 >= ldx*nb
 *   Y^p: mc x mb x ma at Y + p*ldyp, element (i,j,k) at i + ldy*j + ldy2*k,
 *        ldy >= mc, ldy2 >= ldy*mb, ldyp >= ldy2*(ma-1) + ldy*(mb-1) + mc
 *
 * The three mode contractions (Algorithm 1's 2-D step per plane, then the third
 * mode) are fused in one kernel; no intermediate array goes to device memory.
 * Errors: as kron2_batched.
 */
KRON_API kron_status kron3_batched(kron_stream_t stream, char transa, char transb, char transc,
                                   int ma, int na, int mb, int nb, int mc, int nc,
                                   int64_t batch_count, const void* alpha, const void* A, int lda,
                                   const void* B, int ldb, const void* C, int ldc, const void* X,
                                   int ldx, int ldx2, int64_t ldxp, const void* beta, void* Y,
                                   int ldy, int ldy2, int64_t ldyp, kron_dtype io,
                                   kron_compute comp);

/*
 * kron1_batched -- the paper's TKRON1 (Sec. 3), the 1-D product ("almost a
 * batched GEMV"):
 *
 *   y^p <- alpha op(A) x^p + beta y^p,  p = 0 .. batch_count-1
 *
 *   op(A): ma x na (1 <= ma, na <= 16), stored as A, host pointer (FP64 for
 *          KRON_R64F, FP32 otherwise), lda >= ma if transa = 'N', >= na if 'T'
 *   x^p:   na contiguous elements at X + p*ldxp (device), ldxp >= 0
 *   y^p:   ma contiguous elements at Y + p*ldyp (device), ldyp >= ma when
 *          batch_count > 1 (outputs may not overlap)
 *
 * The paper prints both vector strides under one name; they are read as the X
 * and the Y stride.  alpha, beta: host scalars of the compute type; beta = 0
 * means Y is not read.  Storage: any real kron_dtype (complex storage returns
 * KRON_ERR_NOT_SUPPORTED); compute: KRON_COMPUTE_NATIVE only
 * (KRON_ERR_NOT_SUPPORTED otherwise).  Errors: KRON_ERR_INVALID_VALUE
 * (bad size, ld, stride, trans, null pointer with batch_count > 0),
 * KRON_ERR_ALIAS (X and Y ranges overlap), KRON_ERR_CUDA.  batch_count = 0 is a
 * no-op.  It runs on the kron_gemm_a_batched kernel with m = 1.
 */
KRON_API kron_status kron1_batched(kron_stream_t stream, char transa, int ma, int na, int64_t batch_count,
                                   const void* alpha, const void* A, int lda, const void* X, int64_t ldxp,
                                   const void* beta, void* Y, int64_t ldyp, kron_dtype io,
                                   kron_compute comp);

/*
 * kron_gemm_a_batched -- the paper's TGEMM_A (Sec. 3): a batched GEMM whose
 * first factor varies across the batch and whose second is shared,
 *
 *   C^p <- alpha op(A^p) op(B) + beta C^p,  p = 0 .. batch_count-1
 *
 *   op(A^p): m x k (1 <= m <= 2^24, 1 <= k <= 16) at A + p*lda2 (device),
 *            column stride lda >= m if transa = 'N', >= k if 'T'; lda2 >= 0
 *            (instances of A may overlap; 0 repeats one matrix)
 *   op(B):   k x n (1 <= n <= 16), stored as B, host pointer (FP64 for
 *            KRON_R64F, FP32 otherwise), ldb >= k if transb = 'N', >= n if 'T'
 *   C^p:     m x n at C + p*ldc2 (device), column stride ldc >= m,
 *            ldc2 >= ldc*(n-1) + m when batch_count > 1
 *   grid_size: CTAs to launch; 0 = one persistent wave (the paper's interface
 *            carries the same launch knob)
 *
 * The paper uses it for the third mode of its 3-D algorithm (Algorithm 1):
 * with tmp^p the (mc mb) x na result of the 2-D product on every plane,
 * Y^p = tmp^p op(A)^T.  Storage: any real kron_dtype (complex storage returns
 * KRON_ERR_NOT_SUPPORTED); compute: KRON_COMPUTE_NATIVE only.  Errors as kron1_batched (KRON_ERR_ALIAS when the A and C ranges
 * overlap).
 */
KRON_API kron_status kron_gemm_a_batched(kron_stream_t stream, char transa, char transb, int m, int n, int k,
                                         const void* alpha, const void* A, int lda, int64_t lda2,
                                         const void* B, int ldb, const void* beta, void* C, int ldc,
                                         int64_t ldc2, int64_t batch_count, int grid_size, kron_dtype io,
                                         kron_compute comp);

/*
 * kron_device_status -- synchronises `stream`, then reads and clears the
 * device status word of the current device.  Returns KRON_OK, or
 * KRON_ERR_DEVICE_TIMEOUT if a kernel gave up on a bounded wait since the last
 * call (its outputs for that launch are then incomplete), or KRON_ERR_CUDA.
 */
KRON_API kron_status kron_device_status(kron_stream_t stream);

/*
 * kron_set_first_wait_limit_ns -- a test aid for the failure path, off by
 * default (0).  With ns > 0, the first operand wait of every CTA (of every
 * compute group of a CTA) of later launches of the 2-D n = 16 FP32 kernel (kron2_batched, contiguous FP32
 * batches, n = 16) polls for at most ns nanoseconds instead of the normal
 * limit.  A limit shorter than an operand copy takes to land makes that real
 * wait expire on a normal launch: the kernel records the expiry in the device
 * status word (kron_device_status then returns KRON_ERR_DEVICE_TIMEOUT), waits
 * with the normal bound for its copies still in flight, and returns; the
 * outputs of that launch are incomplete.  Every other wait keeps the normal
 * limit (2 s).  Process-wide.  Errors: KRON_ERR_INVALID_VALUE for ns above the
 * normal limit.
 */
KRON_API kron_status kron_set_first_wait_limit_ns(unsigned long long ns);

/*
 * kron_peak_probe -- a measurement aid with no computation of the operation:
 * the roofline of the CUDA-core contraction kernels is the FMA throughput the
 * chip sustains (the paper quotes its GPU's peaks from the data sheet, Sec. 5;
 * here they are measured).  Launches one kernel on `stream` that runs only
 * independent FMA chains, with operands in registers, on every SM, and returns
 * in *flops the floating-point operations of that launch (2 per FMA).  The
 * caller times the launch (CUDA events on `stream`).
 *   unit 0: FP32, packed two-lane fma.rn.f32x2 (the form the FP32 kernels use)
 *   unit 1: FP32, scalar fma.rn.f32
 *   unit 2: FP64, fma.rn.f64
 * iters: loop trips, 1 .. 2^24; each trip is 32 FMA instructions per thread.
 * Errors: KRON_ERR_INVALID_VALUE (unit, iters or flops), KRON_ERR_CUDA (launch).
 */
KRON_API kron_status kron_peak_probe(kron_stream_t stream, int unit, int iters, double* flops);

/*
 * Tile configuration of the fixed-size kernels, per (kind, n, io, comp):
 * instances processed per CTA tile and depth of the bulk-copy pipeline (both 0
 * = built-in default).  kron_autotune times the candidate configurations on the
 * caller's buffers (contiguous X and Y of batch_count instances, minimal
 * leading dimensions; Y is overwritten; each candidate is timed as the best of
 * three rounds of ten launches), keeps the fastest in the process-wide table
 * unless it beats the built-in default by less than 2% (then the default, 0 0,
 * is kept), appends the choice to the file named by KRON_TUNE_CACHE (if set;
 * read at first use; later lines override earlier ones), and returns it.
 *
 * For contiguous batches the tile size also chooses the kernel: the in-place
 * kernels take their own tile shapes (2-D n = 16: FP32 8, 16, 24 or 32
 * instances, 16-bit storage 16; the rest FP32 only: 2-D
 * n = 10, 14: multiples of 8; 3-D n = 16: 1; 3-D n = 10, 14: 4; odd n: multiples
 * of 4), and any other tile size runs the generic kernel of that shape.  Every
 * configuration computes the same result within the documented tolerance.
 *
 * Errors: KRON_ERR_INVALID_VALUE for bad arguments, KRON_ERR_CUDA if a timing
 * call fails.
 */
KRON_API kron_status kron_set_tile_config(int kind, int n, kron_dtype io, kron_compute comp,
                                          int instances_per_tile, int pipeline_depth);
KRON_API kron_status kron_get_tile_config(int kind, int n, kron_dtype io, kron_compute comp,
                                          int* instances_per_tile, int* pipeline_depth);
KRON_API kron_status kron_autotune(kron_stream_t stream, int kind, int n, int64_t batch_count,
                                   const void* X, void* Y, kron_dtype io, kron_compute comp,
                                   int* instances_per_tile, int* pipeline_depth);

/*
 * Full kernel configuration of a fixed-size (kind, n, io, comp), the search
 * space of the autotuner.  The paper fixes one launch shape (5000 thread
 * blocks, Sec. 5); here the body, the tile, the copy pipeline and the register
 * blocking are chosen per configuration and per GPU.
 *
 *   variant:            the kernel body for contiguous batches (kron_variant);
 *                       KRON_VARIANT_AUTO = the built-in choice
 *   instances_per_tile: instances per CTA tile (0 = the body's default; the in-
 *                       place bodies take the tile shapes listed above)
 *   pipeline_depth:     tiles in flight per CTA (0 = default, 1..8)
 *   fibers_per_step:    register blocking of the last contraction of the
 *                       packed-pair bodies: 1 or 2 fibers per thread and step
 *                       (0 = default); for the stacked 2-D split tensor body
 *                       (even n, plain epilogue), 1 or 2 groups of stacked
 *                       instances per warp step
 *   compute_warps:      compute warps per CTA (0 = default).  The FP32 2-D
 *                       in-place bodies take it -- n = 16: groups of
 *                       instances_per_tile / 4 warps; n = 10, 14: groups of
 *                       four warps; each group on its own tile of the ring,
 *                       so compute_warps must be a multiple of the group,
 *                       at most 16; pipeline_depth is then rounded down to
 *                       a multiple of the number of groups (at least one
 *                       tile per group) -- and, with pipeline_depth (up to 12
 *                       tiles for these bodies, 8 for the others), sets the
 *                       split of an SM between
 *                       registers (resident warps) and shared memory (tiles
 *                       in flight).  The 3-D split tensor body
 *                       (KRON_COMPUTE_32F_BF16X3): 1 = one warp per instance
 *                       and CTA; 2, 4 or 8 = that many warps share one
 *                       instance (a CTA barrier between the modes) with the
 *                       next instance's operand arriving meanwhile.
 *
 * kron_set_kernel_config returns KRON_ERR_NOT_SUPPORTED when the body does not
 * exist for (kind, n, io, comp) (CUDA-core bodies, KRON_COMPUTE_NATIVE -- in
 * place: 2-D n = 16 any storage -- FP32 with
 * tiles of 8, 16, 24 or 32 instances, 16-bit with 16 --, FP32 2-D n =
 * 10, 14, FP32 3-D n = 10, 14, 16, FP32 odd n; exchange: even n, FP32 or 16-bit
 * storage; scalar: every real storage type; the split tensor bodies below)
 * and KRON_ERR_INVALID_VALUE for
 * values out of range; all-zero restores the built-in default.  Strided,
 * transposed or misaligned batches always run the scalar body.  The 2-D split
 * tensor path (KRON_COMPUTE_32F_BF16X3, FP32 or 16-bit storage) has two bodies:
 * KRON_VARIANT_IN_PLACE, one zero-padded 16 x 16 tile per instance (n <= 8:
 * several instances on the tile's diagonal), the second product taking the
 * first's accumulators; and KRON_VARIANT_EXCHANGE (9 <= n <= 16), 8 / gcd(n, 8)
 * instances side by side along the MMA's N dimension with the intermediate
 * passed through per-warp exchange rows in shared memory, so that only the
 * contracted dimension and the component rows are padded.  The built-in
 * choice is the stacked body for even n >= 10 except FP32 at n = 16 (with two
 * groups per warp step for 16-bit storage at n = 14, 16) and the padded one
 * otherwise; both give the same bits.  The 3-D split tensor path and complex storage have one body
 * each: only instances_per_tile and pipeline_depth apply there (and
 * compute_warps for the 3-D tensor body).
 *
 * kron_autotune_config times every configuration of that space on the
 * caller's buffers (as kron_autotune; Y is overwritten), keeps the fastest
 * unless the built-in default is within 2%, stores it in the process-wide
 * table and in the tuning cache (KRON_TUNE_CACHE; entries are keyed by GPU
 * name, SM count and driver version, so a cache written on another GPU or
 * driver is ignored) and returns it.  kron_autotune is this search reduced to
 * its instances-per-tile and pipeline-depth result.
 */
typedef enum {
    KRON_VARIANT_AUTO = 0,
    KRON_VARIANT_IN_PLACE = 1,   /* every contraction in place in the operand tile */
    KRON_VARIANT_EXCHANGE = 2,   /* packed pairs, intermediates in separate exchange buffers */
    KRON_VARIANT_SCALAR = 3      /* one fiber per thread, scalar FMA, exchange buffers */
} kron_variant;

typedef struct {
    int variant;
    int instances_per_tile;
    int pipeline_depth;
    int fibers_per_step;
    int compute_warps;
} kron_kernel_config;

KRON_API kron_status kron_set_kernel_config(int kind, int n, kron_dtype io, kron_compute comp,
                                            const kron_kernel_config* config);
KRON_API kron_status kron_get_kernel_config(int kind, int n, kron_dtype io, kron_compute comp,
                                            kron_kernel_config* config);
KRON_API kron_status kron_autotune_config(kron_stream_t stream, int kind, int n, int64_t batch_count,
                                          const void* X, void* Y, kron_dtype io, kron_compute comp,
                                          kron_kernel_config* config);

/*
 * Mixed-size batches (one launch for instances of different sizes and kinds).
 *
 * A class is one (kind, n) pair with its own shared components (square n x n,
 * column-major, host pointers, 'N' op; C only for kind 3).  A plan may hold at
 * most one class per (kind, n).  Instance p belongs to class h_class_of[p];
 * its operand starts at element offset h_x_off[p] of X and its result at
 * h_y_off[p] of Y; instances are contiguous (minimal leading dimensions);
 * alpha and beta are 1 and 0 unless kron_varlen_plan_set_scaling sets them.  Storage: KRON_R32F or KRON_R16BF / KRON_R16F
 * (components float).  X and Y may span at most 2^31 - 1 elements each
 * (KRON_ERR_NOT_SUPPORTED beyond).  X and Y need only element alignment, and
 * the offsets are arbitrary: the kernel copies the 16-byte-aligned span around
 * each operand and writes each result's aligned middle by bulk copy, its ends
 * by plain stores, so nothing outside [h_y_off[p], h_y_off[p] + n^kind) is
 * written.  Results of different instances must not overlap
 * (KRON_ERR_INVALID_VALUE at plan creation); X and Y must not overlap
 * (KRON_ERR_ALIAS at execute).
 *
 * kron_varlen_plan_create copies the host metadata, sorts instances by class,
 * chooses per-class tile sizes (from the tuning cache when present) and
 * prepares the device tables; it launches nothing.  The tables live in the
 * caller's workspace (kron_varlen_workspace_size bytes, 256-byte aligned
 * device memory), written by the first execute on that workspace.
 * kron_varlen_execute launches ONE persistent kernel, captured once into a CUDA
 * graph and replayed with cudaGraphLaunch on later calls.
 * kron_varlen_tune times the candidate tile sizes on the given buffers (it
 * overwrites Y), keeps the fastest per class, records them in the tuning cache
 * (file named by the KRON_TUNE_CACHE environment variable, if set) and
 * re-captures the graph.
 */
typedef struct {
    int kind;          /* 2 or 3 */
    int n;             /* 1..16 */
    const void* A;     /* host, n*n; mode 2 (kind 2) or mode 3 (kind 3) */
    const void* B;     /* host, n*n; mode 1 (kind 2) or mode 2 (kind 3) */
    const void* C;     /* host, n*n; mode 1 (kind 3), ignored for kind 2 */
} kron_class_desc;

typedef struct kron_varlen_plan kron_varlen_plan;

KRON_API kron_status kron_varlen_plan_create(kron_varlen_plan** plan, int num_classes,
                                             const kron_class_desc* classes, int64_t batch_count,
                                             const int32_t* h_class_of, const int64_t* h_x_off,
                                             const int64_t* h_y_off, kron_dtype io,
                                             kron_compute comp);
KRON_API kron_status kron_varlen_workspace_size(const kron_varlen_plan* plan, size_t* bytes);
KRON_API kron_status kron_varlen_execute(kron_varlen_plan* plan, const void* X, void* Y,
                                         void* workspace, size_t workspace_bytes,
                                         kron_stream_t stream);
KRON_API kron_status kron_varlen_tune(kron_varlen_plan* plan, const void* X, void* Y,
                                      void* workspace, size_t workspace_bytes,
                                      kron_stream_t stream);
/*
 * kron_varlen_plan_set_scaling -- alpha and beta of the plan's later executes:
 * Y^p = alpha (K_c X^p) + beta Y^p for every instance (Sec. 2.2's alpha and beta,
 * shared by the whole batch; default alpha = 1, beta = 0).  With beta = 0, Y is
 * not read (NaN or Inf in it are overwritten).  With beta != 0 the outputs must
 * not overlap one another.  alpha and beta enter the kernel as FP32; the scaling
 * is a pass over the staged results, so with 16-bit storage K_c X^p is rounded to
 * the storage type before it is scaled (two roundings).  Errors:
 * KRON_ERR_INVALID_VALUE for a null plan or a non-finite alpha or beta.
 */
KRON_API kron_status kron_varlen_plan_set_scaling(kron_varlen_plan* plan, double alpha, double beta);
KRON_API kron_status kron_varlen_plan_destroy(kron_varlen_plan* plan);

/*
 * kron_varlen_execute_noalloc -- the paper has no counterpart; this entry point
 * is for callers that cannot allocate device memory.  Examples: code that runs
 * while another component owns every byte of device memory through its own
 * allocator and hands out no scratch buffer, and latency-critical loops where
 * cudaMalloc / cudaFree would synchronise the device.  It computes the same
 * result as kron_varlen_execute on the same plan, X and Y, but takes no
 * workspace.  The plan's tables go into one fixed 8 MiB device array inside the
 * library.  Every GPU that loads the library holds that array until the process
 * exits.
 *
 *  - Limit: the plan needs 32 bytes of tables per instance, so at most 262,144
 *    instances.  Larger plans are rejected with KRON_ERR_WORKSPACE before any
 *    device work.
 *  - It calls no cudaMalloc, cudaFree or other allocating routine, and launches
 *    the kernel directly (no graph).
 *  - The first call on a device looks up the array's device address with that
 *    device current and keeps it for the life of the process.  After a
 *    cudaDeviceReset that address is stale: do not call this entry point on a
 *    device that has been reset since its first call.
 *  - Every call copies its tables into the array (a host-to-device copy from
 *    pageable memory) and waits on `stream` for that copy before it launches.
 *    Because each call synchronises its stream, it cannot be used while the
 *    stream is being captured into a CUDA graph.  Nothing is kept between
 *    calls.  All calls on a device share the one array, so calls whose work
 *    overlaps on the GPU (other streams, other host threads) race; serialise
 *    them.
 *  - Errors: as kron_varlen_execute (KRON_ERR_INVALID_VALUE, KRON_ERR_ALIAS,
 *    KRON_ERR_NOT_SUPPORTED, KRON_ERR_CUDA), plus KRON_ERR_WORKSPACE for a batch
 *    above the limit.
 */
KRON_API kron_status kron_varlen_execute_noalloc(kron_varlen_plan* plan, const void* X, void* Y,
                                                 kron_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* KRON_GB300_H */
