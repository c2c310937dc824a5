/*
 * Oracle for the batched Kronecker product action -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct CPU loops.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may call this file; the product path
 * never does.  It shares no code, header or constant with the CUDA library.
 *
 * Conventions (paper Sec. 2 and Sec. 2.1, with the factor order written as
 * (A (x) B) vec(X) = vec(B X A^T), the last Kronecker factor acting on the
 * fastest, column-major mode):
 *
 *   2-D:  Y^p <- alpha * op(B) op(X^p) op(A)^T + beta * Y^p         (Sec. 2.2)
 *         op(A): ma x na, op(B): mb x nb, op(X^p): nb x na, Y^p: mb x ma.
 *   3-D:  Y^p[i,j,k] <- alpha * sum_{l,m,q} op(C)[i,l] op(B)[j,m] op(A)[k,q]
 *                       X^p[l,m,q] + beta * Y^p[i,j,k]                (Sec. 2.1-2.2)
 *         X^p: nc x nb x na, Y^p: mc x mb x ma; C acts on mode 1, B on mode 2,
 *         A on mode 3, i.e. vec(Y) = (op(A) (x) op(B) (x) op(C)) vec(X).
 *
 * Every array is column-major.  Leading dimensions follow the TKRON2/TKRON3
 * interfaces of Sec. 3: ldx (column stride), ldx2 (plane stride, 3-D) and ldxp
 * (offset between consecutive batch instances), all in elements.
 *
 * beta == 0 means Y is not read (BLAS convention), so NaN in Y is ignored.
 *
 * The paper's 1-D interface (TKRON1) and its varying-A batched GEMM (TGEMM_A)
 * are defined further down, as direct sums.
 *
 * Three independent evaluations are provided:
 *   O1 "direct":   the multiple sum written out (Sec. 2.1 sums), O(n^4) / O(n^6)
 *   O2 "factored": one mode at a time in the order of Algorithm 1 (first the
 *                  2-D product on every plane, then the third mode)
 *   O3 "matrix":   the explicit Kronecker matrix from the block definition of
 *                  Sec. 2, for tiny sizes, to be multiplied with vec(X).
 *
 * FP64 and FP32 variants; the FP32 variants accumulate in float and the file
 * is compiled with -ffp-contract=off so no fused multiply-add is formed.
 * Complex variants of O1-O3 (op 'C' = Hermitian transpose) are at the end.
 */
#include <stddef.h>
#include <stdint.h>

#define ORACLE_API __attribute__((visibility("default")))

/* op(M)[r, c] for a column-major stored matrix with leading dimension ld. */
#define OPEL(M, ld, t, r, c) (((t) == 'N' || (t) == 'n') ? (M)[(size_t)(r) + (size_t)(ld) * (size_t)(c)] \
                                                        : (M)[(size_t)(c) + (size_t)(ld) * (size_t)(r)])

#define DEFINE_ORACLE(T, SUF)                                                                  \
/* O1, 2-D: Y[i,j] = alpha * sum_l sum_m opB[i,l] opX[l,m] opA[j,m] + beta Y[i,j] (Sec. 2.1) */ \
ORACLE_API void oracle_kron2_direct_##SUF(char ta, char tb, char tx, int ma, int na, int mb,   \
    int nb, int64_t batch, T alpha, const T* A, int lda, const T* B, int ldb, const T* X,      \
    int ldx, int64_t ldxp, T beta, T* Y, int ldy, int64_t ldyp)                                 \
{                                                                                              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        const T* Xp = X + p * ldxp;                                                            \
        T* Yp = Y + p * ldyp;                                                                  \
        for (int j = 0; j < ma; j++)                                                           \
            for (int i = 0; i < mb; i++) {                                                     \
                T s = 0;                                                                       \
                for (int l = 0; l < nb; l++)                                                   \
                    for (int m = 0; m < na; m++)                                               \
                        s += OPEL(B, ldb, tb, i, l) * OPEL(Xp, ldx, tx, l, m)                  \
                             * OPEL(A, lda, ta, j, m);                                         \
                T* y = &Yp[(size_t)i + (size_t)ldy * j];                                       \
                *y = (beta == (T)0) ? alpha * s : alpha * s + beta * *y;                       \
            }                                                                                  \
    }                                                                                          \
}                                                                                              \
                                                                                               \
/* O2, 2-D: Z = opB * opX (mb x na), then Y = alpha * Z * opA^T + beta * Y.                   \
   The per-plane step of Algorithm 1, one small GEMM after the other. */                       \
ORACLE_API void oracle_kron2_factored_##SUF(char ta, char tb, char tx, int ma, int na, int mb, \
    int nb, int64_t batch, T alpha, const T* A, int lda, const T* B, int ldb, const T* X,      \
    int ldx, int64_t ldxp, T beta, T* Y, int ldy, int64_t ldyp)                                 \
{                                                                                              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        T Z[16 * 16];                                                                          \
        const T* Xp = X + p * ldxp;                                                            \
        T* Yp = Y + p * ldyp;                                                                  \
        for (int m = 0; m < na; m++)                                                           \
            for (int i = 0; i < mb; i++) {                                                     \
                T s = 0;                                                                       \
                for (int l = 0; l < nb; l++)                                                   \
                    s += OPEL(B, ldb, tb, i, l) * OPEL(Xp, ldx, tx, l, m);                     \
                Z[i + 16 * m] = s;                                                             \
            }                                                                                  \
        for (int j = 0; j < ma; j++)                                                           \
            for (int i = 0; i < mb; i++) {                                                     \
                T s = 0;                                                                       \
                for (int m = 0; m < na; m++)                                                   \
                    s += Z[i + 16 * m] * OPEL(A, lda, ta, j, m);                               \
                T* y = &Yp[(size_t)i + (size_t)ldy * j];                                       \
                *y = (beta == (T)0) ? alpha * s : alpha * s + beta * *y;                       \
            }                                                                                  \
    }                                                                                          \
}                                                                                              \
                                                                                               \
/* O1, 3-D: the triple sum of Sec. 2.1, written out. */                                        \
ORACLE_API void oracle_kron3_direct_##SUF(char ta, char tb, char tc, int ma, int na, int mb,   \
    int nb, int mc, int nc, int64_t batch, T alpha, const T* A, int lda, const T* B, int ldb,  \
    const T* C, int ldc, const T* X, int ldx, int ldx2, int64_t ldxp, T beta, T* Y, int ldy,   \
    int ldy2, int64_t ldyp)                                                                    \
{                                                                                              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        const T* Xp = X + p * ldxp;                                                            \
        T* Yp = Y + p * ldyp;                                                                  \
        for (int k = 0; k < ma; k++)                                                           \
            for (int j = 0; j < mb; j++)                                                       \
                for (int i = 0; i < mc; i++) {                                                 \
                    T s = 0;                                                                   \
                    for (int l = 0; l < nc; l++)                                               \
                        for (int m = 0; m < nb; m++)                                           \
                            for (int q = 0; q < na; q++)                                       \
                                s += OPEL(C, ldc, tc, i, l) * OPEL(B, ldb, tb, j, m)           \
                                     * OPEL(A, lda, ta, k, q)                                  \
                                     * Xp[(size_t)l + (size_t)ldx * m + (size_t)ldx2 * q];     \
                    T* y = &Yp[(size_t)i + (size_t)ldy * j + (size_t)ldy2 * k];                \
                    *y = (beta == (T)0) ? alpha * s : alpha * s + beta * *y;                   \
                }                                                                              \
    }                                                                                          \
}                                                                                              \
                                                                                               \
/* O2, 3-D, Algorithm 1: every plane q gets tmp(:,:,q) = opC * X(:,:,q) * opB^T               \
   (the 2-D step), then each slice tmp(:,j,:) is multiplied by opA^T (the batched            \
   GEMM step).  tmp is mc x mb x na. */                                                        \
ORACLE_API void oracle_kron3_factored_##SUF(char ta, char tb, char tc, int ma, int na, int mb, \
    int nb, int mc, int nc, int64_t batch, T alpha, const T* A, int lda, const T* B, int ldb,  \
    const T* C, int ldc, const T* X, int ldx, int ldx2, int64_t ldxp, T beta, T* Y, int ldy,   \
    int ldy2, int64_t ldyp)                                                                    \
{                                                                                              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        T Z[16 * 16];                                                                          \
        T tmp[16 * 16 * 16];                                                                   \
        const T* Xp = X + p * ldxp;                                                            \
        T* Yp = Y + p * ldyp;                                                                  \
        for (int q = 0; q < na; q++) {                                                         \
            const T* Xq = Xp + (size_t)ldx2 * q;                                               \
            for (int m = 0; m < nb; m++)                                                       \
                for (int i = 0; i < mc; i++) {                                                 \
                    T s = 0;                                                                   \
                    for (int l = 0; l < nc; l++)                                               \
                        s += OPEL(C, ldc, tc, i, l) * Xq[(size_t)l + (size_t)ldx * m];         \
                    Z[i + 16 * m] = s;                                                         \
                }                                                                              \
            for (int j = 0; j < mb; j++)                                                       \
                for (int i = 0; i < mc; i++) {                                                 \
                    T s = 0;                                                                   \
                    for (int m = 0; m < nb; m++)                                               \
                        s += Z[i + 16 * m] * OPEL(B, ldb, tb, j, m);                           \
                    tmp[i + 16 * j + 256 * q] = s;                                             \
                }                                                                              \
        }                                                                                      \
        for (int j = 0; j < mb; j++)                                                           \
            for (int k = 0; k < ma; k++)                                                       \
                for (int i = 0; i < mc; i++) {                                                 \
                    T s = 0;                                                                   \
                    for (int q = 0; q < na; q++)                                               \
                        s += tmp[i + 16 * j + 256 * q] * OPEL(A, lda, ta, k, q);               \
                    T* y = &Yp[(size_t)i + (size_t)ldy * j + (size_t)ldy2 * k];                \
                    *y = (beta == (T)0) ? alpha * s : alpha * s + beta * *y;                   \
                }                                                                              \
    }                                                                                          \
}

/* The paper's two other interfaces (Sec. 3), as direct sums.
 *
 * TKRON1 (1-D, "almost a batched GEMV"):
 *   y^p <- alpha * op(A) x^p + beta * y^p,  op(A): ma x na,
 *   x^p: na contiguous elements at X + p*ldxp, y^p: ma at Y + p*ldyp.
 *   (The printed interface names both vector strides "ldp"; they are read as
 *   the X and the Y stride.)
 *
 * TGEMM_A (batched GEMM whose first factor varies across the batch):
 *   C^p <- alpha * op(A^p) op(B) + beta * C^p,  op(A^p): m x k at A + p*lda2,
 *   op(B): k x n (shared), C^p: m x n at C + p*ldc2, column stride ldc.
 */
#define DEFINE_ORACLE_1D_GEMM(T, SUF)                                                          \
ORACLE_API void oracle_kron1_##SUF(char ta, int ma, int na, int64_t batch, T alpha,            \
    const T* A, int lda, const T* X, int64_t ldxp, T beta, T* Y, int64_t ldyp)                  \
{                                                                                              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        const T* xp = X + p * ldxp;                                                            \
        T* yp = Y + p * ldyp;                                                                  \
        for (int i = 0; i < ma; i++) {                                                         \
            T s = 0;                                                                           \
            for (int l = 0; l < na; l++) s += OPEL(A, lda, ta, i, l) * xp[l];                  \
            yp[i] = (beta == (T)0) ? alpha * s : alpha * s + beta * yp[i];                     \
        }                                                                                      \
    }                                                                                          \
}                                                                                              \
                                                                                               \
ORACLE_API void oracle_gemm_a_##SUF(char ta, char tb, int m, int n, int k, T alpha,            \
    const T* A, int lda, int64_t lda2, const T* B, int ldb, T beta, T* C, int ldc,              \
    int64_t ldc2, int64_t batch)                                                               \
{                                                                                              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        const T* Ap = A + p * lda2;                                                            \
        T* Cp = C + p * ldc2;                                                                  \
        for (int j = 0; j < n; j++)                                                            \
            for (int i = 0; i < m; i++) {                                                      \
                T s = 0;                                                                       \
                for (int l = 0; l < k; l++)                                                    \
                    s += OPEL(Ap, lda, ta, i, l) * OPEL(B, ldb, tb, l, j);                     \
                T* c = &Cp[(size_t)i + (size_t)ldc * j];                                       \
                *c = (beta == (T)0) ? alpha * s : alpha * s + beta * *c;                       \
            }                                                                                  \
    }                                                                                          \
}

DEFINE_ORACLE(double, f64)
DEFINE_ORACLE(float, f32)
DEFINE_ORACLE_1D_GEMM(double, f64)
DEFINE_ORACLE_1D_GEMM(float, f32)

/* O3: the Kronecker matrix K = A (x) B from the block definition of Sec. 2:
 * block (r, c) of K is a_{rc} * B, so K[r*mb + i, c*nb + j] = A[r,c] * B[i,j].
 * A is ma x na (lda), B is mb x nb (ldb); K is (ma*mb) x (na*nb), column-major,
 * leading dimension ma*mb.  No op() here: callers transpose beforehand. */
ORACLE_API void oracle_kron_matrix_f64(int ma, int na, int mb, int nb, const double* A, int lda,
                                       const double* B, int ldb, double* K)
{
    const size_t ldk = (size_t)ma * (size_t)mb;
    for (int r = 0; r < ma; r++)
        for (int c = 0; c < na; c++)
            for (int i = 0; i < mb; i++)
                for (int j = 0; j < nb; j++)
                    K[((size_t)r * mb + i) + ldk * ((size_t)c * nb + j)] =
                        A[(size_t)r + (size_t)lda * c] * B[(size_t)i + (size_t)ldb * j];
}

/* Plain matrix-vector product y = K x for a column-major (rows x cols) K. */
ORACLE_API void oracle_matvec_f64(int64_t rows, int64_t cols, const double* K, const double* x,
                                  double* y)
{
    for (int64_t r = 0; r < rows; r++) {
        double s = 0;
        for (int64_t c = 0; c < cols; c++) s += K[r + rows * c] * x[c];
        y[r] = s;
    }
}

/* Threads the OpenMP runtime would use (1 when built without OpenMP). */
ORACLE_API int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ===========================================================================
 * Complex entries (the paper works over the complex field, Sec. 2, and its
 * interfaces take T in {single, double} x {real, complex}, Sec. 3).
 *
 * op(M) is M, M^T or M^* (Hermitian transpose) for 'N', 'T' and 'C' (Sec. 2.2);
 * op(X) of the 2-D case takes the same three values.  Storage is interleaved
 * (real part, imaginary part), the layout of C99 complex types and numpy's
 * complex64 / complex128.  alpha and beta are passed as pointers to their
 * (real, imaginary) pair.  Suffix z = double complex, c = float complex; the
 * arithmetic is C99 complex arithmetic, without fused multiply-adds.
 * ======================================================================== */
#include <complex.h>

/* op(M)[r, c] for a column-major stored complex matrix, conjugated for 'C'. */
#define ZOP(M, ld, t, r, c, CONJ)                                                             \
    (((t) == 'N' || (t) == 'n') ? (M)[(size_t)(r) + (size_t)(ld) * (size_t)(c)]               \
     : ((t) == 'T' || (t) == 't') ? (M)[(size_t)(c) + (size_t)(ld) * (size_t)(r)]             \
     : CONJ((M)[(size_t)(c) + (size_t)(ld) * (size_t)(r)]))

#define DEFINE_ORACLE_COMPLEX(T, R, SUF, CONJ)                                                 \
/* O1, 2-D: Y[i,j] = alpha sum_l sum_m opB[i,l] opX[l,m] opA[j,m] + beta Y[i,j] */            \
ORACLE_API void oracle_kron2_direct_##SUF(char ta, char tb, char tx, int ma, int na, int mb,   \
    int nb, int64_t batch, const R* alpha_ri, const T* A, int lda, const T* B, int ldb,        \
    const T* X, int ldx, int64_t ldxp, const R* beta_ri, T* Y, int ldy, int64_t ldyp)           \
{                                                                                              \
    const T al = alpha_ri[0] + alpha_ri[1] * I, be = beta_ri[0] + beta_ri[1] * I;              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        const T* Xc = X + p * ldxp;                                                            \
        T* Yc = Y + p * ldyp;                                                                  \
        for (int jj = 0; jj < ma; jj++)                                                        \
            for (int ii = 0; ii < mb; ii++) {                                                  \
                T acc = 0;                                                                     \
                for (int ll = 0; ll < nb; ll++)                                                \
                    for (int mm = 0; mm < na; mm++)                                            \
                        acc += ZOP(B, ldb, tb, ii, ll, CONJ) * ZOP(Xc, ldx, tx, ll, mm, CONJ)  \
                               * ZOP(A, lda, ta, jj, mm, CONJ);                                \
                T* yo = &Yc[(size_t)ii + (size_t)ldy * jj];                                    \
                *yo = (be == 0) ? al * acc : al * acc + be * *yo;                              \
            }                                                                                  \
    }                                                                                          \
}                                                                                              \
                                                                                               \
/* O2, 2-D: Z = opB opX, then Y = alpha Z opA^T + beta Y (Algorithm 1's plane step). */      \
ORACLE_API void oracle_kron2_factored_##SUF(char ta, char tb, char tx, int ma, int na, int mb, \
    int nb, int64_t batch, const R* alpha_ri, const T* A, int lda, const T* B, int ldb,        \
    const T* X, int ldx, int64_t ldxp, const R* beta_ri, T* Y, int ldy, int64_t ldyp)           \
{                                                                                              \
    const T al = alpha_ri[0] + alpha_ri[1] * I, be = beta_ri[0] + beta_ri[1] * I;              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        T W[16 * 16];                                                                          \
        const T* Xc = X + p * ldxp;                                                            \
        T* Yc = Y + p * ldyp;                                                                  \
        for (int mm = 0; mm < na; mm++)                                                        \
            for (int ii = 0; ii < mb; ii++) {                                                  \
                T acc = 0;                                                                     \
                for (int ll = 0; ll < nb; ll++)                                                \
                    acc += ZOP(B, ldb, tb, ii, ll, CONJ) * ZOP(Xc, ldx, tx, ll, mm, CONJ);     \
                W[ii + 16 * mm] = acc;                                                         \
            }                                                                                  \
        for (int jj = 0; jj < ma; jj++)                                                        \
            for (int ii = 0; ii < mb; ii++) {                                                  \
                T acc = 0;                                                                     \
                for (int mm = 0; mm < na; mm++)                                                \
                    acc += W[ii + 16 * mm] * ZOP(A, lda, ta, jj, mm, CONJ);                    \
                T* yo = &Yc[(size_t)ii + (size_t)ldy * jj];                                    \
                *yo = (be == 0) ? al * acc : al * acc + be * *yo;                              \
            }                                                                                  \
    }                                                                                          \
}                                                                                              \
                                                                                               \
/* O1, 3-D: the triple sum of Sec. 2.1 (C on mode 1, B on mode 2, A on mode 3). */            \
ORACLE_API void oracle_kron3_direct_##SUF(char ta, char tb, char tc, int ma, int na, int mb,   \
    int nb, int mc, int nc, int64_t batch, const R* alpha_ri, const T* A, int lda, const T* B, \
    int ldb, const T* C, int ldc, const T* X, int ldx, int ldx2, int64_t ldxp,                 \
    const R* beta_ri, T* Y, int ldy, int ldy2, int64_t ldyp)                                   \
{                                                                                              \
    const T al = alpha_ri[0] + alpha_ri[1] * I, be = beta_ri[0] + beta_ri[1] * I;              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        const T* Xc = X + p * ldxp;                                                            \
        T* Yc = Y + p * ldyp;                                                                  \
        for (int kk = 0; kk < ma; kk++)                                                        \
            for (int jj = 0; jj < mb; jj++)                                                    \
                for (int ii = 0; ii < mc; ii++) {                                              \
                    T acc = 0;                                                                 \
                    for (int ll = 0; ll < nc; ll++)                                            \
                        for (int mm = 0; mm < nb; mm++)                                        \
                            for (int qq = 0; qq < na; qq++)                                    \
                                acc += ZOP(C, ldc, tc, ii, ll, CONJ)                           \
                                       * ZOP(B, ldb, tb, jj, mm, CONJ)                         \
                                       * ZOP(A, lda, ta, kk, qq, CONJ)                         \
                                       * Xc[(size_t)ll + (size_t)ldx * mm + (size_t)ldx2 * qq]; \
                    T* yo = &Yc[(size_t)ii + (size_t)ldy * jj + (size_t)ldy2 * kk];            \
                    *yo = (be == 0) ? al * acc : al * acc + be * *yo;                          \
                }                                                                              \
    }                                                                                          \
}                                                                                              \
                                                                                               \
/* O2, 3-D, Algorithm 1: the 2-D step on every plane into tmp, then the third mode. */        \
ORACLE_API void oracle_kron3_factored_##SUF(char ta, char tb, char tc, int ma, int na, int mb, \
    int nb, int mc, int nc, int64_t batch, const R* alpha_ri, const T* A, int lda, const T* B, \
    int ldb, const T* C, int ldc, const T* X, int ldx, int ldx2, int64_t ldxp,                 \
    const R* beta_ri, T* Y, int ldy, int ldy2, int64_t ldyp)                                   \
{                                                                                              \
    const T al = alpha_ri[0] + alpha_ri[1] * I, be = beta_ri[0] + beta_ri[1] * I;              \
    int64_t p;                                                                                 \
    _Pragma("omp parallel for schedule(static)")                                               \
    for (p = 0; p < batch; p++) {                                                              \
        T W[16 * 16];                                                                          \
        T tp[16 * 16 * 16];                                                                    \
        const T* Xc = X + p * ldxp;                                                            \
        T* Yc = Y + p * ldyp;                                                                  \
        for (int qq = 0; qq < na; qq++) {                                                      \
            const T* Xq = Xc + (size_t)ldx2 * qq;                                              \
            for (int mm = 0; mm < nb; mm++)                                                    \
                for (int ii = 0; ii < mc; ii++) {                                              \
                    T acc = 0;                                                                 \
                    for (int ll = 0; ll < nc; ll++)                                            \
                        acc += ZOP(C, ldc, tc, ii, ll, CONJ) * Xq[(size_t)ll + (size_t)ldx * mm]; \
                    W[ii + 16 * mm] = acc;                                                     \
                }                                                                              \
            for (int jj = 0; jj < mb; jj++)                                                    \
                for (int ii = 0; ii < mc; ii++) {                                              \
                    T acc = 0;                                                                 \
                    for (int mm = 0; mm < nb; mm++)                                            \
                        acc += W[ii + 16 * mm] * ZOP(B, ldb, tb, jj, mm, CONJ);                \
                    tp[ii + 16 * jj + 256 * qq] = acc;                                         \
                }                                                                              \
        }                                                                                      \
        for (int jj = 0; jj < mb; jj++)                                                        \
            for (int kk = 0; kk < ma; kk++)                                                    \
                for (int ii = 0; ii < mc; ii++) {                                              \
                    T acc = 0;                                                                 \
                    for (int qq = 0; qq < na; qq++)                                            \
                        acc += tp[ii + 16 * jj + 256 * qq] * ZOP(A, lda, ta, kk, qq, CONJ);    \
                    T* yo = &Yc[(size_t)ii + (size_t)ldy * jj + (size_t)ldy2 * kk];            \
                    *yo = (be == 0) ? al * acc : al * acc + be * *yo;                          \
                }                                                                              \
    }                                                                                          \
}

DEFINE_ORACLE_COMPLEX(double complex, double, z, conj)
DEFINE_ORACLE_COMPLEX(float complex, float, c, conjf)

/* O3, complex: K = A (x) B from the block definition of Sec. 2 (no op()). */
ORACLE_API void oracle_kron_matrix_z(int ma, int na, int mb, int nb, const double complex* A, int lda,
                                     const double complex* B, int ldb, double complex* K)
{
    const size_t ldk = (size_t)ma * (size_t)mb;
    for (int r = 0; r < ma; r++)
        for (int c = 0; c < na; c++)
            for (int i = 0; i < mb; i++)
                for (int j = 0; j < nb; j++)
                    K[((size_t)r * mb + i) + ldk * ((size_t)c * nb + j)] =
                        A[(size_t)r + (size_t)lda * c] * B[(size_t)i + (size_t)ldb * j];
}

/* y = K x for a column-major complex (rows x cols) K. */
ORACLE_API void oracle_matvec_z(int64_t rows, int64_t cols, const double complex* K, const double complex* x,
                                double complex* y)
{
    for (int64_t r = 0; r < rows; r++) {
        double complex s = 0;
        for (int64_t c = 0; c < cols; c++) s += K[r + rows * c] * x[c];
        y[r] = s;
    }
}
