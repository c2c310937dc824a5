"""Oracle for the batched Kronecker product action -- TEST INFRASTRUCTURE ONLY.

Plain CPU loops (``kron_oracle.c``) in FP64 and FP32, loaded through ctypes.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package; the library under
``paper_1304_7054_gb300`` never does, and the two share no code.

Three independent evaluations of the same operation (paper Sec. 2.1 / 2.2):

* ``direct``   -- the double (2-D) or triple (3-D) sum written out;
* ``factored`` -- one mode at a time, in the order of Algorithm 1;
* ``kron_matrix`` + ``matvec`` -- the explicit Kronecker matrix built from the
  block definition of Sec. 2, for tiny sizes.

The complex field (Sec. 2) has its own entries with the same three forms:
``kron2c`` / ``kron3c`` (op 'C' = Hermitian transpose, Sec. 2.2) and
``kron_matrix_c`` + ``matvec_c``.

It also holds the paper's two other interfaces of Sec. 3 as direct sums:
``kron1`` (TKRON1, the 1-D product, a batched GEMV with a shared matrix) and
``gemm_a`` (TGEMM_A, a batched GEMM whose first factor varies across the batch).

Conventions: ``kron2(A, B)`` computes ``vec(Y) = (op(A) (x) op(B)) vec(op(X))``,
i.e. ``Y = op(B) op(X) op(A)^T``; ``kron3(A, B, C)`` applies
``op(A) (x) op(B) (x) op(C)`` with C on mode 1, B on mode 2, A on mode 3.
All buffers are flat, column-major, with explicit leading dimensions as in the
TKRON2/TKRON3 interfaces of Sec. 3.  The factored forms need every dimension
<= 16 (the paper's size range); the direct forms have no limit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kron_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libkron_oracle.so")

_lib = None


def compile_source(src: str, out: str) -> None:
    """Compile an oracle C source into a shared library with gcc.

    -ffp-contract=off keeps the FP32 variants free of fused multiply-adds so the
    FP32 oracle rounds every product and every sum.  OpenMP parallelises over
    batch instances only; the per-instance arithmetic is unchanged by it.
    """
    os.makedirs(os.path.dirname(out), exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", src, "-o", out]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       stdout=subprocess.PIPE, stderr=subprocess.PIPE)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)


def build(force: bool = False) -> str:
    """Compile kron_oracle.c (if stale) and return the library path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


_D = ctypes.c_double
_F = ctypes.c_float
_I = ctypes.c_int
_L = ctypes.c_int64
_C = ctypes.c_char
_P = ctypes.c_void_p


def bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    """Attach argument types to every oracle entry point of ``lib``."""
    for suf, scal in (("f64", _D), ("f32", _F)):
        for name in ("oracle_kron2_direct_", "oracle_kron2_factored_"):
            fn = getattr(lib, name + suf)
            fn.argtypes = [_C, _C, _C, _I, _I, _I, _I, _L, scal, _P, _I, _P, _I, _P, _I, _L,
                           scal, _P, _I, _L]
            fn.restype = None
        for name in ("oracle_kron3_direct_", "oracle_kron3_factored_"):
            fn = getattr(lib, name + suf)
            fn.argtypes = [_C, _C, _C, _I, _I, _I, _I, _I, _I, _L, scal, _P, _I, _P, _I, _P, _I,
                           _P, _I, _I, _L, scal, _P, _I, _I, _L]
            fn.restype = None
    for suf, scal in (("f64", _D), ("f32", _F)):
        fn = getattr(lib, "oracle_kron1_" + suf)
        fn.argtypes = [_C, _I, _I, _L, scal, _P, _I, _P, _L, scal, _P, _L]
        fn.restype = None
        fn = getattr(lib, "oracle_gemm_a_" + suf)
        fn.argtypes = [_C, _C, _I, _I, _I, scal, _P, _I, _L, _P, _I, scal, _P, _I, _L, _L]
        fn.restype = None
    for suf in ("z", "c"):
        for name in ("oracle_kron2_direct_", "oracle_kron2_factored_"):
            fn = getattr(lib, name + suf)
            fn.argtypes = [_C, _C, _C, _I, _I, _I, _I, _L, _P, _P, _I, _P, _I, _P, _I, _L, _P, _P, _I, _L]
            fn.restype = None
        for name in ("oracle_kron3_direct_", "oracle_kron3_factored_"):
            fn = getattr(lib, name + suf)
            fn.argtypes = [_C, _C, _C, _I, _I, _I, _I, _I, _I, _L, _P, _P, _I, _P, _I, _P, _I, _P, _I, _I, _L,
                           _P, _P, _I, _I, _L]
            fn.restype = None
    lib.oracle_kron_matrix_z.argtypes = [_I, _I, _I, _I, _P, _I, _P, _I, _P]
    lib.oracle_kron_matrix_z.restype = None
    lib.oracle_matvec_z.argtypes = [_L, _L, _P, _P, _P]
    lib.oracle_matvec_z.restype = None
    lib.oracle_kron_matrix_f64.argtypes = [_I, _I, _I, _I, _P, _I, _P, _I, _P]
    lib.oracle_kron_matrix_f64.restype = None
    lib.oracle_matvec_f64.argtypes = [_L, _L, _P, _P, _P]
    lib.oracle_matvec_f64.restype = None
    lib.oracle_num_threads.argtypes = []
    lib.oracle_num_threads.restype = _I
    return lib


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = bind(ctypes.CDLL(build()))
    return _lib


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _dt(precision: str):
    if precision == "f64":
        return np.float64
    if precision == "f32":
        return np.float32
    raise ValueError(precision)


def _b(c: str) -> bytes:
    return c.encode() if isinstance(c, str) else c


def kron2(A, B, X, *, ma, na, mb, nb, batch, lda=None, ldb=None, ldx=None, ldxp=None,
          ldy=None, ldyp=None, alpha=1.0, beta=0.0, Y=None, transa="N", transb="N",
          transx="N", method="factored", precision="f64", lib_override=None):
    """Y^p <- alpha op(B) op(X^p) op(A)^T + beta Y^p on flat column-major buffers.

    Returns the output buffer (a new one if ``Y`` is None).  Defaults for the
    leading dimensions are the minimal ones of Sec. 4 ("all the leading
    dimension parameters are the smallest they can logically be").
    """
    dt = _dt(precision)
    ta, tb, tx = (t.upper() for t in (transa, transb, transx))
    lda = lda or (ma if ta == "N" else na)
    ldb = ldb or (mb if tb == "N" else nb)
    ldx = ldx or (nb if tx == "N" else na)
    ldxp = ldx * (na if tx == "N" else nb) if ldxp is None else ldxp
    ldy = ldy or mb
    ldyp = ldy * ma if ldyp is None else ldyp
    A = np.ascontiguousarray(A, dtype=dt).ravel()
    B = np.ascontiguousarray(B, dtype=dt).ravel()
    X = np.ascontiguousarray(X, dtype=dt).ravel()
    if Y is None:
        Y = np.zeros(max(1, (batch - 1) * ldyp + ldy * (ma - 1) + mb), dtype=dt)
    else:
        Y = np.array(Y, dtype=dt, copy=True).ravel()
    L = lib_override or lib()
    fn = getattr(L, f"oracle_kron2_{method}_{precision}")
    fn(_b(ta), _b(tb), _b(tx), ma, na, mb, nb, batch, alpha, _ptr(A), lda, _ptr(B), ldb, _ptr(X),
       ldx, ldxp, beta, _ptr(Y), ldy, ldyp)
    return Y


def kron3(A, B, C, X, *, ma, na, mb, nb, mc, nc, batch, lda=None, ldb=None, ldc=None,
          ldx=None, ldx2=None, ldxp=None, ldy=None, ldy2=None, ldyp=None, alpha=1.0, beta=0.0,
          Y=None, transa="N", transb="N", transc="N", method="factored", precision="f64",
          lib_override=None):
    """Y^p[i,j,k] <- alpha sum op(C)[i,l] op(B)[j,m] op(A)[k,q] X^p[l,m,q] + beta Y^p."""
    dt = _dt(precision)
    ta, tb, tc = (t.upper() for t in (transa, transb, transc))
    lda = lda or (ma if ta == "N" else na)
    ldb = ldb or (mb if tb == "N" else nb)
    ldc = ldc or (mc if tc == "N" else nc)
    ldx = ldx or nc
    ldx2 = ldx2 or ldx * nb
    ldxp = ldx2 * na if ldxp is None else ldxp
    ldy = ldy or mc
    ldy2 = ldy2 or ldy * mb
    ldyp = ldy2 * ma if ldyp is None else ldyp
    A = np.ascontiguousarray(A, dtype=dt).ravel()
    B = np.ascontiguousarray(B, dtype=dt).ravel()
    C = np.ascontiguousarray(C, dtype=dt).ravel()
    X = np.ascontiguousarray(X, dtype=dt).ravel()
    if Y is None:
        Y = np.zeros(max(1, (batch - 1) * ldyp + ldy2 * (ma - 1) + ldy * (mb - 1) + mc), dtype=dt)
    else:
        Y = np.array(Y, dtype=dt, copy=True).ravel()
    L = lib_override or lib()
    fn = getattr(L, f"oracle_kron3_{method}_{precision}")
    fn(_b(ta), _b(tb), _b(tc), ma, na, mb, nb, mc, nc, batch, alpha, _ptr(A), lda, _ptr(B), ldb,
       _ptr(C), ldc, _ptr(X), ldx, ldx2, ldxp, beta, _ptr(Y), ldy, ldy2, ldyp)
    return Y


def kron1(A, X, *, ma, na, batch, lda=None, ldxp=None, ldyp=None, alpha=1.0, beta=0.0, Y=None,
          transa="N", precision="f64", lib_override=None):
    """TKRON1 (Sec. 3): y^p <- alpha op(A) x^p + beta y^p, op(A): ma x na."""
    dt = _dt(precision)
    ta = transa.upper()
    lda = lda or (ma if ta == "N" else na)
    ldxp = na if ldxp is None else ldxp
    ldyp = ma if ldyp is None else ldyp
    A = np.ascontiguousarray(A, dtype=dt).ravel()
    X = np.ascontiguousarray(X, dtype=dt).ravel()
    if Y is None:
        Y = np.zeros(max(1, (batch - 1) * ldyp + ma), dtype=dt)
    else:
        Y = np.array(Y, dtype=dt, copy=True).ravel()
    L = lib_override or lib()
    getattr(L, f"oracle_kron1_{precision}")(_b(ta), ma, na, batch, alpha, _ptr(A), lda, _ptr(X), ldxp,
                                            beta, _ptr(Y), ldyp)
    return Y


def gemm_a(A, B, *, m, n, k, batch, lda=None, lda2=None, ldb=None, ldc=None, ldc2=None, alpha=1.0,
           beta=0.0, C=None, transa="N", transb="N", precision="f64", lib_override=None):
    """TGEMM_A (Sec. 3): C^p <- alpha op(A^p) op(B) + beta C^p; A varies, B is shared."""
    dt = _dt(precision)
    ta, tb = transa.upper(), transb.upper()
    lda = lda or (m if ta == "N" else k)
    lda2 = lda * (k if ta == "N" else m) if lda2 is None else lda2
    ldb = ldb or (k if tb == "N" else n)
    ldc = ldc or m
    ldc2 = ldc * n if ldc2 is None else ldc2
    A = np.ascontiguousarray(A, dtype=dt).ravel()
    B = np.ascontiguousarray(B, dtype=dt).ravel()
    if C is None:
        C = np.zeros(max(1, (batch - 1) * ldc2 + ldc * (n - 1) + m), dtype=dt)
    else:
        C = np.array(C, dtype=dt, copy=True).ravel()
    L = lib_override or lib()
    getattr(L, f"oracle_gemm_a_{precision}")(_b(ta), _b(tb), m, n, k, alpha, _ptr(A), lda, lda2, _ptr(B),
                                             ldb, beta, _ptr(C), ldc, ldc2, batch)
    return C


def kron_matrix(A, B, lib_override=None):
    """Explicit K = A (x) B (block definition, Sec. 2) for 2-D numpy arrays A, B."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    ma, na = A.shape
    mb, nb = B.shape
    Af = np.ascontiguousarray(A.T).ravel()  # column-major storage
    Bf = np.ascontiguousarray(B.T).ravel()
    K = np.zeros(ma * mb * na * nb, dtype=np.float64)
    L = lib_override or lib()
    L.oracle_kron_matrix_f64(ma, na, mb, nb, _ptr(Af), ma, _ptr(Bf), mb, _ptr(K))
    return K.reshape(na * nb, ma * mb).T  # back to a (rows, cols) numpy view


def matvec(K, x, lib_override=None):
    """y = K x with the oracle's own loop (K a 2-D numpy array)."""
    K = np.asarray(K, dtype=np.float64)
    rows, cols = K.shape
    Kf = np.ascontiguousarray(K.T).ravel()
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.zeros(rows, dtype=np.float64)
    L = lib_override or lib()
    L.oracle_matvec_f64(rows, cols, _ptr(Kf), _ptr(x), _ptr(y))
    return y


# ---------------------------------------------------------------------------
# Complex entries: op in {'N', 'T', 'C'} ('C' = Hermitian transpose, Sec. 2.2);
# precision "z" (complex128) or "c" (complex64); alpha, beta complex scalars.
# ---------------------------------------------------------------------------
def _cdt(precision: str):
    if precision == "z":
        return np.complex128, np.float64
    if precision == "c":
        return np.complex64, np.float32
    raise ValueError(precision)


def _scal(v, rdt):
    v = complex(v)
    return np.array([v.real, v.imag], dtype=rdt)


def kron2c(A, B, X, *, ma, na, mb, nb, batch, lda=None, ldb=None, ldx=None, ldxp=None, ldy=None, ldyp=None,
           alpha=1.0, beta=0.0, Y=None, transa="N", transb="N", transx="N", method="factored", precision="z",
           lib_override=None):
    """Complex Y^p <- alpha op(B) op(X^p) op(A)^T + beta Y^p (flat column-major buffers)."""
    dt, rdt = _cdt(precision)
    ta, tb, tx = (t.upper() for t in (transa, transb, transx))
    lda = lda or (ma if ta == "N" else na)
    ldb = ldb or (mb if tb == "N" else nb)
    ldx = ldx or (nb if tx == "N" else na)
    ldxp = ldx * (na if tx == "N" else nb) if ldxp is None else ldxp
    ldy = ldy or mb
    ldyp = ldy * ma if ldyp is None else ldyp
    A = np.ascontiguousarray(A, dtype=dt).ravel()
    B = np.ascontiguousarray(B, dtype=dt).ravel()
    X = np.ascontiguousarray(X, dtype=dt).ravel()
    if Y is None:
        Y = np.zeros(max(1, (batch - 1) * ldyp + ldy * (ma - 1) + mb), dtype=dt)
    else:
        Y = np.array(Y, dtype=dt, copy=True).ravel()
    al, be = _scal(alpha, rdt), _scal(beta, rdt)
    L = lib_override or lib()
    fn = getattr(L, f"oracle_kron2_{method}_{precision}")
    fn(_b(ta), _b(tb), _b(tx), ma, na, mb, nb, batch, _ptr(al), _ptr(A), lda, _ptr(B), ldb, _ptr(X),
       ldx, ldxp, _ptr(be), _ptr(Y), ldy, ldyp)
    return Y


def kron3c(A, B, C, X, *, ma, na, mb, nb, mc, nc, batch, lda=None, ldb=None, ldc=None, ldx=None, ldx2=None,
           ldxp=None, ldy=None, ldy2=None, ldyp=None, alpha=1.0, beta=0.0, Y=None, transa="N", transb="N",
           transc="N", method="factored", precision="z", lib_override=None):
    """Complex Y^p[i,j,k] <- alpha sum op(C)[i,l] op(B)[j,m] op(A)[k,q] X^p[l,m,q] + beta Y^p."""
    dt, rdt = _cdt(precision)
    ta, tb, tc = (t.upper() for t in (transa, transb, transc))
    lda = lda or (ma if ta == "N" else na)
    ldb = ldb or (mb if tb == "N" else nb)
    ldc = ldc or (mc if tc == "N" else nc)
    ldx = ldx or nc
    ldx2 = ldx2 or ldx * nb
    ldxp = ldx2 * na if ldxp is None else ldxp
    ldy = ldy or mc
    ldy2 = ldy2 or ldy * mb
    ldyp = ldy2 * ma if ldyp is None else ldyp
    A = np.ascontiguousarray(A, dtype=dt).ravel()
    B = np.ascontiguousarray(B, dtype=dt).ravel()
    C = np.ascontiguousarray(C, dtype=dt).ravel()
    X = np.ascontiguousarray(X, dtype=dt).ravel()
    if Y is None:
        Y = np.zeros(max(1, (batch - 1) * ldyp + ldy2 * (ma - 1) + ldy * (mb - 1) + mc), dtype=dt)
    else:
        Y = np.array(Y, dtype=dt, copy=True).ravel()
    al, be = _scal(alpha, rdt), _scal(beta, rdt)
    L = lib_override or lib()
    fn = getattr(L, f"oracle_kron3_{method}_{precision}")
    fn(_b(ta), _b(tb), _b(tc), ma, na, mb, nb, mc, nc, batch, _ptr(al), _ptr(A), lda, _ptr(B), ldb,
       _ptr(C), ldc, _ptr(X), ldx, ldx2, ldxp, _ptr(be), _ptr(Y), ldy, ldy2, ldyp)
    return Y


def kron_matrix_c(A, B, lib_override=None):
    """Explicit complex K = A (x) B (block definition, Sec. 2) for 2-D numpy arrays."""
    A = np.asarray(A, dtype=np.complex128)
    B = np.asarray(B, dtype=np.complex128)
    ma, na = A.shape
    mb, nb = B.shape
    Af = np.ascontiguousarray(A.T).ravel()
    Bf = np.ascontiguousarray(B.T).ravel()
    K = np.zeros(ma * mb * na * nb, dtype=np.complex128)
    L = lib_override or lib()
    L.oracle_kron_matrix_z(ma, na, mb, nb, _ptr(Af), ma, _ptr(Bf), mb, _ptr(K))
    return K.reshape(na * nb, ma * mb).T


def matvec_c(K, x, lib_override=None):
    """y = K x for a complex 2-D numpy array K, with the oracle's own loop."""
    K = np.asarray(K, dtype=np.complex128)
    rows, cols = K.shape
    Kf = np.ascontiguousarray(K.T).ravel()
    x = np.ascontiguousarray(x, dtype=np.complex128).ravel()
    y = np.zeros(rows, dtype=np.complex128)
    L = lib_override or lib()
    L.oracle_matvec_z(rows, cols, _ptr(Kf), _ptr(x), _ptr(y))
    return y


def normalized_error(Y, Yref, norms, batch, inst_size, ldyp=None):
    """Per-instance max |Y - Yref| divided by the product of Frobenius norms.

    ``norms`` is an array (batch,) of ||A||_F ||B||_F (||C||_F) ||X^p||_F.  Each
    |Y_ij| is bounded by that product (Cauchy-Schwarz on the sum of Sec. 2.1), so
    the ratio is a scale-free error.  Returns the maximum over instances.
    """
    ldyp = ldyp or inst_size
    Y = np.asarray(Y, dtype=np.float64)
    Yref = np.asarray(Yref, dtype=np.float64)
    idx = (np.arange(batch)[:, None] * ldyp + np.arange(inst_size)[None, :])
    d = np.abs(Y[idx] - Yref[idx]).max(axis=1)
    return float((d / np.asarray(norms, dtype=np.float64)).max()) if batch else 0.0
