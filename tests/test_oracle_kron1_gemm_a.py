"""Pins for the oracle's TKRON1 (1-D product) and TGEMM_A (varying-A batched
GEMM) of Sec. 3, against what the mathematics fixes.

Independent anchors: numpy matrix products on tiny inputs, exact invariants
(identity, powers of two), the 1-D product as the 2-D product with a 1 x 1
unit factor (the 2-D oracle is pinned on its own), TGEMM_A applied twice giving
the 2-D product B X A^T (Sec. 2, vec identity), and the paper's Algorithm 1 --
a 2-D product on every plane followed by one TGEMM_A -- giving the 3-D product.
A last test plants typical mistakes in a copy of the oracle source and checks
that these pins catch each one.
"""
import ctypes

import numpy as np
import pytest

import oracle

from test_oracle_pins import colmaj, rnd


# ---------------------------------------------------------------------------
# TKRON1
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ma,na,ta", [(1, 1, "N"), (4, 4, "N"), (5, 3, "N"), (3, 7, "T"), (16, 16, "T")])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_kron1_against_numpy(ma, na, ta, precision):
    rng = np.random.default_rng(ma * 31 + na)
    batch, ldxp, ldyp = 5, na + 2, ma + 3
    A = rnd(rng, ma, na)
    stored = A if ta == "N" else A.T
    X = rnd(rng, batch * ldxp)
    Y0 = rnd(rng, batch * ldyp)
    Y = oracle.kron1(colmaj(stored), X, ma=ma, na=na, batch=batch, ldxp=ldxp, ldyp=ldyp, alpha=0.75,
                     beta=-1.5, Y=Y0, transa=ta, precision=precision)
    tol = 1e-13 if precision == "f64" else 1e-5
    for p in range(batch):
        ref = 0.75 * A @ X[p * ldxp:p * ldxp + na] - 1.5 * Y0[p * ldyp:p * ldyp + ma]
        np.testing.assert_allclose(Y[p * ldyp:p * ldyp + ma], ref, rtol=0, atol=tol * 4)
        # the gaps between strided outputs are left alone
        gap = Y0[p * ldyp + ma:(p + 1) * ldyp].astype(Y.dtype)
        np.testing.assert_array_equal(Y[p * ldyp + ma:(p + 1) * ldyp], gap)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_kron1_identity_and_pow2_are_exact(precision):
    rng = np.random.default_rng(2)
    n, batch = 9, 40
    X = rnd(rng, n * batch).astype(np.float32 if precision == "f32" else np.float64)
    Y = oracle.kron1(np.eye(n).ravel(), X, ma=n, na=n, batch=batch, precision=precision)
    assert np.array_equal(Y, X)
    Y = oracle.kron1((0.25 * np.eye(n)).ravel(), X, ma=n, na=n, batch=batch, alpha=2.0, precision=precision)
    assert np.array_equal(Y, X * 0.5)


def test_kron1_is_kron2_with_a_unit_factor():
    """(1 (x) A) vec(x) = A x: the 1-D product is the 2-D one with op(A') = [1]."""
    rng = np.random.default_rng(3)
    ma, na, batch = 6, 11, 17
    A = rnd(rng, ma, na)
    X = rnd(rng, na * batch)
    y1 = oracle.kron1(colmaj(A), X, ma=ma, na=na, batch=batch)
    y2 = oracle.kron2(np.ones(1), colmaj(A), X, ma=1, na=1, mb=ma, nb=na, batch=batch)
    np.testing.assert_allclose(y1, y2, rtol=0, atol=1e-14)


def test_kron1_beta_zero_ignores_nan():
    Y0 = np.full(12, np.nan)
    Y = oracle.kron1(np.eye(3).ravel(), np.ones(12), ma=3, na=3, batch=4, beta=0.0, Y=Y0)
    assert np.array_equal(Y, np.ones(12))


# ---------------------------------------------------------------------------
# TGEMM_A
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 3, 5), (40, 16, 16), (256, 10, 10), (5, 16, 2)])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_gemm_a_against_numpy(m, n, k, ta, tb):
    rng = np.random.default_rng(m + 7 * n + 13 * k)
    batch = 3
    lda = (m if ta == "N" else k) + 1
    lda2 = lda * (k if ta == "N" else m) + 5
    ldb = (k if tb == "N" else n) + 2
    ldc = m + 4
    ldc2 = ldc * n + 3
    As = [rnd(rng, m, k) for _ in range(batch)]
    B = rnd(rng, k, n)
    Abuf = rnd(rng, batch * lda2)
    for p, Ap in enumerate(As):
        st = Ap if ta == "N" else Ap.T
        for c in range(st.shape[1]):
            Abuf[p * lda2 + c * lda:p * lda2 + c * lda + st.shape[0]] = st[:, c]
    Bst = B if tb == "N" else B.T
    Bbuf = np.zeros(ldb * Bst.shape[1])
    for c in range(Bst.shape[1]):
        Bbuf[c * ldb:c * ldb + Bst.shape[0]] = Bst[:, c]
    C0 = rnd(rng, batch * ldc2)
    C = oracle.gemm_a(Abuf, Bbuf, m=m, n=n, k=k, batch=batch, lda=lda, lda2=lda2, ldb=ldb, ldc=ldc, ldc2=ldc2,
                      alpha=-0.5, beta=2.0, C=C0, transa=ta, transb=tb)
    for p, Ap in enumerate(As):
        ref = -0.5 * Ap @ B + 2.0 * np.array([[C0[p * ldc2 + j * ldc + i] for j in range(n)] for i in range(m)])
        got = np.array([[C[p * ldc2 + j * ldc + i] for j in range(n)] for i in range(m)])
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
    # padding rows of C are left alone
    assert C[ldc - 1] == C0[ldc - 1]


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_gemm_a_identity_is_exact(precision):
    rng = np.random.default_rng(5)
    m, k, batch = 33, 7, 6
    A = rnd(rng, m * k * batch).astype(np.float32 if precision == "f32" else np.float64)
    C = oracle.gemm_a(A, np.eye(k).ravel(), m=m, n=k, k=k, batch=batch, precision=precision)
    assert np.array_equal(C, A)


def test_gemm_a_twice_is_kron2():
    """Y = B X A^T as two TGEMM_A calls: Z^T = X^T B^T, then Y = (Z^T)^T A^T."""
    rng = np.random.default_rng(6)
    ma, na, mb, nb, batch = 5, 4, 3, 6, 9
    A, B = rnd(rng, ma, na), rnd(rng, mb, nb)
    X = rnd(rng, nb * na * batch)
    Zt = oracle.gemm_a(X, colmaj(B), m=na, n=mb, k=nb, batch=batch, lda=nb, lda2=nb * na, transa="T",
                       transb="T", ldb=mb)
    Y = oracle.gemm_a(Zt, colmaj(A), m=mb, n=ma, k=na, batch=batch, lda=na, lda2=na * mb, transa="T",
                      transb="T", ldb=ma)
    ref = oracle.kron2(colmaj(A), colmaj(B), X, ma=ma, na=na, mb=mb, nb=nb, batch=batch)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [3, 10])
def test_algorithm1_is_kron3(n):
    """Algorithm 1: a 2-D product on every plane into tmp, then tmp (n^2 x n) times A^T."""
    rng = np.random.default_rng(n)
    batch = 4
    A, B, C = rnd(rng, n, n), rnd(rng, n, n), rnd(rng, n, n)
    X = rnd(rng, n ** 3 * batch)
    tmp = oracle.kron2(colmaj(B), colmaj(C), X, ma=n, na=n, mb=n, nb=n, batch=batch * n)
    Y = oracle.gemm_a(tmp, colmaj(A), m=n * n, n=n, k=n, batch=batch, lda=n * n, lda2=n ** 3, transb="T",
                      ldb=n, ldc=n * n, ldc2=n ** 3)
    ref = oracle.kron3(colmaj(A), colmaj(B), colmaj(C), X, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-13)


def test_gemm_a_beta_zero_ignores_nan():
    C0 = np.full(8, np.nan)
    C = oracle.gemm_a(np.ones(8), np.eye(2).ravel(), m=2, n=2, k=2, batch=2, beta=0.0, C=C0)
    assert np.array_equal(C, np.ones(8))


# ---------------------------------------------------------------------------
# Planted mistakes
# ---------------------------------------------------------------------------
MUTANTS = {
    "kron1_transposed": ("OPEL(A, lda, ta, i, l) * xp[l]", "OPEL(A, lda, ta, l, i) * xp[l]"),
    "kron1_dropped_term": ("for (int l = 0; l < na; l++) s +=", "for (int l = 1; l < na; l++) s +="),
    "kron1_beta_sign": ("alpha * s + beta * yp[i]", "alpha * s - beta * yp[i]"),
    "gemm_a_transposed_B": ("OPEL(B, ldb, tb, l, j);", "OPEL(B, ldb, tb, j, l);"),
    "gemm_a_dropped_term": ("for (int l = 0; l < k; l++)", "for (int l = 1; l < k; l++)"),
    "gemm_a_batch_stride": ("const T* Ap = A + p * lda2;", "const T* Ap = A + p * ldc2;"),
}


def _pins_pass(L):
    rng = np.random.default_rng(11)
    try:
        ma, na, batch = 5, 3, 3
        A = rnd(rng, ma, na)
        X = rnd(rng, na * batch)
        Y0 = rnd(rng, ma * batch)
        Y = oracle.kron1(colmaj(A), X, ma=ma, na=na, batch=batch, alpha=0.5, beta=2.0, Y=Y0, lib_override=L)
        ref = np.concatenate([0.5 * A @ X[p * na:(p + 1) * na] + 2.0 * Y0[p * ma:(p + 1) * ma]
                              for p in range(batch)])
        if not np.allclose(Y, ref, atol=1e-12):
            return False
        m, n, k = 4, 2, 3
        As = rnd(rng, batch, m, k)
        B = rnd(rng, k, n)
        Abuf = np.concatenate([colmaj(a) for a in As])
        C = oracle.gemm_a(Abuf, colmaj(B), m=m, n=n, k=k, batch=batch, lib_override=L)
        ref = np.concatenate([colmaj(a @ B) for a in As])
        if not np.allclose(C, ref, atol=1e-12):
            return False
    except Exception:
        return False
    return True


def test_pins_pass_on_real_oracle():
    assert _pins_pass(oracle.lib())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutant_src = tmp_path / "mutant.c"
    mutant_src.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    oracle.compile_source(str(mutant_src), so)
    L = oracle.bind(ctypes.CDLL(so))
    assert not _pins_pass(L), f"planted mistake {name} was not caught by the pins"
