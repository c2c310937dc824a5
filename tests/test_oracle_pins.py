"""Pins for the oracle: checks against what the paper and the mathematics fix.

None of these compares the oracle with itself.  Independent anchors are:
numpy.kron (a library routine for the block definition of Sec. 2), values worked
by hand (tests/golden), closed forms (rank-1 and separable operands), exact
invariants (identity, permutation, power-of-two scaling), the mixed-product rule,
linearity, and the 1-D reduction to a plain matrix-vector product (Sec. 2.1).
A last test plants typical mistakes in a copy of the oracle source and checks
that these pins catch every one of them.
"""
import json
import os
import zlib

import numpy as np
import pytest

import oracle
from paper_1304_7054_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rnd(rng, *shape):
    return rng.uniform(-1, 1, shape)


def colmaj(M):
    """numpy 2-D array -> flat column-major buffer."""
    return np.ascontiguousarray(np.asarray(M).T).ravel()


def from_colmaj(v, rows, cols):
    return np.asarray(v).reshape(cols, rows).T


def ref2_numpy(A, B, X):
    """(A kron B) vec(X) with numpy.kron, reshaped to Y (mb x ma)."""
    y = np.kron(A, B) @ colmaj(X)
    return from_colmaj(y, B.shape[0], A.shape[0])


def ref3_numpy(A, B, C, Xflat, nc, nb, na):
    """(A kron B kron C) vec(X) with numpy.kron; returns vec(Y)."""
    return np.kron(A, np.kron(B, C)) @ Xflat


# ---------------------------------------------------------------------------
# Block definition of Sec. 2 against numpy.kron
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (2, 3, 3, 2), (3, 3, 3, 3), (4, 2, 1, 3), (2, 2, 4, 4)])
def test_kron_matrix_is_numpy_kron(shape):
    rng = np.random.default_rng(1)
    ma, na, mb, nb = shape
    A, B = rnd(rng, ma, na), rnd(rng, mb, nb)
    K = oracle.kron_matrix(A, B)
    assert np.array_equal(K, np.kron(A, B))  # single products: bitwise equal


def test_matvec_against_numpy():
    rng = np.random.default_rng(2)
    K, x = rnd(rng, 7, 5), rnd(rng, 5)
    np.testing.assert_allclose(oracle.matvec(K, x), K @ x, rtol=1e-15, atol=1e-15)


# ---------------------------------------------------------------------------
# Hand-worked examples
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["direct", "factored"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_hand_example_2d(method, precision):
    g = json.load(open(os.path.join(GOLDEN, "hand_kron2_2x2.json")))
    Y = oracle.kron2(g["A_colmajor"], g["B_colmajor"], g["X_colmajor"], ma=2, na=2, mb=2, nb=2,
                     batch=1, method=method, precision=precision)
    assert Y.tolist() == g["Y_colmajor"]
    A = from_colmaj(g["A_colmajor"], 2, 2)
    B = from_colmaj(g["B_colmajor"], 2, 2)
    assert oracle.kron_matrix(A, B).tolist() == g["kron_AB_rows"]


@pytest.mark.parametrize("method", ["direct", "factored"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_hand_example_3d(method, precision):
    g = json.load(open(os.path.join(GOLDEN, "hand_kron3_2x2x2.json")))
    Y = oracle.kron3(g["A_colmajor"], g["B_colmajor"], g["C_colmajor"], g["X_colmajor"], ma=2, na=2,
                     mb=2, nb=2, mc=2, nc=2, batch=1, method=method, precision=precision)
    assert Y.tolist() == g["Y_colmajor"]


# ---------------------------------------------------------------------------
# The vec identity (A kron B) vec(X) = vec(B X A^T), Sec. 2, incl. op() and
# rectangular shapes (Sec. 2.2)
# ---------------------------------------------------------------------------
SHAPES2 = [(1, 1, 1, 1), (2, 2, 2, 2), (3, 3, 3, 3), (4, 4, 4, 4), (2, 3, 4, 1), (3, 1, 2, 4), (4, 2, 3, 3)]


@pytest.mark.parametrize("shape", SHAPES2)
@pytest.mark.parametrize("trans", ["NNN", "TNN", "NTN", "NNT", "TTT"])
@pytest.mark.parametrize("method", ["direct", "factored"])
def test_vec_identity_2d(shape, trans, method):
    rng = np.random.default_rng(zlib.crc32(repr((shape, trans)).encode()))
    ma, na, mb, nb = shape
    batch = 3
    opA, opB = rnd(rng, ma, na), rnd(rng, mb, nb)
    opX = [rnd(rng, nb, na) for _ in range(batch)]
    ta, tb, tx = trans
    Ast = opA.T if ta == "T" else opA
    Bst = opB.T if tb == "T" else opB
    Xst = np.concatenate([colmaj(x.T if tx == "T" else x) for x in opX])
    Y = oracle.kron2(colmaj(Ast), colmaj(Bst), Xst, ma=ma, na=na, mb=mb, nb=nb, batch=batch,
                     transa=ta, transb=tb, transx=tx, method=method)
    for p in range(batch):
        ref = ref2_numpy(opA, opB, opX[p])
        got = from_colmaj(Y[p * ma * mb:(p + 1) * ma * mb], mb, ma)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


SHAPES3 = [(1, 1, 1, 1, 1, 1), (2, 2, 2, 2, 2, 2), (3, 3, 3, 3, 3, 3), (2, 3, 1, 2, 3, 2), (3, 2, 2, 1, 1, 3)]


@pytest.mark.parametrize("shape", SHAPES3)
@pytest.mark.parametrize("trans", ["NNN", "TNN", "NTN", "NNT"])
@pytest.mark.parametrize("method", ["direct", "factored"])
def test_vec_identity_3d(shape, trans, method):
    rng = np.random.default_rng(zlib.crc32(repr((shape, trans, 3)).encode()))
    ma, na, mb, nb, mc, nc = shape
    batch = 2
    opA, opB, opC = rnd(rng, ma, na), rnd(rng, mb, nb), rnd(rng, mc, nc)
    X = rnd(rng, batch * nc * nb * na)
    ta, tb, tc = trans
    st = lambda M, t: colmaj(M.T if t == "T" else M)
    Y = oracle.kron3(st(opA, ta), st(opB, tb), st(opC, tc), X, ma=ma, na=na, mb=mb, nb=nb, mc=mc,
                     nc=nc, batch=batch, transa=ta, transb=tb, transc=tc, method=method)
    isz, osz = nc * nb * na, mc * mb * ma
    for p in range(batch):
        ref = ref3_numpy(opA, opB, opC, X[p * isz:(p + 1) * isz], nc, nb, na)
        np.testing.assert_allclose(Y[p * osz:(p + 1) * osz], ref, rtol=0, atol=1e-14)


def test_explicit_kron_path_3d():
    """O3 (oracle's own explicit matrix + matvec) against the triple sum (O1)."""
    rng = np.random.default_rng(5)
    n = 3
    A, B, C = rnd(rng, n, n), rnd(rng, n, n), rnd(rng, n, n)
    X = rnd(rng, n ** 3)
    K = oracle.kron_matrix(A, oracle.kron_matrix(B, C))
    y3 = oracle.matvec(K, X)
    y1 = oracle.kron3(colmaj(A), colmaj(B), colmaj(C), X, ma=n, na=n, mb=n, nb=n, mc=n, nc=n,
                      batch=1, method="direct")
    np.testing.assert_allclose(y1, y3, rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# Exact invariants
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("n", [1, 4, 7, 16])
def test_identity_is_bitwise(precision, n):
    dt = np.float64 if precision == "f64" else np.float32
    b = inputs.make_batch(2, n, 5, seed=3, dtype=dt)
    I = colmaj(np.eye(n))
    Y = oracle.kron2(I, I, b.X, ma=n, na=n, mb=n, nb=n, batch=5, precision=precision)
    assert np.array_equal(Y, b.X)
    if n <= 10:
        b3 = inputs.make_batch(3, n, 2, seed=4, dtype=dt)
        Y3 = oracle.kron3(I, I, I, b3.X, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=2, precision=precision)
        assert np.array_equal(Y3, b3.X)


@pytest.mark.parametrize("n", [3, 8, 16])
def test_permutation_and_pow2_scaling_are_exact(n):
    rng = np.random.default_rng(n)
    pa, pb = rng.permutation(n), rng.permutation(n)
    PA, PB = np.eye(n)[pa], np.eye(n)[pb]       # (P x)[i] = x[p[i]]
    da = 2.0 ** rng.integers(-4, 5, n)
    db = 2.0 ** rng.integers(-4, 5, n)
    A, B = PA * da[:, None], PB * db[:, None]   # diag(d) P: row i scaled by d[i]
    X = rnd(rng, n, n)
    Y = from_colmaj(oracle.kron2(colmaj(A), colmaj(B), colmaj(X), ma=n, na=n, mb=n, nb=n, batch=1),
                    n, n)
    expect = db[:, None] * X[np.ix_(pb, pa)] * da[None, :]   # Y = B X A^T
    assert np.array_equal(Y, expect)


# ---------------------------------------------------------------------------
# Closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [2, 5, 16])
def test_rank_one_closed_form(n):
    """X = u v^T  =>  B X A^T = (B u)(A v)^T."""
    rng = np.random.default_rng(10 + n)
    A, B, u, v = rnd(rng, n, n), rnd(rng, n, n), rnd(rng, n), rnd(rng, n)
    Y = from_colmaj(oracle.kron2(colmaj(A), colmaj(B), colmaj(np.outer(u, v)), ma=n, na=n, mb=n,
                                 nb=n, batch=1, method="factored"), n, n)
    np.testing.assert_allclose(Y, np.outer(B @ u, A @ v), rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [2, 4, 9])
def test_separable_closed_form_3d(n):
    """X = u o v o w  =>  Y = (C u) o (B v) o (A w)."""
    rng = np.random.default_rng(20 + n)
    A, B, C = rnd(rng, n, n), rnd(rng, n, n), rnd(rng, n, n)
    u, v, w = rnd(rng, n), rnd(rng, n), rnd(rng, n)
    X = np.einsum("l,m,q->lmq", u, v, w).ravel(order="F")
    Y = oracle.kron3(colmaj(A), colmaj(B), colmaj(C), X, ma=n, na=n, mb=n, nb=n, mc=n, nc=n,
                     batch=1, method="factored")
    ref = np.einsum("i,j,k->ijk", C @ u, B @ v, A @ w).ravel(order="F")
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-13)


def test_one_dimensional_reduction():
    """With A = [1] (ma = na = 1) the 2-D action is the plain product Y = op(B) x
    (the 1-D case of Sec. 2.1); with A = B = [1] the 3-D action is Y = C x."""
    rng = np.random.default_rng(30)
    B, x = rnd(rng, 5, 3), rnd(rng, 3)
    Y = oracle.kron2([1.0], colmaj(B), x, ma=1, na=1, mb=5, nb=3, batch=1)
    np.testing.assert_allclose(Y, B @ x, rtol=0, atol=1e-15)
    C = rnd(rng, 4, 6)
    x6 = rnd(rng, 6)
    Y3 = oracle.kron3([1.0], [1.0], colmaj(C), x6, ma=1, na=1, mb=1, nb=1, mc=4, nc=6, batch=1,
                      method="direct")
    np.testing.assert_allclose(Y3, C @ x6, rtol=0, atol=1e-15)


def test_mixed_product_rule():
    """(A kron B)(C kron D) = (AC) kron (BD), applied to vec(X)."""
    rng = np.random.default_rng(40)
    n = 6
    A, B, C, D = (rnd(rng, n, n) for _ in range(4))
    X = rnd(rng, 4 * n * n)
    kw = dict(ma=n, na=n, mb=n, nb=n, batch=4)
    inner = oracle.kron2(colmaj(C), colmaj(D), X, **kw)
    two = oracle.kron2(colmaj(A), colmaj(B), inner, **kw)
    one = oracle.kron2(colmaj(A @ C), colmaj(B @ D), X, **kw)
    np.testing.assert_allclose(two, one, rtol=0, atol=1e-13)
    E, F, G = (rnd(rng, 4, 4) for _ in range(3))
    X3 = rnd(rng, 2 * 64)
    kw3 = dict(ma=4, na=4, mb=4, nb=4, mc=4, nc=4, batch=2)
    t = oracle.kron3(colmaj(E), colmaj(F), colmaj(G), X3, **kw3)
    t = oracle.kron3(colmaj(A[:4, :4]), colmaj(B[:4, :4]), colmaj(C[:4, :4]), t, **kw3)
    o = oracle.kron3(colmaj(A[:4, :4] @ E), colmaj(B[:4, :4] @ F), colmaj(C[:4, :4] @ G), X3, **kw3)
    np.testing.assert_allclose(t, o, rtol=0, atol=1e-13)


# ---------------------------------------------------------------------------
# alpha / beta and linearity (Sec. 2.2); beta = 0 does not read Y
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["direct", "factored"])
def test_alpha_beta_linearity(method):
    rng = np.random.default_rng(50)
    n = 5
    A, B = colmaj(rnd(rng, n, n)), colmaj(rnd(rng, n, n))
    X1, X2, Y0 = rnd(rng, 3 * n * n), rnd(rng, 3 * n * n), rnd(rng, 3 * n * n)
    kw = dict(ma=n, na=n, mb=n, nb=n, batch=3, method=method)
    base1 = oracle.kron2(A, B, X1, **kw)
    base2 = oracle.kron2(A, B, X2, **kw)
    lin = oracle.kron2(A, B, 2.0 * X1 - 3.0 * X2, **kw)
    np.testing.assert_allclose(lin, 2.0 * base1 - 3.0 * base2, rtol=0, atol=1e-13)
    ab = oracle.kron2(A, B, X1, alpha=-1.5, beta=0.25, Y=Y0, **kw)
    np.testing.assert_allclose(ab, -1.5 * base1 + 0.25 * Y0, rtol=0, atol=1e-14)
    nan = np.full_like(Y0, np.nan)
    z = oracle.kron2(A, B, X1, alpha=1.0, beta=0.0, Y=nan, **kw)
    assert np.array_equal(z, base1)


def test_alpha_beta_3d():
    rng = np.random.default_rng(51)
    n = 3
    A, B, C = (colmaj(rnd(rng, n, n)) for _ in range(3))
    X, Y0 = rnd(rng, 2 * n ** 3), rnd(rng, 2 * n ** 3)
    kw = dict(ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=2)
    base = oracle.kron3(A, B, C, X, **kw)
    for method in ("direct", "factored"):
        ab = oracle.kron3(A, B, C, X, alpha=2.0, beta=-0.5, Y=Y0, method=method, **kw)
        np.testing.assert_allclose(ab, 2.0 * base - 0.5 * Y0, rtol=0, atol=1e-14)
        z = oracle.kron3(A, B, C, X, beta=0.0, Y=np.full_like(Y0, np.nan), method=method, **kw)
        assert not np.isnan(z).any()


# ---------------------------------------------------------------------------
# Leading dimensions (Sec. 3): padded strides give the same values, padding untouched
# ---------------------------------------------------------------------------
def test_leading_dimensions_2d():
    rng = np.random.default_rng(60)
    ma, na, mb, nb, batch = 3, 4, 5, 2, 3
    A, B = rnd(rng, ma, na), rnd(rng, mb, nb)
    Xs = [rnd(rng, nb, na) for _ in range(batch)]
    lda, ldb, ldx, ldxp, ldy, ldyp = 5, 7, 3, 17, 6, 23
    Ab = np.zeros(lda * na); Bb = np.zeros(ldb * nb); Xb = np.zeros(ldxp * batch)
    for c in range(na):
        Ab[c * lda:c * lda + ma] = A[:, c]
    for c in range(nb):
        Bb[c * ldb:c * ldb + mb] = B[:, c]
    for p in range(batch):
        for c in range(na):
            Xb[p * ldxp + c * ldx:p * ldxp + c * ldx + nb] = Xs[p][:, c]
    sentinel = 12345.0
    Y0 = np.full(ldyp * batch, sentinel)
    Y = oracle.kron2(Ab, Bb, Xb, ma=ma, na=na, mb=mb, nb=nb, batch=batch, lda=lda, ldb=ldb, ldx=ldx,
                     ldxp=ldxp, ldy=ldy, ldyp=ldyp, Y=Y0, beta=0.0)
    touched = np.zeros_like(Y, dtype=bool)
    for p in range(batch):
        ref = B @ Xs[p] @ A.T
        for c in range(ma):
            s = p * ldyp + c * ldy
            np.testing.assert_allclose(Y[s:s + mb], ref[:, c], rtol=0, atol=1e-14)
            touched[s:s + mb] = True
    assert np.all(Y[~touched] == sentinel)


def test_leading_dimensions_3d():
    rng = np.random.default_rng(61)
    n, batch = 3, 2
    A, B, C = rnd(rng, n, n), rnd(rng, n, n), rnd(rng, n, n)
    X = rnd(rng, batch * n ** 3)
    ldx, ldx2, ldxp, ldy, ldy2, ldyp = 4, 13, 60, 5, 16, 50
    Xb = np.zeros(ldxp * batch)
    for p in range(batch):
        for q in range(n):
            for m in range(n):
                s = p * ldxp + q * ldx2 + m * ldx
                Xb[s:s + n] = X[p * 27 + q * 9 + m * 3:p * 27 + q * 9 + m * 3 + 3]
    Y = oracle.kron3(colmaj(A), colmaj(B), colmaj(C), Xb, ma=n, na=n, mb=n, nb=n, mc=n, nc=n,
                     batch=batch, ldx=ldx, ldx2=ldx2, ldxp=ldxp, ldy=ldy, ldy2=ldy2, ldyp=ldyp,
                     Y=np.full(ldyp * batch, -7.0))
    Ymin = oracle.kron3(colmaj(A), colmaj(B), colmaj(C), X, ma=n, na=n, mb=n, nb=n, mc=n, nc=n,
                        batch=batch)
    for p in range(batch):
        for k in range(n):
            for j in range(n):
                s = p * ldyp + k * ldy2 + j * ldy
                np.testing.assert_allclose(Y[s:s + n], Ymin[p * 27 + k * 9 + j * 3:][:3], atol=1e-14)


# ---------------------------------------------------------------------------
# FP32 oracle within the a-priori error bound of the FP64 one
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,n", [(2, 16), (2, 10), (3, 8), (3, 16)])
def test_f32_within_bound(kind, n):
    b32 = inputs.make_batch(kind, n, 16, seed=70, x_dist="normal", dtype=np.float32)
    kw = dict(ma=n, na=n, mb=n, nb=n, batch=16)
    if kind == 2:
        y32 = oracle.kron2(b32.A, b32.B, b32.X, precision="f32", **kw)
        y64 = oracle.kron2(b32.A, b32.B, b32.X, precision="f64", **kw)
        cn = np.linalg.norm(b32.A) * np.linalg.norm(b32.B)
    else:
        kw.update(mc=n, nc=n)
        y32 = oracle.kron3(b32.A, b32.B, b32.C, b32.X, precision="f32", **kw)
        y64 = oracle.kron3(b32.A, b32.B, b32.C, b32.X, precision="f64", **kw)
        cn = np.linalg.norm(b32.A) * np.linalg.norm(b32.B) * np.linalg.norm(b32.C)
    sz = n ** kind
    xn = np.linalg.norm(b32.X.astype(np.float64).reshape(16, sz), axis=1)
    err = oracle.normalized_error(y32, y64, cn * xn, 16, sz)
    # kind contractions of length n, each adding at most ~n unit roundoffs per term
    assert err < kind * n * 2.0 ** -24
    assert err > 0  # FP32 really rounded


# ---------------------------------------------------------------------------
# Planted mistakes: each mutant of the oracle source must fail a pin above
# ---------------------------------------------------------------------------
MUTANTS = {
    "transposed_A_2d": ("OPEL(A, lda, ta, j, m)", "OPEL(A, lda, ta, m, j)"),
    "dropped_term_2d": ("for (int l = 0; l < nb; l++)", "for (int l = 1; l < nb; l++)"),
    "beta_sign": ("alpha * s + beta * *y", "alpha * s - beta * *y"),
    "tmp_index_3d": ("tmp[i + 16 * j + 256 * q] * OPEL(A", "tmp[j + 16 * i + 256 * q] * OPEL(A"),
    "transposed_C_3d": ("OPEL(C, ldc, tc, i, l) * Xq", "OPEL(C, ldc, tc, l, i) * Xq"),
    "mode_swap_3d": ("Z[i + 16 * m] * OPEL(B, ldb, tb, j, m)", "Z[i + 16 * m] * OPEL(B, ldb, tb, m, j)"),
}


def _pins_pass(L):
    """A compact run of the independent pins against a (possibly mutated) library."""
    rng = np.random.default_rng(99)
    try:
        for method in ("direct", "factored"):
            for (ma, na, mb, nb) in [(3, 3, 3, 3), (2, 3, 4, 2)]:
                A, B, X = rnd(rng, ma, na), rnd(rng, mb, nb), rnd(rng, nb, na)
                Y = oracle.kron2(colmaj(A), colmaj(B), colmaj(X), ma=ma, na=na, mb=mb, nb=nb,
                                 batch=1, method=method, lib_override=L)
                if not np.allclose(from_colmaj(Y, mb, ma), ref2_numpy(A, B, X), atol=1e-12):
                    return False
            Y0 = rnd(rng, 9)
            Y = oracle.kron2(colmaj(A[:3, :3] if A.shape == (3, 3) else np.eye(3)), colmaj(np.eye(3)),
                             colmaj(np.eye(3)), ma=3, na=3, mb=3, nb=3, batch=1, alpha=0.0, beta=2.0,
                             Y=Y0, method=method, lib_override=L)
            if not np.allclose(Y, 2.0 * Y0):
                return False
            n = 3
            A, B, C = rnd(rng, n, n), rnd(rng, n, n), rnd(rng, n, n)
            X = rnd(rng, n ** 3)
            Y = oracle.kron3(colmaj(A), colmaj(B), colmaj(C), X, ma=n, na=n, mb=n, nb=n, mc=n, nc=n,
                             batch=1, method=method, lib_override=L)
            if not np.allclose(Y, ref3_numpy(A, B, C, X, n, n, n), atol=1e-12):
                return False
            Y0 = rnd(rng, n ** 3)
            Y = oracle.kron3(colmaj(A), colmaj(B), colmaj(C), X, ma=n, na=n, mb=n, nb=n, mc=n, nc=n,
                             batch=1, alpha=0.0, beta=-1.0, Y=Y0, method=method, lib_override=L)
            if not np.allclose(Y, -Y0):
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
    assert old in src, f"mutation anchor not found: {old!r}"
    mutant_src = tmp_path / "mutant.c"
    mutant_src.write_text(src.replace(old, new))
    so = str(tmp_path / "libmutant.so")
    oracle.compile_source(str(mutant_src), so)
    import ctypes
    L = oracle.bind(ctypes.CDLL(so))
    assert not _pins_pass(L), f"planted mistake {name} was not caught by the pins"
