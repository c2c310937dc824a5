"""Pins for the complex oracle (paper Sec. 2: the complex field; Sec. 2.2: op in
{N, T, C}, C = Hermitian transpose; Sec. 3: T in {single, double} x {real,
complex}).

Independent anchors: numpy.kron on complex matrices (the block definition of
Sec. 2), a hand-worked complex example (tests/golden), the real oracle on
real-valued complex input, exact invariants (op 'C' of a real-valued matrix is
op 'T'; op 'C' is op 'T' of the conjugated matrix; multiplying X by i multiplies
Y by i), the rank-1 closed form, alpha / beta, and the FP32 complex oracle within
its a-priori bound of the FP64 one.  Planted mistakes in a copy of the complex
oracle source are caught.
"""
import ctypes
import json
import os
import zlib

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def crnd(rng, *shape):
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


def colmaj(M):
    return np.ascontiguousarray(np.asarray(M).T).ravel()


def from_colmaj(v, rows, cols):
    return np.asarray(v).reshape(cols, rows).T


def op(M, t):
    return {"N": M, "T": M.T, "C": M.conj().T}[t]


def stored(opM, t):
    """The stored matrix whose op(., t) is opM."""
    return {"N": opM, "T": opM.T, "C": opM.conj().T}[t]


def pair(v):
    return np.array([complex(*e) for e in v])


# ---------------------------------------------------------------------------
# Block definition against numpy.kron; hand-worked example
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(1, 1, 1, 1), (2, 3, 3, 2), (3, 3, 3, 3), (2, 2, 4, 1)])
def test_kron_matrix_is_numpy_kron(shape):
    rng = np.random.default_rng(3)
    ma, na, mb, nb = shape
    A, B = crnd(rng, ma, na), crnd(rng, mb, nb)
    np.testing.assert_allclose(oracle.kron_matrix_c(A, B), np.kron(A, B), rtol=0, atol=4e-16)


@pytest.mark.parametrize("method", ["direct", "factored"])
@pytest.mark.parametrize("precision", ["z", "c"])
def test_hand_example(method, precision):
    g = json.load(open(os.path.join(GOLDEN, "hand_kron2_complex_2x2.json")))
    A, B, X = pair(g["A_colmajor"]), pair(g["B_colmajor"]), pair(g["X_colmajor"])
    kw = dict(ma=2, na=2, mb=2, nb=2, batch=1, method=method, precision=precision)
    assert np.array_equal(oracle.kron2c(A, B, X, **kw), pair(g["Y_NNN_colmajor"]))
    assert np.array_equal(oracle.kron2c(A, B, X, transa="C", **kw), pair(g["Y_transa_C_colmajor"]))
    assert np.array_equal(oracle.kron2c(A, B, X, transa="T", **kw), pair(g["Y_transa_T_colmajor"]))
    assert np.array_equal(oracle.kron2c(A, B, X, transx="C", **kw), pair(g["Y_transx_C_colmajor"]))


# ---------------------------------------------------------------------------
# The vec identity over every op combination, rectangular shapes
# ---------------------------------------------------------------------------
SHAPES2 = [(1, 1, 1, 1), (3, 3, 3, 3), (2, 3, 4, 1), (4, 2, 3, 3)]
OPS2 = ["NNN", "CNN", "NCN", "NNC", "CCC", "TCN", "CTT", "NTC"]


@pytest.mark.parametrize("shape", SHAPES2)
@pytest.mark.parametrize("trans", OPS2)
@pytest.mark.parametrize("method", ["direct", "factored"])
def test_vec_identity_2d(shape, trans, method):
    rng = np.random.default_rng(zlib.crc32(repr((shape, trans, "c")).encode()))
    ma, na, mb, nb = shape
    batch = 3
    opA, opB = crnd(rng, ma, na), crnd(rng, mb, nb)
    opX = [crnd(rng, nb, na) for _ in range(batch)]
    ta, tb, tx = trans
    Xst = np.concatenate([colmaj(stored(x, tx)) for x in opX])
    Y = oracle.kron2c(colmaj(stored(opA, ta)), colmaj(stored(opB, tb)), Xst, ma=ma, na=na, mb=mb, nb=nb,
                      batch=batch, transa=ta, transb=tb, transx=tx, method=method)
    for p in range(batch):
        ref = np.kron(opA, opB) @ colmaj(opX[p])
        np.testing.assert_allclose(Y[p * ma * mb:(p + 1) * ma * mb], ref, rtol=0, atol=1e-14)


SHAPES3 = [(1, 1, 1, 1, 1, 1), (2, 2, 2, 2, 2, 2), (3, 3, 3, 3, 3, 3), (2, 3, 1, 2, 3, 2)]


@pytest.mark.parametrize("shape", SHAPES3)
@pytest.mark.parametrize("trans", ["NNN", "CNN", "NCN", "NNC", "CTC"])
@pytest.mark.parametrize("method", ["direct", "factored"])
def test_triple_sum_3d(shape, trans, method):
    rng = np.random.default_rng(zlib.crc32(repr((shape, trans, "c3")).encode()))
    ma, na, mb, nb, mc, nc = shape
    opA, opB, opC = crnd(rng, ma, na), crnd(rng, mb, nb), crnd(rng, mc, nc)
    X = crnd(rng, 2 * nc * nb * na)
    ta, tb, tc = trans
    Y = oracle.kron3c(colmaj(stored(opA, ta)), colmaj(stored(opB, tb)), colmaj(stored(opC, tc)), X, ma=ma, na=na,
                      mb=mb, nb=nb, mc=mc, nc=nc, batch=2, transa=ta, transb=tb, transc=tc, method=method)
    K = np.kron(opA, np.kron(opB, opC))
    sx, sy = nc * nb * na, mc * mb * ma
    for p in range(2):
        np.testing.assert_allclose(Y[p * sy:(p + 1) * sy], K @ X[p * sx:(p + 1) * sx], rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# Exact invariants and reductions
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("method", ["direct", "factored"])
@pytest.mark.parametrize("precision", ["z", "c"])
def test_real_valued_input_equals_real_oracle(method, precision):
    rng = np.random.default_rng(11)
    n, batch = 5, 4
    A, B, C = (rng.uniform(-1, 1, (n, n)) for _ in range(3))
    X = rng.uniform(-1, 1, batch * n ** 3)
    real = {"z": "f64", "c": "f32"}[precision]
    kw2 = dict(ma=n, na=n, mb=n, nb=n, batch=batch * n, method=method)
    y2 = oracle.kron2c(colmaj(A), colmaj(B), X.astype(complex), precision=precision, **kw2)
    r2 = oracle.kron2(colmaj(A), colmaj(B), X, precision=real, **kw2)
    assert np.array_equal(y2.real, r2) and not y2.imag.any()
    kw3 = dict(ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch, method=method)
    y3 = oracle.kron3c(colmaj(A), colmaj(B), colmaj(C), X.astype(complex), precision=precision, **kw3)
    r3 = oracle.kron3(colmaj(A), colmaj(B), colmaj(C), X, precision=real, **kw3)
    assert np.array_equal(y3.real, r3) and not y3.imag.any()


@pytest.mark.parametrize("method", ["direct", "factored"])
def test_hermitian_op_rules(method):
    rng = np.random.default_rng(12)
    n = 4
    A, B, X = crnd(rng, n, n), crnd(rng, n, n), crnd(rng, 3 * n * n)
    kw = dict(ma=n, na=n, mb=n, nb=n, batch=3, method=method)
    # 'C' on the stored matrix is 'T' on its conjugate
    for which in ("a", "b", "x"):
        t = {"transa": "N", "transb": "N", "transx": "N"}
        tc, tt = dict(t), dict(t)
        tc["trans" + which] = "C"
        tt["trans" + which] = "T"
        args_c = [colmaj(A), colmaj(B), X]
        args_t = [colmaj(A), colmaj(B), X]
        i = "abx".index(which)
        args_t[i] = np.conj(args_t[i])
        assert np.array_equal(oracle.kron2c(*args_c, **kw, **tc), oracle.kron2c(*args_t, **kw, **tt))
    # 'C' of a real-valued complex matrix is 'T'
    Ar = rng.uniform(-1, 1, (n, n)).astype(complex)
    assert np.array_equal(oracle.kron2c(colmaj(Ar), colmaj(B), X, transa="C", **kw),
                          oracle.kron2c(colmaj(Ar), colmaj(B), X, transa="T", **kw))


@pytest.mark.parametrize("method", ["direct", "factored"])
def test_times_i_is_exact(method):
    """Multiplying every operand by i multiplies every result by i, exactly
    (multiplication by i only swaps and negates parts)."""
    rng = np.random.default_rng(13)
    n = 6
    A, B, C = crnd(rng, n, n), crnd(rng, n, n), crnd(rng, n, n)
    X = crnd(rng, 2 * n ** 3)
    kw = dict(ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=2, method=method)
    y = oracle.kron3c(colmaj(A), colmaj(B), colmaj(C), X, **kw)
    yi = oracle.kron3c(colmaj(A), colmaj(B), colmaj(C), 1j * X, **kw)
    assert np.array_equal(yi, 1j * y)


def test_rank_one_closed_form():
    rng = np.random.default_rng(14)
    ma, na, mb, nb = 5, 4, 3, 6
    A, B = crnd(rng, ma, na), crnd(rng, mb, nb)
    u, v = crnd(rng, nb), crnd(rng, na)
    X = np.outer(u, v)
    for t in ("N", "C"):
        Y = oracle.kron2c(colmaj(stored(A, t)), colmaj(stored(B, t)), colmaj(X), ma=ma, na=na, mb=mb, nb=nb,
                          batch=1, transa=t, transb=t)
        np.testing.assert_allclose(from_colmaj(Y, mb, ma), np.outer(B @ u, A @ v), rtol=0, atol=1e-14)


@pytest.mark.parametrize("method", ["direct", "factored"])
def test_alpha_beta(method):
    rng = np.random.default_rng(15)
    n, batch = 3, 2
    A, B, C = crnd(rng, n, n), crnd(rng, n, n), crnd(rng, n, n)
    X, Y0 = crnd(rng, batch * n ** 3), crnd(rng, batch * n ** 3)
    al, be = 0.5 - 1.25j, -0.75 + 2j
    kw = dict(ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch, method=method)
    Y = oracle.kron3c(colmaj(A), colmaj(B), colmaj(C), X, alpha=al, beta=be, Y=Y0, **kw)
    K = np.kron(A, np.kron(B, C))
    ref = np.concatenate([al * (K @ X[p * 27:(p + 1) * 27]) + be * Y0[p * 27:(p + 1) * 27] for p in range(batch)])
    np.testing.assert_allclose(Y, ref, rtol=0, atol=1e-14)
    # beta = 0: Y is not read
    Ynan = np.full(batch * 27, np.nan + 1j * np.nan)
    Y = oracle.kron3c(colmaj(A), colmaj(B), colmaj(C), X, alpha=al, beta=0.0, Y=Ynan, **kw)
    assert not np.isnan(Y).any()


@pytest.mark.parametrize("kind,n", [(2, 16), (3, 8)])
def test_c_within_bound_of_z(kind, n):
    rng = np.random.default_rng(16)
    batch = 8
    comps = [crnd(rng, n, n).astype(np.complex64) for _ in range(kind)]
    X = crnd(rng, batch * n ** kind).astype(np.complex64)
    kw = dict(ma=n, na=n, mb=n, nb=n, batch=batch)
    if kind == 2:
        yc = oracle.kron2c(colmaj(comps[0]), colmaj(comps[1]), X, precision="c", **kw)
        yz = oracle.kron2c(colmaj(comps[0]), colmaj(comps[1]), X, precision="z", **kw)
    else:
        kw.update(mc=n, nc=n)
        yc = oracle.kron3c(*(colmaj(M) for M in comps), X, precision="c", **kw)
        yz = oracle.kron3c(*(colmaj(M) for M in comps), X, precision="z", **kw)
    cn = np.prod([np.linalg.norm(M.astype(np.complex128)) for M in comps])
    sz = n ** kind
    xn = np.linalg.norm(X.astype(np.complex128).reshape(batch, sz), axis=1)
    err = (np.abs(yc - yz).reshape(batch, sz).max(axis=1) / (cn * xn)).max()
    # a complex product and sum cost a few real roundings: 4 per term and contraction at most
    assert 0 < err < 4 * kind * n * 2.0 ** -24


# ---------------------------------------------------------------------------
# Planted mistakes in the complex oracle source
# ---------------------------------------------------------------------------
MUTANTS = {
    "conjugate_dropped": (": CONJ((M)[(size_t)(c) + (size_t)(ld) * (size_t)(r)]))",
                          ": ((M)[(size_t)(c) + (size_t)(ld) * (size_t)(r)]))"),
    "conjugate_for_T": ("? (M)[(size_t)(c) + (size_t)(ld) * (size_t)(r)]             \\",
                        "? CONJ((M)[(size_t)(c) + (size_t)(ld) * (size_t)(r)])       \\"),
    "alpha_imag_sign": ("const T al = alpha_ri[0] + alpha_ri[1] * I,",
                        "const T al = alpha_ri[0] - alpha_ri[1] * I,"),
    "transposed_A_2d": ("acc += W[ii + 16 * mm] * ZOP(A, lda, ta, jj, mm, CONJ);",
                        "acc += W[ii + 16 * mm] * ZOP(A, lda, ta, mm, jj, CONJ);"),
    "plane_index_3d": ("acc += tp[ii + 16 * jj + 256 * qq] * ZOP(A",
                       "acc += tp[jj + 16 * ii + 256 * qq] * ZOP(A"),
}


def _pins_pass(L):
    rng = np.random.default_rng(98)
    try:
        for method in ("direct", "factored"):
            for trans in ("NNN", "CTC", "TCN"):
                ma, na, mb, nb = 3, 2, 2, 3
                opA, opB, opX = crnd(rng, ma, na), crnd(rng, mb, nb), crnd(rng, nb, na)
                ta, tb, tx = trans
                Y = oracle.kron2c(colmaj(stored(opA, ta)), colmaj(stored(opB, tb)), colmaj(stored(opX, tx)), ma=ma,
                                  na=na, mb=mb, nb=nb, batch=1, transa=ta, transb=tb, transx=tx, alpha=0.5 + 0.25j,
                                  method=method, lib_override=L)
                if not np.allclose(Y, (0.5 + 0.25j) * (np.kron(opA, opB) @ colmaj(opX)), atol=1e-12):
                    return False
            n = 3
            opA, opB, opC = crnd(rng, n, n), crnd(rng, n, n), crnd(rng, n, n)
            X = crnd(rng, n ** 3)
            Y = oracle.kron3c(colmaj(opA.conj().T), colmaj(opB), colmaj(opC), X, ma=n, na=n, mb=n, nb=n, mc=n,
                              nc=n, batch=1, transa="C", alpha=-1j, method=method, lib_override=L)
            if not np.allclose(Y, -1j * (np.kron(opA, np.kron(opB, opC)) @ X), atol=1e-12):
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
    L = oracle.bind(ctypes.CDLL(so))
    assert not _pins_pass(L), f"planted mistake {name} was not caught by the pins"
