"""Shared helpers of the tests: run the CUDA path and the oracle on the same inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1304_7054_gb300 import inputs

# Normalised error bars (max |Y - Y_ref| / (||A|| ||B|| (||C||) ||X^p||)) of the
# FP32 and FP64 paths.  16-bit storage is checked element by element instead
# (storage_excess below); its entries here are the normalised form of the same
# rounding and serve only the reports.
TOL = {"f32": 1e-5, "f64": 1e-13,
       "bf16": 2.0 ** -8 + 1e-5, "f16": 2.0 ** -11 + 1e-5}
# Below the smallest normal float16 (2^-14) rounding is absolute: half the
# subnormal spacing, 2^-25 (bfloat16 shares FP32's exponent range).
ABS_FLOOR = {"f16": 2.0 ** -25}

# ---------------------------------------------------------------------------
# Element-wise check of 16-bit storage.  A correct kernel computes each output in
# FP32, y_k = y + e with |e| <= E (the componentwise bound of the FP32 arithmetic,
# a multiple of (|M1| |X| |M2|^T)_ij in 2-D and likewise in 3-D), then rounds y_k
# once to the storage type with round-to-nearest-even.  Hence
#     |Y - y| <= 1/2 ulp_s(|y| + E) + E,
# y being the exact result (the FP64 oracle on the stored operand values).  The
# bar is per element, so a kernel that loses even a fraction of an ulp on some
# outputs fails, unlike a bar normalised by the product of norms.
# ---------------------------------------------------------------------------
U32 = 2.0 ** -24
# precision in bits (with the implicit one) and smallest normal exponent
FORMAT = {"bf16": (8, -126), "f16": (11, -14), "f32": (24, -126)}


def ulp(v, io):
    """Spacing of the storage format io at magnitude |v| (subnormals included)."""
    p, emin = FORMAT[io]
    a = np.abs(np.asarray(v, dtype=np.float64))
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.where(a > 0, np.maximum(e, emin), emin)
    return np.ldexp(1.0, (e - (p - 1)).astype(np.int64))


def arith_factor(kind, n, compute="native"):
    """Bound of the FP32 arithmetic error as a multiple of the absolute-value
    product: `kind` contractions of length n, each within gamma_n = n u/(1 - n u)
    of its absolute sum (u = 2^-24); the split path adds 3 * 2^-16 per contraction
    (hi/lo residual and the dropped lo*lo term, bfloat16 u = 2^-8)."""
    g = n * U32 / (1.0 - n * U32)
    if compute == "bf16x3":
        return kind * (3 * 2.0 ** -16 + 2.0 * g)
    return 1.01 * kind * g


def storage_excess(got, ref, absref, io, factor, absextra=None):
    """max |got - ref| / (1/2 ulp_io(|ref| + E) + E) with E = factor * absref
    (+ 3 u |absextra| for an alpha/beta epilogue); <= 1 passes."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    absref = np.asarray(absref, np.float64)
    E = factor * absref + 2.0 ** -50 * absref
    if absextra is not None:
        E = E + 3 * U32 * (absref + np.asarray(absextra, np.float64))
    allowed = 0.5 * ulp(np.abs(ref) + E, io) + E
    d = np.abs(got - ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(d == 0, 0.0, d / allowed)
    return float(r.max()) if r.size else 0.0


def abs_batch(b):
    """The batch with every component replaced by its absolute values."""
    return inputs.Batch(b.kind, b.n, b.batch, np.abs(b.A), np.abs(b.B),
                        None if b.C is None else np.abs(b.C), None)


def storage_check(Y, b, X64, io, compute="native", alpha=1.0, beta=0.0, Y0=None, ref=None):
    """storage_excess of a whole batch against the FP64 oracle on the stored
    operands (X64): the exact result and its absolute-value product both come
    from the oracle."""
    n = b.n
    if ref is None:
        kw = {} if beta == 0.0 else dict(Y=np.array(Y0, np.float64))
        ref = oracle_ref(b, X64, alpha=alpha, beta=beta, **kw)
    absref = abs(alpha) * oracle_ref(abs_batch(b), np.abs(X64))
    extra = None if beta == 0.0 else abs(beta) * np.abs(np.asarray(Y0, np.float64))
    inst = n ** b.kind
    m = b.batch * inst
    return storage_excess(np.asarray(Y, np.float64)[:m], np.asarray(ref)[:m], absref[:m], io,
                          arith_factor(b.kind, n, compute), None if extra is None else extra[:m])


def torch_dtype(io):
    import torch
    return {"f32": torch.float32, "f64": torch.float64, "bf16": torch.bfloat16, "f16": torch.float16}[io]


def np_dtype(io):
    return np.float64 if io == "f64" else np.float32


def comp_norm(b):
    r = 1.0
    for M in b.comps():
        r *= float(np.linalg.norm(np.asarray(M, dtype=np.float64)))
    return r


def x_norms(X64, batch, inst):
    return np.linalg.norm(np.asarray(X64, dtype=np.float64)[: batch * inst].reshape(batch, inst), axis=1)


def storage_x(b, io):
    """(device-ready CPU torch tensor of X in storage type, X as exact float64)."""
    import torch
    if io in ("bf16", "f16"):
        t = inputs.to_storage(b.X, io)
        return t, inputs.storage_to_f64(t)
    t = torch.from_numpy(np.ascontiguousarray(b.X))
    return t, b.X.astype(np.float64)


def oracle_ref(b, X64, **kw):
    n = b.n
    if b.kind == 2:
        return oracle.kron2(b.A, b.B, X64, ma=n, na=n, mb=n, nb=n, batch=b.batch, **kw)
    return oracle.kron3(b.A, b.B, b.C, X64, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=b.batch, **kw)


def max_norm_err(Y, Yref, b, X64, io=None):
    inst = b.n ** b.kind
    Y = np.asarray(Y, dtype=np.float64)[: b.batch * inst].reshape(b.batch, inst)
    R = np.asarray(Yref, dtype=np.float64)[: b.batch * inst].reshape(b.batch, inst)
    d = np.maximum(np.abs(Y - R) - ABS_FLOOR.get(io, 0.0), 0.0).max(axis=1)
    return float((d / (comp_norm(b) * x_norms(X64, b.batch, inst))).max())
