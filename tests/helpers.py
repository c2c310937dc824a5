"""Shared helpers of the tests: run the CUDA path and the oracle on the same inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1304_7054_gb300 import inputs

TOL = {"f32": 1e-5, "f64": 1e-13,
       # output rounding to the 16-bit storage type: half an ulp relative to |y|,
       # |y| <= ||A|| ||B|| ||X|| (Cauchy-Schwarz), plus the FP32 accumulation error
       "bf16": 2.0 ** -8 + 1e-5, "f16": 2.0 ** -11 + 1e-5}
# Below the smallest normal float16 (2^-14) rounding is absolute: half the
# subnormal spacing, 2^-25.  It is subtracted from each difference before the
# normalisation (bfloat16 shares FP32's exponent range, so it has no such floor).
ABS_FLOOR = {"f16": 2.0 ** -25}


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
