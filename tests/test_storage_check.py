"""The element-wise parity check of 16-bit storage, pinned on the CPU.

A kernel that is correct in the sense of the check computes every output in FP32
and rounds it once to the storage type with round-to-nearest-even.  The FP32
oracle (plain float loops) is such a computation, so its result rounded to bf16 /
f16 must pass; the same result with a mistake planted in the oracle's inputs (one
coefficient scaled by 1 + 2^-8) or rounded toward zero instead of to nearest must
fail.  The ulp helper is checked against the formats' definitions.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1304_7054_gb300 import inputs

from helpers import abs_batch, arith_factor, oracle_ref, storage_check, storage_excess, ulp


def test_ulp_matches_format_definitions():
    # bf16: 8 significant bits; f16: 11 bits, normal range from 2^-14, subnormal spacing 2^-24
    assert ulp(1.0, "bf16") == 2.0 ** -7
    assert ulp(1.5, "bf16") == 2.0 ** -7
    assert ulp(2.0 ** -126, "bf16") == 2.0 ** -133
    assert ulp(1.0, "f16") == 2.0 ** -10
    assert ulp(65504.0, "f16") == 32.0
    assert ulp(2.0 ** -14, "f16") == 2.0 ** -24
    assert ulp(2.0 ** -20, "f16") == 2.0 ** -24
    assert ulp(0.0, "f16") == 2.0 ** -24
    # the spacing is the distance to the next representable value
    for io, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        for v in (0.3, 1.0, 7.25, 1e-3, 123.0):
            t = torch.tensor([v], dtype=torch.float64).to(dt)
            nxt = torch.nextafter(t.float(), torch.tensor([np.inf])).to(dt)   # float32 step rounds up
            a, b = float(t.double()), float(nxt.double())
            if b == a:   # the float32 step vanished in rounding: step by the format's own bits
                bits = t.view(torch.int16) + 1
                b = float(bits.view(dt).double())
            assert b - a == ulp(a, io), (io, v)


def _rounded(y32, io):
    dt = torch.bfloat16 if io == "bf16" else torch.float16
    return torch.from_numpy(np.asarray(y32, np.float32)).to(dt).double().numpy()


def _truncated(y32, io):
    """Round toward zero: the wrong rounding mode."""
    dt = torch.bfloat16 if io == "bf16" else torch.float16
    y = torch.from_numpy(np.asarray(y32, np.float32))
    r = y.to(dt)
    over = r.double().abs() > y.double().abs()
    # sign and magnitude: one step down in the bit pattern is one ulp less magnitude
    fixed = (r.view(torch.int16) - 1).view(dt)
    return torch.where(over, fixed, r).double().numpy()


def _simulate(b, io):
    """FP32 oracle on the stored operands, rounded once to the storage type."""
    Xs = inputs.storage_to_f64(inputs.to_storage(b.X, io))
    n = b.n
    kw = dict(batch=b.batch, precision="f32")
    if b.kind == 2:
        y32 = oracle.kron2(b.A, b.B, Xs, ma=n, na=n, mb=n, nb=n, **kw)
    else:
        y32 = oracle.kron3(b.A, b.B, b.C, Xs, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, **kw)
    return y32, Xs


CASES = [(2, 16, 600), (2, 8, 900), (3, 8, 40), (3, 5, 80)]


@pytest.mark.parametrize("io", ["bf16", "f16"])
@pytest.mark.parametrize("kind,n,batch", CASES)
def test_correctly_rounded_fp32_result_passes(io, kind, n, batch):
    b = inputs.make_batch(kind, n, batch, seed=500 + n + kind, x_dist="normal")
    y32, Xs = _simulate(b, io)
    assert storage_check(_rounded(y32, io), b, Xs, io) <= 1.0


@pytest.mark.parametrize("io", ["bf16", "f16"])
@pytest.mark.parametrize("kind,n,batch", CASES)
def test_planted_coefficient_error_fails(io, kind, n, batch):
    """One coefficient of A scaled by 1 + 2^-8 in the oracle's copy of the
    components: the correct result must now fail the check."""
    b = inputs.make_batch(kind, n, batch, seed=500 + n + kind, x_dist="normal")
    y32, Xs = _simulate(b, io)
    bad = inputs.Batch(b.kind, n, b.batch, b.A.astype(np.float64).copy(), b.B, b.C, None)
    bad.A[0] *= 1.0 + 2.0 ** -8
    ref_bad = oracle_ref(bad, Xs)
    absref = oracle_ref(abs_batch(b), np.abs(Xs))
    assert storage_excess(_rounded(y32, io), ref_bad, absref, io, arith_factor(kind, n)) > 1.0


@pytest.mark.parametrize("io", ["bf16", "f16"])
@pytest.mark.parametrize("kind,n,batch", CASES[:2])
def test_wrong_rounding_mode_fails(io, kind, n, batch):
    b = inputs.make_batch(kind, n, batch, seed=700 + n, x_dist="normal")
    y32, Xs = _simulate(b, io)
    assert storage_check(_truncated(y32, io), b, Xs, io) > 1.0


def test_normalised_bar_misses_what_the_elementwise_check_catches():
    """The planted error stays within the old normalised bar (2^-8 + 1e-5 of
    ||A|| ||B|| ||X^p||), which is why the check is element-wise."""
    b = inputs.make_batch(2, 16, 600, seed=516, x_dist="normal")
    y32, Xs = _simulate(b, "bf16")
    bad = inputs.Batch(2, 16, b.batch, b.A.astype(np.float64).copy(), b.B, None, None)
    bad.A[0] *= 1.0 + 2.0 ** -8
    ref_bad = oracle_ref(bad, Xs).reshape(600, 256)
    got = _rounded(y32, "bf16").reshape(600, 256)
    norm = np.linalg.norm(b.A) * np.linalg.norm(b.B) * np.linalg.norm(Xs.reshape(600, 256), axis=1)
    assert float((np.abs(got - ref_bad).max(axis=1) / norm).max()) <= 2.0 ** -8 + 1e-5
