"""Parity of the 2-D n = 16 in-place kernel on 16-bit storage (bf16, f16;
FP32 arithmetic) with the FP64 oracle, and agreement with the generic pair
kernel.

The operands arrive in 16-bit slots by one bulk copy per instance, W is
staged in a separate FP32 buffer, and the 16-bit results overwrite the
operand slots before they leave by bulk copy.  Batch sizes cover a single
instance, ragged last tiles, exact multiples of the 16-instance tile and
enough tiles that every CTA wraps its ring several times; each run checks
that nothing beyond Y is written and that X is left as it was.  Every output
must lie within half an ulp of the storage type of the exact result, plus the
componentwise bound of the FP32 arithmetic (helpers.storage_check)."""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import storage_check
from test_gpu_fiber import run_gpu

pytestmark = pytest.mark.gpu

IO = ["bf16", "f16"]


@pytest.mark.parametrize("io", IO)
@pytest.mark.parametrize("P,depth", [(0, 0), (16, 1), (16, 2), (16, 4)])
@pytest.mark.parametrize("batch", [1, 15, 16, 1037, 40000])
def test_depths_and_ragged_batches(io, P, depth, batch):
    b = inputs.make_batch(2, 16, batch, seed=1200 + batch % 89 + depth, x_dist="normal")
    try:
        kg.set_tile_config(2, 16, io, "native", P, depth)
        Y, X64 = run_gpu(b, io=io, guard=64)
    finally:
        kg.set_tile_config(2, 16, io, "native", 0, 0)
    assert storage_check(Y, b, X64, io) <= 1.0


@pytest.mark.parametrize("io", IO)
@pytest.mark.parametrize("alpha,beta", [(-0.75, 0.0), (0.5, 2.0), (1.0, -1.0)])
def test_alpha_beta_ragged(io, alpha, beta):
    batch = 1037
    b = inputs.make_batch(2, 16, batch, seed=91, x_dist="uniform")
    y0 = np.random.default_rng(5).standard_normal(batch * 256)
    Y0 = inputs.storage_to_f64(inputs.to_storage(y0, io))   # beta Y0 with the stored Y0
    Y, X64 = run_gpu(b, io=io, alpha=alpha, beta=beta, Y0=Y0.copy(), guard=16)
    assert storage_check(Y, b, X64, io, alpha=alpha, beta=beta, Y0=Y0) <= 1.0


@pytest.mark.parametrize("io", IO)
def test_same_bits_as_generic_pair_kernel(io):
    """A tile of 7 instances goes to the generic pair kernel; both kernels run
    the same FP32 FMA sequence per output and round it once to the storage
    type, so the bits agree."""
    b = inputs.make_batch(2, 16, 333, seed=47, x_dist="normal")
    out = []
    for P in (0, 7):
        try:
            kg.set_tile_config(2, 16, io, "native", P, 1 if P else 0)
            out.append(run_gpu(b, io=io, guard=8))
        finally:
            kg.set_tile_config(2, 16, io, "native", 0, 0)
    Y0, X64 = out[0]
    assert storage_check(Y0, b, X64, io) <= 1.0
    assert np.array_equal(out[0][0], out[1][0])
