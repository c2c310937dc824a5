"""Parity of the 3-D FP32 kernels whose three contractions run in place (n = 16:
one instance per tile, planes 260 words apart; n = 10, 14: four packed
instances per tile; a ring of 1 to 4 buffers fed by a producer warp, results
leaving by bulk copy) with the FP64 oracle, and agreement with the generic 3-D
pair kernel.

Batch sizes cover a single instance, counts below and above the grid, and
enough instances that every CTA wraps its ring several times; each run checks
that nothing beyond Y is written and that X is left as it was."""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, max_norm_err, oracle_ref
from test_gpu_fiber import run_gpu

pytestmark = pytest.mark.gpu


TILE = {16: 1, 10: 4, 14: 4}   # instances per tile of the in-place kernels


@pytest.mark.parametrize("n", [16, 10, 14])
@pytest.mark.parametrize("depth", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("batch", [1, 3, 203, 5000])
def test_ring_depths_and_batches(n, depth, batch):
    if n == 14 and batch == 5000:
        batch = 2001
    b = inputs.make_batch(3, n, batch, seed=700 + batch % 89 + depth + n, x_dist="normal")
    try:
        kg.set_tile_config(3, n, "f32", "native", TILE[n] if depth else 0, depth)
        Y, X64 = run_gpu(b, guard=64)
    finally:
        kg.set_tile_config(3, n, "f32", "native", 0, 0)
    assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= TOL["f32"]


@pytest.mark.parametrize("n", [16, 10, 14])
@pytest.mark.parametrize("alpha,beta", [(-0.75, 0.0), (0.5, 2.0), (1.0, -1.0)])
def test_alpha_beta(n, alpha, beta):
    batch = 211
    b = inputs.make_batch(3, n, batch, seed=71 + n, x_dist="uniform")
    Y0 = np.random.default_rng(4).standard_normal(batch * n ** 3).astype(np.float32).astype(np.float64)
    Y, X64 = run_gpu(b, alpha=alpha, beta=beta, Y0=Y0.copy(), guard=16)
    ref = oracle_ref(b, X64, alpha=alpha, beta=beta, Y=Y0.copy())
    err = np.abs(ref - Y).reshape(batch, -1).max(axis=1)
    cn = np.linalg.norm(np.asarray(b.A, np.float64)) * np.linalg.norm(np.asarray(b.B, np.float64)) * \
        np.linalg.norm(np.asarray(b.C, np.float64))
    scale = cn * np.linalg.norm(X64.reshape(batch, -1), axis=1) * abs(alpha) + \
        abs(beta) * np.linalg.norm(Y0.reshape(batch, -1), axis=1)
    assert float((err / scale).max()) <= TOL["f32"]


@pytest.mark.parametrize("n", [16, 10, 14])
def test_same_bits_as_generic_pair_kernel(n):
    """Other tile sizes go to the generic 3-D pair kernel; both run the same FMA
    sequence per output, so the bits agree."""
    b = inputs.make_batch(3, n, 77, seed=72 + n, x_dist="normal")
    out = []
    for P in (0, 2):
        try:
            kg.set_tile_config(3, n, "f32", "native", P, 1 if P else 0)
            out.append(run_gpu(b, guard=8))
        finally:
            kg.set_tile_config(3, n, "f32", "native", 0, 0)
    Y0, X64 = out[0]
    assert max_norm_err(Y0, oracle_ref(b, X64), b, X64) <= TOL["f32"]
    assert np.array_equal(out[0][0], out[1][0])
