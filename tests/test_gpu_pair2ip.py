"""Parity of the 2-D FP32 kernels whose exchange is done in place (n = 10, 14
and 16: a ring of 1 to 4 tile buffers fed by a producer warp, results leaving
by bulk copy) with the FP64 oracle, and agreement with the generic pair kernel.

Every even n runs through the tile configurations: tiles of a multiple of 8
instances (16 at n = 16) go to the in-place kernels where they exist, other
tiles and sizes to the generic pair kernel.  Batch sizes cover a single
instance, ragged last tiles, exact multiples of the tile, and enough tiles that
every CTA wraps its ring of buffers several times; each run checks that nothing
beyond Y is written and that X is left as it was."""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, max_norm_err, oracle_ref
from test_gpu_fiber import run_gpu

pytestmark = pytest.mark.gpu

EVEN = [4, 6, 8, 10, 12, 14, 16]


@pytest.mark.parametrize("n", EVEN)
@pytest.mark.parametrize("P,depth", [(0, 0), (8, 1), (24, 2), (0, 3), (16, 4)])
@pytest.mark.parametrize("batch", [1, 7, 9, 1037, 40000])
def test_tiles_depths_and_ragged_batches(n, P, depth, batch):
    b = inputs.make_batch(2, n, batch, seed=900 + batch % 97 + depth + n, x_dist="normal")
    try:
        kg.set_tile_config(2, n, "f32", "native", P, depth)
        Y, X64 = run_gpu(b, guard=64)
    finally:
        kg.set_tile_config(2, n, "f32", "native", 0, 0)
    assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= TOL["f32"]


@pytest.mark.parametrize("n", [6, 10, 16])
@pytest.mark.parametrize("alpha,beta", [(-0.75, 0.0), (0.5, 2.0), (1.0, -1.0)])
def test_alpha_beta_ragged(n, alpha, beta):
    batch = 1037
    b = inputs.make_batch(2, n, batch, seed=77 + n, x_dist="uniform")
    Y0 = np.random.default_rng(3).standard_normal(batch * n * n).astype(np.float32).astype(np.float64)
    Y, X64 = run_gpu(b, alpha=alpha, beta=beta, Y0=Y0.copy(), guard=16)
    ref = oracle_ref(b, X64, alpha=alpha, beta=beta, Y=Y0.copy())
    # beta * Y0 adds |beta| ||Y0_p|| to the scale of each instance's result
    err = np.abs(ref - Y).reshape(batch, n * n).max(axis=1)
    scale = np.linalg.norm(np.asarray(b.A, np.float64)) * np.linalg.norm(np.asarray(b.B, np.float64)) * \
        np.linalg.norm(X64.reshape(batch, n * n), axis=1) * abs(alpha) + \
        abs(beta) * np.linalg.norm(Y0.reshape(batch, n * n), axis=1)
    assert float((err / scale).max()) <= TOL["f32"]


@pytest.mark.parametrize("n", EVEN)
def test_same_bits_as_generic_pair_kernel(n):
    """A tile of 7 instances goes to the generic pair kernel.  The in-place
    kernels run the same FMA sequence per output, so the bits agree."""
    b = inputs.make_batch(2, n, 333, seed=31 + n, x_dist="normal")
    out = []
    for P in (0, 7):
        try:
            kg.set_tile_config(2, n, "f32", "native", P, 1 if P else 0)
            out.append(run_gpu(b, guard=8))
        finally:
            kg.set_tile_config(2, n, "f32", "native", 0, 0)
    Y0, X64 = out[0]
    assert max_norm_err(Y0, oracle_ref(b, X64), b, X64) <= TOL["f32"]
    assert np.array_equal(out[0][0], out[1][0])
