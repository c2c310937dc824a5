"""Parity of the 2-D n = 16 FP32 kernel whose exchange is done in place
(16 instances per tile, a ring of 1 to 4 tile buffers fed by a producer warp)
with the FP64 oracle.

Batch sizes cover a single instance, ragged last tiles (1, 15, 17, 1037), an
exact multiple of the tile, and enough tiles that every CTA wraps its ring of
buffers several times; each run checks that nothing beyond Y is written and
that X is left as it was."""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, max_norm_err, oracle_ref
from test_gpu_fiber import run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("depth", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("batch", [1, 15, 16, 17, 1037, 40000])
def test_ring_depths_and_ragged_tiles(depth, batch):
    b = inputs.make_batch(2, 16, batch, seed=900 + batch % 97 + depth, x_dist="normal")
    try:
        kg.set_tile_config(2, 16, "f32", "native", 16 if depth else 0, depth)
        Y, X64 = run_gpu(b, guard=64)
    finally:
        kg.set_tile_config(2, 16, "f32", "native", 0, 0)
    assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= TOL["f32"]


@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.75, 0.0), (0.5, 2.0), (1.0, -1.0)])
def test_alpha_beta_ragged(alpha, beta):
    b = inputs.make_batch(2, 16, 1037, seed=77, x_dist="uniform")
    Y0 = np.random.default_rng(3).standard_normal(1037 * 256)
    Y, X64 = run_gpu(b, alpha=alpha, beta=beta, Y0=Y0.astype(np.float32).astype(np.float64), guard=16)
    ref = oracle_ref(b, X64, alpha=alpha, beta=beta, Y=Y0.astype(np.float32).astype(np.float64))
    # beta * Y0 adds |beta| ||Y0_p|| to the scale of each instance's result
    scale = np.abs(ref - Y).reshape(1037, 256).max(axis=1)
    norm = np.linalg.norm(np.asarray(b.A, np.float64)) * np.linalg.norm(np.asarray(b.B, np.float64)) * \
        np.linalg.norm(X64.reshape(1037, 256), axis=1) * abs(alpha) + \
        abs(beta) * np.linalg.norm(Y0.reshape(1037, 256), axis=1)
    assert float((scale / norm).max()) <= TOL["f32"]


def test_tile_size_other_than_16_uses_generic_kernel():
    """Instances per tile != 16 go to the generic pair kernel; same answer."""
    b = inputs.make_batch(2, 16, 333, seed=31, x_dist="normal")
    out = []
    for P in (0, 8):
        try:
            kg.set_tile_config(2, 16, "f32", "native", P, 1 if P else 0)
            out.append(run_gpu(b, guard=8))
        finally:
            kg.set_tile_config(2, 16, "f32", "native", 0, 0)
    for Y, X64 in out:
        assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= TOL["f32"]
    # both kernels run the same FMA sequence per output: results agree bit for bit
    assert np.array_equal(out[0][0], out[1][0])
