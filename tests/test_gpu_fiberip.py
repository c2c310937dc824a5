"""Parity of the 2-D and 3-D FP32 kernels for odd n whose contractions run in
place (one thread per fiber, tiles of a multiple of 4 packed instances, a ring
of buffers fed by a producer warp) with the FP64 oracle.

Batch sizes cover a single instance, ragged last tiles whose bytes are not a
whole number of 16-byte chunks (the tail is moved by the compute threads), and
enough tiles that every CTA wraps its ring; tile sizes that are not a multiple
of 4 go to the scalar fiber kernel and must agree within the same tolerance."""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, max_norm_err, oracle_ref
from test_gpu_fiber import run_gpu

pytestmark = pytest.mark.gpu

ODD = [3, 5, 7, 9, 11, 13, 15]


@pytest.mark.parametrize("kind", [3, 2])
@pytest.mark.parametrize("n", ODD)
@pytest.mark.parametrize("P,depth", [(0, 0), (4, 1), (8, 2), (12, 3)])
@pytest.mark.parametrize("batch", [1, 5, 203, 2001])
def test_tiles_depths_and_ragged_batches(kind, n, P, depth, batch):
    b = inputs.make_batch(kind, n, batch, seed=800 + n + batch % 53 + P + kind, x_dist="normal")
    try:
        kg.set_tile_config(kind, n, "f32", "native", P, depth)
        Y, X64 = run_gpu(b, guard=64)
    finally:
        kg.set_tile_config(kind, n, "f32", "native", 0, 0)
    assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= TOL["f32"]


@pytest.mark.parametrize("n", [5, 15])
@pytest.mark.parametrize("alpha,beta", [(-0.75, 0.0), (0.5, 2.0)])
def test_alpha_beta(n, alpha, beta):
    batch = 99
    b = inputs.make_batch(3, n, batch, seed=81 + n, x_dist="uniform")
    Y0 = np.random.default_rng(5).standard_normal(batch * n ** 3).astype(np.float32).astype(np.float64)
    Y, X64 = run_gpu(b, alpha=alpha, beta=beta, Y0=Y0.copy(), guard=16)
    ref = oracle_ref(b, X64, alpha=alpha, beta=beta, Y=Y0.copy())
    err = np.abs(ref - Y).reshape(batch, -1).max(axis=1)
    cn = np.prod([np.linalg.norm(np.asarray(M, np.float64)) for M in (b.A, b.B, b.C)])
    scale = cn * np.linalg.norm(X64.reshape(batch, -1), axis=1) * abs(alpha) + \
        abs(beta) * np.linalg.norm(Y0.reshape(batch, -1), axis=1)
    assert float((err / scale).max()) <= TOL["f32"]


@pytest.mark.parametrize("kind", [3, 2])
@pytest.mark.parametrize("n", [7, 15])
def test_agrees_with_fiber_kernel(kind, n):
    b = inputs.make_batch(kind, n, 301, seed=90 + n + kind, x_dist="normal")
    out = []
    for P in (0, 3):
        try:
            kg.set_tile_config(kind, n, "f32", "native", P, 1 if P else 0)
            out.append(run_gpu(b, guard=8))
        finally:
            kg.set_tile_config(kind, n, "f32", "native", 0, 0)
    for Y, X64 in out:
        assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= TOL["f32"]
    assert max_norm_err(out[0][0], out[1][0], b, out[0][1]) <= TOL["f32"]
