"""Results do not depend on the launch configuration: every tile size / pipeline
depth the tuning table can hold gives the oracle's answer, and the autotuner
leaves a configuration that does too."""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, max_norm_err, oracle_ref
from test_gpu_fiber import run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,n,io", [(2, 16, "f32"), (2, 10, "f32"), (3, 16, "f32"), (3, 10, "f32"),
                                       (2, 16, "bf16"), (3, 7, "f32"), (2, 5, "f64"), (3, 12, "f16")])
@pytest.mark.parametrize("P,depth", [(1, 1), (3, 2), (7, 1), (16, 3), (40, 2)])
def test_tile_configs_give_the_same_result(kind, n, io, P, depth):
    b = inputs.make_batch(kind, n, 333 if kind == 2 else 45, seed=500 + n, x_dist="normal",
                          dtype=np.float64 if io == "f64" else np.float32)
    try:
        kg.set_tile_config(kind, n, io, "native", P, depth)
        Y, X64 = run_gpu(b, io=io, guard=8)
    finally:
        kg.set_tile_config(kind, n, io, "native", 0, 0)
    assert max_norm_err(Y, oracle_ref(b, X64), b, X64, io) <= TOL[io]


@pytest.mark.parametrize("kind,n", [(2, 16), (3, 16), (2, 9)])
def test_autotune_then_correct(kind, n):
    import torch
    b = inputs.make_batch(kind, n, 4096 if kind == 2 else 512, seed=520 + n, x_dist="normal")
    X = torch.from_numpy(b.X).cuda()
    scratch = torch.empty_like(X)
    P, depth = kg.autotune(kind, n, b.batch, X, scratch)
    # (0, 0) means no candidate beat the built-in default clearly enough.
    assert (P, depth) == (0, 0) or (P >= 1 and depth >= 1)
    assert kg.get_tile_config(kind, n, "f32") == (P, depth)
    try:
        Y, X64 = run_gpu(b)
    finally:
        kg.set_tile_config(kind, n, "f32", "native", 0, 0)
    assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= TOL["f32"]
