"""Results do not depend on the launch configuration: every tile size / pipeline
depth the tuning table can hold gives the oracle's answer, and the autotuner
leaves a configuration that does too."""
import numpy as np
import pytest

import oracle
import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, max_norm_err, oracle_ref, storage_check
from test_gpu_fiber import run_gpu


def check(Y, b, X64, io):
    if io in ("bf16", "f16"):
        assert storage_check(Y, b, X64, io) <= 1.0
    else:
        assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= TOL[io]

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
    check(Y, b, X64, io)


@pytest.mark.parametrize("kind,n", [(2, 16), (3, 16), (2, 9)])
def test_autotune_then_correct(kind, n):
    import torch
    b = inputs.make_batch(kind, n, 4096 if kind == 2 else 512, seed=520 + n, x_dist="normal")
    X = torch.from_numpy(b.X).cuda()
    scratch = torch.empty_like(X)
    P, depth = kg.autotune(kind, n, b.batch, X, scratch)
    # (0, 0) means no candidate beat the built-in default clearly enough; a tile
    # of 0 with a depth is a body's own tile shape with another pipeline depth.
    assert P >= 0 and 0 <= depth <= 8
    assert kg.get_tile_config(kind, n, "f32") == (P, depth)
    try:
        Y, X64 = run_gpu(b)
    finally:
        kg.set_kernel_config(kind, n, "f32")
    assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= TOL["f32"]


# Every kernel body the tuner can choose, with tiles, pipeline depths and fibers
# per step, computes the same operation (a body that does not exist for the
# configuration is refused when it is set).
CONFIGS = [("in_place", 0, 1, 0), ("in_place", 0, 2, 0), ("exchange", 0, 1, 1), ("exchange", 0, 2, 2),
           ("exchange", 7, 1, 2), ("scalar", 0, 1, 0), ("scalar", 5, 2, 0)]


@pytest.mark.parametrize("kind,n,io", [(2, 16, "f32"), (3, 16, "f32"), (2, 10, "f32"), (3, 10, "f32"), (2, 16, "bf16"),
                                       (3, 12, "f16"), (2, 15, "f32"), (3, 7, "f32"), (2, 8, "f64")])
@pytest.mark.parametrize("variant,P,depth,fps", CONFIGS)
def test_kernel_configs_give_the_same_result(kind, n, io, variant, P, depth, fps):
    b = inputs.make_batch(kind, n, 333 if kind == 2 else 45, seed=540 + n, x_dist="normal",
                          dtype=np.float64 if io == "f64" else np.float32)
    try:
        kg.set_kernel_config(kind, n, io, "native", variant, P, depth, fps)
    except kg.KronError as e:
        assert e.status == 2   # KRON_ERR_NOT_SUPPORTED: no such body here
        return
    try:
        assert kg.get_kernel_config(kind, n, io)["variant"] == variant
        Y, X64 = run_gpu(b, io=io, guard=8)
    finally:
        kg.set_kernel_config(kind, n, io)
    check(Y, b, X64, io)


# The FP32 2-D n = 16 in-place body (tiles moved by tensor copies): tiles,
# ring depths and compute-warp groups, on a batch whose last tile is partial,
# with alpha and beta.
@pytest.mark.parametrize("P,depth,warps", [(8, 8, 8), (16, 8, 16), (24, 3, 12), (32, 5, 16), (32, 2, 8), (16, 2, 4),
                                           (8, 1, 2), (32, 12, 16)])
@pytest.mark.parametrize("batch", [1, 7, 1003])
def test_tensor_copy_body_configs(P, depth, warps, batch):
    import torch
    b = inputs.make_batch(2, 16, batch, seed=580 + P + batch, x_dist="normal")
    kg.set_kernel_config(2, 16, "f32", "native", "in_place", P, depth, 0, warps)
    try:
        assert kg.get_kernel_config(2, 16, "f32")["compute_warps"] == warps
        Y, X64 = run_gpu(b, io="f32", guard=8)
        check(Y, b, X64, "f32")
        # beta != 0 reads Y for the live instances of the last tile only
        rng = np.random.default_rng(batch)
        Y0 = rng.standard_normal(batch * 256).astype(np.float32)
        Yd = torch.from_numpy(Y0.copy()).cuda()
        X = torch.from_numpy(b.X).cuda()
        kg.kron2_batched(b.A, b.B, X, Yd, ma=16, na=16, mb=16, nb=16, batch=batch, alpha=0.5, beta=-2.0)
        torch.cuda.synchronize()
        assert kg.device_status() == 0
        R = oracle.kron2(b.A.astype(np.float64), b.B.astype(np.float64), b.X.astype(np.float64), ma=16, na=16, mb=16,
                         nb=16, batch=batch, alpha=0.5, beta=-2.0, Y=Y0.astype(np.float64))
        scale = np.abs(R).max() + 1.0
        assert np.abs(Yd.cpu().numpy().astype(np.float64) - R).max() <= 1e-5 * scale * 16
    finally:
        kg.set_kernel_config(2, 16, "f32")


@pytest.mark.parametrize("kind,n,io", [(3, 16, "f32"), (2, 12, "bf16"), (3, 9, "f32")])
def test_autotune_config_then_correct(kind, n, io):
    import torch
    from paper_1304_7054_gb300 import inputs as inp
    b = inputs.make_batch(kind, n, 4096 if kind == 2 else 600, seed=560 + n, x_dist="normal")
    xt = inp.to_storage(b.X, io) if io != "f32" else torch.from_numpy(b.X)
    X = xt.cuda()
    cfg = kg.autotune_config(kind, n, b.batch, X, torch.empty_like(X))
    assert cfg == kg.get_kernel_config(kind, n, io)
    assert cfg["variant"] in kg.VARIANTS
    try:
        Y, X64 = run_gpu(b, io=io)
    finally:
        kg.set_kernel_config(kind, n, io)
    check(Y, b, X64, io)


# The FP32 2-D in-place bodies for n = 10, 14 and odd n: one to four compute groups of four warps
# sharing a CTA's ring, tiles of multiples of 8 instances, several ring depths;
# every configuration gives the same bits (the same arithmetic per instance).
@pytest.mark.parametrize("n", [10, 14, 15, 7])
@pytest.mark.parametrize("batch", [5, 1001])
def test_in_place_groups_same_bits(n, batch):
    b = inputs.make_batch(2, n, batch, seed=600 + n + batch, x_dist="normal")
    outs = []
    try:
        shapes = [(48, 1, 4), (48, 10, 16), (40, 5, 16), (16, 6, 12), (8, 3, 8), (24, 12, 16)]
        if n % 2:   # odd n: tiles of a multiple of 4 instances
            shapes = [(24, 2, 4), (24, 8, 16), (12, 6, 12), (4, 3, 8), (8, 12, 16), (44, 1, 16)]
        for P, depth, warps in shapes:
            kg.set_kernel_config(2, n, "f32", "native", "in_place", P, depth, 0, warps)
            Y, X64 = run_gpu(b, io="f32", guard=8)
            outs.append(Y)
    finally:
        kg.set_kernel_config(2, n, "f32")
    for Y in outs[1:]:
        assert np.array_equal(Y, outs[0])
    check(outs[0], b, X64, "f32")
