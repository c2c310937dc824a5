"""Parity of the tensor-core split-precision path (KRON_COMPUTE_32F_BF16X3).

Error bound (derived from the split): with bfloat16 unit roundoff u = 2^-8, the
parts hi = bf16(v), lo = bf16(v - hi) leave a residual below u^2 |v|, and the
dropped lo*lo product is below u^2 |a b|, so each contraction adds at most
3 u^2 = 3 * 2^-16 relative to sum |a||b|; summed over the contractions of a
2-D (two) or 3-D (three) action and normalised as in the FP32 tests
(|Y_ij| <= ||A|| ||B|| (||C||) ||X||), the normalised error is at most
kind * 3 * 2^-16 plus FP32 accumulation.  From n >= 2 on, the seeded inputs
must also meet the FP32 target of 1e-5 ("recovers FP32-level accuracy"); at
n = 1 an output is a single product, nothing averages, and only the bound holds.
"""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, max_norm_err, oracle_ref, storage_check, storage_x, torch_dtype
from test_gpu_fiber import run_gpu

pytestmark = pytest.mark.gpu


def bound(kind, n):
    return kind * 3 * 2.0 ** -16 + 2 * kind * n * 2.0 ** -24


@pytest.mark.parametrize("n", list(range(1, 17)))
def test_bf16x3_2d_all_sizes(n):
    b = inputs.make_batch(2, n, 1037, seed=300 + n, x_dist="normal")
    Y, X64 = run_gpu(b, io="f32", compute="bf16x3", guard=16)
    err = max_norm_err(Y, oracle_ref(b, X64), b, X64)
    assert err <= bound(2, n)
    if n >= 2:
        assert err <= 1e-5, err


@pytest.mark.parametrize("n", [4, 8, 12, 16, 7])
def test_bf16x3_2d_bf16_storage(n):
    b = inputs.make_batch(2, n, 513, seed=320 + n, x_dist="normal")
    Y, X64 = run_gpu(b, io="bf16", compute="bf16x3", guard=16)
    assert storage_check(Y, b, X64, "bf16", compute="bf16x3") <= 1.0


@pytest.mark.parametrize("n", [3, 4, 6, 8, 16])
def test_bf16x3_bf16_storage_identity_is_exact(n):
    """Small n share a tile (instances on its diagonal); identity stays exact."""
    b = inputs.make_batch(2, n, 201, seed=330)
    b.A = np.eye(n).ravel(order="F").astype(np.float32)
    b.B = b.A.copy()
    Y, X64 = run_gpu(b, io="bf16", compute="bf16x3")
    assert np.array_equal(Y, X64)


@pytest.mark.parametrize("kind,n", [(2, 16), (2, 5)])
def test_bf16x3_alpha_beta(kind, n):
    b = inputs.make_batch(kind, n, 99, seed=340 + n, x_dist="normal")
    rng = np.random.default_rng(1)
    Y0 = rng.standard_normal(b.batch * n ** kind).astype(np.float32).astype(np.float64)
    Y, X64 = run_gpu(b, io="f32", compute="bf16x3", alpha=0.75, beta=-2.0, Y0=Y0, guard=8)
    ref = oracle_ref(b, X64, alpha=0.75, beta=-2.0, Y=Y0)
    assert max_norm_err(Y, ref, b, X64) <= 2 * bound(kind, n) + 1e-6


@pytest.mark.parametrize("n", [3, 6, 8])
@pytest.mark.parametrize("P,depth", [(3, 1), (7, 2), (33, 3)])
def test_bf16x3_2d_packed_tiles_any_tile_size(n, P, depth):
    """Odd tile sizes leave the last pair / quadruple of a tile half filled."""
    b = inputs.make_batch(2, n, 1001, seed=350 + n + P, x_dist="normal")
    try:
        kg.set_tile_config(2, n, "f32", "bf16x3", P, depth)
        Y, X64 = run_gpu(b, io="f32", compute="bf16x3", guard=16)
    finally:
        kg.set_tile_config(2, n, "f32", "bf16x3", 0, 0)
    assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= 1e-5


def test_bf16x3_full_size_sampled():
    import torch
    batch, n = 1 << 20, 16
    b = inputs.make_batch(2, n, batch, seed=4, x_dist="normal")
    X = torch.from_numpy(b.X).cuda()
    Y = torch.empty_like(X)
    kg.kron2_batched(b.A, b.B, X, Y, ma=n, na=n, mb=n, nb=n, batch=batch, compute="bf16x3")
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(6).choice(batch, 1024, replace=False))
    idx[-1] = batch - 1
    Xs = b.X.reshape(batch, 256)[idx].astype(np.float64).ravel()
    sub = inputs.Batch(2, n, len(idx), b.A, b.B, None, Xs)
    got = Y.view(batch, 256)[torch.from_numpy(idx).cuda()].double().cpu().numpy().ravel()
    assert max_norm_err(got, oracle_ref(sub, Xs), sub, Xs) <= 1e-5


def test_bf16x3_rejects_unsupported_layouts():
    import torch
    X = torch.zeros(64 * 20, device="cuda")
    Y = torch.zeros(64 * 20, device="cuda")
    with pytest.raises(kg.KronError) as e:
        kg.kron2_batched(np.eye(8), np.eye(8), X, Y, ma=8, na=8, mb=8, nb=8, batch=10, ldx=9, ldxp=80,
                         compute="bf16x3")
    assert e.value.status == 2
    Xd = torch.zeros(8 * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(kg.KronError) as e:
        kg.kron2_batched(np.eye(8), np.eye(8), Xd, torch.zeros_like(Xd), ma=8, na=8, mb=8, nb=8, batch=8,
                         compute="bf16x3")
    assert e.value.status == 2


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12, 14, 16])
def test_bf16x3_3d_even_sizes(n):
    b = inputs.make_batch(3, n, 203, seed=400 + n, x_dist="normal")
    Y, X64 = run_gpu(b, io="f32", compute="bf16x3", guard=16)
    err = max_norm_err(Y, oracle_ref(b, X64), b, X64)
    assert err <= bound(3, n)
    assert err <= 1e-5, err


@pytest.mark.parametrize("n", [10, 16])
@pytest.mark.parametrize("batch", [1, 3, 4099])
def test_bf16x3_3d_ragged_and_wrapping_batches(n, batch):
    """Batches that leave warps idle and batches that wrap every warp several
    times (n = 10 fetches the next instance while mode 3 runs, n = 16 after it)."""
    b = inputs.make_batch(3, n, batch, seed=420 + batch + n, x_dist="normal")
    Y, X64 = run_gpu(b, io="f32", compute="bf16x3", guard=16)
    assert max_norm_err(Y, oracle_ref(b, X64), b, X64) <= 1e-5


def test_bf16x3_3d_alpha_beta():
    n = 16
    b = inputs.make_batch(3, n, 37, seed=410, x_dist="normal")
    Y0 = np.random.default_rng(2).standard_normal(b.batch * n ** 3).astype(np.float32).astype(np.float64)
    Y, X64 = run_gpu(b, io="f32", compute="bf16x3", alpha=-0.5, beta=1.5, Y0=Y0, guard=8)
    ref = oracle_ref(b, X64, alpha=-0.5, beta=1.5, Y=Y0)
    assert max_norm_err(Y, ref, b, X64) <= 2 * bound(3, n) + 1e-6


def test_bf16x3_3d_full_size_sampled():
    import torch
    batch, n = 1 << 16, 16
    b = inputs.make_batch(3, n, batch, seed=5, x_dist="normal")
    X = torch.from_numpy(b.X).cuda()
    Y = torch.empty_like(X)
    kg.kron3_batched(b.A, b.B, b.C, X, Y, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch, compute="bf16x3")
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    idx = np.sort(np.random.default_rng(7).choice(batch, 256, replace=False))
    idx[-1] = batch - 1
    Xs = b.X.reshape(batch, 4096)[idx].astype(np.float64).ravel()
    sub = inputs.Batch(3, n, len(idx), b.A, b.B, b.C, Xs)
    got = Y.view(batch, 4096)[torch.from_numpy(idx).cuda()].double().cpu().numpy().ravel()
    assert max_norm_err(got, oracle_ref(sub, Xs), sub, Xs) <= 1e-5


def test_bf16x3_3d_odd_size_not_supported():
    import torch
    X = torch.zeros(5 * 125, device="cuda")
    with pytest.raises(kg.KronError) as e:
        kg.kron3_batched(np.eye(5), np.eye(5), np.eye(5), X, torch.zeros_like(X), ma=5, na=5, mb=5, nb=5, mc=5,
                         nc=5, batch=5, compute="bf16x3")
    assert e.value.status == 2
