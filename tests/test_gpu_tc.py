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


@pytest.mark.parametrize("io", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n", [1, 3, 5, 7, 9, 11, 13, 15])
def test_bf16x3_3d_odd_sizes(n, io):
    """Odd n: an instance is not a whole number of 16-byte units, so each copy takes
    the aligned span around it and the instance sits at its phase; a ragged
    batch puts every phase in play."""
    b = inputs.make_batch(3, n, 71, seed=400 + n, x_dist="normal")
    Y, X64 = run_gpu(b, io=io, compute="bf16x3", guard=16)
    if io == "f32":
        err = max_norm_err(Y, oracle_ref(b, X64), b, X64)
        assert err <= bound(3, n)
        if n >= 2:
            assert err <= 1e-5, err
    else:
        assert storage_check(Y, b, X64, io, compute="bf16x3") <= 1.0


# --- 16-bit storage on the tensor cores: the stored operand is exact in the split
# (bf16: lo = 0; f16: 11 significant bits = bf16 hi + lo), so the arithmetic error
# is the components' split and the FP32 accumulation; every output must lie within
# the storage type's rounding of the exact result (helpers.storage_check) ---------
@pytest.mark.parametrize("io", ["bf16", "f16"])
@pytest.mark.parametrize("n", [2, 5, 8, 12, 15, 16])
def test_bf16x3_2d_16bit_storage(io, n):
    b = inputs.make_batch(2, n, 777, seed=360 + n, x_dist="normal")
    Y, X64 = run_gpu(b, io=io, compute="bf16x3", guard=16)
    assert storage_check(Y, b, X64, io, compute="bf16x3") <= 1.0


@pytest.mark.parametrize("io", ["bf16", "f16"])
@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12, 14, 16])
def test_bf16x3_3d_16bit_storage(io, n):
    b = inputs.make_batch(3, n, 67, seed=380 + n, x_dist="normal")
    Y, X64 = run_gpu(b, io=io, compute="bf16x3", guard=16)
    assert storage_check(Y, b, X64, io, compute="bf16x3") <= 1.0


@pytest.mark.parametrize("io", ["bf16", "f16"])
@pytest.mark.parametrize("kind,n", [(2, 16), (2, 6), (3, 16), (3, 8)])
def test_bf16x3_16bit_storage_identity_is_exact(io, kind, n):
    b = inputs.make_batch(kind, n, 41, seed=390)
    I = np.eye(n).ravel(order="F").astype(np.float32)
    b.A, b.B = I, I.copy()
    if kind == 3:
        b.C = I.copy()
    Y, X64 = run_gpu(b, io=io, compute="bf16x3")
    assert np.array_equal(Y, X64)


@pytest.mark.parametrize("kind,n,batch,io", [(3, 16, 1 << 16, "bf16"), (3, 16, 1 << 16, "f16"),
                                             (2, 16, 1 << 20, "f16"), (2, 12, 1 << 20, "bf16")])
def test_bf16x3_16bit_storage_full_size_sampled(kind, n, batch, io):
    """The 16-bit tensor-core launches the benchmark times, on sampled instances."""
    import torch
    b = inputs.make_batch(kind, n, batch, seed=4, x_dist="normal")
    inst = n ** kind
    xt, X64 = storage_x(b, io)
    X = xt.to(torch_dtype(io)).cuda()
    Y = torch.empty_like(X)
    if kind == 2:
        kg.kron2_batched(b.A, b.B, X, Y, ma=n, na=n, mb=n, nb=n, batch=batch, compute="bf16x3")
    else:
        kg.kron3_batched(b.A, b.B, b.C, X, Y, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch, compute="bf16x3")
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(batch, 512, replace=False))
    idx[-1] = batch - 1
    Xs = X64.reshape(batch, inst)[idx].ravel()
    sub = inputs.Batch(kind, n, len(idx), b.A, b.B, b.C, Xs)
    got = Y.view(batch, inst)[torch.from_numpy(idx).cuda()].double().cpu().numpy().ravel()
    assert storage_check(got, sub, Xs, io, compute="bf16x3") <= 1.0
    del X, Y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("io", ["bf16", "f16"])
@pytest.mark.parametrize("guard", [7, 8])
def test_bf16x3_3d_16bit_results_at_any_alignment(io, guard):
    """16-bit results leave as 32-bit pairs when Y is 4-byte aligned (guard 8) and
    element by element otherwise (guard 7: Y two bytes past a 4-byte boundary)."""
    b = inputs.make_batch(3, 16, 37, seed=395 + guard, x_dist="normal")
    Y, X64 = run_gpu(b, io=io, compute="bf16x3", guard=guard)
    assert storage_check(Y, b, X64, io, compute="bf16x3") <= 1.0


@pytest.mark.parametrize("io", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n", [16, 15, 13, 10, 6])
def test_bf16x3_3d_warps_per_instance(io, n):
    """The single-warp kernel and 2, 4, 8 warps sharing an instance give the same bits."""
    b = inputs.make_batch(3, n, 43, seed=397 + n, x_dist="normal")
    outs = []
    try:
        for w in (1, 2, 4, 8):
            kg.set_kernel_config(3, n, io, "bf16x3", compute_warps=w)
            assert kg.get_kernel_config(3, n, io, "bf16x3")["compute_warps"] == w
            Y, X64 = run_gpu(b, io=io, compute="bf16x3", guard=8)
            outs.append(Y)
    finally:
        kg.set_kernel_config(3, n, io, "bf16x3")
    for Y in outs[1:]:
        assert np.array_equal(Y, outs[0])
    if io == "f32":
        assert max_norm_err(outs[0], oracle_ref(b, X64), b, X64) <= 1e-5
    else:
        assert storage_check(outs[0], b, X64, io, compute="bf16x3") <= 1.0


# --- 2-D stacked body: G = 8 / gcd(n, 8) instances side by side along the MMA's N
# dimension, intermediates through per-warp exchange rows (variant "exchange") ---------
def _stacked_and_padded(b, io, guard, alpha=1.0, beta=0.0, Y0=None, P=0, depth=0, groups=0):
    n, outs = b.n, {}
    try:
        for var in ("in_place", "exchange"):
            kg.set_kernel_config(2, n, io, "bf16x3", variant=var, instances_per_tile=P, pipeline_depth=depth,
                                 fibers_per_step=groups if var == "exchange" else 0)
            assert kg.get_kernel_config(2, n, io, "bf16x3")["variant"] == var
            outs[var], X64 = run_gpu(b, io=io, compute="bf16x3", alpha=alpha, beta=beta, Y0=Y0, guard=guard)
    finally:
        kg.set_kernel_config(2, n, io, "bf16x3")
    return outs, X64


def _check_tc(Y, b, X64, io, **kw):
    if io == "f32":
        ref = oracle_ref(b, X64, **({} if kw.get("beta", 0.0) == 0.0 else
                                    dict(alpha=kw["alpha"], beta=kw["beta"], Y=np.array(kw["Y0"], np.float64))))
        tol = 1e-5 if kw.get("beta", 0.0) == 0.0 else 2 * bound(2, b.n) + 1e-6
        assert max_norm_err(Y, ref, b, X64) <= tol
    else:
        assert storage_check(Y, b, X64, io, compute="bf16x3", **kw) <= 1.0


@pytest.mark.parametrize("io", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n", [9, 10, 11, 12, 13, 14, 15, 16])
@pytest.mark.parametrize("guard", [8, 7])
def test_bf16x3_2d_stacked_body(io, n, guard):
    """Ragged batch (the last tile and the last group half filled); Y at an offset
    where results leave as pairs (guard 8) and where they cannot (guard 7).  The two
    bodies form every output from the same MMA products in the same order, so they
    agree bit for bit."""
    b = inputs.make_batch(2, n, 1037, seed=410 + n, x_dist="normal")
    outs, X64 = _stacked_and_padded(b, io, guard)
    _check_tc(outs["exchange"], b, X64, io)
    assert np.array_equal(outs["exchange"], outs["in_place"])


@pytest.mark.parametrize("io", ["f32", "bf16"])
@pytest.mark.parametrize("n", [12, 13])
@pytest.mark.parametrize("P,depth", [(5, 1), (24, 2), (40, 3), (128, 1)])
def test_bf16x3_2d_stacked_any_tile(io, n, P, depth):
    """Tiles that are not a whole number of groups, and every ring depth."""
    b = inputs.make_batch(2, n, 2003, seed=430 + n + P, x_dist="normal")
    outs, X64 = _stacked_and_padded(b, io, 8, P=P, depth=depth)
    _check_tc(outs["exchange"], b, X64, io)


@pytest.mark.parametrize("io", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n", [12, 15])
def test_bf16x3_2d_stacked_alpha_beta(io, n):
    b = inputs.make_batch(2, n, 301, seed=440 + n, x_dist="normal")
    rng = np.random.default_rng(3)
    Y0 = rng.standard_normal(b.batch * n * n).astype(np.float32)
    if io != "f32":
        Y0 = storage_x(inputs.Batch(2, n, b.batch, b.A, b.B, None, Y0), io)[1]
    Y0 = np.asarray(Y0, np.float64)
    outs, X64 = _stacked_and_padded(b, io, 8, alpha=0.75, beta=-2.0, Y0=Y0)
    _check_tc(outs["exchange"], b, X64, io, alpha=0.75, beta=-2.0, Y0=Y0)


@pytest.mark.parametrize("io", ["bf16", "f16"])
def test_bf16x3_2d_stacked_identity_is_exact(io):
    b = inputs.make_batch(2, 12, 203, seed=450)
    I = np.eye(12).ravel(order="F").astype(np.float32)
    b.A, b.B = I, I.copy()
    outs, X64 = _stacked_and_padded(b, io, 8)
    assert np.array_equal(outs["exchange"], X64)


@pytest.mark.parametrize("io", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("n", [10, 12, 14, 16])
@pytest.mark.parametrize("P", [0, 40])
def test_bf16x3_2d_stacked_two_groups_per_step(io, n, P):
    """Two groups of stacked instances per warp step (fibers_per_step 2): the same bits as
    the padded tile, with the last groups of a ragged batch partly or wholly absent."""
    b = inputs.make_batch(2, n, 1037, seed=460 + n + P, x_dist="normal")
    outs, X64 = _stacked_and_padded(b, io, 8, P=P, depth=2 if P else 0, groups=2)
    _check_tc(outs["exchange"], b, X64, io)
    assert np.array_equal(outs["exchange"], outs["in_place"])
