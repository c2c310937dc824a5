"""Parity of the CUDA-core kernels (KRON_COMPUTE_NATIVE) with the oracle.

Every call goes through the C ABI (ctypes binding).  Floating-point parity is
checked per instance against the FP64 oracle with the normalised error of the
target accuracy (max |Y - Y_ref| / (||A|| ||B|| (||C||) ||X^p||)): FP32 <= 1e-5,
FP64 <= 1e-13.  16-bit storage is checked element by element: within half an
ulp of the storage type of the exact result, plus the componentwise bound of
the FP32 arithmetic before that one rounding (helpers.storage_check).  Exact
cases (identity, permutations, powers of two) are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, max_norm_err, oracle_ref, storage_check, storage_x, torch_dtype, np_dtype

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def run_gpu(b, io="f32", compute="native", alpha=1.0, beta=0.0, Y0=None, guard=0):
    """Run one batch through the library; returns (Y as float64 numpy, X as float64)."""
    torch = _torch()
    xt, X64 = storage_x(b, io)
    X = xt.to(torch_dtype(io)).cuda()
    total = b.batch * b.n ** b.kind
    if Y0 is None:
        Ybuf = torch.full((total + 2 * guard,), float("nan"), dtype=torch_dtype(io), device="cuda")
    else:
        Ybuf = torch.tensor(np.concatenate([np.full(guard, np.nan), Y0, np.full(guard, np.nan)]),
                            dtype=torch_dtype(io), device="cuda")
    Y = Ybuf[guard:guard + total]
    n = b.n
    if b.kind == 2:
        kg.kron2_batched(b.A, b.B, X, Y, ma=n, na=n, mb=n, nb=n, batch=b.batch, alpha=alpha, beta=beta,
                         compute=compute)
    else:
        kg.kron3_batched(b.A, b.B, b.C, X, Y, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=b.batch,
                         alpha=alpha, beta=beta, compute=compute)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    out = Ybuf.to(torch.float64).cpu().numpy()
    if guard:
        assert np.isnan(out[:guard]).all() and np.isnan(out[-guard:]).all(), "guard band written"
    assert torch.equal(X.cpu(), xt.to(torch_dtype(io))), "X modified"
    return out[guard:guard + total], X64


# --- config 1: 2-D n=4, batch 1024, uniform[-1,1] from seed 0 ---------------------------------
def test_config1_vs_oracle_and_explicit_kron():
    b = inputs.make_batch(2, 4, 1024, seed=0, x_dist="uniform")
    Y, X64 = run_gpu(b, guard=64)
    ref = oracle_ref(b, X64)
    assert max_norm_err(Y, ref, b, X64) <= TOL["f32"]
    # brute force: the explicit 16 x 16 A (x) B of the paper's block definition
    A = np.asarray(b.A, np.float64).reshape(4, 4).T
    B = np.asarray(b.B, np.float64).reshape(4, 4).T
    K = oracle.kron_matrix(A, B)
    for p in range(0, 1024, 37):
        y = oracle.matvec(K, X64[16 * p:16 * p + 16])
        np.testing.assert_allclose(Y[16 * p:16 * p + 16], y, rtol=0, atol=1e-5 * np.abs(y).max() + 1e-6)


# --- every size, both kinds, FP32 and FP64, ragged batch -------------------------------------
@pytest.mark.parametrize("io", ["f32", "f64"])
@pytest.mark.parametrize("n", list(range(1, 17)))
@pytest.mark.parametrize("kind", [2, 3])
def test_all_sizes(kind, n, io):
    batch = 1037 if kind == 2 else 203
    b = inputs.make_batch(kind, n, batch, seed=100 + n + 17 * kind, x_dist="normal", dtype=np_dtype(io))
    Y, X64 = run_gpu(b, io=io, guard=32)
    ref = oracle_ref(b, X64)
    assert max_norm_err(Y, ref, b, X64) <= TOL[io]


@pytest.mark.parametrize("io", ["bf16", "f16"])
@pytest.mark.parametrize("n", list(range(1, 17)))
@pytest.mark.parametrize("kind", [2, 3])
def test_16bit_storage(kind, n, io):
    batch = 777 if kind == 2 else 65
    b = inputs.make_batch(kind, n, batch, seed=200 + n + kind, x_dist="normal")
    Y, X64 = run_gpu(b, io=io, guard=16)
    assert storage_check(Y, b, X64, io) <= 1.0   # oracle on the stored (rounded) operand values


@pytest.mark.parametrize("io", ["bf16", "f16"])
@pytest.mark.parametrize("kind,n", [(2, 16), (2, 12), (3, 16)])
def test_16bit_check_catches_planted_coefficient_error(kind, n, io):
    """The check that passes the kernel's result must fail it against an oracle
    whose copy of A has one coefficient scaled by 1 + 2^-8 (the mistake is
    planted in the oracle's inputs, on the CPU)."""
    b = inputs.make_batch(kind, n, 777 if kind == 2 else 65, seed=216 + n, x_dist="normal")
    Y, X64 = run_gpu(b, io=io)
    assert storage_check(Y, b, X64, io) <= 1.0
    bad = inputs.Batch(kind, n, b.batch, b.A.astype(np.float64).copy(), b.B, b.C, None)
    bad.A[0] *= 1.0 + 2.0 ** -8
    assert storage_check(Y, b, X64, io, ref=oracle_ref(bad, X64)) > 1.0


# --- exact cases ------------------------------------------------------------------------------
@pytest.mark.parametrize("io", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("kind,n", [(2, 4), (2, 7), (2, 16), (3, 5), (3, 16)])
def test_identity_bitwise(kind, n, io):
    b = inputs.make_batch(kind, n, 300, seed=7, x_dist="normal", dtype=np_dtype(io))
    I = np.eye(n).ravel(order="F").astype(np_dtype(io))
    b.A, b.B = I, I.copy()
    if kind == 3:
        b.C = I.copy()
    Y, X64 = run_gpu(b, io=io)
    assert np.array_equal(Y, X64)


@pytest.mark.parametrize("kind,n", [(2, 8), (2, 16), (3, 6), (3, 16)])
def test_permutation_pow2_bitwise(kind, n):
    rng = np.random.default_rng(n + kind)
    b = inputs.make_batch(kind, n, 64, seed=9, x_dist="normal")
    mats = []
    for _ in range(kind):
        P = np.eye(n)[rng.permutation(n)] * (2.0 ** rng.integers(-3, 4, n))[:, None]
        mats.append(P)
    b.A = mats[0].ravel(order="F").astype(np.float32)
    b.B = mats[1].ravel(order="F").astype(np.float32)
    if kind == 3:
        b.C = mats[2].ravel(order="F").astype(np.float32)
    Y, X64 = run_gpu(b)
    ref = oracle_ref(b, X64)   # a single nonzero product per output: exact in any precision
    assert np.array_equal(Y, ref)


# --- alpha / beta (Sec. 2.2) ------------------------------------------------------------------
@pytest.mark.parametrize("io", ["f32", "f64"])
@pytest.mark.parametrize("kind,n", [(2, 16), (2, 5), (3, 16), (3, 7)])
def test_alpha_beta(kind, n, io):
    b = inputs.make_batch(kind, n, 129, seed=11, x_dist="normal", dtype=np_dtype(io))
    rng = np.random.default_rng(3)
    Y0 = rng.standard_normal(b.batch * n ** kind)
    if io == "f32":
        Y0 = Y0.astype(np.float32).astype(np.float64)
    Y, X64 = run_gpu(b, io=io, alpha=-1.25, beta=0.5, Y0=Y0, guard=8)
    ref = oracle_ref(b, X64, alpha=-1.25, beta=0.5, Y=Y0)
    assert max_norm_err(Y, ref, b, X64) <= 2 * TOL[io]


def test_beta_zero_ignores_nan():
    b = inputs.make_batch(2, 16, 50, seed=12)
    Y, X64 = run_gpu(b, beta=0.0)   # Y starts NaN-filled
    assert not np.isnan(Y).any()


# --- strided / transposed / rectangular / misaligned operands (generic loader) ------------------
def _colmaj(M):
    return np.ascontiguousarray(np.asarray(M).T).ravel()


@pytest.mark.parametrize("io", ["f32", "f64"])
@pytest.mark.parametrize("shape,trans,lds", [
    ((16, 16, 16, 16), "NNN", (19, 300, 17, 290)),
    ((5, 7, 3, 9), "NNN", (11, 80, 4, 30)),
    ((8, 8, 8, 8), "TTT", (8, 64, 8, 64)),
    ((12, 3, 6, 10), "TNT", (5, 60, 7, 100)),
    ((1, 16, 16, 1), "NTN", (1, 16, 16, 16)),
])
def test_general_2d(shape, trans, lds, io):
    torch = _torch()
    ma, na, mb, nb = shape
    ta, tb, tx = trans
    ldx, ldxp, ldy, ldyp = lds
    batch = 91
    rng = np.random.default_rng(sum(shape))
    dt = np_dtype(io)
    A = rng.uniform(-1, 1, (ma, na)).astype(dt)
    B = rng.uniform(-1, 1, (mb, nb)).astype(dt)
    Ast = A.T if ta == "T" else A
    Bst = B.T if tb == "T" else B
    X = rng.standard_normal(batch * ldxp + 3).astype(dt)
    Y = torch.full((batch * ldyp + 5,), float("nan"), dtype=torch_dtype(io), device="cuda")
    Xd = torch.from_numpy(X).cuda()
    kg.kron2_batched(Ast, Bst, Xd, Y, ma=ma, na=na, mb=mb, nb=nb, batch=batch, transa=ta, transb=tb,
                     transx=tx, ldx=ldx, ldxp=ldxp, ldy=ldy, ldyp=ldyp)
    ref = oracle.kron2(_colmaj(Ast), _colmaj(Bst), X.astype(np.float64), ma=ma, na=na, mb=mb, nb=nb,
                       batch=batch, transa=ta, transb=tb, transx=tx, ldx=ldx, ldxp=ldxp, ldy=ldy,
                       ldyp=ldyp, Y=np.full(batch * ldyp + 5, np.nan))
    got = Y.to(torch.float64).cpu().numpy()
    written = ~np.isnan(ref)
    assert np.array_equal(np.isnan(got), ~written), "written set differs from the oracle's"
    scale = np.linalg.norm(A) * np.linalg.norm(B) * np.abs(X).max() * max(na, nb)
    assert np.abs(got[written] - ref[written]).max() <= TOL[io] * scale


@pytest.mark.parametrize("io", ["f32", "f64"])
@pytest.mark.parametrize("shape,trans,lds", [
    ((16, 16, 16, 16, 16, 16), "NNN", (17, 290, 4700, 16, 300, 5000)),
    ((4, 6, 5, 3, 7, 2), "TNT", (3, 9, 70, 8, 50, 300)),
    ((10, 10, 10, 10, 10, 10), "TTT", (10, 100, 1000, 10, 100, 1000)),
])
def test_general_3d(shape, trans, lds, io):
    torch = _torch()
    ma, na, mb, nb, mc, nc = shape
    ta, tb, tc = trans
    ldx, ldx2, ldxp, ldy, ldy2, ldyp = lds
    batch = 23
    rng = np.random.default_rng(sum(shape) + 1)
    dt = np_dtype(io)
    A, B, C = (rng.uniform(-1, 1, s).astype(dt) for s in ((ma, na), (mb, nb), (mc, nc)))
    st = lambda M, t: M.T if t == "T" else M
    X = rng.standard_normal(batch * ldxp + 3).astype(dt)
    Y = torch.full((batch * ldyp + 5,), float("nan"), dtype=torch_dtype(io), device="cuda")
    kg.kron3_batched(st(A, ta), st(B, tb), st(C, tc), torch.from_numpy(X).cuda(), Y, ma=ma, na=na, mb=mb,
                     nb=nb, mc=mc, nc=nc, batch=batch, transa=ta, transb=tb, transc=tc, ldx=ldx, ldx2=ldx2,
                     ldxp=ldxp, ldy=ldy, ldy2=ldy2, ldyp=ldyp)
    ref = oracle.kron3(_colmaj(st(A, ta)), _colmaj(st(B, tb)), _colmaj(st(C, tc)), X.astype(np.float64),
                       ma=ma, na=na, mb=mb, nb=nb, mc=mc, nc=nc, batch=batch, transa=ta, transb=tb,
                       transc=tc, ldx=ldx, ldx2=ldx2, ldxp=ldxp, ldy=ldy, ldy2=ldy2, ldyp=ldyp,
                       Y=np.full(batch * ldyp + 5, np.nan))
    got = Y.to(torch.float64).cpu().numpy()
    written = ~np.isnan(ref)
    assert np.array_equal(np.isnan(got), ~written)
    scale = np.linalg.norm(A) * np.linalg.norm(B) * np.linalg.norm(C) * np.abs(X).max() * 16
    assert np.abs(got[written] - ref[written]).max() <= TOL[io] * scale


def test_misaligned_operand_uses_generic_path():
    torch = _torch()
    b = inputs.make_batch(2, 16, 100, seed=13)
    X = torch.from_numpy(np.concatenate([[0.0], b.X]).astype(np.float32)).cuda()[1:]   # 4-byte offset
    Y = torch.empty(100 * 256, dtype=torch.float32, device="cuda")
    kg.kron2_batched(b.A, b.B, X, Y, ma=16, na=16, mb=16, nb=16, batch=100)
    ref = oracle_ref(b, b.X.astype(np.float64))
    assert max_norm_err(Y.double().cpu().numpy(), ref, b, b.X) <= TOL["f32"]


def test_shared_operand_ldxp_zero():
    torch = _torch()
    b = inputs.make_batch(2, 8, 1, seed=14)
    X = torch.from_numpy(b.X).cuda()
    Y = torch.empty(40 * 64, dtype=torch.float32, device="cuda")
    kg.kron2_batched(b.A, b.B, X, Y, ma=8, na=8, mb=8, nb=8, batch=40, ldxp=0)
    ref = oracle_ref(b, b.X.astype(np.float64))
    out = Y.double().cpu().numpy().reshape(40, 64)
    assert np.abs(out - ref[None, :]).max() <= 1e-5 * np.abs(ref).max()


def test_empty_batch_is_noop():
    torch = _torch()
    X = torch.zeros(16, device="cuda")
    Y = torch.full((16,), 7.0, device="cuda")
    kg.kron2_batched(np.eye(4), np.eye(4), X, Y, ma=4, na=4, mb=4, nb=4, batch=0)
    assert (Y == 7.0).all()


# --- full-size launches (the configurations the benchmark times), sampled instances -----------------
@pytest.mark.parametrize("io", ["f32", "f64"])
@pytest.mark.parametrize("kind,n,batch", [(2, 16, 1 << 20), (2, 10, 1 << 20), (3, 16, 1 << 16), (3, 10, 1 << 18)])
def test_full_size_sampled(kind, n, batch, io):
    torch = _torch()
    b = inputs.make_batch(kind, n, batch, seed=1 + (kind == 3), x_dist="normal", dtype=np_dtype(io))
    inst = n ** kind
    X = torch.from_numpy(b.X).cuda()
    Y = torch.empty(batch * inst, dtype=torch_dtype(io), device="cuda")
    if kind == 2:
        kg.kron2_batched(b.A, b.B, X, Y, ma=n, na=n, mb=n, nb=n, batch=batch)
    else:
        kg.kron3_batched(b.A, b.B, b.C, X, Y, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(batch, 2048, replace=False))
    idx[-1] = batch - 1   # include the last instance (ragged end of the tile loop)
    Xs = b.X.reshape(batch, inst)[idx].astype(np.float64).ravel()
    sub = inputs.Batch(kind, n, len(idx), b.A, b.B, b.C, Xs)
    ref = oracle_ref(sub, Xs)
    got = Y.view(batch, inst)[torch.from_numpy(idx).cuda()].double().cpu().numpy().ravel()
    assert max_norm_err(got, ref, sub, Xs) <= TOL[io]
    del X, Y
    torch.cuda.empty_cache()


# the other variants the benchmark times at full size: 16-bit storage (FP32 arithmetic)
# and the odd-n in-place kernels, sampled instances against the FP64 oracle
@pytest.mark.parametrize("kind,n,batch,io", [(2, 16, 1 << 20, "bf16"), (2, 16, 1 << 20, "f16"),
                                             (2, 12, 1 << 20, "bf16"), (2, 12, 1 << 20, "f16"),
                                             (2, 8, 1 << 20, "bf16"), (3, 16, 1 << 16, "bf16"),
                                             (2, 15, 1 << 20, "f32"), (3, 15, 1 << 16, "f32")])
def test_full_size_sampled_other_variants(kind, n, batch, io):
    torch = _torch()
    b = inputs.make_batch(kind, n, batch, seed=4, x_dist="normal", dtype=np.float32)
    inst = n ** kind
    xt, X64 = storage_x(b, io)
    X = xt.to(torch_dtype(io)).cuda()
    Y = torch.empty(batch * inst, dtype=torch_dtype(io), device="cuda")
    if kind == 2:
        kg.kron2_batched(b.A, b.B, X, Y, ma=n, na=n, mb=n, nb=n, batch=batch)
    else:
        kg.kron3_batched(b.A, b.B, b.C, X, Y, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    rng = np.random.default_rng(6)
    idx = np.sort(rng.choice(batch, 2048, replace=False))
    idx[-1] = batch - 1
    Xs = X64.reshape(batch, inst)[idx].ravel()
    sub = inputs.Batch(kind, n, len(idx), b.A, b.B, b.C, Xs)
    got = Y.view(batch, inst)[torch.from_numpy(idx).cuda()].double().cpu().numpy().ravel()
    if io in ("bf16", "f16"):
        assert storage_check(got, sub, Xs, io) <= 1.0
    else:
        assert max_norm_err(got, oracle_ref(sub, Xs), sub, Xs) <= TOL[io]
    del X, Y
    torch.cuda.empty_cache()
