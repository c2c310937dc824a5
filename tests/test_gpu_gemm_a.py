"""Parity of TGEMM_A (kron_gemm_a_batched) and TKRON1 (kron1_batched) with the
FP64 oracle, through the C ABI.

The error of C^p is normalised by ||op(A^p)||_F ||op(B)||_F (each |C_ij| is at
most that, by Cauchy-Schwarz), with the tolerances of the Kronecker entry
points: FP32 1e-5, FP64 1e-13.  16-bit storage is checked element by element:
within half an ulp of the storage type of the exact result plus the
componentwise bound of the FP32 arithmetic (helpers.storage_excess).  Exact cases (identity factors) are compared bit for bit, and
the paper's Algorithm 1 -- the 2-D product on every plane, then one TGEMM_A --
is checked against the fused 3-D kernel.
"""
import numpy as np
import pytest

import oracle
import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, arith_factor, storage_excess, torch_dtype

STORAGE16 = ("bf16", "f16")


def bar(io):
    """Pass mark of a case: the normalised tolerance, or 1 for the 16-bit element-wise check."""
    return 1.0 if io in STORAGE16 else TOL[io]

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def dev_buffer(vals64, io):
    """(device tensor in the storage type, the stored values as float64)."""
    torch = _torch()
    if io in ("bf16", "f16"):
        t = inputs.to_storage(np.asarray(vals64, np.float64), io)
        return t.cuda(), inputs.storage_to_f64(t)
    dt = np.float64 if io == "f64" else np.float32
    v = np.asarray(vals64, dt)
    return torch.from_numpy(v.copy()).cuda(), v.astype(np.float64)


def comp(M, io):
    """Host component in the compute type (FP32 unless FP64 storage)."""
    return np.asarray(M, np.float64 if io == "f64" else np.float32)


def ga_case(io, m, n, k, ta, tb, batch, pad=(0, 0, 0, 0), alpha=1.0, beta=0.0, grid_size=0, seed=0):
    torch = _torch()
    rng = np.random.default_rng(seed)
    lda = (m if ta == "N" else k) + pad[0]
    lda2 = lda * (k if ta == "N" else m) + pad[1]
    ldc = m + pad[2]
    ldc2 = ldc * n + pad[3]
    Abuf = rng.standard_normal(max(1, (batch - 1) * lda2 + lda * ((k if ta == "N" else m) - 1) + lda))
    Bst = comp(rng.uniform(-1, 1, (k, n) if tb == "N" else (n, k)), io)
    ldb = Bst.shape[0]
    Bflat = np.ascontiguousarray(Bst.T).ravel()
    C0 = rng.standard_normal(max(1, (batch - 1) * ldc2 + ldc * (n - 1) + m))
    At, A64 = dev_buffer(Abuf, io)
    Ct, C64 = dev_buffer(C0, io)
    kg.gemm_a_batched(At, Bflat, Ct, m=m, n=n, k=k, batch=batch, alpha=alpha, beta=beta, transa=ta, transb=tb,
                      lda=lda, lda2=lda2, ldb=ldb, ldc=ldc, ldc2=ldc2, grid_size=grid_size)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    got = Ct.double().cpu().numpy()
    ref = oracle.gemm_a(A64, Bflat.astype(np.float64), m=m, n=n, k=k, batch=batch, lda=lda, lda2=lda2, ldb=ldb,
                        ldc=ldc, ldc2=ldc2, alpha=alpha, beta=beta, C=C64, transa=ta, transb=tb)
    assert torch.equal(At.cpu(), dev_buffer(Abuf, io)[0].cpu()), "A modified"
    # entries of C outside the m x n blocks are untouched
    mask = np.zeros(len(C0), bool)
    for p in range(batch):
        for j in range(n):
            mask[p * ldc2 + j * ldc:p * ldc2 + j * ldc + m] = True
    assert np.array_equal(got[~mask], C64[~mask])
    if io in STORAGE16:
        absref = oracle.gemm_a(np.abs(A64), np.abs(Bflat.astype(np.float64)), m=m, n=n, k=k, batch=batch,
                               lda=lda, lda2=lda2, ldb=ldb, ldc=ldc, ldc2=ldc2, alpha=abs(alpha), beta=0.0,
                               transa=ta, transb=tb)
        return storage_excess(got[mask], ref[mask], absref[mask], io, arith_factor(1, k),
                              None if beta == 0.0 else abs(beta) * np.abs(C64[mask]))
    # normalised error per instance
    bn = np.linalg.norm(Bflat.astype(np.float64))
    worst = 0.0
    for p in range(batch):
        if ta == "N":
            Ap = np.array([[A64[p * lda2 + i + lda * l] for l in range(k)] for i in range(m)])
        else:
            Ap = np.array([[A64[p * lda2 + l + lda * i] for l in range(k)] for i in range(m)])
        idx = np.array([p * ldc2 + j * ldc + i for j in range(n) for i in range(m)])
        d = np.abs(got[idx] - ref[idx]).max()
        scale = abs(alpha) * np.linalg.norm(Ap) * bn + abs(beta) * np.abs(C64[idx]).max()
        worst = max(worst, d / scale if scale else d)
    return worst


@pytest.mark.parametrize("io", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 3, 5), (33, 16, 16), (256, 10, 10), (5, 16, 2), (100, 15, 16)])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
def test_gemm_a_parity(io, m, n, k, ta, tb):
    assert ga_case(io, m, n, k, ta, tb, batch=37, seed=m + n + k) <= bar(io)


@pytest.mark.parametrize("ta,tb", [("N", "T"), ("T", "N")])
@pytest.mark.parametrize("pad", [(0, 0, 0, 0), (3, 5, 2, 7)])
def test_gemm_a_strides_and_alpha_beta(ta, tb, pad):
    assert ga_case("f32", 45, 9, 12, ta, tb, batch=23, pad=pad, alpha=-0.5, beta=1.5, seed=3) <= 2 * TOL["f32"]


@pytest.mark.parametrize("grid_size", [1, 2, 3, 7])
@pytest.mark.parametrize("m", [1, 5, 256, 1000])
def test_gemm_a_small_grids_walk_every_row(grid_size, m):
    """A grid smaller than the rows makes each thread walk rows with the
    (instances, rows) stride; every row must be reached exactly once."""
    assert ga_case("f32", m, 4, 3, "N", "N", batch=29, grid_size=grid_size, seed=m) <= TOL["f32"]


@pytest.mark.parametrize("m,n,k", [(32, 16, 16), (64, 8, 12), (256, 16, 16), (100, 15, 16), (1536, 4, 16)])
@pytest.mark.parametrize("grid_size", [0, 1, 3])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.5, 1.5)])
def test_gemm_a_packed_batches(m, n, k, grid_size, alpha, beta):
    """Packed FP32 batches (contiguous A^p and C^p, the layout of the paper's
    Algorithm 1) with grids smaller than the row count and alpha / beta."""
    assert ga_case("f32", m, n, k, "N", "N", batch=37, alpha=alpha, beta=beta, grid_size=grid_size,
                   seed=m + n) <= 2 * TOL["f32"]


@pytest.mark.parametrize("io", ["f32", "f64", "bf16"])
def test_gemm_a_identity_is_exact(io):
    torch = _torch()
    m, k, batch = 70, 9, 12
    rng = np.random.default_rng(9)
    At, A64 = dev_buffer(rng.standard_normal(m * k * batch), io)
    Ct = torch.empty_like(At)
    kg.gemm_a_batched(At, comp(np.eye(k), io), Ct, m=m, n=k, k=k, batch=batch)
    torch.cuda.synchronize()
    assert torch.equal(Ct, At)


def test_gemm_a_beta_zero_ignores_nan():
    torch = _torch()
    At = torch.ones(2 * 4 * 3, device="cuda")
    Ct = torch.full((2 * 4 * 2,), float("nan"), device="cuda")
    kg.gemm_a_batched(At, np.ones((3, 2), np.float32), Ct, m=4, n=2, k=3, batch=2, beta=0.0)
    torch.cuda.synchronize()
    assert torch.equal(Ct, torch.full_like(Ct, 3.0))


@pytest.mark.parametrize("n", [4, 10, 16])
def test_algorithm1_on_gpu_equals_fused_kron3(n):
    """The paper's unfused 3-D product (2-D on every plane into tmp, then
    tmp op(A)^T with TGEMM_A) against the fused 3-D kernel and the oracle."""
    torch = _torch()
    b = inputs.make_batch(3, n, 300, seed=40 + n, x_dist="normal")
    X = torch.from_numpy(b.X).cuda()
    tmp = torch.empty_like(X)
    Y1 = torch.empty_like(X)
    Y2 = torch.empty_like(X)
    kg.kron2_batched(b.B, b.C, X, tmp, ma=n, na=n, mb=n, nb=n, batch=300 * n)
    kg.gemm_a_batched(tmp, b.A, Y1, m=n * n, n=n, k=n, batch=300, transb="T", lda=n * n, lda2=n ** 3,
                      ldc=n * n, ldc2=n ** 3)
    kg.kron3_batched(b.A, b.B, b.C, X, Y2, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=300)
    torch.cuda.synchronize()
    X64 = b.X.astype(np.float64)
    ref = oracle.kron3(b.A, b.B, b.C, X64, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=300)
    norm = (np.linalg.norm(b.A) * np.linalg.norm(b.B) * np.linalg.norm(b.C) *
            np.linalg.norm(X64.reshape(300, -1), axis=1))
    for Y in (Y1, Y2):
        d = np.abs(Y.double().cpu().numpy() - ref).reshape(300, -1).max(axis=1)
        assert float((d / norm).max()) <= TOL["f32"]


def test_gemm_a_full_size_sampled():
    """The benchmark's TGEMM_A launch (m = 256, n = k = 16, 2^16 instances),
    checked on sampled instances."""
    torch = _torch()
    m, n, k, batch = 256, 16, 16, 1 << 16
    rng = np.random.default_rng(12)
    A = torch.randn(batch * m * k, device="cuda")
    B = rng.uniform(-1, 1, (k, n)).astype(np.float32)
    C = torch.empty(batch * m * n, device="cuda")
    kg.gemm_a_batched(A, B, C, m=m, n=n, k=k, batch=batch)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    idx = np.sort(rng.choice(batch, 256, replace=False))
    idx[-1] = batch - 1
    As = A.view(batch, m * k)[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    ref = oracle.gemm_a(As.ravel(), np.ascontiguousarray(B.T).ravel().astype(np.float64), m=m, n=n, k=k,
                        batch=len(idx))
    got = C.view(batch, m * n)[torch.from_numpy(idx).cuda()].double().cpu().numpy().ravel()
    d = np.abs(got - ref).reshape(len(idx), -1).max(axis=1)
    norm = np.linalg.norm(As, axis=1) * np.linalg.norm(B)
    assert float((d / norm).max()) <= TOL["f32"]
    del A, C
    torch.cuda.empty_cache()


# ---------------------------------------------------------------------------
# TKRON1
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("io", ["f32", "f64", "bf16", "f16"])
@pytest.mark.parametrize("ma,na,ta", [(1, 1, "N"), (16, 16, "N"), (5, 12, "T"), (13, 3, "N")])
@pytest.mark.parametrize("strides", [(0, 0), (3, 1)])
def test_kron1_parity(io, ma, na, ta, strides):
    torch = _torch()
    rng = np.random.default_rng(ma * 17 + na)
    batch = 1001
    ldxp, ldyp = na + strides[0], ma + strides[1]
    A = comp(rng.uniform(-1, 1, (ma, na)), io)
    stored = A if ta == "N" else A.T
    Xt, X64 = dev_buffer(rng.standard_normal((batch - 1) * ldxp + na), io)
    Y0 = rng.standard_normal((batch - 1) * ldyp + ma)
    Yt, Y64 = dev_buffer(Y0, io)
    kg.kron1_batched(np.ascontiguousarray(stored.T).ravel(), Xt, Yt, ma=ma, na=na, batch=batch, transa=ta,
                     lda=stored.shape[0], ldxp=ldxp, ldyp=ldyp, alpha=0.5, beta=-1.0)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    got = Yt.double().cpu().numpy()
    ref = oracle.kron1(np.ascontiguousarray(stored.T).ravel().astype(np.float64), X64, ma=ma, na=na, batch=batch,
                       lda=stored.shape[0], ldxp=ldxp, ldyp=ldyp, alpha=0.5, beta=-1.0, Y=Y64, transa=ta)
    an = np.linalg.norm(A.astype(np.float64))
    worst = 0.0
    for p in range(batch):
        d = np.abs(got[p * ldyp:p * ldyp + ma] - ref[p * ldyp:p * ldyp + ma]).max()
        scale = 0.5 * an * np.linalg.norm(X64[p * ldxp:p * ldxp + na]) + np.abs(Y64[p * ldyp:p * ldyp + ma]).max()
        worst = max(worst, d / scale)
        assert np.array_equal(got[p * ldyp + ma:(p + 1) * ldyp], Y64[p * ldyp + ma:(p + 1) * ldyp])
    if io in STORAGE16:
        absref = oracle.kron1(np.abs(np.ascontiguousarray(stored.T).ravel().astype(np.float64)), np.abs(X64), ma=ma,
                              na=na, batch=batch, lda=stored.shape[0], ldxp=ldxp, ldyp=ldyp, alpha=0.5, beta=0.0,
                              transa=ta)
        sel = (np.arange(batch)[:, None] * ldyp + np.arange(ma)[None, :]).ravel()
        assert storage_excess(got[sel], ref[sel], absref[sel], io, arith_factor(1, na), np.abs(Y64[sel])) <= 1.0
    else:
        assert worst <= 2 * TOL[io]


def test_kron1_identity_is_exact():
    torch = _torch()
    X = torch.randn(16 * 5000, device="cuda")
    Y = torch.empty_like(X)
    kg.kron1_batched(np.eye(16, dtype=np.float32), X, Y, ma=16, na=16, batch=5000)
    torch.cuda.synchronize()
    assert torch.equal(X, Y)


def test_kron1_full_size_sampled():
    """TKRON1 at the benchmark's launch: 2^24 vectors of n = 16, sampled instances."""
    torch = _torch()
    n, batch = 16, 1 << 24
    rng = np.random.default_rng(21)
    A1 = rng.uniform(-1, 1, (n, n)).astype(np.float32)
    X = torch.randn(batch * n, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    Y = torch.empty_like(X)
    kg.kron1_batched(A1, X, Y, ma=n, na=n, batch=batch)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    idx = np.sort(rng.choice(batch, 2048, replace=False))
    idx[-1] = batch - 1
    sel = torch.from_numpy(idx).cuda()
    Xs = X.view(batch, n)[sel].double().cpu().numpy()
    ref = oracle.kron1(np.ascontiguousarray(A1.T).ravel().astype(np.float64), Xs.ravel(), ma=n, na=n,
                       batch=len(idx))
    got = Y.view(batch, n)[sel].double().cpu().numpy().ravel()
    err = (np.abs(got - ref).reshape(len(idx), n).max(axis=1) /
           (np.linalg.norm(Xs, axis=1) * np.linalg.norm(A1.astype(np.float64)))).max()
    assert err <= TOL["f32"]
    del X, Y
    torch.cuda.empty_cache()
