"""Parity of complex storage (KRON_C32F, KRON_C64F) with the complex oracle.

The operation over the complex field (paper Sec. 2) with op in {N, T, C}, C the
Hermitian transpose (Sec. 2.2), through the C ABI.  The error of an instance is
normalised as for real data, max |Y - Y_ref| / (||A|| ||B|| (||C||) ||X^p||)
with Frobenius norms of the complex arrays: complex float <= 1e-5, complex double
<= 1e-13, against the complex128 oracle.  Exact cases (identity, i times the
identity) are compared bit for bit.
"""
import numpy as np
import pytest

import oracle
import paper_1304_7054_gb300 as kg

pytestmark = pytest.mark.gpu

TOLC = {"c64": 1e-5, "c128": 1e-13}
NPC = {"c64": np.complex64, "c128": np.complex128}


def _torch():
    import torch
    assert torch.cuda.is_available()
    return torch


def tdt(io):
    import torch
    return {"c64": torch.complex64, "c128": torch.complex128}[io]


def crnd(rng, *shape):
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


def colmaj(M):
    return np.ascontiguousarray(np.asarray(M).T).ravel()


def stored(opM, t):
    return {"N": opM, "T": opM.T, "C": opM.conj().T}[t]


def cbatch(kind, n, batch, seed, io):
    rng = np.random.default_rng(seed)
    comps = [crnd(rng, n, n).astype(NPC[io]) for _ in range(kind)]
    X = (rng.standard_normal(batch * n ** kind) + 1j * rng.standard_normal(batch * n ** kind)).astype(NPC[io])
    return comps, X


def run(kind, n, batch, comps, X, io, guard=0, **kw):
    torch = _torch()
    total = batch * n ** kind
    Xd = torch.from_numpy(X).cuda()
    Ybuf = torch.full((total + 2 * guard,), complex(np.nan, np.nan), dtype=tdt(io), device="cuda")
    Y = Ybuf[guard:guard + total]
    if kind == 2:
        kg.kron2_batched(comps[0], comps[1], Xd, Y, ma=n, na=n, mb=n, nb=n, batch=batch, **kw)
    else:
        kg.kron3_batched(comps[0], comps[1], comps[2], Xd, Y, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch, **kw)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    out = Ybuf.cpu().numpy().astype(np.complex128)
    if guard:
        assert np.isnan(out[:guard]).all() and np.isnan(out[-guard:]).all(), "guard band written"
    return out[guard:guard + total]


def ref(kind, n, batch, comps, X, **kw):
    c = [colmaj(M.astype(np.complex128)) for M in comps]
    X = X.astype(np.complex128)
    if kind == 2:
        return oracle.kron2c(c[0], c[1], X, ma=n, na=n, mb=n, nb=n, batch=batch, **kw)
    return oracle.kron3c(c[0], c[1], c[2], X, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch, **kw)


def norm_err(Y, R, kind, n, batch, comps, X, extra=None):
    sz = n ** kind
    cn = np.prod([np.linalg.norm(M.astype(np.complex128)) for M in comps])
    xn = np.linalg.norm(X.astype(np.complex128).reshape(batch, sz), axis=1)
    scale = cn * xn if extra is None else cn * xn + extra
    d = np.abs(Y - R).reshape(batch, sz).max(axis=1)
    return float((d / scale).max())


@pytest.mark.parametrize("io", ["c64", "c128"])
@pytest.mark.parametrize("n", list(range(1, 17)))
@pytest.mark.parametrize("kind", [2, 3])
def test_all_sizes(kind, n, io):
    batch = 517 if kind == 2 else 67
    comps, X = cbatch(kind, n, batch, 900 + n + 17 * kind, io)
    Y = run(kind, n, batch, comps, X, io, guard=8)
    assert norm_err(Y, ref(kind, n, batch, comps, X), kind, n, batch, comps, X) <= TOLC[io]


@pytest.mark.parametrize("io", ["c64", "c128"])
@pytest.mark.parametrize("trans", ["CNN", "NCN", "NNC", "CCC", "TCN", "CTT"])
@pytest.mark.parametrize("shape,lds", [((16, 16, 16, 16), (19, 300, 17, 290)), ((5, 7, 3, 9), (11, 80, 4, 30)),
                                       ((8, 8, 8, 8), (8, 64, 8, 64))])
def test_ops_and_strides_2d(io, trans, shape, lds):
    torch = _torch()
    ma, na, mb, nb = shape
    ldx, ldxp, ldy, ldyp = lds
    ta, tb, tx = trans
    if tx != "N":
        ldx = max(ldx, na)
        ldxp = max(ldxp, ldx * nb)
    batch = 37
    rng = np.random.default_rng(sum(shape) + len(trans))
    opA, opB = crnd(rng, ma, na).astype(NPC[io]), crnd(rng, mb, nb).astype(NPC[io])
    X = crnd(rng, batch * ldxp + 3).astype(NPC[io])
    Y = torch.full((batch * ldyp + 5,), complex(np.nan, np.nan), dtype=tdt(io), device="cuda")
    Ast, Bst = stored(opA, ta), stored(opB, tb)
    kg.kron2_batched(Ast, Bst, torch.from_numpy(X).cuda(), Y, ma=ma, na=na, mb=mb, nb=nb, batch=batch,
                     transa=ta, transb=tb, transx=tx, ldx=ldx, ldxp=ldxp, ldy=ldy, ldyp=ldyp)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    R = oracle.kron2c(colmaj(Ast.astype(np.complex128)), colmaj(Bst.astype(np.complex128)),
                      X.astype(np.complex128), ma=ma, na=na, mb=mb, nb=nb, batch=batch, transa=ta, transb=tb,
                      transx=tx, ldx=ldx, ldxp=ldxp, ldy=ldy, ldyp=ldyp,
                      Y=np.full(batch * ldyp + 5, complex(np.nan, np.nan)))
    got = Y.cpu().numpy().astype(np.complex128)
    written = ~np.isnan(R)
    assert np.array_equal(np.isnan(got), ~written), "written set differs from the oracle's"
    scale = np.linalg.norm(opA) * np.linalg.norm(opB) * np.abs(X).max() * max(na, nb)
    assert np.abs(got[written] - R[written]).max() <= TOLC[io] * scale


@pytest.mark.parametrize("io", ["c64", "c128"])
@pytest.mark.parametrize("trans", ["CNN", "NCT", "CCC"])
def test_ops_3d(io, trans):
    n, batch = 7, 41
    rng = np.random.default_rng(77 + len(trans))
    ops = [crnd(rng, n, n).astype(NPC[io]) for _ in range(3)]
    X = crnd(rng, batch * n ** 3).astype(NPC[io])
    st = [stored(M, t) for M, t in zip(ops, trans)]
    Y = run(3, n, batch, st, X, io, transa=trans[0], transb=trans[1], transc=trans[2])
    R = ref(3, n, batch, st, X, transa=trans[0], transb=trans[1], transc=trans[2])
    assert norm_err(Y, R, 3, n, batch, ops, X) <= TOLC[io]


@pytest.mark.parametrize("io", ["c64", "c128"])
@pytest.mark.parametrize("kind,n", [(2, 16), (2, 5), (3, 16), (3, 6)])
def test_alpha_beta(io, kind, n):
    torch = _torch()
    batch = 33
    comps, X = cbatch(kind, n, batch, 31 + n, io)
    rng = np.random.default_rng(4)
    Y0 = crnd(rng, batch * n ** kind).astype(NPC[io])
    al, be = 0.75 - 0.5j, -1.25 + 0.25j
    total = batch * n ** kind
    Yd = torch.from_numpy(Y0.copy()).cuda()
    Xd = torch.from_numpy(X).cuda()
    if kind == 2:
        kg.kron2_batched(comps[0], comps[1], Xd, Yd, ma=n, na=n, mb=n, nb=n, batch=batch, alpha=al, beta=be)
    else:
        kg.kron3_batched(comps[0], comps[1], comps[2], Xd, Yd, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch,
                         alpha=al, beta=be)
    torch.cuda.synchronize()
    got = Yd.cpu().numpy().astype(np.complex128)
    R = ref(kind, n, batch, comps, X, alpha=al, beta=be, Y=Y0.astype(np.complex128))
    extra = abs(be) * np.linalg.norm(Y0.astype(np.complex128).reshape(batch, -1), axis=1)
    assert norm_err(got, R, kind, n, batch, comps, X, extra) <= 2 * TOLC[io]
    assert total == len(got)


@pytest.mark.parametrize("io", ["c64", "c128"])
@pytest.mark.parametrize("kind,n", [(2, 16), (2, 7), (3, 16), (3, 5)])
def test_identity_and_i_identity_are_exact(io, kind, n):
    comps, X = cbatch(kind, n, 50, 5, io)
    eye = np.eye(n).astype(NPC[io])
    Y = run(kind, n, 50, [eye] * kind, X, io)
    assert np.array_equal(Y, X.astype(np.complex128))
    Y = run(kind, n, 50, [1j * eye] + [eye] * (kind - 1), X, io)   # one factor i I: Y = i X
    assert np.array_equal(Y, 1j * X.astype(np.complex128))


def test_beta_zero_ignores_nan_and_misaligned_operand():
    torch = _torch()
    n, batch = 16, 64
    comps, X = cbatch(2, n, batch, 8, "c64")
    Y = run(2, n, batch, comps, X, "c64")   # Y starts NaN-filled, beta = 0
    assert not np.isnan(Y).any()
    # X one complex element past a 16-byte boundary: the element-wise loader
    Xb = torch.from_numpy(np.concatenate([[0], X]).astype(np.complex64)).cuda()[1:]
    Yd = torch.empty(batch * 256, dtype=torch.complex64, device="cuda")
    kg.kron2_batched(comps[0], comps[1], Xb, Yd, ma=n, na=n, mb=n, nb=n, batch=batch)
    torch.cuda.synchronize()
    assert norm_err(Yd.cpu().numpy().astype(np.complex128), ref(2, n, batch, comps, X), 2, n, batch, comps,
                    X) <= TOLC["c64"]


@pytest.mark.parametrize("io,kind,n,batch", [("c64", 2, 16, 1 << 20), ("c64", 3, 16, 1 << 15),
                                             ("c128", 2, 16, 1 << 18)])
def test_full_size_sampled(io, kind, n, batch):
    """The complex launches the benchmark times, checked on sampled instances."""
    torch = _torch()
    rng = np.random.default_rng(3)
    comps = [crnd(rng, n, n).astype(NPC[io]) for _ in range(kind)]
    sz = n ** kind
    g = torch.Generator(device="cuda").manual_seed(11)
    X = torch.randn(batch * sz, dtype=tdt(io), device="cuda", generator=g)
    Y = torch.empty_like(X)
    if kind == 2:
        kg.kron2_batched(comps[0], comps[1], X, Y, ma=n, na=n, mb=n, nb=n, batch=batch)
    else:
        kg.kron3_batched(comps[0], comps[1], comps[2], X, Y, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=batch)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    idx = np.sort(rng.choice(batch, 512, replace=False))
    idx[-1] = batch - 1
    sel = torch.from_numpy(idx).cuda()
    Xs = X.view(batch, sz)[sel].cpu().numpy().astype(np.complex128).ravel()
    got = Y.view(batch, sz)[sel].cpu().numpy().astype(np.complex128).ravel()
    R = ref(kind, n, len(idx), comps, Xs)
    assert norm_err(got, R, kind, n, len(idx), comps, Xs) <= TOLC[io]
    del X, Y
    torch.cuda.empty_cache()
