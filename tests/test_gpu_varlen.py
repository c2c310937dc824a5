"""Parity of the mixed-size persistent path (one graph-captured launch) with the oracle.

FP32 results are checked with the normalised error (<= 1e-5); 16-bit storage
element by element: within half an ulp of the storage type of the exact result
plus the componentwise bound of the FP32 arithmetic (helpers.storage_excess)."""
import numpy as np
import pytest

import oracle
import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, arith_factor, storage_excess, torch_dtype, ulp

pytestmark = pytest.mark.gpu


def classes_of(v):
    return [(k, n, *cs) for (k, n), cs in zip(v.classes, v.comps)]


def reference(v, X64, idx=None):
    """Oracle output per instance (dict p -> flat array), the normalising factor,
    and the oracle's absolute-value product (|K| |x^p|, dict p -> flat array)."""
    idx = np.arange(len(v.class_of)) if idx is None else idx
    out, norm, absref = {}, {}, {}
    for c, (kind, n) in enumerate(v.classes):
        sel = idx[v.class_of[idx] == c]
        if len(sel) == 0:
            continue
        nx = n ** kind
        Xs = np.concatenate([X64[v.x_off[p]:v.x_off[p] + nx] for p in sel])
        cs = v.comps[c]
        acs = [np.abs(np.asarray(M, np.float64)) for M in cs]
        if kind == 2:
            Y = oracle.kron2(cs[0], cs[1], Xs, ma=n, na=n, mb=n, nb=n, batch=len(sel))
            Ya = oracle.kron2(acs[0], acs[1], np.abs(Xs), ma=n, na=n, mb=n, nb=n, batch=len(sel))
        else:
            Y = oracle.kron3(cs[0], cs[1], cs[2], Xs, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=len(sel))
            Ya = oracle.kron3(acs[0], acs[1], acs[2], np.abs(Xs), ma=n, na=n, mb=n, nb=n, mc=n, nc=n,
                              batch=len(sel))
        cn = np.prod([np.linalg.norm(np.asarray(M, np.float64)) for M in cs])
        for r, p in enumerate(sel):
            out[p] = Y[r * nx:(r + 1) * nx]
            absref[p] = Ya[r * nx:(r + 1) * nx]
            norm[p] = cn * np.linalg.norm(Xs[r * nx:(r + 1) * nx])
    return out, norm, absref


def max_err(v, Y, refs, io="f32", y_off=None):
    """FP32: the largest normalised error; 16-bit storage: the largest element-wise
    excess over the rounding bar (passes at <= 1)."""
    ref, norm, absref = refs
    y_off = v.y_off if y_off is None else y_off
    e = 0.0
    for p, r in ref.items():
        kind, n = v.classes[v.class_of[p]]
        got = Y[y_off[p]:y_off[p] + n ** kind]
        if io in ("bf16", "f16"):
            e = max(e, storage_excess(got, r, absref[p], io, arith_factor(kind, n)))
        else:
            e = max(e, np.abs(got - r).max() / max(norm[p], 1e-300))
    return e


def bar(io):
    return 1.0 if io in ("bf16", "f16") else TOL[io]


def run(v, io="f32", plan=None, Y=None, ws=None):
    import torch
    if io == "f32":
        X = torch.from_numpy(v.X).cuda()
        X64 = v.X.astype(np.float64)
    else:
        t = inputs.to_storage(v.X, io)
        X, X64 = t.cuda(), inputs.storage_to_f64(t)
    plan = plan or kg.VarlenPlan(classes_of(v), v.class_of, v.x_off, v.y_off, io=io)
    Y = Y if Y is not None else torch.full((v.total,), float("nan"), dtype=torch_dtype(io), device="cuda")
    ws = ws if ws is not None else plan.alloc_workspace()
    plan.execute(X, Y, ws)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    return plan, X, Y, ws, X64


@pytest.mark.parametrize("io", ["f32", "bf16", "f16"])
def test_varlen_all_classes(io):
    v = inputs.make_varlen(3000, seed=11, nmin=1, nmax=16)
    plan, X, Y, ws, X64 = run(v, io)
    Yh = Y.double().cpu().numpy()
    assert not np.isnan(Yh).any()
    err = max_err(v, Yh, reference(v, X64), io)
    assert err <= bar(io), err
    plan.close()


def test_varlen_graph_replay_is_deterministic_and_pointers_update():
    import torch
    v = inputs.make_varlen(2000, seed=12)
    plan, X, Y, ws, X64 = run(v)
    Y1 = Y.clone()
    plan.execute(X, Y, ws)
    torch.cuda.synchronize()
    assert torch.equal(Y, Y1)
    Y2 = torch.zeros_like(Y)   # another output buffer: the graph's kernel node is updated
    plan.execute(X, Y2, ws)
    torch.cuda.synchronize()
    assert torch.equal(Y2, Y1)
    plan.close()


def test_varlen_matches_per_size_launches():
    import torch
    v = inputs.make_varlen(2500, seed=13)
    plan, X, Y, ws, X64 = run(v)
    Yh = Y.double().cpu().numpy()
    for c, (kind, n) in enumerate(v.classes):
        sel = np.nonzero(v.class_of == c)[0]
        if len(sel) == 0:
            continue
        nx = n ** kind
        Xs = torch.from_numpy(np.concatenate([v.X[v.x_off[p]:v.x_off[p] + nx] for p in sel])).cuda()
        Ys = torch.empty_like(Xs)
        cs = v.comps[c]
        if kind == 2:
            kg.kron2_batched(cs[0], cs[1], Xs, Ys, ma=n, na=n, mb=n, nb=n, batch=len(sel))
        else:
            kg.kron3_batched(cs[0], cs[1], cs[2], Xs, Ys, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=len(sel))
        got = np.concatenate([Yh[v.y_off[p]:v.y_off[p] + nx] for p in sel])
        exp = Ys.double().cpu().numpy()
        assert np.abs(got - exp).max() <= 1e-5 * max(1.0, np.abs(exp).max()) * n
    plan.close()


def test_varlen_single_instance_class_and_missing_classes():
    import torch
    rng = np.random.default_rng(3)
    A2, B2 = rng.uniform(-1, 1, (5, 5)), rng.uniform(-1, 1, (5, 5))
    A3, B3, C3 = (rng.uniform(-1, 1, (3, 3)) for _ in range(3))
    classes = [(2, 5, A2, B2), (3, 3, A3, B3, C3), (2, 16, np.eye(16), np.eye(16))]   # class 2 unused
    class_of = [1, 0, 0, 0]
    sizes = [27, 25, 25, 25]
    x_off = np.concatenate([[0], np.cumsum(sizes)[:-1]])
    total = int(sum(sizes))
    X = rng.standard_normal(total).astype(np.float32)
    plan = kg.VarlenPlan(classes, class_of, x_off, x_off)
    ws = plan.alloc_workspace()
    Y = torch.full((total,), float("nan"), device="cuda")
    plan.execute(torch.from_numpy(X).cuda(), Y, ws)
    torch.cuda.synchronize()
    Yh = Y.double().cpu().numpy()
    col = lambda M: np.ascontiguousarray(np.asarray(M).T).ravel()
    r3 = oracle.kron3(col(A3), col(B3), col(C3), X[:27].astype(np.float64), ma=3, na=3, mb=3, nb=3, mc=3, nc=3,
                      batch=1)
    np.testing.assert_allclose(Yh[:27], r3, atol=1e-5)
    r2 = oracle.kron2(col(A2), col(B2), X[27:].astype(np.float64), ma=5, na=5, mb=5, nb=5, batch=3)
    np.testing.assert_allclose(Yh[27:], r2, atol=1e-5)
    plan.close()


def test_varlen_tune_keeps_results():
    import torch
    v = inputs.make_varlen(4000, seed=14)
    plan, X, Y, ws, X64 = run(v)
    Y1 = Y.clone()
    plan.tune(X, Y, ws)
    Y.fill_(float("nan"))
    plan.execute(X, Y, ws)
    torch.cuda.synchronize()
    assert max_err(v, Y.double().cpu().numpy(), reference(v, X64)) <= TOL["f32"]
    plan.close()


@pytest.mark.parametrize("io", ["f32", "bf16"])
def test_varlen_full_size_sampled(io):
    """The mixed-size workload the benchmark times: 200,000 instances, n ~ U{4..16}."""
    v = inputs.make_varlen(200000, seed=5)
    plan, X, Y, ws, X64 = run(v, io)
    rng = np.random.default_rng(8)
    idx = np.sort(rng.choice(200000, 3000, replace=False))
    idx[-1] = 199999
    assert max_err(v, Y.double().cpu().numpy(), reference(v, X64, idx), io) <= bar(io)
    plan.close()


@pytest.mark.parametrize("io", ["f32", "bf16"])
def test_varlen_unaligned_bases_and_permuted_output(io):
    """Instances start at arbitrary element offsets: X and Y begin one element past
    a 16-byte boundary, and Y holds the instances in another order with gaps of
    0..5 elements, so an instance's alignment phase in Y differs from its phase
    in X.  Every instance matches the oracle and no gap element is written."""
    import torch
    v = inputs.make_varlen(3000, seed=15, nmin=1, nmax=16)
    rng = np.random.default_rng(16)
    sizes = np.array([v.classes[c][1] ** v.classes[c][0] for c in v.class_of], np.int64)
    y_off = np.zeros(len(sizes), np.int64)
    pos = 0
    for p in rng.permutation(len(sizes)):
        pos += int(rng.integers(0, 6))
        y_off[p] = pos
        pos += int(sizes[p])
    ytotal = pos + 5
    if io == "f32":
        xs, X64 = torch.from_numpy(v.X), v.X.astype(np.float64)
    else:
        xs = inputs.to_storage(v.X, io)
        X64 = inputs.storage_to_f64(xs)
    xb = torch.zeros(v.total + 1, dtype=torch_dtype(io), device="cuda")
    xb[1:] = xs.cuda()
    yb = torch.full((ytotal + 1,), float("nan"), dtype=torch_dtype(io), device="cuda")
    X, Y = xb[1:], yb[1:]
    plan = kg.VarlenPlan(classes_of(v), v.class_of, v.x_off, y_off, io=io)
    ws = plan.alloc_workspace()
    plan.execute(X, Y, ws)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    Yh = Y.double().cpu().numpy()
    covered = np.zeros(ytotal, bool)
    for p in range(len(sizes)):
        covered[y_off[p]:y_off[p] + sizes[p]] = True
    assert np.isnan(Yh[~covered]).all(), "gap written"
    assert np.isnan(yb[:1].double().cpu().numpy()).all()
    e = max_err(v, Yh, reference(v, X64), io, y_off=y_off)
    assert e <= bar(io), e
    plan.close()


@pytest.mark.parametrize("io", ["f32", "bf16"])
def test_varlen_alpha_beta(io):
    """Y = alpha (K X) + beta Y per instance (kron_varlen_plan_set_scaling), against
    the oracle with the same alpha, beta and starting Y; back to the plain action
    after alpha = 1, beta = 0."""
    import torch
    v = inputs.make_varlen(1500, seed=14, nmin=1, nmax=16)
    al, be = 0.75, -1.5
    rng = np.random.default_rng(9)
    Y0 = rng.standard_normal(v.total).astype(np.float32)
    if io == "f32":
        Yd, Y064 = torch.from_numpy(Y0.copy()).cuda(), Y0.astype(np.float64)
        X, X64 = torch.from_numpy(v.X).cuda(), v.X.astype(np.float64)
    else:
        t0 = inputs.to_storage(Y0, io)
        Yd, Y064 = t0.cuda(), inputs.storage_to_f64(t0)
        t = inputs.to_storage(v.X, io)
        X, X64 = t.cuda(), inputs.storage_to_f64(t)
    plan = kg.VarlenPlan(classes_of(v), v.class_of, v.x_off, v.y_off, io=io)
    ws = plan.alloc_workspace()
    plan.set_scaling(al, be)
    plan.execute(X, Yd, ws)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    got = Yd.double().cpu().numpy()
    ref, norm, absref = reference(v, X64)
    worst = 0.0
    for p, r in ref.items():
        kind, n = v.classes[v.class_of[p]]
        nx = n ** kind
        y0 = Y064[v.y_off[p]:v.y_off[p] + nx]
        want = al * r + be * y0
        g = got[v.y_off[p]:v.y_off[p] + nx]
        if io == "f32":
            scale = abs(al) * norm[p] + abs(be) * np.abs(y0).max() + 1e-300
            worst = max(worst, np.abs(g - want).max() / scale)
        else:
            # the kernel rounds K x to the storage type, then forms alpha (K x) + beta y0
            # in FP32 and rounds again: one more half ulp of |alpha K x| than the bar
            # (the first rounding also enters the argument of the second one's ulp)
            ka = abs(al) * absref[p]
            E = arith_factor(kind, n) * ka + 3 * 2.0 ** -24 * (ka + abs(be) * np.abs(y0))
            d1 = abs(al) * 0.5 * ulp(np.abs(r) + arith_factor(kind, n) * absref[p], io)
            allowed = 0.5 * ulp(np.abs(want) + E + d1, io) + E + d1
            worst = max(worst, float((np.abs(g - want) / allowed).max()))
    assert worst <= (2 * TOL["f32"] if io == "f32" else 1.0), worst
    # alpha = 1, beta = 0 again: the plain action on the same plan and graph
    plan.set_scaling(1.0, 0.0)
    Yn = torch.full((v.total,), float("nan"), dtype=torch_dtype(io), device="cuda")
    plan.execute(X, Yn, ws)
    torch.cuda.synchronize()
    assert max_err(v, Yn.double().cpu().numpy(), (ref, norm, absref), io) <= bar(io)
    with pytest.raises(kg.KronError):
        plan.set_scaling(float("nan"), 0.0)
    plan.close()
