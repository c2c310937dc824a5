"""The allocation-free mixed-size entry point (kron_varlen_execute_noalloc).

Some callers cannot allocate device memory: code whose device memory is all
owned by another allocator that hands out no scratch buffer, and loops where a
cudaMalloc / cudaFree would synchronise the device.  For them the library runs a
mixed-size plan on a fixed device array of its own instead of a caller
workspace.  It runs the same kernel on the same tables as kron_varlen_execute,
so the two must agree bit for bit, call after call, although every call
rewrites the shared array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

pytestmark = pytest.mark.gpu


def _classes(v):
    return [(k, n, *cs) for (k, n), cs in zip(v.classes, v.comps)]


def test_noalloc_matches_workspace_entry_point_twice():
    import torch
    v = inputs.make_varlen(20000, seed=21, nmin=1, nmax=16)
    w = inputs.make_varlen(7000, seed=22)   # a second plan writes the shared array in between
    X = torch.from_numpy(v.X).cuda()
    XW = torch.from_numpy(w.X).cuda()
    plan = kg.VarlenPlan(_classes(v), v.class_of, v.x_off, v.y_off)
    other = kg.VarlenPlan(_classes(w), w.class_of, w.x_off, w.y_off)
    ws = plan.alloc_workspace()
    Yref = torch.full((v.total,), float("nan"), device="cuda")
    plan.execute(X, Yref, ws)
    torch.cuda.synchronize()
    assert not torch.isnan(Yref).any()
    for call in range(2):
        Y = torch.full((v.total,), float("nan"), device="cuda")
        plan.execute_noalloc(X, Y)
        other.execute_noalloc(XW, torch.empty_like(XW))
        torch.cuda.synchronize()
        assert kg.device_status() == 0
        assert torch.equal(Y, Yref), f"call {call}: differs from the workspace entry point"
    plan.close()
    other.close()


def test_noalloc_between_workspace_calls_of_a_larger_plan():
    """A plan that needs more shared memory runs through the workspace entry point,
    a smaller one through the allocation-free one, then the first again: the
    kernel's shared-memory limit must still cover the first plan."""
    import torch
    big = inputs.make_varlen(6000, seed=31, nmin=12, nmax=16)
    small = inputs.make_varlen(6000, seed=32, nmin=2, nmax=4)
    Xb = torch.from_numpy(big.X).cuda()
    Xs = torch.from_numpy(small.X).cuda()
    pb = kg.VarlenPlan(_classes(big), big.class_of, big.x_off, big.y_off)
    ps = kg.VarlenPlan(_classes(small), small.class_of, small.x_off, small.y_off)
    ws_b, ws_s = pb.alloc_workspace(), ps.alloc_workspace()
    Yb1 = torch.full((big.total,), float("nan"), device="cuda")
    pb.execute(Xb, Yb1, ws_b)
    Ys_ref = torch.full((small.total,), float("nan"), device="cuda")
    ps.execute(Xs, Ys_ref, ws_s)
    Ys = torch.full((small.total,), float("nan"), device="cuda")
    ps.execute_noalloc(Xs, Ys)
    Yb2 = torch.full((big.total,), float("nan"), device="cuda")
    pb.execute(Xb, Yb2, ws_b)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    assert not torch.isnan(Yb1).any() and not torch.isnan(Ys_ref).any()
    assert torch.equal(Ys, Ys_ref)
    assert torch.equal(Yb2, Yb1)
    pb.close()
    ps.close()


def test_noalloc_rejects_batches_above_the_limit():
    import torch
    count = 262145   # one instance more than the fixed array holds
    I = np.eye(2)
    off = np.arange(count, dtype=np.int64) * 4
    plan = kg.VarlenPlan([(2, 2, I, I)], np.zeros(count, np.int32), off, off)
    X = torch.zeros(4 * count, device="cuda")
    with pytest.raises(kg.KronError) as e:
        plan.execute_noalloc(X, torch.zeros_like(X))
    assert e.value.status == 4   # KRON_ERR_WORKSPACE
    plan.close()
