"""The allocation-free mixed-size entry point (kron_varlen_execute_noalloc).

It is for callers that cannot allocate device memory (all memory owned by
another allocator, or loops where cudaMalloc/cudaFree would synchronise the
device).  It must give the same result as kron_varlen_execute with a
caller-allocated workspace, call after call, since the fixed device array it
uses is rewritten by every call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL

pytestmark = pytest.mark.gpu


def _classes(v):
    return [(k, n, *cs) for (k, n), cs in zip(v.classes, v.comps)]


def _norm_diff(v, Y, R):
    e = 0.0
    for p in range(len(v.class_of)):
        k, n = v.classes[v.class_of[p]]
        nx = n ** k
        a = Y[v.y_off[p]:v.y_off[p] + nx]
        b = R[v.y_off[p]:v.y_off[p] + nx]
        e = max(e, float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)))
    return e


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
    R = Yref.double().cpu().numpy()
    for call in range(2):
        Y = torch.full((v.total,), float("nan"), device="cuda")
        plan.execute_noalloc(X, Y)
        other.execute_noalloc(XW, torch.empty_like(XW))
        torch.cuda.synchronize()
        assert kg.device_status() == 0
        got = Y.double().cpu().numpy()
        assert not np.isnan(got).any(), f"call {call}: outputs missing"
        assert _norm_diff(v, got, R) <= TOL["f32"], f"call {call}"
    plan.close()
    other.close()


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
