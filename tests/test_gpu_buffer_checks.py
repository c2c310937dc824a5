"""The pre-launch buffer checks: a host pointer, or a range past the end of its
allocation, is rejected before anything is launched (such a launch would fault
the GPU).  The library's check is exercised on its own first (it launches
nothing), then through an entry point with the same kind of argument."""
import ctypes

import numpy as np
import pytest

import paper_1304_7054_gb300 as kg

pytestmark = pytest.mark.gpu


def test_check_device_buffer_accepts_device_memory_only():
    import torch
    t = torch.zeros(1 << 20, device="cuda")
    assert kg.check_device_buffer(t) == 0
    assert kg.check_device_buffer(t.data_ptr(), 16) == 0
    assert kg.check_device_buffer(t.data_ptr(), 1 << 42) == 1          # past the allocation
    h = np.zeros(1024, np.float32)
    assert kg.check_device_buffer(h.ctypes.data, h.nbytes) == 1         # pageable host memory
    assert kg.check_device_buffer(0, 16) == 1


def test_entry_points_reject_host_pointers_before_launch():
    import torch
    assert kg.check_device_buffer(np.zeros(4, np.float32).ctypes.data, 16) == 1   # the check itself first
    L = kg.load_library()
    n, batch = 4, 8
    h = np.zeros(batch * n * n, np.float32)
    Y = torch.zeros(batch * n * n, device="cuda")
    eye = np.eye(n, dtype=np.float32).ravel()
    one, zero = ctypes.c_float(1.0), ctypes.c_float(0.0)
    st = L.kron2_batched(0, b"N", b"N", b"N", n, n, n, n, batch, ctypes.addressof(one), eye.ctypes.data, n,
                         eye.ctypes.data, n, h.ctypes.data, n, n * n, ctypes.addressof(zero), Y.data_ptr(), n,
                         n * n, kg.DTYPES["f32"], 0)
    assert st == 1
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    assert torch.count_nonzero(Y) == 0   # nothing was written


def test_binding_rejects_host_and_short_tensors():
    import torch
    n, batch = 4, 8
    eye = np.eye(n)
    X = torch.zeros(batch * n * n, device="cuda")
    with pytest.raises(TypeError):
        kg.kron2_batched(eye, eye, X.cpu(), X.clone(), ma=n, na=n, mb=n, nb=n, batch=batch)
    with pytest.raises(ValueError):
        kg.kron2_batched(eye, eye, X, X[: n * n].clone(), ma=n, na=n, mb=n, nb=n, batch=batch)
    with pytest.raises(ValueError):
        kg.kron3_batched(eye, eye, eye, X, torch.zeros(batch * n ** 3 - 1, device="cuda"), ma=n, na=n, mb=n, nb=n,
                         mc=n, nc=n, batch=batch)


_EXPANDABLE = r"""
import os, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, os.path.join(sys.argv[1], "tests"))
import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs
from helpers import TOL, max_norm_err, oracle_ref
assert "expandable_segments:True" in os.environ.get("PYTORCH_CUDA_ALLOC_CONF", "")
n, batch = 16, 1 << 18                         # 256 MB per operand: many mapped chunks
small = [torch.empty(1 << 18, device="cuda") for _ in range(3)]   # the segment is already in use
b = inputs.make_batch(2, n, batch, seed=77)
X = torch.from_numpy(b.X).cuda()
Y = torch.empty_like(X)
assert kg.check_device_buffer(X) == 0, "whole tensor rejected"
assert kg.check_device_buffer(Y) == 0
kg.kron2_batched(b.A, b.B, X, Y, ma=n, na=n, mb=n, nb=n, batch=batch)
torch.cuda.synchronize()
assert kg.device_status() == 0
idx = np.sort(np.random.default_rng(1).choice(batch, 256, replace=False))
idx[-1] = batch - 1
Xs = b.X.reshape(batch, 256)[idx].astype(np.float64).ravel()
sub = inputs.Batch(2, n, len(idx), b.A, b.B, None, Xs)
got = Y.view(batch, 256)[torch.from_numpy(idx).cuda()].double().cpu().numpy().ravel()
assert max_norm_err(got, oracle_ref(sub, Xs), sub, Xs) <= TOL["f32"]
print("expandable ok")
"""


def test_tensors_of_an_expandable_segment_allocator_are_accepted():
    """PyTorch's expandable segments map device memory in chunks through the
    virtual memory management API, so one tensor can span several mapped
    ranges; the pre-launch check must accept it (fresh process: the allocator
    setting is read at start-up)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTORCH_CUDA_ALLOC_CONF="expandable_segments:True")
    r = subprocess.run([sys.executable, "-c", _EXPANDABLE, root], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "expandable ok" in r.stdout
