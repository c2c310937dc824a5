"""The device-side failure path: a bounded wait that runs out is reported, and
the library stays usable.

Every wait of the kernels on a bulk copy is bounded.  The test shortens the
limit of the first operand wait of the 2-D n = 16 FP32 kernel
(kron_set_first_wait_limit_ns) below the time a copy takes to land, so that real
wait expires on a normal launch: no fault, no hang, only an expired wait.  The
kernel then drains its copies in flight with the normal bound and returns; the
status word reports KRON_ERR_DEVICE_TIMEOUT once and is cleared by the read, and
the next normal call matches the oracle.
"""
import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import inputs

from helpers import TOL, max_norm_err, oracle_ref

pytestmark = pytest.mark.gpu

TIMEOUT = 6


def test_expired_wait_is_reported_and_the_next_call_is_correct():
    import torch
    n, batch = 16, 2048
    b = inputs.make_batch(2, n, batch, seed=61)
    X = torch.from_numpy(b.X).cuda()
    Y = torch.empty_like(X)
    assert kg.device_status() == 0
    seen = []
    try:
        kg.set_first_wait_limit_ns(1)
        for _ in range(3):   # a copy landing within the first poll would let a launch through
            kg.kron2_batched(b.A, b.B, X, Y, ma=n, na=n, mb=n, nb=n, batch=batch)
            seen.append(kg.device_status())
            if seen[-1] == TIMEOUT:
                break
    finally:
        kg.set_first_wait_limit_ns(0)
    assert TIMEOUT in seen, seen
    assert kg.device_status() == 0, "the status word is cleared by the read"
    Y.fill_(float("nan"))
    kg.kron2_batched(b.A, b.B, X, Y, ma=n, na=n, mb=n, nb=n, batch=batch)
    torch.cuda.synchronize()
    assert kg.device_status() == 0
    X64 = b.X.astype(np.float64)
    assert max_norm_err(Y.double().cpu().numpy(), oracle_ref(b, X64), b, X64) <= TOL["f32"]

