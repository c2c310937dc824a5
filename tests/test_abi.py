"""The C ABI on the host: the library loads, exports every declared entry point,
and rejects invalid arguments with the documented status codes before touching
the GPU (these calls run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1304_7054_gb300 as kg
from paper_1304_7054_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()   # incremental: a no-op when up to date
    return kg.load_library()


def declared_symbols():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"KRON_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "kron2_batched" in names and "kron3_batched" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(kg.SIGNATURES), "binding misses a declared entry point"


def test_status_strings(lib):
    for code, name in kg.STATUS.items():
        assert kg.status_string(code) == name


F = ctypes.c_float(1.0)
ZERO = ctypes.c_float(0.0)
COMP = np.eye(16, dtype=np.float32).ravel()


def k2(lib, **over):
    a = dict(stream=None, ta=b"N", tb=b"N", tx=b"N", ma=4, na=4, mb=4, nb=4, batch=10,
             alpha=ctypes.addressof(F), A=COMP.ctypes.data, lda=4, B=COMP.ctypes.data, ldb=4,
             X=0x10000, ldx=4, ldxp=16, beta=ctypes.addressof(ZERO), Y=0x90000, ldy=4, ldyp=16,
             io=0, comp=0)
    a.update(over)
    return lib.kron2_batched(*a.values())


def k3(lib, **over):
    a = dict(stream=None, ta=b"N", tb=b"N", tc=b"N", ma=3, na=3, mb=3, nb=3, mc=3, nc=3, batch=10,
             alpha=ctypes.addressof(F), A=COMP.ctypes.data, lda=3, B=COMP.ctypes.data, ldb=3,
             C=COMP.ctypes.data, ldc=3, X=0x10000, ldx=3, ldx2=9, ldxp=27, beta=ctypes.addressof(ZERO),
             Y=0x90000, ldy=3, ldy2=9, ldyp=27, io=0, comp=0)
    a.update(over)
    return lib.kron3_batched(*a.values())


INVALID, NOTSUP, ALIAS = 1, 2, 3


@pytest.mark.parametrize("over,code", [
    (dict(ma=0), INVALID), (dict(nb=17), INVALID), (dict(ta=b"X"), INVALID), (dict(tx=b"Q"), INVALID),
    (dict(batch=-1), INVALID), (dict(lda=3), INVALID), (dict(ldb=2), INVALID), (dict(ldx=3), INVALID),
    (dict(ldy=3), INVALID), (dict(ldyp=15), INVALID), (dict(ldxp=-1), INVALID),
    (dict(alpha=None), INVALID), (dict(beta=None), INVALID), (dict(X=None), INVALID), (dict(Y=None), INVALID),
    (dict(A=None), INVALID), (dict(io=7), INVALID), (dict(comp=9), INVALID),
    (dict(io=1, comp=1), NOTSUP), (dict(io=4, comp=1), NOTSUP),
    (dict(io=5, comp=1), NOTSUP), (dict(io=6), INVALID),
    (dict(Y=0x10000 + 4 * 100), ALIAS), (dict(X=0x90000), ALIAS),
    (dict(X=0x10002), INVALID),            # not aligned to the element size
    (dict(ta=b"T", lda=3, ma=3, na=4), INVALID),   # stored A is na x ma: lda >= na
    (dict(batch=0, X=None, Y=None), 0),    # empty batch: no-op
])
def test_kron2_validation(lib, over, code):
    assert k2(lib, **over) == code


@pytest.mark.parametrize("over,code", [
    (dict(mc=0), INVALID), (dict(ldx2=8), INVALID), (dict(ldy2=8), INVALID), (dict(ldyp=26), INVALID),
    (dict(C=None), INVALID), (dict(ldc=2), INVALID), (dict(Y=0x10000 + 8), ALIAS),
    (dict(io=2, comp=0, X=0x10000, Y=0x90000), "launch"), (dict(batch=0), 0),
])
def test_kron3_validation(lib, over, code):
    r = k3(lib, **over)
    if code == "launch":
        import torch
        if torch.cuda.is_available():
            # with a GPU the pre-launch check sees that the made-up addresses are
            # not device memory and returns INVALID_VALUE, as it must
            assert r == INVALID
            return
        assert r != INVALID and r != NOTSUP   # valid arguments: only the launch itself can fail here
    else:
        assert r == code


def k1(lib, **over):
    a = dict(stream=None, ta=b"N", ma=4, na=5, batch=10, alpha=ctypes.addressof(F), A=COMP.ctypes.data, lda=4,
             X=0x10000, ldxp=5, beta=ctypes.addressof(ZERO), Y=0x90000, ldyp=4, io=0, comp=0)
    a.update(over)
    return lib.kron1_batched(*a.values())


def ga(lib, **over):
    a = dict(stream=None, ta=b"N", tb=b"N", m=100, n=6, k=5, alpha=ctypes.addressof(F), A=0x10000, lda=100,
             lda2=500, B=COMP.ctypes.data, ldb=5, beta=ctypes.addressof(ZERO), C=0x900000, ldc=100, ldc2=600,
             batch=10, grid=0, io=0, comp=0)
    a.update(over)
    return lib.kron_gemm_a_batched(*a.values())


@pytest.mark.parametrize("over,code", [
    (dict(ma=0), INVALID), (dict(na=17), INVALID), (dict(ta=b"X"), INVALID), (dict(batch=-1), INVALID),
    (dict(lda=3), INVALID), (dict(ta=b"T", lda=4), INVALID), (dict(ldyp=3), INVALID), (dict(ldxp=-1), INVALID),
    (dict(alpha=None), INVALID), (dict(A=None), INVALID), (dict(X=None), INVALID), (dict(Y=None), INVALID),
    (dict(io=7), INVALID), (dict(comp=1), NOTSUP), (dict(io=2, comp=1), NOTSUP),
    (dict(Y=0x10000 + 4 * 40), ALIAS), (dict(X=0x10002), INVALID),
    (dict(batch=0, X=None, Y=None), 0), (dict(batch=1, ldyp=0), "launch"),
])
def test_kron1_validation(lib, over, code):
    r = k1(lib, **over)
    if code == "launch":
        import torch
        if torch.cuda.is_available():   # the made-up addresses are not device memory
            assert r == INVALID
            return
        assert r not in (INVALID, NOTSUP, ALIAS)
    else:
        assert r == code


@pytest.mark.parametrize("over,code", [
    (dict(m=0), INVALID), (dict(m=(1 << 24) + 1), INVALID), (dict(n=17), INVALID), (dict(k=0), INVALID),
    (dict(ta=b"Z"), INVALID), (dict(tb=b"Z"), INVALID), (dict(lda=99), INVALID), (dict(ta=b"T", lda=4), INVALID),
    (dict(ldb=4), INVALID), (dict(tb=b"T", ldb=5), INVALID), (dict(ldc=99), INVALID), (dict(ldc2=599), INVALID),
    (dict(lda2=-1), INVALID), (dict(grid=-1), INVALID), (dict(batch=-1), INVALID), (dict(beta=None), INVALID),
    (dict(B=None), INVALID), (dict(C=None), INVALID), (dict(comp=1), NOTSUP),
    (dict(C=0x10000 + 4 * 4000), ALIAS), (dict(C=0x900002), INVALID),
    (dict(batch=0, A=None, C=None), 0), (dict(lda2=0), "launch"), (dict(batch=1, ldc2=0), "launch"),
])
def test_gemm_a_validation(lib, over, code):
    r = ga(lib, **over)
    if code == "launch":
        import torch
        if torch.cuda.is_available():   # the made-up addresses are not device memory
            assert r == INVALID
            return
        assert r not in (INVALID, NOTSUP, ALIAS)
    else:
        assert r == code


def test_binding_rejects_cpu_tensors_without_a_gpu():
    """A CPU tensor never reaches the library: its address would be a host pointer."""
    import torch
    n = 4
    X = torch.zeros(2 * n * n)
    with pytest.raises(TypeError):
        kg.kron2_batched(np.eye(n), np.eye(n), X, X.clone(), ma=n, na=n, mb=n, nb=n, batch=2)
    with pytest.raises(TypeError):
        kg.kron1_batched(np.eye(n), X, X.clone(), ma=n, na=n, batch=2)


def test_check_device_buffer_without_a_gpu():
    """A null pointer is rejected outright; any other range needs the runtime,
    which answers KRON_ERR_CUDA when no device is usable (a GPU run checks the
    device cases)."""
    import torch
    assert kg.check_device_buffer(0, 16) == 1
    if not torch.cuda.is_available():
        h = np.zeros(4, np.float32)
        assert kg.check_device_buffer(h.ctypes.data, h.nbytes) in (1, 5)


def test_first_wait_limit_is_validated(lib):
    assert lib.kron_set_first_wait_limit_ns(10 ** 12) == INVALID   # above the normal 2 s limit
    assert lib.kron_set_first_wait_limit_ns(5) == 0
    assert lib.kron_set_first_wait_limit_ns(0) == 0


def test_peak_probe_rejects_bad_arguments(lib):
    f = ctypes.c_double()
    assert lib.kron_peak_probe(None, 3, 10, ctypes.byref(f)) == INVALID
    assert lib.kron_peak_probe(None, 0, 0, ctypes.byref(f)) == INVALID
    assert lib.kron_peak_probe(None, 0, 10, None) == INVALID


NOTSUP_ = 2


def test_kernel_config_validation_and_round_trip(lib):
    cfg = kg.KernelConfig
    f32 = kg.DTYPES["f32"]
    # out of range
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg(9, 0, 0, 0))) == INVALID
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg(2, 0, 13, 0))) == INVALID
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg(1, 32, 5, 0, 17))) == INVALID
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg(1, 32, 5, 0, -1))) == INVALID
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg(2, 0, 0, 3))) == INVALID
    assert lib.kron_set_kernel_config(2, 17, f32, 0, ctypes.byref(cfg(0, 0, 0, 0))) == INVALID
    assert lib.kron_set_kernel_config(2, 16, f32, 0, None) == INVALID
    # bodies that do not exist for the configuration
    assert lib.kron_set_kernel_config(2, 12, f32, 0, ctypes.byref(cfg(1, 0, 0, 0))) == NOTSUP_   # no in-place 2-D n=12
    assert lib.kron_set_kernel_config(2, 7, f32, 0, ctypes.byref(cfg(2, 0, 0, 0))) == NOTSUP_    # pairs need even n
    assert lib.kron_set_kernel_config(2, 16, kg.DTYPES["f64"], 0, ctypes.byref(cfg(2, 0, 0, 0))) == NOTSUP_
    # split tensor path: 2-D padded tile (any n) or stacked (9 <= n <= 16); 3-D one body
    assert lib.kron_set_kernel_config(2, 16, f32, 1, ctypes.byref(cfg(3, 0, 0, 0))) == NOTSUP_
    assert lib.kron_set_kernel_config(2, 8, f32, 1, ctypes.byref(cfg(2, 0, 0, 0))) == NOTSUP_
    assert lib.kron_set_kernel_config(3, 16, f32, 1, ctypes.byref(cfg(2, 0, 0, 0))) == NOTSUP_
    assert lib.kron_set_kernel_config(2, 16, kg.DTYPES["f64"], 1, ctypes.byref(cfg(1, 0, 0, 0))) == NOTSUP_
    for n, var, groups in ((8, 1, 0), (9, 2, 0), (12, 1, 0), (16, 2, 2), (14, 2, 1)):
        assert lib.kron_set_kernel_config(2, n, kg.DTYPES["bf16"], 1, ctypes.byref(cfg(var, 64, 2, groups))) == 0
        got = cfg()
        assert lib.kron_get_kernel_config(2, n, kg.DTYPES["bf16"], 1, ctypes.byref(got)) == 0
        assert (got.variant, got.instances_per_tile, got.pipeline_depth, got.fibers_per_step) == (var, 64, 2, groups)
        assert lib.kron_set_kernel_config(2, n, kg.DTYPES["bf16"], 1, ctypes.byref(cfg())) == 0
    assert lib.kron_set_kernel_config(2, 16, kg.DTYPES["bf16"], 1, ctypes.byref(cfg(2, 64, 2, 3))) == INVALID
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg(1, 7, 0, 0))) == NOTSUP_   # in place: 8..32 by 8
    assert lib.kron_set_kernel_config(2, 16, kg.DTYPES["bf16"], 0, ctypes.byref(cfg(1, 32, 0, 0))) == NOTSUP_
    # compute warps: only the FP32 2-D n = 16 in-place body, in groups of P / 4
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg(1, 32, 5, 0, 12))) == NOTSUP_
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg(2, 0, 2, 0, 8))) == NOTSUP_
    assert lib.kron_set_kernel_config(2, 12, f32, 0, ctypes.byref(cfg(0, 0, 0, 0, 8))) == NOTSUP_
    assert lib.kron_set_kernel_config(2, 16, kg.DTYPES["bf16"], 0, ctypes.byref(cfg(1, 16, 0, 0, 4))) == NOTSUP_
    assert lib.kron_set_kernel_config(3, 16, f32, 1, ctypes.byref(cfg(0, 0, 0, 0, 3))) == NOTSUP_   # 1, 2, 4, 8
    assert lib.kron_set_kernel_config(2, 10, f32, 0, ctypes.byref(cfg(1, 48, 10, 0, 6))) == NOTSUP_  # groups of 4
    assert lib.kron_set_kernel_config(2, 10, f32, 0, ctypes.byref(cfg(1, 48, 10, 0, 16))) == 0
    assert lib.kron_set_kernel_config(2, 10, f32, 0, ctypes.byref(cfg())) == 0
    assert lib.kron_set_kernel_config(3, 16, f32, 1, ctypes.byref(cfg(0, 0, 0, 0, 8))) == 0
    assert lib.kron_set_kernel_config(3, 16, f32, 1, ctypes.byref(cfg())) == 0
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg(1, 24, 3, 0, 12))) == 0
    got = cfg()
    assert lib.kron_get_kernel_config(2, 16, f32, 0, ctypes.byref(got)) == 0
    assert (got.variant, got.instances_per_tile, got.pipeline_depth, got.compute_warps) == (1, 24, 3, 12)
    assert lib.kron_set_kernel_config(2, 16, f32, 0, ctypes.byref(cfg())) == 0
    # round trip, then back to the default
    assert lib.kron_set_kernel_config(3, 12, f32, 0, ctypes.byref(cfg(2, 6, 2, 2))) == 0
    got = cfg()
    assert lib.kron_get_kernel_config(3, 12, f32, 0, ctypes.byref(got)) == 0
    assert (got.variant, got.instances_per_tile, got.pipeline_depth, got.fibers_per_step) == (2, 6, 2, 2)
    p, d = ctypes.c_int(), ctypes.c_int()
    assert lib.kron_get_tile_config(3, 12, f32, 0, ctypes.byref(p), ctypes.byref(d)) == 0
    assert (p.value, d.value) == (6, 2)
    assert lib.kron_set_kernel_config(3, 12, f32, 0, ctypes.byref(cfg(0, 0, 0, 0))) == 0
    assert lib.kron_get_kernel_config(3, 12, f32, 0, ctypes.byref(got)) == 0
    assert (got.variant, got.instances_per_tile, got.pipeline_depth, got.fibers_per_step) == (0, 0, 0, 0)


def test_varlen_set_scaling_validation(lib):
    """kron_varlen_plan_set_scaling validates before touching the plan (no GPU needed)."""
    assert lib.kron_varlen_plan_set_scaling(None, 1.0, 0.0) == INVALID
    assert lib.kron_varlen_plan_set_scaling(None, float("nan"), 0.0) == INVALID
