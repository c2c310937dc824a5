"""Python binding of the GB300 batched Kronecker product library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``_build/libkron_gb300.so`` (C ABI in ``include/kron.h``).  PyTorch
provides device memory and streams.  There is no CPU fallback: if the library
is missing or cannot be loaded, every call raises.

Operation (paper Sec. 2.2):
    kron2_batched:  Y^p <- alpha op(B) op(X^p) op(A)^T + beta Y^p
                    ( = alpha (op(A) (x) op(B)) vec(op(X^p)) + beta vec(Y^p) )
    kron3_batched:  Y^p <- alpha (op(A) (x) op(B) (x) op(C)) vec(X^p) + beta Y^p
                    (C on mode 1, B on mode 2, A on mode 3)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkron_gb300.so")

KRON_OK = 0
STATUS = {0: "KRON_OK", 1: "KRON_ERR_INVALID_VALUE", 2: "KRON_ERR_NOT_SUPPORTED", 3: "KRON_ERR_ALIAS",
          4: "KRON_ERR_WORKSPACE", 5: "KRON_ERR_CUDA", 6: "KRON_ERR_DEVICE_TIMEOUT"}
DTYPES = {"f32": 0, "f64": 1, "bf16": 2, "f16": 3, "c64": 4, "c128": 5}
COMPUTE = {"native": 0, "bf16x3": 1}

# Every entry point declared in include/kron.h, with its ctypes signature.
_I, _L, _P, _C, _S = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_char, ctypes.c_size_t
SIGNATURES = {
    "kron_status_string": ([_I], ctypes.c_char_p),
    "kron_version": ([], _I),
    "kron_check_device_buffer": ([_P, _S], _I),
    "kron2_batched": ([_P, _C, _C, _C, _I, _I, _I, _I, _L, _P, _P, _I, _P, _I, _P, _I, _L, _P, _P, _I, _L,
                       _I, _I], _I),
    "kron3_batched": ([_P, _C, _C, _C, _I, _I, _I, _I, _I, _I, _L, _P, _P, _I, _P, _I, _P, _I, _P, _I, _I,
                       _L, _P, _P, _I, _I, _L, _I, _I], _I),
    "kron1_batched": ([_P, _C, _I, _I, _L, _P, _P, _I, _P, _L, _P, _P, _L, _I, _I], _I),
    "kron_gemm_a_batched": ([_P, _C, _C, _I, _I, _I, _P, _P, _I, _L, _P, _I, _P, _P, _I, _L, _L, _I, _I, _I],
                            _I),
    "kron_device_status": ([_P], _I),
    "kron_set_first_wait_limit_ns": ([ctypes.c_ulonglong], _I),
    "kron_peak_probe": ([_P, _I, _I, ctypes.POINTER(ctypes.c_double)], _I),
    "kron_set_tile_config": ([_I, _I, _I, _I, _I, _I], _I),
    "kron_get_tile_config": ([_I, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "kron_autotune": ([_P, _I, _I, _L, _P, _P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "kron_set_kernel_config": ([_I, _I, _I, _I, _P], _I),
    "kron_get_kernel_config": ([_I, _I, _I, _I, _P], _I),
    "kron_autotune_config": ([_P, _I, _I, _L, _P, _P, _I, _I, _P], _I),
    "kron_varlen_plan_create": ([ctypes.POINTER(_P), _I, _P, _L, _P, _P, _P, _I, _I], _I),
    "kron_varlen_workspace_size": ([_P, ctypes.POINTER(_S)], _I),
    "kron_varlen_execute": ([_P, _P, _P, _P, _S, _P], _I),
    "kron_varlen_tune": ([_P, _P, _P, _P, _S, _P], _I),
    "kron_varlen_plan_destroy": ([_P], _I),
    "kron_varlen_plan_set_scaling": ([_P, ctypes.c_double, ctypes.c_double], _I),
    "kron_varlen_execute_noalloc": ([_P, _P, _P, _P], _I),
}

_lib = None


class KronError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the CUDA library and bind the C ABI (raises if it is not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built: {path} is missing "
                               "(run __graft_entry__.build() or paper_1304_7054_gb300/build.py)")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def status_string(status: int) -> str:
    return load_library().kron_status_string(status).decode()


def _check(status: int, what: str):
    if status != KRON_OK:
        raise KronError(status, what)


def _torch():
    import torch
    return torch


def _io_of(t) -> int:
    torch = _torch()
    m = {torch.float32: "f32", torch.float64: "f64", torch.bfloat16: "bf16", torch.float16: "f16",
         torch.complex64: "c64", torch.complex128: "c128"}
    if t.dtype not in m:
        raise TypeError(f"unsupported storage dtype {t.dtype}")
    return DTYPES[m[t.dtype]]


def _stream_handle(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _comp_buffer(M, ctype):
    """A component as a host buffer: 2-D arrays become column-major (ld = rows);
    1-D arrays are taken as already column-major.  Returns (array, ld)."""
    if hasattr(M, "detach"):
        M = M.detach().cpu().numpy()
    M = np.asarray(M, dtype=ctype)
    if M.ndim == 2:
        return np.ascontiguousarray(M.T).ravel(), M.shape[0]
    return np.ascontiguousarray(M.ravel()), None


def _device_operand(t, need, name):
    """Device address of tensor t, after checking that it lives on a GPU and, when
    contiguous, holds the `need` elements the call touches (the library checks
    the same range against the allocation before it launches anything)."""
    if not getattr(t, "is_cuda", False):
        raise TypeError(f"{name} must be a CUDA tensor")
    if need > 0 and t.is_contiguous() and t.numel() < need:
        raise ValueError(f"{name} holds {t.numel()} elements but the call reaches element {need - 1}")
    return t.data_ptr()


def _scalar(v, ctype):
    """A host scalar of the compute type; complex scalars as their (re, im) pair."""
    if ctype in (np.complex64, np.complex128):
        v = complex(v)
        return ((ctypes.c_double if ctype == np.complex128 else ctypes.c_float) * 2)(v.real, v.imag)
    return (ctypes.c_double if ctype == np.float64 else ctypes.c_float)(v)


def _ctype_of(io):
    """Host type of the components, alpha and beta for storage type io."""
    return {DTYPES["f64"]: np.float64, DTYPES["c64"]: np.complex64, DTYPES["c128"]: np.complex128}.get(io, np.float32)


def kron2_batched(A, B, X, Y, *, ma, na, mb, nb, batch, alpha=1.0, beta=0.0, transa="N", transb="N",
                  transx="N", lda=None, ldb=None, ldx=None, ldxp=None, ldy=None, ldyp=None,
                  compute="native", stream=None):
    """Y^p <- alpha op(B) op(X^p) op(A)^T + beta Y^p on CUDA tensors X, Y (storage
    f32/f64/bf16/f16, flat column-major instances); A, B host arrays."""
    L = load_library()
    io = _io_of(X)
    if _io_of(Y) != io:
        raise TypeError("X and Y must have the same dtype")
    ctype = _ctype_of(io)
    Ab, lda0 = _comp_buffer(A, ctype)
    Bb, ldb0 = _comp_buffer(B, ctype)
    ta, tb, tx = transa.upper(), transb.upper(), transx.upper()
    lda = lda or lda0 or (ma if ta == "N" else na)
    ldb = ldb or ldb0 or (mb if tb == "N" else nb)
    ldx = ldx or (nb if tx == "N" else na)
    ldxp = ldx * (na if tx == "N" else nb) if ldxp is None else ldxp
    ldy = ldy or mb
    ldyp = ldy * ma if ldyp is None else ldyp
    al, be = _scalar(alpha, ctype), _scalar(beta, ctype)
    xr, xc = (nb, na) if tx == "N" else (na, nb)
    xp = _device_operand(X, (batch - 1) * ldxp + ldx * (xc - 1) + xr if batch > 0 else 0, "X")
    yp = _device_operand(Y, (batch - 1) * ldyp + ldy * (ma - 1) + mb if batch > 0 else 0, "Y")
    st = L.kron2_batched(_stream_handle(stream), ta.encode(), tb.encode(), tx.encode(), ma, na, mb, nb, batch,
                         ctypes.addressof(al), Ab.ctypes.data, lda, Bb.ctypes.data, ldb, xp, ldx, ldxp,
                         ctypes.addressof(be), yp, ldy, ldyp, io, COMPUTE[compute])
    _check(st, "kron2_batched")
    return Y


def kron3_batched(A, B, C, X, Y, *, ma, na, mb, nb, mc, nc, batch, alpha=1.0, beta=0.0, transa="N",
                  transb="N", transc="N", lda=None, ldb=None, ldc=None, ldx=None, ldx2=None, ldxp=None,
                  ldy=None, ldy2=None, ldyp=None, compute="native", stream=None):
    """Y^p <- alpha (op(A) (x) op(B) (x) op(C)) vec(X^p) + beta Y^p (C on mode 1)."""
    L = load_library()
    io = _io_of(X)
    if _io_of(Y) != io:
        raise TypeError("X and Y must have the same dtype")
    ctype = _ctype_of(io)
    Ab, lda0 = _comp_buffer(A, ctype)
    Bb, ldb0 = _comp_buffer(B, ctype)
    Cb, ldc0 = _comp_buffer(C, ctype)
    ta, tb, tc = transa.upper(), transb.upper(), transc.upper()
    lda = lda or lda0 or (ma if ta == "N" else na)
    ldb = ldb or ldb0 or (mb if tb == "N" else nb)
    ldc = ldc or ldc0 or (mc if tc == "N" else nc)
    ldx = ldx or nc
    ldx2 = ldx2 or ldx * nb
    ldxp = ldx2 * na if ldxp is None else ldxp
    ldy = ldy or mc
    ldy2 = ldy2 or ldy * mb
    ldyp = ldy2 * ma if ldyp is None else ldyp
    al, be = _scalar(alpha, ctype), _scalar(beta, ctype)
    xp = _device_operand(X, (batch - 1) * ldxp + ldx2 * (na - 1) + ldx * (nb - 1) + nc if batch > 0 else 0, "X")
    yp = _device_operand(Y, (batch - 1) * ldyp + ldy2 * (ma - 1) + ldy * (mb - 1) + mc if batch > 0 else 0, "Y")
    st = L.kron3_batched(_stream_handle(stream), ta.encode(), tb.encode(), tc.encode(), ma, na, mb, nb, mc, nc,
                         batch, ctypes.addressof(al), Ab.ctypes.data, lda, Bb.ctypes.data, ldb, Cb.ctypes.data,
                         ldc, xp, ldx, ldx2, ldxp, ctypes.addressof(be), yp, ldy, ldy2, ldyp,
                         io, COMPUTE[compute])
    _check(st, "kron3_batched")
    return Y


def kron1_batched(A, X, Y, *, ma, na, batch, alpha=1.0, beta=0.0, transa="N", lda=None, ldxp=None, ldyp=None,
                  compute="native", stream=None):
    """TKRON1: y^p <- alpha op(A) x^p + beta y^p on CUDA tensors X, Y; A a host array."""
    L = load_library()
    io = _io_of(X)
    if _io_of(Y) != io:
        raise TypeError("X and Y must have the same dtype")
    ctype = _ctype_of(io)
    Ab, lda0 = _comp_buffer(A, ctype)
    ta = transa.upper()
    lda = lda or lda0 or (ma if ta == "N" else na)
    ldxp = na if ldxp is None else ldxp
    ldyp = ma if ldyp is None else ldyp
    al, be = _scalar(alpha, ctype), _scalar(beta, ctype)
    xp = _device_operand(X, (batch - 1) * ldxp + na if batch > 0 else 0, "X")
    yp = _device_operand(Y, (batch - 1) * ldyp + ma if batch > 0 else 0, "Y")
    st = L.kron1_batched(_stream_handle(stream), ta.encode(), ma, na, batch, ctypes.addressof(al), Ab.ctypes.data,
                         lda, xp, ldxp, ctypes.addressof(be), yp, ldyp, io, COMPUTE[compute])
    _check(st, "kron1_batched")
    return Y


def gemm_a_batched(A, B, C, *, m, n, k, batch, alpha=1.0, beta=0.0, transa="N", transb="N", lda=None, lda2=None,
                   ldb=None, ldc=None, ldc2=None, grid_size=0, compute="native", stream=None):
    """TGEMM_A: C^p <- alpha op(A^p) op(B) + beta C^p on CUDA tensors A, C; B a host array."""
    L = load_library()
    io = _io_of(A)
    if _io_of(C) != io:
        raise TypeError("A and C must have the same dtype")
    ctype = _ctype_of(io)
    Bb, ldb0 = _comp_buffer(B, ctype)
    ta, tb = transa.upper(), transb.upper()
    lda = lda or (m if ta == "N" else k)
    lda2 = lda * (k if ta == "N" else m) if lda2 is None else lda2
    ldb = ldb or ldb0 or (k if tb == "N" else n)
    ldc = ldc or m
    ldc2 = ldc * n if ldc2 is None else ldc2
    al, be = _scalar(alpha, ctype), _scalar(beta, ctype)
    aext = lda * (m - 1) + k if ta == "T" else lda * (k - 1) + m
    ap = _device_operand(A, (batch - 1) * lda2 + aext if batch > 0 else 0, "A")
    cp = _device_operand(C, (batch - 1) * ldc2 + ldc * (n - 1) + m if batch > 0 else 0, "C")
    st = L.kron_gemm_a_batched(_stream_handle(stream), ta.encode(), tb.encode(), m, n, k, ctypes.addressof(al),
                               ap, lda, lda2, Bb.ctypes.data, ldb, ctypes.addressof(be), cp,
                               ldc, ldc2, batch, grid_size, io, COMPUTE[compute])
    _check(st, "kron_gemm_a_batched")
    return C


def check_device_buffer(t, nbytes=None) -> int:
    """kron_check_device_buffer on tensor t (or a raw address with nbytes): the
    status the library's own pre-launch check gives for that range."""
    ptr = t.data_ptr() if hasattr(t, "data_ptr") else int(t)
    if nbytes is None:
        nbytes = t.numel() * t.element_size()
    return load_library().kron_check_device_buffer(ptr, nbytes)


def device_status(stream=None) -> int:
    """Synchronise and read/clear the device status word (0 = OK)."""
    return load_library().kron_device_status(_stream_handle(stream))


def set_first_wait_limit_ns(ns: int) -> None:
    """Failure-path test aid: the first operand wait of each CTA of the 2-D n = 16
    FP32 kernel polls for at most ns nanoseconds (0 restores the normal limit)."""
    _check(load_library().kron_set_first_wait_limit_ns(ns), "kron_set_first_wait_limit_ns")


PEAK_UNITS = {"ffma2": 0, "ffma": 1, "dfma": 2}


def peak_probe(unit, iters, stream=None) -> float:
    """Launch the FMA-throughput probe of `unit` ("ffma2", "ffma", "dfma") on the
    stream; returns the flops of that launch (the caller times it)."""
    f = ctypes.c_double()
    _check(load_library().kron_peak_probe(_stream_handle(stream), PEAK_UNITS[unit], iters, ctypes.byref(f)),
           "kron_peak_probe")
    return f.value


def set_tile_config(kind, n, io, compute="native", instances_per_tile=0, pipeline_depth=0):
    """Launch configuration of the fixed-size kernels for one (kind, n, storage, compute)."""
    _check(load_library().kron_set_tile_config(kind, n, DTYPES[io], COMPUTE[compute], instances_per_tile,
                                                pipeline_depth), "kron_set_tile_config")


def get_tile_config(kind, n, io, compute="native"):
    p, d = ctypes.c_int(), ctypes.c_int()
    _check(load_library().kron_get_tile_config(kind, n, DTYPES[io], COMPUTE[compute], ctypes.byref(p),
                                                ctypes.byref(d)), "kron_get_tile_config")
    return p.value, d.value


def autotune(kind, n, batch, X, Y, compute="native", stream=None):
    """Time the candidate tile configurations on X -> Y and keep the fastest."""
    p, d = ctypes.c_int(), ctypes.c_int()
    need = batch * n ** kind
    xp, yp = _device_operand(X, need, "X"), _device_operand(Y, need, "Y")
    _check(load_library().kron_autotune(_stream_handle(stream), kind, n, batch, xp, yp,
                                        _io_of(X), COMPUTE[compute], ctypes.byref(p), ctypes.byref(d)),
           "kron_autotune")
    return p.value, d.value


VARIANTS = {"auto": 0, "in_place": 1, "exchange": 2, "scalar": 3}


class KernelConfig(ctypes.Structure):
    """kron_kernel_config: kernel body, instances per tile, pipeline depth,
    fibers per step and compute warps of one fixed-size (kind, n, storage, compute)."""
    _fields_ = [("variant", ctypes.c_int), ("instances_per_tile", ctypes.c_int), ("pipeline_depth", ctypes.c_int),
                ("fibers_per_step", ctypes.c_int), ("compute_warps", ctypes.c_int)]

    def as_dict(self):
        names = {v: k for k, v in VARIANTS.items()}
        return {"variant": names.get(self.variant, self.variant), "instances_per_tile": self.instances_per_tile,
                "pipeline_depth": self.pipeline_depth, "fibers_per_step": self.fibers_per_step,
                "compute_warps": self.compute_warps}


def set_kernel_config(kind, n, io, compute="native", variant="auto", instances_per_tile=0, pipeline_depth=0,
                      fibers_per_step=0, compute_warps=0):
    c = KernelConfig(VARIANTS[variant], instances_per_tile, pipeline_depth, fibers_per_step, compute_warps)
    _check(load_library().kron_set_kernel_config(kind, n, DTYPES[io], COMPUTE[compute], ctypes.byref(c)),
           "kron_set_kernel_config")


def get_kernel_config(kind, n, io, compute="native") -> dict:
    c = KernelConfig()
    _check(load_library().kron_get_kernel_config(kind, n, DTYPES[io], COMPUTE[compute], ctypes.byref(c)),
           "kron_get_kernel_config")
    return c.as_dict()


def autotune_config(kind, n, batch, X, Y, compute="native", stream=None) -> dict:
    """Search kernel bodies, tiles, pipeline depths and fibers per step on X -> Y;
    keeps the fastest (Y is overwritten) and returns it."""
    c = KernelConfig()
    need = batch * n ** kind
    xp, yp = _device_operand(X, need, "X"), _device_operand(Y, need, "Y")
    _check(load_library().kron_autotune_config(_stream_handle(stream), kind, n, batch, xp, yp, _io_of(X),
                                               COMPUTE[compute], ctypes.byref(c)), "kron_autotune_config")
    return c.as_dict()


class _ClassDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("C", ctypes.c_void_p)]


class VarlenPlan:
    """Mixed-size batch plan (kron_varlen_plan_*): one persistent, graph-captured launch.

    classes: list of (kind, n, A, B[, C]) with n x n host components (2-D arrays are
    taken as matrices, 1-D as column-major); class_of[p], x_off[p], y_off[p] give each
    instance's class and element offsets into X and Y.
    """

    def __init__(self, classes, class_of, x_off, y_off, io="f32", compute="native"):
        L = load_library()
        self._keep = []
        descs = (_ClassDesc * max(1, len(classes)))()
        for i, c in enumerate(classes):
            kind, n = int(c[0]), int(c[1])
            mats = []
            for M in c[2:2 + kind]:
                buf, _ = _comp_buffer(M, np.float32)
                self._keep.append(buf)
                mats.append(buf.ctypes.data)
            A, B = mats[0], mats[1]
            C = mats[2] if kind == 3 else None
            descs[i] = _ClassDesc(kind, n, A, B, C)
        self._cls = np.ascontiguousarray(class_of, dtype=np.int32)
        self._xo = np.ascontiguousarray(x_off, dtype=np.int64)
        self._yo = np.ascontiguousarray(y_off, dtype=np.int64)
        self.batch = len(self._cls)
        h = ctypes.c_void_p()
        _check(L.kron_varlen_plan_create(ctypes.byref(h), len(classes), ctypes.addressof(descs), self.batch,
                                         self._cls.ctypes.data, self._xo.ctypes.data, self._yo.ctypes.data,
                                         DTYPES[io], COMPUTE[compute]), "kron_varlen_plan_create")
        self.handle = h
        self.io = io
        # elements of X and Y the plan reaches (the library has validated the metadata)
        sizes = np.array([int(c[1]) ** int(c[0]) for c in classes] or [0], dtype=np.int64)
        nx = sizes[self._cls] if self.batch else np.zeros(0, np.int64)
        self.x_extent = int((self._xo + nx).max()) if self.batch else 0
        self.y_extent = int((self._yo + nx).max()) if self.batch else 0

    def workspace_size(self) -> int:
        s = ctypes.c_size_t()
        _check(load_library().kron_varlen_workspace_size(self.handle, ctypes.byref(s)),
               "kron_varlen_workspace_size")
        return s.value

    def alloc_workspace(self, device=None):
        torch = _torch()
        return torch.empty(max(1, self.workspace_size()), dtype=torch.uint8, device=device or "cuda")

    def _operands(self, X, Y):
        return _device_operand(X, self.x_extent, "X"), _device_operand(Y, self.y_extent, "Y")

    def execute(self, X, Y, workspace, stream=None):
        xp, yp = self._operands(X, Y)
        _check(load_library().kron_varlen_execute(self.handle, xp, yp, _device_operand(workspace, 0, "workspace"),
                                                  workspace.numel() * workspace.element_size(),
                                                  _stream_handle(stream)),
               "kron_varlen_execute")
        return Y

    def execute_noalloc(self, X, Y, stream=None):
        """Same result as execute(), with the library's fixed device array as the
        workspace (no allocation anywhere; at most 262,144 instances)."""
        xp, yp = self._operands(X, Y)
        _check(load_library().kron_varlen_execute_noalloc(self.handle, xp, yp, _stream_handle(stream)),
               "kron_varlen_execute_noalloc")
        return Y

    def set_scaling(self, alpha=1.0, beta=0.0):
        """alpha and beta of later executes: Y = alpha (K X) + beta Y per instance."""
        _check(load_library().kron_varlen_plan_set_scaling(self.handle, float(alpha), float(beta)),
               "kron_varlen_plan_set_scaling")

    def tune(self, X, Y, workspace, stream=None):
        xp, yp = self._operands(X, Y)
        _check(load_library().kron_varlen_tune(self.handle, xp, yp, _device_operand(workspace, 0, "workspace"),
                                               workspace.numel() * workspace.element_size(),
                                               _stream_handle(stream)), "kron_varlen_tune")

    def close(self):
        if getattr(self, "handle", None):
            load_library().kron_varlen_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
