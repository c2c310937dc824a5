"""Seeded synthetic inputs for the batched Kronecker product action.

This module only draws random numbers and lays them out; it contains none of
the method's arithmetic, so both the CUDA library's tests and the oracle can be
fed from it.  Workloads follow the paper's experiments (Sec. 5: real square
components of size n <= 16 shared by the whole batch, per-instance operands,
minimal leading dimensions) with synthetic values standing in for high-order
finite-element operands:

* components ~ U[-1, 1], drawn in the order A, B, C (C only for 3-D);
* operands X^p ~ U[-1, 1] (``x_dist="uniform"``) or N(0, 1) (``"normal"``),
  drawn after the components, batch-major, column-major inside an instance;
* generator: numpy PCG64 (``numpy.random.default_rng(seed)``);
* complex data (``dtype`` complex64 / complex128): every array draws its real
  parts, then its imaginary parts, from the same distribution.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Batch:
    kind: int                 # 2 or 3
    n: int                    # component size (square n x n)
    batch: int
    A: np.ndarray             # n*n, column-major
    B: np.ndarray
    C: np.ndarray | None      # 3-D only
    X: np.ndarray             # batch * n**kind, contiguous instances
    seed: int = 0
    x_dist: str = "normal"

    @property
    def inst(self) -> int:
        return self.n ** self.kind

    def comps(self):
        return (self.A, self.B) if self.kind == 2 else (self.A, self.B, self.C)


def _is_complex(dtype):
    return np.dtype(dtype).kind == "c"


def _real_of(dtype):
    return np.float64 if np.dtype(dtype) == np.complex128 else np.float32


def _uniform(rng, size, dtype):
    if _is_complex(dtype):
        r = rng.uniform(-1.0, 1.0, size)
        return (r + 1j * rng.uniform(-1.0, 1.0, size)).astype(dtype)
    return rng.uniform(-1.0, 1.0, size).astype(dtype)


def _draw_x(rng, size, x_dist, dtype):
    if _is_complex(dtype):
        re = _draw_x(rng, size, x_dist, _real_of(dtype))
        im = _draw_x(rng, size, x_dist, _real_of(dtype))
        out = np.empty(size, dtype=dtype)
        out.real, out.imag = re, im
        return out
    if x_dist == "uniform":
        return rng.uniform(-1.0, 1.0, size).astype(dtype)
    if x_dist == "normal":
        if dtype in (np.float32, np.float64):
            return rng.standard_normal(size, dtype=dtype)
        return rng.standard_normal(size).astype(dtype)
    raise ValueError(x_dist)


def make_batch(kind: int, n: int, batch: int, seed: int, x_dist: str = "normal",
               dtype=np.float32) -> Batch:
    """Components then operands from one PCG64 stream (draw order A, B, C, X)."""
    rng = np.random.default_rng(seed)
    A = _uniform(rng, n * n, dtype)
    B = _uniform(rng, n * n, dtype)
    C = _uniform(rng, n * n, dtype) if kind == 3 else None
    X = _draw_x(rng, batch * n ** kind, x_dist, dtype)
    return Batch(kind, n, batch, A, B, C, X, seed, x_dist)


@dataclass
class VarlenBatch:
    """A mixed-size batch: every instance has its own (kind, n) class.

    ``classes`` lists (kind, n) once per class with one shared component set each;
    ``class_of[p]`` is the class of instance p; instances are stored back to back
    in draw order, ``x_off[p]`` / ``y_off[p]`` being element offsets.
    """
    classes: list
    comps: list               # per class: (A, B) or (A, B, C), each n*n column-major
    class_of: np.ndarray      # int32 [batch]
    x_off: np.ndarray         # int64 [batch]
    y_off: np.ndarray         # int64 [batch]
    X: np.ndarray             # total elements
    total: int
    seed: int = 0
    extra: dict = field(default_factory=dict)


def make_varlen(count: int, seed: int, nmin: int = 4, nmax: int = 16, p3: float = 0.5,
                x_dist: str = "normal", dtype=np.float32) -> VarlenBatch:
    """``count`` instances with n ~ U{nmin..nmax} and kind 3 with probability p3.

    Classes are every (kind, n) pair, 2-D first, in increasing n; each gets its
    own components (draw order: for each class A, B, C; then the per-instance
    n, then kind, then X).
    """
    rng = np.random.default_rng(seed)
    classes = [(k, n) for k in (2, 3) for n in range(nmin, nmax + 1)]
    comps = []
    for k, n in classes:
        cs = [rng.uniform(-1.0, 1.0, n * n).astype(dtype) for _ in range(k)]
        comps.append(tuple(cs))
    ns = rng.integers(nmin, nmax + 1, size=count)
    kinds = np.where(rng.random(count) < p3, 3, 2)
    index = {c: i for i, c in enumerate(classes)}
    class_of = np.array([index[(int(k), int(n))] for k, n in zip(kinds, ns)], dtype=np.int32)
    sizes = ns.astype(np.int64) ** kinds.astype(np.int64)
    x_off = np.zeros(count, dtype=np.int64)
    if count:
        x_off[1:] = np.cumsum(sizes)[:-1]
    total = int(sizes.sum())
    X = _draw_x(rng, total, x_dist, dtype)
    return VarlenBatch(classes, comps, class_of, x_off, x_off.copy(), X, total, seed)


def to_storage(x: np.ndarray, storage: str):
    """Round an FP32 array to a 16-bit storage type (round-to-nearest-even).

    Returns a CPU torch tensor of dtype bfloat16 or float16 (numpy has no
    bfloat16).  This is input preparation shared by the library and the oracle:
    both then see exactly the same stored operand values.
    """
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    if storage == "bf16":
        return t.to(torch.bfloat16)
    if storage == "f16":
        return t.to(torch.float16)
    raise ValueError(storage)


def storage_to_f64(t) -> np.ndarray:
    """Exact widening of a 16-bit torch tensor to a float64 numpy array."""
    import torch
    return t.to(torch.float64).cpu().numpy()
