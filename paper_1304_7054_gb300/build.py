"""Builds the CUDA library ``_build/libkron_gb300.so`` for sm_103a with nvcc.

Every translation unit under ``csrc/`` is compiled in parallel, then linked
into one shared library exporting the C ABI of ``include/kron.h``.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libkron_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
                     "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                     "-Xcompiler", "-Wall", "-I", os.path.join(HERE, "..", "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(obj: str, src: str, headers) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(f) > t for f in [src, *headers])


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    srcs = _sources()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    todo = [(s, o) for s, o in zip(srcs, objs) if force or _stale(o, s, headers)]
    cc = nvcc()

    def one(so):
        s, o = so
        cmd = [cc, *NVCC_FLAGS, *extra, "-c", s, "-o", o]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(s)}:\n{r.stdout}")
        if verbose and r.stdout.strip():
            print(r.stdout)
        return r.stdout

    jobs = jobs or max(1, min(len(todo), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        list(ex.map(one, todo))
    if todo or not os.path.exists(LIB):
        cmd = [cc, *ARCH, "-shared", "-o", LIB, *objs, "-cudart", "static"]
        subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))


# Sources that define each kernel family: its device code and its launcher (tile
# size, pipeline depth, grid).  Argument checking and dispatch are left out: they
# decide which kernel runs, not what a launch of it does.
FAMILY_SOURCES = {
    "pair_kernel": ["kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "pair16_kernel": ["kron_pair16.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "pair16h_kernel": ["kron_pair16.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "pair16t_kernel": ["kron_pair16.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh", "kron_internal.h"],
    "pair2ip_kernel": ["kron_pair2ip.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "pair3ip_kernel": ["kron_pair3ip.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "pair3pk_kernel": ["kron_pair3ip.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "fiber_kernel": ["kron_fiber.cuh", "kron_device.cuh"],
    "fiberip_kernel": ["kron_fiberip.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "gemm_a_kernel": ["kron_gemm_a.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "gemm_a_pair_kernel": ["kron_gemm_a.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "kron1_kernel": ["kron_kron1.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "kron1t_kernel": ["kron_kron1.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "gemm_a_tma_kernel": ["kron_gemm_a.cu", "kron_pair.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "tc2_kernel": ["kron_tc2.cu", "kron_tc.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "tc2s_kernel": ["kron_tc2.cu", "kron_tc.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "tc3_kernel": ["kron_tc3.cu", "kron_tc.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "tc3g_kernel": ["kron_tc3.cu", "kron_tc.cuh", "kron_fiber.cuh", "kron_device.cuh"],
    "varlen_kernel": ["kron_varlen.cu", "kron_fiber.cuh", "kron_device.cuh"],
}


def strip_comments(src: str) -> str:
    """C/C++ source without its comments (string and character literals kept),
    so that a comment edit leaves the code's hash unchanged."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return "".join(out)


def source_hash(family: str | None = None) -> str:
    """Hash of the code (comments removed, whitespace runs collapsed) of one kernel
    family's sources, or of all sources if None; a stored profile applies only
    while it is unchanged."""
    import hashlib
    h = hashlib.sha256()
    files = ([os.path.join(CSRC, f) for f in FAMILY_SOURCES[family]] if family
             else sorted(glob.glob(os.path.join(CSRC, "*"))))
    for f in files:
        h.update(os.path.basename(f).encode())
        h.update(" ".join(strip_comments(open(f, encoding="utf-8").read()).split()).encode())
    return h.hexdigest()[:16]
