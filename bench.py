#!/usr/bin/env python
"""Throughput of the batched Kronecker product action on GB300.

One step = one pass of the whole hot path over one batch: component
preparation, operand stream-in, every mode contraction, epilogue and store
(one kernel launch).  The headline workload is the 2-D FP32 action at n = 16
over 2^20 instances (shared A, B ~ U[-1,1], X^p ~ N(0,1), seeded); the other
workloads (3-D, FP64, 16-bit storage, split-precision tensor cores, mixed
sizes) are measured the same way and reported under "variants".

Flops follow the paper's convention (Sec. 5): 4 n^3 per 2-D and 6 n^4 per 3-D
instance.  Algorithmic bytes are X read + Y written once (beta = 0).  Inputs
(>= 0.5 GB per pass) are larger than the 129 MB L2, so no flush is needed.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own batch (weak scaling, no collective in
the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GFlop/s & HBM GB/s (% roofline), 2-D/3-D Kronecker, n=16, FP32 vs BF16/varlen"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0

WORKLOADS = {
    # name: kind, n, batch, storage, compute, seed
    "kron2-f32-n16": dict(kind=2, n=16, batch=1 << 20, io="f32", compute="native", seed=1),
    "kron2-f32-n10": dict(kind=2, n=10, batch=1 << 20, io="f32", compute="native", seed=1),
    "kron3-f32-n16": dict(kind=3, n=16, batch=1 << 16, io="f32", compute="native", seed=2),
    "kron3-f32-n10": dict(kind=3, n=10, batch=1 << 18, io="f32", compute="native", seed=2),
    "kron2-f64-n16": dict(kind=2, n=16, batch=1 << 20, io="f64", compute="native", seed=1),
    "kron3-f64-n16": dict(kind=3, n=16, batch=1 << 16, io="f64", compute="native", seed=2),
    "kron2-bf16-n16": dict(kind=2, n=16, batch=1 << 20, io="bf16", compute="native", seed=4),
    "kron2-f16-n16": dict(kind=2, n=16, batch=1 << 20, io="f16", compute="native", seed=4),
    "kron2-bf16x3-n16": dict(kind=2, n=16, batch=1 << 20, io="f32", compute="bf16x3", seed=4),
    "kron3-bf16x3-n16": dict(kind=3, n=16, batch=1 << 16, io="f32", compute="bf16x3", seed=4),
    "kron2-bf16-bf16x3-n16": dict(kind=2, n=16, batch=1 << 20, io="bf16", compute="bf16x3", seed=4),
    "kron2-f16-bf16x3-n16": dict(kind=2, n=16, batch=1 << 20, io="f16", compute="bf16x3", seed=4),
    "kron2-bf16-bf16x3-n12": dict(kind=2, n=12, batch=1 << 20, io="bf16", compute="bf16x3", seed=4),
    "kron2-f16-bf16x3-n12": dict(kind=2, n=12, batch=1 << 20, io="f16", compute="bf16x3", seed=4),
    "kron3-bf16-bf16x3-n16": dict(kind=3, n=16, batch=1 << 16, io="bf16", compute="bf16x3", seed=4),
    "kron3-f16-bf16x3-n16": dict(kind=3, n=16, batch=1 << 16, io="f16", compute="bf16x3", seed=4),
    "kron3-bf16x3-n15": dict(kind=3, n=15, batch=1 << 16, io="f32", compute="bf16x3", seed=4),
    "kron2-bf16-n8": dict(kind=2, n=8, batch=1 << 20, io="bf16", compute="native", seed=4),
    "kron2-f16-n8": dict(kind=2, n=8, batch=1 << 20, io="f16", compute="native", seed=4),
    "kron2-bf16-bf16x3-n8": dict(kind=2, n=8, batch=1 << 20, io="bf16", compute="bf16x3", seed=4),
    "kron2-f16-bf16x3-n8": dict(kind=2, n=8, batch=1 << 20, io="f16", compute="bf16x3", seed=4),
    "kron2-bf16-n12": dict(kind=2, n=12, batch=1 << 20, io="bf16", compute="native", seed=4),
    "kron2-f16-n12": dict(kind=2, n=12, batch=1 << 20, io="f16", compute="native", seed=4),
    "kron2-bf16x3-n8": dict(kind=2, n=8, batch=1 << 20, io="f32", compute="bf16x3", seed=4),
    "kron2-bf16x3-n12": dict(kind=2, n=12, batch=1 << 20, io="f32", compute="bf16x3", seed=4),
    "kron3-bf16x3-n10": dict(kind=3, n=10, batch=1 << 18, io="f32", compute="bf16x3", seed=4),
    "kron3-bf16-n16": dict(kind=3, n=16, batch=1 << 16, io="bf16", compute="native", seed=4),
    "kron3-f64-n10": dict(kind=3, n=10, batch=1 << 18, io="f64", compute="native", seed=2),
    "kron2-f64-n10": dict(kind=2, n=10, batch=1 << 20, io="f64", compute="native", seed=1),
    # complex storage (the paper's complex field, Sec. 2), interleaved
    "kron2-c64-n16": dict(kind=2, n=16, batch=1 << 20, io="c64", compute="native", seed=6),
    "kron3-c64-n16": dict(kind=3, n=16, batch=1 << 15, io="c64", compute="native", seed=6),
    "kron2-c128-n16": dict(kind=2, n=16, batch=1 << 19, io="c128", compute="native", seed=6),
    # odd sizes (the mixed-size batch draws n from 4..16)
    "kron3-f32-n15": dict(kind=3, n=15, batch=1 << 16, io="f32", compute="native", seed=2),
    "kron2-f32-n15": dict(kind=2, n=15, batch=1 << 20, io="f32", compute="native", seed=1),
}
HEADLINE = "kron2-f32-n16"
ESIZE = {"f32": 4, "f64": 8, "bf16": 2, "f16": 2, "c64": 8, "c128": 16}
NP_DTYPE = {"f64": np.float64, "c64": np.complex64, "c128": np.complex128}


def flops_per_instance(kind, n, io="f32"):
    """The paper's count (Sec. 5): 4 n^3 (2-D) or 6 n^4 (3-D) real flops per
    instance.  A complex multiply-add is 8 real flops where a real one is 2, so
    complex storage counts four times as many."""
    f = 4 * n ** 3 if kind == 2 else 6 * n ** 4
    return 4 * f if io in ("c64", "c128") else f


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sustained=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), src="measured")
    return dict(hbm=FALLBACK_HBM_GBS, bf16=FALLBACK_BF16_TFLOPS, bf16_sustained=1700.0, src="fallback")


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t_on = self.t_off = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu=timestamp,{self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark_on(self):
        self.t_on = time.time()

    def mark_off(self):
        self.t_off = time.time()

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((t, parts))
        if not rows:
            return None
        inside = [r for t, r in rows if self.t_on is not None and self.t_on - 0.06 <= t <= (self.t_off or t) + 0.06]
        use = inside or [r for _, r in rows]
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in use if num(r[1]) is not None]
        mx = [num(r[2]) for r in use if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(inside),
                "power_w_max": max([num(r[3]) for r in use if num(r[3]) is not None] or [0])}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------
def rank_seed(seed, rank):
    """Each rank draws its own batch (weak scaling: the work per GPU is fixed)."""
    return seed + 1000 * rank


def reduce_time_max(ms, dist, device):
    """The step time of a multi-rank run is the slowest rank's (no data-path collective)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms):
    """Aggregate throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def make_inputs(wl, rank=0):
    from paper_1304_7054_gb300 import inputs
    b = inputs.make_batch(wl["kind"], wl["n"], wl["batch"], seed=rank_seed(wl["seed"], rank), x_dist="normal",
                          dtype=NP_DTYPE.get(wl["io"], np.float32))
    return b


def to_device_storage(b, io, torch, dev):
    from paper_1304_7054_gb300 import inputs
    if io in ("bf16", "f16"):
        return inputs.to_storage(b.X, io).to(dev)
    return torch.from_numpy(b.X).to(dev)


def call(kg, b, X, Y, compute):
    n = b.n
    if b.kind == 2:
        kg.kron2_batched(b.A, b.B, X, Y, ma=n, na=n, mb=n, nb=n, batch=b.batch, compute=compute)
    else:
        kg.kron3_batched(b.A, b.B, b.C, X, Y, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=b.batch,
                         compute=compute)


def sample_error(kg, b, Y, io, torch):
    """Max normalised error vs the FP64 oracle on 512 seeded instances."""
    import oracle
    from paper_1304_7054_gb300 import inputs
    inst = b.n ** b.kind
    rng = np.random.default_rng(17)
    idx = np.sort(rng.choice(b.batch, min(512, b.batch), replace=False))
    n = b.n
    cplx = io in ("c64", "c128")
    k2, k3 = (oracle.kron2c, oracle.kron3c) if cplx else (oracle.kron2, oracle.kron3)
    if io in ("bf16", "f16"):
        Xs = inputs.storage_to_f64(inputs.to_storage(b.X.reshape(b.batch, inst)[idx].ravel(), io))
    else:
        Xs = b.X.reshape(b.batch, inst)[idx].astype(np.complex128 if cplx else np.float64).ravel()
    if b.kind == 2:
        ref = k2(b.A, b.B, Xs, ma=n, na=n, mb=n, nb=n, batch=len(idx))
    else:
        ref = k3(b.A, b.B, b.C, Xs, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=len(idx))
    sel = Y.view(b.batch, inst)[torch.from_numpy(idx).to(Y.device)]
    got = sel.cpu().numpy().astype(np.complex128) if cplx else sel.double().cpu().numpy()
    cn = 1.0
    for M in b.comps():
        cn *= float(np.linalg.norm(np.asarray(M, np.complex128 if cplx else np.float64)))
    xn = np.linalg.norm(Xs.reshape(len(idx), inst), axis=1)
    d = np.abs(got - ref.reshape(len(idx), inst)).max(axis=1)
    return float((d / (cn * xn)).max())


def storage_report(b, Y, io, torch, compute="native", samples=256):
    """Accuracy of a 16-bit-storage result on seeded instances, against the FP64
    oracle, in both readings of the error:
      kernel: the oracle on the STORED operands.  A correct kernel computes each
              output in FP32 (error at most E = kind * gamma_n * (|K| |x|)_i,
              gamma_n = n u / (1 - n u), u = 2^-24; the split tensor path adds
              3 * 2^-16 per contraction) and rounds it once to the storage type.
              Reported: the fraction of outputs equal to the exact result rounded
              to the storage type, and the largest |Y - y| / (1/2 ulp(|y| + E) + E),
              which is <= 1 for a correct kernel.  (The FP32 value before the
              rounding never leaves the kernel.)
      end to end: the oracle on the original FP32 operands against the stored
              result, normalised like the FP32 error (by ||A|| ||B|| (||C||) ||X^p||).
    """
    import oracle
    from paper_1304_7054_gb300 import inputs
    inst, n = b.n ** b.kind, b.n
    rng = np.random.default_rng(19)
    idx = np.sort(rng.choice(b.batch, min(samples, b.batch), replace=False))
    X32 = b.X.reshape(b.batch, inst)[idx].ravel()
    Xs = inputs.storage_to_f64(inputs.to_storage(X32, io))

    def ref(X64, comps):
        if b.kind == 2:
            return oracle.kron2(comps[0], comps[1], X64, ma=n, na=n, mb=n, nb=n, batch=len(idx))
        return oracle.kron3(comps[0], comps[1], comps[2], X64, ma=n, na=n, mb=n, nb=n, mc=n, nc=n,
                            batch=len(idx))
    comps = [np.asarray(M, np.float64) for M in b.comps()]
    got = Y.view(b.batch, inst)[torch.from_numpy(idx).to(Y.device)].double().cpu().numpy().ravel()
    y = ref(Xs, comps)
    absref = ref(np.abs(Xs), [np.abs(M) for M in comps])
    u = 2.0 ** -24
    g = n * u / (1 - n * u)
    factor = b.kind * (3 * 2.0 ** -16 + 2 * g) if compute == "bf16x3" else 1.01 * b.kind * g
    E = factor * absref
    p, emin = (8, -126) if io == "bf16" else (11, -14)
    mag = np.abs(y) + E
    e = np.where(mag > 0, np.maximum(np.floor(np.log2(np.where(mag > 0, mag, 1.0))), emin), emin)
    allowed = 0.5 * np.ldexp(1.0, (e - (p - 1)).astype(np.int64)) + E
    rounded = inputs.storage_to_f64(inputs.to_storage(y.astype(np.float32), io))
    r_e2e = ref(X32.astype(np.float64), comps)
    cn = float(np.prod([np.linalg.norm(M) for M in comps]))
    xn = np.linalg.norm(X32.astype(np.float64).reshape(len(idx), inst), axis=1)
    e2e = float((np.abs(got - r_e2e).reshape(len(idx), inst).max(axis=1) / (cn * xn)).max())
    return {"instances": len(idx), "outputs_equal_to_rounded_exact": round(float(np.mean(got == rounded)), 6),
            "max_excess_over_rounding_bar": round(float((np.abs(got - y) / allowed).max()), 4),
            "end_to_end_max_norm_err_vs_fp32_operands": e2e}


def time_device(kg, b, X, Y, compute, steps, warmup, torch, sampler=None, dist=None):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        call(kg, b, X, Y, compute)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    if sampler:
        sampler.mark_on()
    t0.record(stream)
    for i in range(steps):
        ev[i][0].record(stream)
        call(kg, b, X, Y, compute)
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if sampler:
        sampler.mark_off()
    total_ms = t0.elapsed_time(t1)
    kern_ms = sum(a.elapsed_time(c) for a, c in ev) / steps
    return total_ms, kern_ms


def time_e2e(kg, b, io, compute, steps, warmup, torch, dev, chunks=16, nstreams=3):
    """Public API with host buffers: every step copies the pinned host operands to the
    device, runs the action and copies the results back to pinned host memory.  The
    batch is cut into `chunks` sub-batches issued round-robin on `nstreams` streams, so
    the copies of one chunk overlap the computation of another (each chunk is an
    ordinary kron2_batched / kron3_batched call on its stream)."""
    from paper_1304_7054_gb300 import inputs
    if io in ("bf16", "f16"):
        Xh = inputs.to_storage(b.X, io).pin_memory()
    else:
        Xh = torch.from_numpy(b.X).pin_memory()
    Xd = torch.empty_like(Xh, device=dev)
    Yd = torch.empty_like(Xd)
    Yh = torch.empty_like(Xh).pin_memory()
    inst = b.n ** b.kind
    streams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)]
    bounds = [round(c * b.batch / chunks) for c in range(chunks + 1)]
    main = torch.cuda.current_stream()

    def step():
        ev = torch.cuda.Event()
        ev.record(main)
        for c in range(chunks):
            s = streams[c % nstreams]
            s.wait_event(ev)
            lo, hi = bounds[c] * inst, bounds[c + 1] * inst
            with torch.cuda.stream(s):
                Xd[lo:hi].copy_(Xh[lo:hi], non_blocking=True)
                sub = inputs.Batch(b.kind, b.n, bounds[c + 1] - bounds[c], b.A, b.B, b.C, None)
                call(kg, sub, Xd[lo:hi], Yd[lo:hi], compute)
                Yh[lo:hi].copy_(Yd[lo:hi], non_blocking=True)
        for s in streams:
            done = torch.cuda.Event()
            done.record(s)
            main.wait_event(done)

    for _ in range(max(1, warmup)):
        step()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(main)
    for _ in range(steps):
        step()
    t1.record(main)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    nbytes = Xh.numel() * Xh.element_size()
    return ms, nbytes, nbytes


def cpu_baseline(b, seconds=8.0):
    """The FP32 oracle (sum-factorised loops, OpenMP over instances) on host cores,
    on a bounded sample of the same workload; returns GFlop/s."""
    import oracle
    oracle.build()
    n, inst = b.n, b.n ** b.kind
    f = flops_per_instance(b.kind, n)
    chunk = min(b.batch, max(64, int(2e8 // f)))
    done, t_used = 0, 0.0
    out = np.empty(chunk * inst, np.float32)
    while t_used < seconds and done + chunk <= b.batch:
        Xs = b.X[done * inst:(done + chunk) * inst]
        t = time.perf_counter()
        if b.kind == 2:
            oracle.kron2(b.A, b.B, Xs, ma=n, na=n, mb=n, nb=n, batch=chunk, precision="f32", Y=out)
        else:
            oracle.kron3(b.A, b.B, b.C, Xs, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=chunk, precision="f32",
                         Y=out)
        t_used += time.perf_counter() - t
        done += chunk
    gf = done * f / t_used / 1e9
    return {"value": round(gf, 3), "unit": "GFlop/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{done} of {b.batch} instances ({b.kind}-D n={n}, FP32 sum-factorised loops), "
                      f"{t_used:.1f} s"}


def measure_variant(kg, name, steps, warmup, torch, dev, peaks, tune=True):
    wl = WORKLOADS[name]
    b = make_inputs(wl)
    try:
        X = to_device_storage(b, wl["io"], torch, dev)
        Y = torch.empty_like(X)
        call(kg, b, X, Y, wl["compute"])
    except kg.KronError as e:
        return {"unavailable": str(e)}
    tile = None
    if tune:   # the library's autotuner picks body, tile, pipeline depth, fibers per step (untimed)
        tile = kg.autotune_config(b.kind, b.n, b.batch, X, Y, compute=wl["compute"])
    total_ms, kern_ms = time_device(kg, b, X, Y, wl["compute"], steps, warmup, torch)
    err = sample_error(kg, b, Y, wl["io"], torch)
    fl = flops_per_instance(b.kind, b.n, wl["io"]) * b.batch
    by = 2 * ESIZE[wl["io"]] * b.n ** b.kind * b.batch
    gbs = by / (kern_ms * 1e-3) / 1e9
    r = {"gflops": round(fl / (kern_ms * 1e-3) / 1e9, 1), "hbm_gbs": round(gbs, 1),
         "hbm_frac": round(gbs / peaks["hbm"], 4), "ms": round(kern_ms, 4), "batch": b.batch,
         "kernel": kernel_of(b.kind, b.n, wl["io"], wl["compute"], (tile or {}).get("variant", "auto"),
                             (tile or {}).get("compute_warps", 0)),
         "max_norm_err_vs_fp64_oracle": err,
         "tuned_config": tile}
    if wl["io"] in ("bf16", "f16"):
        r["storage_rounding"] = storage_report(b, Y, wl["io"], torch, wl["compute"])
    del X, Y
    torch.cuda.empty_cache()
    return r


ALU_ITERS = {"ffma2": 8192, "ffma": 8192, "dfma": 512}


def measure_alu_peaks(kg, torch, dev, repeats=5):
    """FMA throughput of the CUDA cores (the probe kernels of kron_peak_probe:
    independent FMA chains on every SM), best of `repeats` launches timed with
    CUDA events on the launching stream, with the SM clock sampled meanwhile."""
    stream = torch.cuda.current_stream()
    out = {}
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.2)
    sampler.mark_on()
    for unit, iters in ALU_ITERS.items():
        kg.peak_probe(unit, iters)   # warm-up
        best = None
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fl = kg.peak_probe(unit, iters)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
        out[unit] = {"tflops": round(fl / (best * 1e-3) / 1e12, 2), "ms": round(best, 4)}
    sampler.mark_off()
    clocks = sampler.stop()
    out["clocks"] = clocks
    out["how"] = ("kron_peak_probe: 8 independent FMA chains per thread, 32 FMA instructions per loop trip, "
                  "all resident CTAs on every SM; best of %d launches (CUDA events)" % repeats)
    return out


def _time_calls(fn, steps, warmup, torch):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for i in range(steps):
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(c) for a, c in ev) / steps


def measure_interfaces(kg, steps, warmup, torch, dev, peaks):
    """The paper's other two interfaces (Sec. 3) and its unfused 3-D algorithm
    (Algorithm 1: the 2-D product on every plane into tmp in HBM, then TGEMM_A
    for the third mode), next to the fused 3-D kernel.  FP32, inputs > L2."""
    import oracle
    out = {}
    rng = np.random.default_rng(21)

    def line(ms, fl, by, kernel, err, extra=None):
        gbs = by / (ms * 1e-3) / 1e9
        r = {"gflops": round(fl / (ms * 1e-3) / 1e9, 1), "hbm_gbs": round(gbs, 1),
             "hbm_frac": round(gbs / peaks["hbm"], 4), "ms": round(ms, 4), "kernel": kernel,
             "max_norm_err_vs_fp64_oracle": err}
        r.update(extra or {})
        return r

    # TGEMM_A at the shape Algorithm 1 gives it for n = 16: m = n^2, k = n = 16
    m, n, k, batch = 256, 16, 16, 1 << 16
    A = torch.randn(batch * m * k, device=dev)
    B = rng.uniform(-1, 1, (k, n)).astype(np.float32)
    C = torch.empty(batch * m * n, device=dev)
    ms = _time_calls(lambda: kg.gemm_a_batched(A, B, C, m=m, n=n, k=k, batch=batch), steps, warmup, torch)
    idx = np.sort(rng.choice(batch, 128, replace=False))
    As = A.view(batch, -1)[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
    ref = oracle.gemm_a(As.ravel(), np.ascontiguousarray(B.T).ravel().astype(np.float64), m=m, n=n, k=k,
                        batch=len(idx))
    got = C.view(batch, -1)[torch.from_numpy(idx).to(dev)].double().cpu().numpy().ravel()
    err = float((np.abs(got - ref).reshape(len(idx), -1).max(axis=1) /
                 (np.linalg.norm(As, axis=1) * np.linalg.norm(B))).max())
    out["tgemm_a-f32-m256-n16-k16"] = line(ms, 2.0 * m * n * k * batch, 4.0 * (m * k + m * n) * batch,
                                           "gemm_a_tma_kernel<f32,n=16>", err, {"batch": batch})
    del A, C

    # TKRON1, n = 16
    nn, batch = 16, 1 << 24
    A1 = rng.uniform(-1, 1, (nn, nn)).astype(np.float32)
    X = torch.randn(batch * nn, device=dev)
    Y = torch.empty_like(X)
    ms = _time_calls(lambda: kg.kron1_batched(A1, X, Y, ma=nn, na=nn, batch=batch), steps, warmup, torch)
    idx = np.sort(rng.choice(batch, 1024, replace=False))
    Xs = X.view(batch, -1)[torch.from_numpy(idx).to(dev)].double().cpu().numpy()
    ref = oracle.kron1(np.ascontiguousarray(A1.T).ravel().astype(np.float64), Xs.ravel(), ma=nn, na=nn,
                       batch=len(idx))
    got = Y.view(batch, -1)[torch.from_numpy(idx).to(dev)].double().cpu().numpy().ravel()
    err = float((np.abs(got - ref).reshape(len(idx), -1).max(axis=1) /
                 (np.linalg.norm(Xs, axis=1) * np.linalg.norm(A1))).max())
    out["tkron1-f32-n16"] = line(ms, 2.0 * nn * nn * batch, 8.0 * nn * batch, "kron1t_kernel<f32,n=16>",
                                 err, {"batch": batch})
    del X, Y

    # Algorithm 1 (unfused 3-D) next to the fused kernel, same data
    for n3, batch in ((16, 1 << 16), (10, 1 << 18)):
        from paper_1304_7054_gb300 import inputs
        b = inputs.make_batch(3, n3, batch, seed=3, x_dist="normal", dtype=np.float32)
        X = torch.from_numpy(b.X).to(dev)
        tmp = torch.empty_like(X)
        Y = torch.empty_like(X)

        def unfused():
            kg.kron2_batched(b.B, b.C, X, tmp, ma=n3, na=n3, mb=n3, nb=n3, batch=batch * n3)
            kg.gemm_a_batched(tmp, b.A, Y, m=n3 * n3, n=n3, k=n3, batch=batch, transb="T", lda=n3 * n3,
                              lda2=n3 ** 3, ldc=n3 * n3, ldc2=n3 ** 3)
        ms_u = _time_calls(unfused, steps, warmup, torch)
        err = sample_error(kg, b, Y, "f32", torch)
        ms_f = _time_calls(lambda: call(kg, b, X, Y, "native"), steps, warmup, torch)
        fl = flops_per_instance(3, n3) * batch
        by = 2 * 4 * n3 ** 3 * batch
        out[f"kron3-f32-n{n3}-unfused-algorithm1"] = line(
            ms_u, fl, by, "pair2ip/pair16/pair_kernel (2-D on planes) + gemm_a_kernel", err,
            {"batch": batch, "hbm_bytes_moved": 2 * by, "hbm_gbs_moved": round(2 * by / (ms_u * 1e-3) / 1e9, 1),
             "fused_kernel_ms": round(ms_f, 4), "unfused_over_fused_time": round(ms_u / ms_f, 3)})
        del X, tmp, Y
    torch.cuda.empty_cache()
    return out


def kernel_of(kind, n, io, compute, variant="auto", warps=0):
    """Name of the kernel the library dispatches a contiguous batch to (with the
    kernel body and compute warps the tuning table holds for it)."""
    if compute == "bf16x3":
        if kind == 3 and (warps > 1 or (warps == 0 and (
                (n >= 14 and not (io == "f16" and n != 16)) or (io == "f32" and n >= 10 and n % 2 == 0)))):
            return f"tc3g_kernel<n={n},{io}>"   # several warps share an instance
        if kind == 2 and (variant == "exchange" or (
                variant == "auto" and n >= 10 and n % 2 == 0 and not (n == 16 and io == "f32"))):
            return f"tc2s_kernel<n={n},{io}>"   # instances stacked along the MMA's N dimension
        return f"tc{kind}_kernel<n={n},{io}>"
    if io in ("c64", "c128") or variant == "scalar":
        return f"fiber_kernel<{io},n={n},{kind}-D>"
    if variant == "exchange":
        return f"pair_kernel<{io},n={n},{kind}-D>"
    if kind == 2 and n == 16 and io == "f32":
        return "pair16t_kernel<f32,n=16,2-D>"
    if kind == 2 and n == 16 and io in ("bf16", "f16"):
        return f"pair16h_kernel<{io},n=16,2-D>"
    if kind == 2 and n in (10, 14) and io == "f32":
        return f"pair2ip_kernel<f32,n={n},2-D>"
    if kind == 3 and n == 16 and io == "f32":
        return "pair3ip_kernel<f32,n=16,3-D>"
    if kind == 3 and n in (10, 14) and io == "f32":
        return f"pair3pk_kernel<f32,n={n},3-D>"
    if n % 2 == 1 and n >= 3 and io == "f32":
        return f"fiberip_kernel<f32,n={n},{kind}-D>"
    if io != "f64" and n % 2 == 0:
        return f"pair_kernel<{io},n={n},{kind}-D>"
    return f"fiber_kernel<{io},n={n},{kind}-D>"


def varlen_stats(v, io):
    fl = sum(4 * n ** 3 if k == 2 else 6 * n ** 4 for k, n in (v.classes[c] for c in v.class_of))
    by = 2 * ESIZE[io] * v.total
    return fl, by


def measure_varlen(kg, io, steps, warmup, torch, dev, peaks, count=200000, seed=5):
    """Mixed-size batch (n ~ U{4..16}, 2-D/3-D 50/50): one graph launch, tuned tiles;
    next to it, the same instances as 26 per-size plain launches (one per class)."""
    from paper_1304_7054_gb300 import inputs
    v = inputs.make_varlen(count, seed=seed)
    X = (torch.from_numpy(v.X) if io == "f32" else inputs.to_storage(v.X, io)).to(dev)
    Y = torch.empty_like(X)
    classes = [(k, n, *cs) for (k, n), cs in zip(v.classes, v.comps)]
    plan = kg.VarlenPlan(classes, v.class_of, v.x_off, v.y_off, io=io)
    ws = plan.alloc_workspace(dev)
    plan.execute(X, Y, ws)
    plan.tune(X, Y, ws)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        plan.execute(X, Y, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        plan.execute(X, Y, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    fl, by = varlen_stats(v, io)
    # error on a seeded sample against the FP64 oracle
    import oracle
    rng = np.random.default_rng(8)
    idx = np.sort(rng.choice(count, 512, replace=False))
    Yh = Y.double().cpu().numpy()
    Xh = X.double().cpu().numpy()
    err = 0.0
    for p in idx:
        k, n = v.classes[v.class_of[p]]
        cs = v.comps[v.class_of[p]]
        nx = n ** k
        xp = Xh[v.x_off[p]:v.x_off[p] + nx]
        if k == 2:
            r = oracle.kron2(cs[0], cs[1], xp, ma=n, na=n, mb=n, nb=n, batch=1)
        else:
            r = oracle.kron3(cs[0], cs[1], cs[2], xp, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=1)
        nrm = np.prod([np.linalg.norm(np.asarray(M, np.float64)) for M in cs]) * np.linalg.norm(xp)
        err = max(err, float(np.abs(Yh[v.y_off[p]:v.y_off[p] + nx] - r).max() / nrm))
    # per-size plain launches on class-contiguous copies of the same instances
    groups = []
    for c, (k, n) in enumerate(v.classes):
        sel = np.nonzero(v.class_of == c)[0]
        if len(sel):
            nx = n ** k
            gx = np.concatenate([v.X[v.x_off[p]:v.x_off[p] + nx] for p in sel])
            gX = (torch.from_numpy(gx) if io == "f32" else inputs.to_storage(gx, io)).to(dev)
            groups.append((k, n, v.comps[c], gX, torch.empty_like(gX), len(sel)))

    groups.sort(key=lambda g: -g[3].numel())   # largest classes first
    side = [torch.cuda.Stream(device=dev) for _ in range(4)]

    def per_size(nstreams=1):
        if nstreams > 1:
            ev = torch.cuda.Event()
            ev.record(stream)
            for sd in side[:nstreams]:
                sd.wait_event(ev)
        for i, (k, n, cs, gX, gY, cnt) in enumerate(groups):
            st = side[i % nstreams] if nstreams > 1 else None
            if k == 2:
                kg.kron2_batched(cs[0], cs[1], gX, gY, ma=n, na=n, mb=n, nb=n, batch=cnt, stream=st)
            else:
                kg.kron3_batched(cs[0], cs[1], cs[2], gX, gY, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=cnt,
                                 stream=st)
        if nstreams > 1:
            for sd in side[:nstreams]:
                done = torch.cuda.Event()
                done.record(sd)
                stream.wait_event(done)

    ms_ps = {}
    try:
        for ns in (1, 4):
            for _ in range(warmup):
                per_size(ns)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                per_size(ns)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_ps[ns] = e0.elapsed_time(e1) / steps
    except kg.KronError as e:
        ms_ps = {1: float("nan"), 4: float("nan")}
        print(f"per-size launches failed: {e}", file=sys.stderr)
    plan.close()
    gbs = by / (ms * 1e-3) / 1e9
    return {"gflops": round(fl / (ms * 1e-3) / 1e9, 1), "hbm_gbs": round(gbs, 1),
            "hbm_frac": round(gbs / peaks["hbm"], 4), "ms": round(ms, 4), "instances": count,
            "launches_per_step": 1, "max_norm_err_vs_fp64_oracle": err,
            "per_size_plain_launches": {"launches_per_step": len(groups), "ms": round(ms_ps[1], 4),
                                        "gflops": round(fl / (ms_ps[1] * 1e-3) / 1e9, 1),
                                        "data": "class-contiguous copies made before timing"},
            "per_size_plain_launches_4_streams": {"ms": round(ms_ps[4], 4),
                                                  "gflops": round(fl / (ms_ps[4] * 1e-3) / 1e9, 1)}}


def traffic_for(kernel_name):
    """DRAM bytes per launch from a committed ncu summary, if the kernel sources are unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(kernel_name)
    if not e:
        return None
    from paper_1304_7054_gb300 import build as lb
    if e.get("source_hash") != lb.source_hash(kernel_name.split("<")[0]):
        return None
    return e.get("dram_bytes_per_launch")


def run_ours(args):
    import torch
    import paper_1304_7054_gb300 as kg
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    torch.cuda.set_device(dev)
    kg.load_library()
    peaks = load_peaks()
    wl = WORKLOADS[args.workload]
    b = make_inputs(wl, rank)
    X = to_device_storage(b, wl["io"], torch, dev)
    Y = torch.empty_like(X)
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    total_ms, kern_ms = time_device(kg, b, X, Y, wl["compute"], args.steps, args.warmup, torch, sampler, dist)
    clocks = sampler.stop() if sampler else None
    total_ms = reduce_time_max(total_ms, dist, dev)
    err = sample_error(kg, b, Y, wl["io"], torch)
    ms = total_ms / args.steps
    fl = flops_per_instance(b.kind, b.n, wl["io"]) * b.batch
    by = 2 * ESIZE[wl["io"]] * b.n ** b.kind * b.batch
    value = whole_job_rate(world, fl, ms) / 1e9
    kernel_name = kernel_of(b.kind, b.n, wl["io"], wl["compute"])
    achieved = by / (kern_ms * 1e-3) / 1e9
    del X, Y
    torch.cuda.empty_cache()
    e2e_ms, h2d, d2h = time_e2e(kg, b, wl["io"], wl["compute"], max(3, min(args.steps, 20)), 2, torch, dev)
    out = None
    if rank == 0:
        variants = {}
        alu = measure_alu_peaks(kg, torch, dev)
        if not args.no_variants:
            for name in WORKLOADS:
                if name != args.workload:
                    variants[name] = measure_variant(kg, name, max(5, min(args.steps, 30)), 3, torch, dev, peaks)
            for io in ("f32", "bf16"):
                variants[f"varlen-{io}"] = measure_varlen(kg, io, max(5, min(args.steps, 30)), 3, torch, dev,
                                                          peaks)
            variants.update(measure_interfaces(kg, max(5, min(args.steps, 30)), 3, torch, dev, peaks))
        # share of the measured FMA throughput that the CUDA-core variants use
        for name, r in variants.items():
            w = WORKLOADS.get(name)
            if w and "gflops" in r and w["compute"] == "native":
                unit = {"f64": "dfma", "c128": "dfma"}.get(w["io"], "ffma2")
                r["of_measured_fma_peak"] = round(r["gflops"] / (alu[unit]["tflops"] * 1e3), 4)
        cpu = cpu_baseline(b, seconds=args.cpu_seconds)
        out = {
            "metric": METRIC, "value": round(value, 1), "unit": "GFlop/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": wl["io"], "data": "synthetic (seeded PCG64: A,B ~ U[-1,1], X ~ N(0,1))",
            "config": {"workload": f"{b.kind}-D batched Kronecker action, n={b.n}, batch={b.batch}, "
                                   f"{wl['io']} storage, {wl['compute']} compute",
                       "kind": b.kind, "n": b.n, "batch_per_gpu": b.batch, "alpha": 1.0, "beta": 0.0,
                       "layout": "contiguous column-major, minimal leading dimensions",
                       "l2": "inputs larger than L2 (no flush)",
                       "paper_k20c_gflops_context": 285 if (b.kind, b.n, wl["io"]) == (2, 16, "f32") else None},
            "hbm_gbs": round(world * by / (ms * 1e-3) / 1e9, 1),
            "max_norm_err_vs_fp64_oracle": err,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm"], "unit": "GB/s",
                         "frac": round(achieved / peaks["hbm"], 4), "traffic": traffic_for(kernel_name),
                         "kernel": kernel_name, "peak_source": peaks["src"],
                         "algorithmic_bytes_per_launch": by},
            "cpu_baseline": cpu,
            "e2e": {"value": round(world * fl / (e2e_ms * 1e-3) / 1e9, 1), "unit": "GFlop/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 4),
                    "how": "pinned host X -> device, the call, device -> pinned host Y, every step; "
                           "16 sub-batch calls on 3 streams overlap copies with compute"},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "alu_peaks_measured": alu,
            "variants": variants,
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return out


def run_profile(args):
    """Warm-up and timed steps of one workload only (the command profiled with ncu)."""
    import torch
    import paper_1304_7054_gb300 as kg
    dev = torch.device("cuda", torch.cuda.current_device())
    kg.load_library()
    if args.workload.startswith("varlen-"):
        from paper_1304_7054_gb300 import inputs
        io = args.workload.split("-", 1)[1]
        v = inputs.make_varlen(args.batch or 200000, seed=5)
        X = (torch.from_numpy(v.X) if io == "f32" else inputs.to_storage(v.X, io)).to(dev)
        Y = torch.empty_like(X)
        plan = kg.VarlenPlan([(k, n, *cs) for (k, n), cs in zip(v.classes, v.comps)], v.class_of, v.x_off,
                             v.y_off, io=io)
        ws = plan.alloc_workspace(dev)
        for _ in range(args.warmup):
            plan.execute(X, Y, ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            plan.execute(X, Y, ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        fl, by = varlen_stats(v, io)
        print(json.dumps({"workload": args.workload, "instances": len(v.class_of), "kernel_ms": ms,
                          "gflops": fl / (ms * 1e-3) / 1e9, "hbm_gbs": by / (ms * 1e-3) / 1e9}))
        plan.close()
        return
    if args.workload in ("tkron1-f32-n16", "tgemm_a-f32-m256-n16-k16"):
        rng = np.random.default_rng(21)
        if args.workload == "tkron1-f32-n16":
            batch = args.batch or (1 << 24)
            A1 = rng.uniform(-1, 1, (16, 16)).astype(np.float32)
            X = torch.randn(batch * 16, device=dev)
            Y = torch.empty_like(X)
            fn = lambda: kg.kron1_batched(A1, X, Y, ma=16, na=16, batch=batch)
            fl, by = 2.0 * 256 * batch, 8.0 * 16 * batch
        else:
            batch = args.batch or (1 << 16)
            A = torch.randn(batch * 256 * 16, device=dev)
            B = rng.uniform(-1, 1, (16, 16)).astype(np.float32)
            C = torch.empty_like(A)
            fn = lambda: kg.gemm_a_batched(A, B, C, m=256, n=16, k=16, batch=batch)
            fl, by = 2.0 * 256 * 16 * 16 * batch, 4.0 * 2 * 256 * 16 * batch
        kern_ms = _time_calls(fn, args.steps, args.warmup, torch)
        print(json.dumps({"workload": args.workload, "batch": batch, "kernel_ms": kern_ms,
                          "gflops": fl / (kern_ms * 1e-3) / 1e9, "hbm_gbs": by / (kern_ms * 1e-3) / 1e9}))
        return
    wl = WORKLOADS[args.workload]
    b = make_inputs(wl)
    X = to_device_storage(b, wl["io"], torch, dev)
    Y = torch.empty_like(X)
    total_ms, kern_ms = time_device(kg, b, X, Y, wl["compute"], args.steps, args.warmup, torch)
    fl = flops_per_instance(b.kind, b.n, wl["io"]) * b.batch
    by = 2 * ESIZE[wl["io"]] * b.n ** b.kind * b.batch
    print(json.dumps({"workload": args.workload, "batch": b.batch, "kernel_ms": kern_ms,
                      "gflops": fl / (kern_ms * 1e-3) / 1e9, "hbm_gbs": by / (kern_ms * 1e-3) / 1e9}))


def run_reference(args):
    """The oracle, as it stands, on the host cores (the reference arm of this benchmark)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    oracle.build()
    wl = WORKLOADS[args.workload]
    b = make_inputs(wl)
    n, inst = b.n, b.n ** b.kind
    f = flops_per_instance(b.kind, n)
    # a bounded sample per step, sized so that warm-up + timed steps take about a minute
    probe = min(b.batch, max(16, int(2e8 // f)))
    t = time.perf_counter()
    pout = np.empty(probe * inst, np.float32)
    if b.kind == 2:
        oracle.kron2(b.A, b.B, b.X[:probe * inst], ma=n, na=n, mb=n, nb=n, batch=probe, precision="f32", Y=pout)
    else:
        oracle.kron3(b.A, b.B, b.C, b.X[:probe * inst], ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=probe,
                     precision="f32", Y=pout)
    rate = probe / max(1e-6, time.perf_counter() - t)          # instances per second
    per_step = int(max(1, min(b.batch // 2 or 1, rate * 60.0 / (args.steps + args.warmup))))
    out = np.empty(per_step * inst, np.float32)

    def step(i):
        o = (i * per_step) % max(1, b.batch - per_step)
        Xs = b.X[o * inst:(o + per_step) * inst]
        if b.kind == 2:
            oracle.kron2(b.A, b.B, Xs, ma=n, na=n, mb=n, nb=n, batch=per_step, precision="f32", Y=out)
        else:
            oracle.kron3(b.A, b.B, b.C, Xs, ma=n, na=n, mb=n, nb=n, mc=n, nc=n, batch=per_step,
                         precision="f32", Y=out)

    for i in range(args.warmup):
        step(i)
    t = time.perf_counter()
    for i in range(args.steps):
        step(i)
    dt = (time.perf_counter() - t) / args.steps
    value = per_step * f / dt / 1e9
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GFlop/s",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": wl["io"], "data": "synthetic (seeded PCG64: A,B ~ U[-1,1], X ~ N(0,1))",
        "config": {"workload": f"{b.kind}-D batched Kronecker action, n={b.n}, batch={b.batch}, "
                               f"{wl['io']} storage", "kind": b.kind, "n": b.n, "batch_per_gpu": b.batch},
        "cpu_baseline": {"value": round(value, 3), "unit": "GFlop/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} instances per step of the {b.batch}-instance batch"},
        "e2e": {"value": round(value, 3), "unit": "GFlop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["varlen-f32", "varlen-bf16", "tkron1-f32-n16",
                                                               "tgemm_a-f32-m256-n16-k16"], default=HEADLINE)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--batch", type=int, default=0, help="override the batch (profiling a smaller case)")
    ap.add_argument("--profile", action="store_true",
                    help="only warm-up + timed steps of the workload, no extra legs (for ncu captures)")
    args = ap.parse_args()
    if args.workload not in WORKLOADS and not args.profile:
        ap.error(f"--workload {args.workload} is measured as a variant of the default run; alone it needs --profile")
    if args.warmup < 3:
        args.warmup = 3
    if args.batch:
        for wl in WORKLOADS.values():
            wl["batch"] = args.batch
    if args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
