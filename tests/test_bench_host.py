"""The benchmark's host-side legs on CPU: the reference arm (the oracle timed on
the host cores) prints one well-formed JSON line."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3", "--warmup", "3",
                        "--batch", "4096"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GFlop/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["higher_is_better"] is True and line["steps"] == 3


def test_kernel_names_follow_dispatch():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.kernel_of(2, 16, "f32", "native").startswith("pair16t_kernel")
    assert bench.kernel_of(2, 16, "f32", "bf16x3").startswith("tc2_kernel")
    assert bench.kernel_of(2, 12, "bf16", "bf16x3").startswith("tc2s_kernel")
    assert bench.kernel_of(2, 12, "bf16", "bf16x3", "in_place").startswith("tc2_kernel")
    assert bench.kernel_of(2, 13, "f16", "bf16x3").startswith("tc2_kernel")
    assert bench.kernel_of(2, 16, "bf16", "bf16x3").startswith("tc2s_kernel")
    assert bench.kernel_of(2, 16, "bf16", "bf16x3", "in_place").startswith("tc2_kernel")
    assert bench.kernel_of(2, 14, "f32", "bf16x3").startswith("tc2s_kernel")
    assert bench.kernel_of(2, 16, "bf16", "native").startswith("pair16h_kernel")
    assert bench.kernel_of(2, 10, "f32", "native").startswith("pair2ip_kernel")
    assert bench.kernel_of(2, 12, "f32", "native").startswith("pair_kernel")
    assert bench.kernel_of(2, 12, "bf16", "native").startswith("pair_kernel")
    assert bench.kernel_of(3, 15, "f32", "native").startswith("fiberip_kernel")
    assert bench.kernel_of(2, 15, "f32", "native").startswith("fiberip_kernel")
    assert bench.kernel_of(2, 15, "f64", "native").startswith("fiber_kernel")
    assert bench.kernel_of(3, 16, "f32", "native").startswith("pair3ip_kernel")
    assert bench.kernel_of(3, 10, "f32", "native").startswith("pair3pk_kernel")
    assert bench.kernel_of(2, 16, "f64", "native").startswith("fiber_kernel")
    assert bench.kernel_of(3, 16, "f32", "bf16x3").startswith("tc3g_kernel")
    assert bench.kernel_of(3, 10, "f32", "bf16x3").startswith("tc3g_kernel")
    assert bench.kernel_of(3, 10, "bf16", "bf16x3").startswith("tc3_kernel")
    assert bench.kernel_of(3, 10, "f32", "bf16x3", "auto", 4).startswith("tc3g_kernel")
    assert bench.kernel_of(3, 16, "f32", "bf16x3", "auto", 1).startswith("tc3_kernel")
    assert bench.kernel_of(3, 15, "f16", "bf16x3").startswith("tc3_kernel")
