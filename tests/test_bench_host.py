"""bench.py's host arithmetic, on the CPU: the roofline fields of the JSON line
follow from the numbers in it.

The work per row is counted from the network's layer shapes (multiply-adds of
one back-substitution row through every affine layer below the objective),
the achieved rate is algorithmic flops over the class's summed event time,
the 3xTF32 peak is the measured TF32 rate / 3, and an HBM-bound class is
measured in bytes against the copy bandwidth.
"""
import pytest

import bench
import synth


def test_chain_macs_of_the_bench_network():
    """conv16 4x4 s2 on 1x28x28 -> 16x13x13 (16 MACs per output), conv32 4x4 s2
    -> 32x5x5 (256 MACs per output), FC 800 -> 100; the last ReLU layer is 100 wide."""
    C, dR = bench.chain_macs(synth.make_network(1))
    assert C == 16 * 13 * 13 * 16 + 32 * 5 * 5 * 16 * 16 + 800 * 100
    assert dR == 100


def test_roofline_fields_follow_from_the_stats():
    layers = synth.make_network(1)
    stats = {"opt_fused_chain_tc": {"launches": 8, "ms": 17.6, "flops": 9.5e10, "bytes": 1e9},
             "acs": {"launches": 8, "ms": 0.2, "flops": 0.0, "bytes": 4e8},
             "step_optimize_wall": {"launches": 0, "ms": 99.0, "flops": 0.0, "bytes": 0.0}}
    peaks = {"tf32_tflops": 1063.5, "hbm_gbs": 6756.5, "bf16_tflops": 1945.8,
             "sm_max_mhz": 2070.0}
    r = bench.roofline(stats, peaks, "measured", None, layers=layers)
    # phase timers are not kernels; the largest kernel class is the fused loop
    assert r["kernel"] == "opt_fused_chain_tc" and r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(9.5e10 / 17.6e-3 / 1e12)
    assert r["peak"] == pytest.approx(1063.5 / 3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["avg_launch_us"] == pytest.approx(17.6 / 8 * 1e3)
    assert r["simt_fp32"]["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    # the three-sweep count per row (a sweep plus a two-sweep adjoint per Adam
    # step) against the library's ((steps + 1) sweeps with the objective row,
    # steps adjoints)
    C, dR = bench.chain_macs(layers)
    ours, three = 21 * (C + dR) + 20 * C, 3 * 20 * C
    assert r["three_sweep_count"]["achieved"] == pytest.approx(r["achieved"] * three / ours)
    assert r["three_sweep_count"]["flops_per_row"] == 2 * three
    assert r["three_sweep_count"]["library_flops_per_row"] == 2 * ours


def test_hbm_bound_class_and_derived_peak():
    peaks = {"hbm_gbs": 6756.5, "bf16_tflops": 1945.8, "sm_max_mhz": 2070.0}
    r = bench.roofline({"acs": {"launches": 4, "ms": 0.2, "flops": 0.0, "bytes": 4e8}}, peaks,
                       "measured", None)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(4e8 / 0.2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6756.5)
    # without a measured TF32 rate the 3xTF32 peak is BF16 x 1/2 / 3
    p, src = bench.tf32x3_peak(peaks, "measured")
    assert p == pytest.approx(1945.8 / 2 / 3) and "derived" in src


def test_reference_arm_line():
    """--impl reference times the FP64 oracle on the host cores (no GPU) and
    prints one JSON line with the same metric and unit, impl "reference", a
    cpu_baseline block and an e2e block without host-device copies; under a
    multi-process launch only rank 0 prints."""
    import json
    import os
    import subprocess
    import sys
    cmd = [sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
           "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.5"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "nodes/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "nodes/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    other = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env)
    assert other.returncode == 0 and other.stdout.strip() == ""
