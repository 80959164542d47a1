"""Host-side helpers of bench.py (no GPU): the leaf-flop count behind the roofline, the lookup of
a profile's DRAM traffic (only for the kernel source it was captured on), the reduction of the
clock record taken during the timed region, and the config both bench arms share."""
import hashlib
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("n", [256, 4096, 8192])
@pytest.mark.parametrize("L", [0, 1, 2, 3])
def test_leaf_flops_is_seven_eighths_per_level(n, L):
    # 7^L leaves of (n / 2^L)^3 multiply-adds: 2 n^3 (7/8)^L
    assert bench.leaf_flops(n, L) == pytest.approx(2.0 * n ** 3 * (7 / 8) ** L, rel=1e-15)


def test_traffic_is_read_only_for_the_profiled_kernel_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    csrc = tmp_path / "paper_2309_00628_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_bytes(b"kernel v1")
    sha = hashlib.sha1(b"kernel v1").hexdigest()[:12]
    (tmp_path / "profiles" / "w.md").write_text(f"kernel_source_sha1: {sha}\ndram_bytes_per_launch: 2.5e9\n")
    assert bench.traffic_from_profiles("k.cu", "w") == 2.5e9
    (csrc / "k.cu").write_bytes(b"kernel v2")  # the kernel changed since the capture: no traffic
    assert bench.traffic_from_profiles("k.cu", "w") is None
    assert bench.traffic_from_profiles("k.cu", "missing") is None


def test_clock_record_reduction(tmp_path):
    # nvidia-smi rows: index, sm clock, max sm clock, power, reasons mask, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    p = tmp_path / "clocks.csv"
    p.write_text("0, 2070, 2070, 900.5, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 1900, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 2000, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "not a record\n")
    s = bench.ClockSampler(0)
    s.path = str(p)
    s.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: None, kill=lambda: None)
    assert s.stop() == {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not p.exists()


def test_both_arms_share_the_workload_config():
    args = types.SimpleNamespace(n=8192, algo="winograd", sched="fused")
    c = bench.workload_config(args, 1)
    assert c["n"] == 8192 and c["depth"] == 1 and c["algo"] == "winograd" and c["schedule"] == "fused"
    assert "n=8192" in c["workload"] and "L=1" in c["workload"]


def test_serving_latency_summaries():
    import bench
    assert bench.size_class(512, 512, 512) == bench.SIZE_CLASSES[0]
    assert bench.size_class(2048, 2048, 2048) == bench.SIZE_CLASSES[1]
    assert bench.size_class(8192, 1024, 8192) == bench.SIZE_CLASSES[2]
    s = bench.latency_summary([0.004, 0.001, 0.002, 0.003])
    assert s["requests"] == 4 and s["p50_ms"] == 2.5 and s["p99_ms"] == 4.0
    assert bench.latency_summary([])["p50_ms"] is None


def test_reference_arm_line_and_other_ranks():
    # the reference arm times the FP64 oracle on the host's cores and prints the contract's line
    # (a small n keeps it quick); under torchrun, ranks other than 0 exit 0 without a line
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--n", "512", "--steps", "1",
           "--warmup", "3", "--cpu-seconds", "0.1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    r1 = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=root, env=dict(os.environ, RANK="1"))
    assert r1.returncode == 0 and not [x for x in r1.stdout.splitlines() if x.startswith("{")]
