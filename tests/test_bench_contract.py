"""bench.py on the CPU: the reference arm (the oracle timed on the host cores)
prints one JSON line with the keys of the benchmark contract, and the helpers
behind the GPU arm's line behave: the harmonic mean of per-root rates, and
the ncu traffic of a committed profile, which counts only while the kernel
sources still hash to the value recorded with it."""
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "rmat16",
                        "--steps", "2", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["unit"] == "GTEPS" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert "scale 16" in d["config"]["workload"] and d["config"]["n"] == 1 << 16
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_harmonic_mean_of_rates():
    # two roots: 1e9 edges in 1 s and 1e9 edges in 0.5 s -> 1 and 2 GTEPS -> harmonic mean 4/3
    assert bench.harmonic_gteps([1e9, 1e9], [1.0, 0.5]) == pytest.approx(4.0 / 3.0)
    assert bench.harmonic_gteps([5e8] * 4, [0.25] * 4) == pytest.approx(2.0)
    assert bench.harmonic_gteps([], []) == 0.0


def test_profile_traffic_counts_only_for_the_recorded_kernel_source(monkeypatch):
    name = "level_loop_rmat23.md"
    text = open(os.path.join(ROOT, "profiles", name)).read()
    recorded = [ln.split("`")[1] for ln in text.splitlines() if ln.startswith("- source_sha256:")][0]
    traffic = float([ln.split(":")[1] for ln in text.splitlines() if ln.startswith("- traffic_bytes_per_launch:")][0])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: recorded)
    assert bench.profile_traffic(name) == traffic
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.profile_traffic(name) is None
    assert bench.profile_traffic("no_such_profile.md") is None


def test_reference_arm_under_torchrun_prints_once():
    """Launched like the multi-GPU bench (torchrun, 2 ranks): rank 0 alone times the
    oracle and prints; the other rank exits 0 without work."""
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", "29517", os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--workload", "rmat16", "--steps", "1", "--warmup", "3", "--gpus", "2"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_traffic_of_a_larger_workload_is_scaled_from_the_small_capture(monkeypatch):
    """A workload without its own capture takes the scale-23 capture's traffic times the
    ratio of algorithmic bytes per launch; a stale capture gives no traffic."""
    kv = bench.profile_summary(bench.SCALED_CAPTURE)
    t23, a23 = float(kv["traffic_bytes_per_launch"]), float(kv["algorithmic_bytes_per_launch"])
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: kv["source_sha256"])
    t, how = bench.traffic_estimate("rmat26", 8 * a23)
    assert t == pytest.approx(8 * t23) and "scaled" in how
    t, how = bench.traffic_estimate("rmat23", a23)
    assert t == pytest.approx(t23) and "this workload" in how
    assert bench.traffic_estimate("grid128", 1e9)[0] is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.traffic_estimate("rmat26", 8 * a23)[0] is None
