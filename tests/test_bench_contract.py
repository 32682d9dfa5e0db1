"""bench.py on the CPU: the reference arm (the FP64 oracle timed on the host
cores, a measured bounded sample per step and its extrapolation to the
whole step) prints one JSON line with the keys and units of the GPU arm's line,
and the GPU arm fails loudly, printing no number, where no GPU exists."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    p = _bench("--impl", "reference", "--n", "64", "--steps", "2", "--warmup", "1")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    sys.path.insert(0, ROOT)
    import bench
    assert d["metric"] == bench.METRIC and d["unit"] == "solves/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    # ms_per_step is the measured bounded sample; the solves/s value is its
    # extrapolation to the whole step (two solves), reported apart
    ex = d["extrapolation"]
    assert ex["measured_ms_per_sample"] == pytest.approx(d["ms_per_step"])
    assert d["value"] == pytest.approx(2000.0 / ex["est_ms_per_full_step"])
    assert len(ex["oracle_iterations"]) == 2 and min(ex["oracle_iterations"]) >= 1
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 1)
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == bench.WORKLOAD and d["config"]["n"] == 64
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    assert cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_gpu_arm_fails_loudly_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = _bench("--n", "64", "--steps", "1", "--warmup", "0", "--no-cpu-baseline")
    assert p.returncode != 0
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_traffic_figure_is_used_only_for_the_kernels_it_was_taken_on(monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu capture; it is
    reported only for the workload it was taken on (n = 1024, rank 4) and
    only while the K application's CUDA sources hash to the recorded digest."""
    sys.path.insert(0, ROOT)
    import bench
    rec = json.load(open(os.path.join(ROOT, "profiles", "kapply_deblur1024_traffic.json")))
    current = bench.sources_digest() == rec["sources_sha256"]
    assert bench.kapply_traffic(1024, 4) == (rec["dram_bytes_per_k_application"] if current else None)
    monkeypatch.setattr(bench, "sources_digest", lambda: rec["sources_sha256"])  # sources as captured
    assert bench.kapply_traffic(1024, 4) == rec["dram_bytes_per_k_application"]
    assert bench.kapply_traffic(512, 4) is None
    assert bench.kapply_traffic(1024, 3) is None
    monkeypatch.setattr(bench, "sources_digest", lambda: "0" * 64)          # sources changed since
    assert bench.kapply_traffic(1024, 4) is None
