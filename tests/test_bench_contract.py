"""bench.py's output contract, checked without a GPU.

The reference arm times the oracle on the host cores and prints one JSON line with the same
metric, unit and config as the CUDA arm, plus its own cpu_baseline and an e2e object with no
host-device traffic.  The CUDA arm has no CPU path: on a machine without a GPU it must fail,
not print a number.
"""
import json
import os
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _run(*args, timeout=600):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    return subprocess.run([sys.executable, str(ROOT / "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_default_workload_is_rmat_scale24():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.DEFAULT_WORKLOAD == "rmat_s24_m256M"
    import graphgen
    assert bench.DEFAULT_WORKLOAD in graphgen.WORKLOADS and bench.SECONDARY_WORKLOAD in graphgen.WORKLOADS


def test_reference_arm_prints_one_contract_line():
    r = _run("--impl", "reference", "--steps", "1", "--warmup", "1", "--workload", "chunglu_n1M_m10M")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    assert d["metric"] == "sampled edge-sketch pairs/s" and d["unit"] == "pairs/s"
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 1
    assert d["vs_baseline"] is None and d["data"] == "synthetic" and d["dtype"] == "u64"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cfg = d["config"]
    assert cfg["workload"] == "chunglu_n1M_m10M"
    assert (cfg["n"], cfg["m"], cfg["R"], cfg["k"]) == (1_000_000, 10_000_000, 256, 100)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_cuda_arm_fails_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    r = _run("--steps", "1", "--warmup", "0")
    assert r.returncode != 0
    assert not _json_lines(r.stdout)


def test_dram_traffic_entries_match_the_current_kernels():
    # every committed ncu figure names the kernel it was taken on and that kernel's source
    # digest; a kernel edited since its capture makes the bench report null traffic, so the
    # committed table is checked to be current.  Builds on the bucketed path take the
    # "@buckets" entries (their own sampling, union and compression kernels).
    sys.path.insert(0, str(ROOT))
    import bench
    table = json.loads((ROOT / "profiles" / "dram_traffic.json").read_text())
    for key, d in table.items():
        assert d["kernel_sha1"] == bench._kernel_digest(d["source"], d["function"]), key
        assert (ROOT / "profiles" / d["profile"]).exists(), key
    for name in ("sample_emit", "union", "compress_count"):
        b = table[name + "@buckets"]["bytes_per_unit"]
        assert bench._traffic(name, 1000.0, "buckets") == pytest.approx(1000.0 * b)
        r = table[name]["bytes_per_unit"]
        assert bench._traffic(name, 1000.0, "records") == pytest.approx(1000.0 * r)
    assert table["sample_emit@buckets"]["function"] == "k_sample_bucket"
    assert table["union@buckets"]["function"] == "k_union_bucket"
    assert table["compress_count"]["function"] == "k_compress_queue"
