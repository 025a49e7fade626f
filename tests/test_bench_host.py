"""Host logic of the benchmark that decides what its JSON line may claim, checked on the CPU:
the DRAM traffic of a kernel is reported only while the kernel source still matches the
ncu capture it came from, the peaks fall back (and say so) without the measured file, the
HMULT oracle timing is bounded and labelled, the variant names and CPU description are well
formed, and the reference arm prints one contract line on rank 0 and nothing elsewhere."""
import hashlib
import json
import os

import pytest

import bench


def _write(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        f.write(data)


def test_traffic_is_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    src = "csrc/kernel.cu"
    _write(str(tmp_path / src), "__global__ void k() {}\n")
    h = hashlib.sha256(open(tmp_path / src, "rb").read()).hexdigest()[:16]
    _write(str(tmp_path / "profiles" / "traffic.json"),
           json.dumps({"k_n65536": {"dram_bytes_per_launch": 123456, "source_sha256_16": h}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for(src, "k_n65536") == 123456
    assert bench.traffic_for(src, "other_key") is None
    _write(str(tmp_path / src), "__global__ void k() { /* changed */ }\n")
    assert bench.traffic_for(src, "k_n65536") is None          # the capture no longer applies
    assert bench.traffic_for("csrc/missing.cu", "k_n65536") is None


def test_committed_traffic_records_are_well_formed():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        recs = json.load(f)
    assert recs
    for key, rec in recs.items():
        assert rec["dram_bytes_per_launch"] > 0, key
        assert len(rec["source_sha256_16"]) == 16, key
        assert os.path.exists(os.path.join(bench.ROOT, rec["source"])), key
        assert "--clock-control none" in rec["command"], key


def test_peaks_fall_back_and_say_so(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench.measured_peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] > 0 and peaks["bf16_tflops"] > 0
    _write(str(tmp_path / "MEASURED_PEAKS.json"), json.dumps({"hbm_gbs": 7000.0, "bf16_tflops": 2000.0}))
    peaks, kind = bench.measured_peaks()
    assert kind == "measured" and peaks["hbm_gbs"] == 7000.0


@pytest.mark.parametrize("v", [0, 1, 6, 7, 8, 16, 31])
def test_variant_names(v):
    name = bench.variant_name(v)
    assert name.startswith("variant %d:" % v)
    assert ("512-thread" in name) == (v & 1 == 0)
    assert ("two-pass" in name) == (((v >> 1) & 3) == 3)


@pytest.mark.parametrize("v", [32, 33])
def test_tensor_core_variant_names(v):
    name = bench.variant_name(v)
    assert name.startswith("variant %d:" % v) and "tensor-core" in name
    assert ("64-column" in name) == (v == 32)


def test_host_cpu_description():
    d = bench.host_cpu()
    assert "logical cores" in d and str(os.cpu_count()) in d


def test_hmult_oracle_timing_is_bounded_and_labelled():
    r = bench.cpu_oracle_hmult(budget_s=0.5, n=1 << 11)
    assert r["kind"] == "oracle" and r["value"] > 0 and "HMULT" in r["unit"]
    assert "N=2048" in r["sample"] and "24 + 8 limbs" in r["sample"]


def _run_reference(env_extra):
    import subprocess
    import sys
    env = {**os.environ, **env_extra}
    return subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
                           "--steps", "1", "--warmup", "1"], cwd=bench.ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    """The reference arm times the oracle on the CPU and prints one JSON line with the CUDA
    arm's metric, unit and direction, its own cpu_baseline and an e2e with no copies."""
    r = _run_reference({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "KOPS"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "KOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]
