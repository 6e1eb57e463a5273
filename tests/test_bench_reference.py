"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one JSON line with
the contract's keys, on the CPU: the same metric and unit as the GPU arm, its own cpu_baseline
and an e2e entry with no host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_step_seconds_agree_with_ms_per_step():
    """s_to_converged and ms_per_step are the same timed region over the same steps."""
    import bench
    ms, s = bench.step_seconds(1.79, 20)
    assert abs(ms - 89.5) < 1e-9 and abs(s * 1e3 - ms) < 1e-12


def test_traffic_records_are_read_only_for_the_current_source(tmp_path, monkeypatch):
    """The DRAM traffic of a committed ncu record enters the roofline only while the hash of
    the kernel's source matches the one the counters were taken on."""
    import hashlib
    import os
    import bench
    src = os.path.join(bench.ROOT, "paper_2109_08547_gb300", "csrc", "vertex_tc.cu")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "rec.txt").write_text(f"source_sha256_16: {h}\nunit: launch\ndram_bytes_per_unit: 123.5\n")
    (prof / "old.txt").write_text("source_sha256_16: 0000000000000000\nunit: launch\ndram_bytes_per_unit: 7\n")
    (tmp_path / "paper_2109_08547_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_2109_08547_gb300" / "csrc" / "vertex_tc.cu").write_bytes(open(src, "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("rec.txt", "vertex_tc.cu") == (123.5, "launch")
    assert bench.profile_traffic("old.txt", "vertex_tc.cu") is None
    assert bench.profile_traffic("missing.txt", "vertex_tc.cu") is None
