"""Host-side parts of bench.py: the reference arm (the oracle on the host cores) prints
one well-formed JSON line, the byte models are what their docstrings say, and stored
ncu counters are used only for the kernel source they were taken on."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--workload", "chain16"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "chain16"], capture_output=True, text=True, timeout=120,
                         cwd=ROOT, env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_byte_models():
    D, T = 1000, 50000
    # per row: state 8, |Stab| 2, x_i and y_i; per term one gathered entry
    assert bench.alg_bytes(D, T, 8) == D * 26 + T * 8
    assert bench.alg_bytes(D, T, 4) == D * 18 + T * 4
    # a random gather costs a whole 32-byte sector whatever the entry size
    assert bench.sector_bytes(D, T, 4) == D * 18 + T * 32
    assert bench.sector_bytes(D, T, 8) == D * 26 + T * 32


def test_profiled_counters_follow_the_source_hash(tmp_path, monkeypatch):
    sha = bench.kernel_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "apply_h_demo.md").write_text(
        f"traffic_bytes_per_launch[mixed]: 12345 source_sha: {sha}\n"
        f"warp_instructions_per_launch[mixed]: 777 source_sha: 0000000000000000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: sha)
    assert bench.profiled("demo", "traffic_bytes_per_launch", "mixed") == 12345
    # a counter taken on other sources is not reported
    assert bench.profiled("demo", "warp_instructions_per_launch", "mixed") is None
    assert bench.profiled("demo", "traffic_bytes_per_launch", "f64") is None
    assert bench.profiled("absent", "traffic_bytes_per_launch", "mixed") is None


def test_kernel_hash_ignores_comments(tmp_path, monkeypatch):
    """The counters' key follows the code, not its comments or layout."""
    src = tmp_path / "k.cu"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", ["k.cu"])
    src.write_text("int f(int a) { return a + 1; }  // one\n")
    h0 = bench.kernel_hash()
    src.write_text("/* header */\nint f(int a) {\n  return a + 1;   // two\n}\n")
    assert bench.kernel_hash() == h0
    src.write_text("int f(int a) { return a + 2; }\n")
    assert bench.kernel_hash() != h0


def test_reference_config_names_the_sector():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--workload", "chain16"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    cfg = json.loads(out.stdout.strip().splitlines()[-1])["config"]
    assert cfg["workload"] == "chain16" and cfg["dim"] == 810
    assert cfg["n_sublat"] >= 1 and cfg["n_sym"] == 16


def test_stored_matrix_record_from_golden():
    rec = bench.stored_matrix_record("square36")
    assert rec is not None and rec["value"] > 0 and rec["cores"] >= 1
    assert "not in this run" in rec["note"]
    assert bench.stored_matrix_record("chain16") is None
