"""bench.py's contract on the CPU: the reference arm's JSON line (the FP64 oracle timed on a
bounded sample of the step), silence of the other ranks, and the guard that keeps a stale
DRAM-traffic figure out of the roofline."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None, timeout=600):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--small", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["unit"] == "it/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "it/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] and d["metric"] == bench.METRIC


def test_reference_arm_other_ranks_exit_silently():
    r = _run(["--impl", "reference", "--small", "--steps", "1", "--warmup", "0"],
             {"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"}, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_traffic_guard_rejects_changed_sources(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel source\n")
    import hashlib
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    (tmp_path / "profiles").mkdir()
    md = tmp_path / "profiles" / "k_x_dram_level5_3M_1080p.md"
    md.write_text(f"# k_x\n\ntraffic_bytes_per_launch: 1234\nsources_sha256: {sha}\nsources: k.cu\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic("k_x") == 1234
    src.write_bytes(b"kernel source, edited\n")
    assert bench.measured_traffic("k_x") is None
    assert bench.measured_traffic("k_missing") is None
