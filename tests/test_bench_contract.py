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


def test_stage_work_and_rooflines():
    w = bench.stage_work(n=1000, n_vis=600, pairs=5000, tiles=100, depth_passes=3, tile_passes=2,
                         deg=3, evals=(1e6, 9e5, 4e5), pixels=200)
    assert w["preprocess"] == ("hbm", 1000 * (236 + 84), "B")
    assert w["tile_sort"] == ("hbm", 20 * 5000 * 2, "B")
    assert w["bwd_adam"] == ("hbm", 1000 * (6 * 236 + 4) + 600 * 52, "B")
    assert w["render_fwd"] == ("alu", 1e6 * bench.FLOP_FWD_EVAL + 4e5 * bench.FLOP_FWD_BLEND, "FLOP")
    assert w["loss"][1] == 3 * 200 * bench.FLOP_LOSS_PX
    roof = bench.rooflines({"preprocess": 0.5, "render_fwd": 2.0}, w, 6000.0, 80.0)
    assert set(roof) == {"preprocess", "render_fwd"}
    p = roof["preprocess"]
    assert abs(p["achieved"] - 320000 / 0.5e-3 / 1e9) < 1e-9 and abs(p["frac"] - p["achieved"] / 6000.0) < 1e-12
    assert roof["render_fwd"]["unit"] == "TFLOP/s"
    assert abs(bench.alu_peak_tflops(152, 2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9


def test_oracle_step_strata_cover_every_tile():
    from paper_2408_12894_gb300 import synth
    g = synth.gaussian_set(3, 3000, k=8, radius=20.0, sh_degree=3, s_mean=-2.0)
    cam = synth.camera((0.0, 0.0, -40.0), 320, 180)
    ost = bench.OracleStep(g, cam, 0.03125, slice_n=500, tiles=16)
    assert ost.weight.sum() == ost.n_tiles == 20 * 12
    assert len(ost.sample) == 16 and ost.sample.max() < ost.n_tiles
    # ordered by pair count: the strata's representatives are non-decreasing in it
    assert (ost.sample_pairs[1:] >= ost.sample_pairs[:-1]).all()
    assert ost.step_seconds(threads=1) > 0
