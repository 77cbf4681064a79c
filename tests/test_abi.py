"""The C-ABI library builds, loads and exports every entry point include/flod.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "flod.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(flod_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2408_12894_gb300 import _build
    return _build.build()


def test_header_declares_the_path_entry_points():
    names = _declared()
    for need in ("flod_preprocess", "flod_bin_sort", "flod_render_fwd", "flod_render_bwd",
                 "flod_select_levels", "flod_adjust_scale", "flod_workspace_size",
                 "flod_workspace_layout"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (flod_\w+)", out))
    assert set(_declared()) <= exported


def test_host_side_checks_without_a_device(libpath):
    from paper_2408_12894_gb300 import flod
    import ctypes as C
    cfg = flod.default_config()
    assert (cfg.tile_w, cfg.tile_h, cfg.batch) == (16, 16, 128)
    assert abs(cfg.dilation - 0.3) < 1e-7 and abs(cfg.z_near - 0.2) < 1e-7
    # a fake set/view description: the size query is pure host arithmetic
    g = flod.Gaussians()
    g.n, g.sh_degree, g.s_min = 0, 3, 0.0
    v = flod.View()
    v.cam.width, v.cam.height, v.cam.fx, v.cam.fy = 1920, 1080, 1000.0, 1000.0
    v.set = 0
    sets = (flod.Gaussians * 1)(g)
    views = (flod.View * 1)(v)
    n = flod.flod_workspace_size(sets, views, 1 << 20, cfg)
    lay, uo, to, po = flod.flod_workspace_layout(sets, views, 1 << 20, cfg)
    assert lay.total == n and lay.tiles == 120 * 68 and lay.pixels == 1920 * 1080
    assert to == [0, 8160] and po == [0, 1920 * 1080]
    for name in ("xy", "depth", "conic_o", "rgb", "ranges", "grad2d"):
        assert getattr(lay, name) % 256 == 0
    # invalid arguments are refused before anything is enqueued
    bad = flod.default_config(tile_w=12)
    assert flod.lib().flod_workspace_size(sets, 1, views, 1, 1 << 20, C.byref(bad)) == 0
    assert flod.lib().flod_workspace_size(sets, 1, views, 1, 1 << 32, C.byref(cfg)) == 0
    v2 = flod.View()
    v2.cam.width = 0
    assert flod.lib().flod_workspace_size(sets, 1, (flod.View * 1)(v2), 1, 1024, C.byref(cfg)) == 0
    assert flod.lib().flod_adjust_scale(None, 10, 0.5, 0.25, None) == 1
    assert flod.lib().flod_adjust_scale(None, 0, 0.25, 0.5, None) == 1
    assert flod.lib().flod_status_string(6) == b"workspace too small"


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    from paper_2408_12894_gb300 import flod
    monkeypatch.setattr(flod, "_lib", None)
    monkeypatch.setattr(flod, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(flod.FlodError):
        flod.lib()
