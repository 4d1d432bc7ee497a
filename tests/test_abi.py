"""Host-only checks of the C ABI: the library builds, loads and exports every
declared entry point; argument validation rejects bad input before any CUDA
work (no compute call is made here)."""
import ctypes
import os
import re

import pytest

import paper_2004_13475_gb300 as fr
from paper_2004_13475_gb300 import build as fbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    fbuild.build()
    return fr._load()


def _declared():
    with open(os.path.join(ROOT, "include", "fractal.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fractal_[a-z0-9_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert sorted(fr.EXPORTS) == _declared()


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_synth_device_twin_builds():
    import synth
    fbuild.build()
    assert hasattr(synth.load_device_lib(), "synth_fill")


def test_strerror(lib):
    assert fr.fractal_strerror(0) == "ok"
    assert fr.fractal_strerror(-1) == "invalid argument"
    assert fr.fractal_strerror(-3) == "CUDA error"
    assert fr.fractal_strerror(12345) == "unknown status"


@pytest.mark.parametrize("k,rho,mode", [
    (-1, 1, 0), (17, 8, 0), (3, 16, 0), (5, 3, 0), (5, 0, 0), (10, 64, 0), (6, 8, 2), (6, 8, -1),
])
def test_map_rejects_bad_arguments(lib, k, rho, mode):
    h = ctypes.c_void_p()
    assert lib.fractal_map(k, rho, mode, ctypes.byref(h)) == fr.FRACTAL_EINVAL
    assert not h.value


def test_map_rejects_null_out(lib):
    assert lib.fractal_map(4, 4, 0, None) == fr.FRACTAL_EINVAL


def test_null_plan_is_rejected(lib):
    assert lib.fractal_plan_destroy(None) == fr.FRACTAL_OK
    assert lib.fractal_plan_get_info(None, None) == fr.FRACTAL_EINVAL
    assert lib.fractal_plan_set_cta_levels(None, 0, 0) == fr.FRACTAL_EINVAL
    assert lib.fractal_map_blocks(None, 16, None) == fr.FRACTAL_EINVAL
    assert lib.fractal_map_write(None, 16, 0, 1.0, None) == fr.FRACTAL_EINVAL
    assert lib.fractal_step_ca(None, 16, 32, 1, None) == fr.FRACTAL_EINVAL
    assert lib.fractal_step_diffusion(None, 16, 32, 0.2, 1, None) == fr.FRACTAL_EINVAL
    out = ctypes.c_double()
    assert lib.fractal_reduce(None, 16, 0, ctypes.byref(out), None) == fr.FRACTAL_EINVAL
    assert lib.fractal_reduce_async(None, 16, 0, 32, None) == fr.FRACTAL_EINVAL


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(fr, "_lib", None)
    monkeypatch.setattr(fr, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        fr.fractal_map(4, 4)
