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


def _box_blocks_brute(T, M, R):
    """Most member blocks of the margin boxes within each reach 1..M of a
    super-tile of side T, over every member super-tile of a level-R grid of
    super-tiles, by direct enumeration (numpy)."""
    import numpy as np
    B, side, W = 8, T // 8, M // 8
    q = []
    for by in range(-W, side + W):
        for bx in range(-W, side + W):
            inside = 0 <= bx < side and 0 <= by < side
            left = -W <= bx < 0 and 0 <= by < W
            top = 0 <= bx < W and -W <= by < 0
            right = side <= bx < side + W and -W <= by < W
            bottom = -W <= bx < W and side <= by < side + W
            if inside or not (left or top or right or bottom):
                continue
            xs, ys = np.arange(bx * B, bx * B + B), np.arange(by * B, by * B + B)
            dx = np.maximum(0, np.maximum(-xs, xs - (T - 1))).min()
            dy = np.maximum(0, np.maximum(-ys, ys - (T - 1))).min()
            q.append((bx, by, dx + dy))
    q = np.array(q)
    g = 1 << R
    nblk = g * side
    sx, sy = np.meshgrid(np.arange(g), np.arange(g))
    keep = (sx & sy) == 0
    sx, sy = sx[keep], sy[keep]
    gx = sx[:, None] * side + q[None, :, 0]
    gy = sy[:, None] * side + q[None, :, 1]
    member = (gx >= 0) & (gy >= 0) & (gx < nblk) & (gy < nblk) & ((gx & gy) == 0)
    return {r: int((member & (q[None, :, 2] <= r)).sum(axis=1).max()) for r in range(1, M + 1)}


@pytest.mark.parametrize("T,M", [(16, 8), (64, 32), (128, 64), (256, 64), (256, 32), (256, 128)])
def test_fused_box_blocks_match_brute_force(lib, T, M):
    """The staged margin-box blocks per super-tile: the library's count (taken
    over a 64 x 64 grid of super-tiles) equals a brute-force maximum over every
    member super-tile of a 128 x 128 grid, for every reach; at reach = margin
    it is the whole boxes' member count, three gasket fragments of side M."""
    want = _box_blocks_brute(T, M, 7)
    for r in range(1, M + 1):
        assert fr.fractal_fused_box_blocks(T, M, r) == want[r], (T, M, r)
    assert want[M] == 3 ** (1 + (M // 8).bit_length() - 1)


@pytest.mark.parametrize("args", [(8, 8, 8), (24, 8, 8), (512, 64, 64), (256, 12, 8), (64, 64, 8), (256, 64, 0),
                                  (256, 64, 65)])
def test_fused_box_blocks_rejects_bad_arguments(lib, args):
    assert lib.fractal_fused_box_blocks(*args) == -1  # FRACTAL_EINVAL
