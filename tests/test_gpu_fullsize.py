"""Parity at the full workload sizes, in the launch configuration the benchmark
times (the plans' default CTA levels), on sampled outputs the oracle computes
one window at a time.

A window of the embedding is exact in the oracle at every cell farther than
`steps` from its inner edges (information moves one cell per step), so each
sample compares the whole valid interior of its window element by element.
Whole-array invariants (the member count, the conserved heat) are checked
against sums the oracle forms from the members' generator values."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SEED = 0


@pytest.fixture(scope="module")
def fr():
    from paper_2004_13475_gb300 import build as fbuild
    fbuild.build()
    import paper_2004_13475_gb300 as m
    assert torch.cuda.is_available()
    return m


def valid_region(n, x0, y0, w, h, steps):
    """Slices (rows, cols) of the window that the oracle gets exactly right."""
    lo_x = 0 if x0 <= 0 else steps
    lo_y = 0 if y0 <= 0 else steps
    hi_x = w if x0 + w >= n else w - steps
    hi_y = h if y0 + h >= n else h - steps
    assert hi_x > lo_x and hi_y > lo_y
    return slice(lo_y, hi_y), slice(lo_x, hi_x)


def windows(n, steps, inner=192):
    """Sample windows around inner squares that start on member blocks: the
    three corners of the gasket's bounding triangle and points inside the
    right and upper level-1 replicas.  Windows are clipped to the array."""
    corners = [(0, 0), (n - inner, 0), (0, n - inner),
               (n // 2 + n // 8, n // 16), (n // 64, n // 2 + n // 4)]
    return windows_at(n, steps, corners, inner)


def seam_windows(n, steps, inner=128):
    """Windows whose inner squares are centred on contacts between super-tiles
    of every side up to 256 (the fused kernels' CTA tiles): seams along the
    bottom row and the left column, an interior contact, the two seams of the
    level-15 replicas (the highest lambda digit) and their diagonal contact."""
    h = inner // 2
    centres = [(3 * 256, 0), (0, 5 * 256), (n // 2 + 256, 256),
               (n // 2, 0), (0, n // 2), (n // 2, n // 2)]
    return windows_at(n, steps, [(cx - h, cy - h) for cx, cy in centres], inner)


def windows_at(n, steps, origins, inner):
    out = []
    for X, Y in origins:
        x0, y0 = max(0, X - steps), max(0, Y - steps)
        x1, y1 = min(n, X + inner + steps), min(n, Y + inner + steps)
        out.append((x0, y0, x1 - x0, y1 - y0))
    return out


_ORACLE = {}


def oracle_window(kind, n, x0, y0, w, h, steps):
    """The oracle's state of a window after ``steps`` steps (cached: the same
    window serves every rho, mode and fusion setting of a test)."""
    key = (kind, n, x0, y0, w, h, steps)
    if key not in _ORACLE:
        dom = oracle.Domain.build(n, x0, y0, w, h)
        if kind == "ca":
            want = oracle.ca_run(synth.bernoulli_u8(SEED, n, x0, y0, w, h), steps, dom)
        else:
            u0 = synth.uniform_f32(SEED, n, x0, y0, w, h).astype(np.float64)
            want = oracle.diffusion_run(u0, steps, 0.2, dom)
        _ORACLE[key] = (dom, want)
    return _ORACLE[key]


def _member_sum(n, dist, seed):
    """Oracle-side sum over all members of the generated state, row by row."""
    total = 0.0 if dist == "uniform" else 0
    xs_all = np.arange(n, dtype=np.int64)
    for y in range(n):
        xs = xs_all[(xs_all & y) == 0]
        vals = synth.values_at(seed, n, xs, np.full(xs.size, y), dist)
        total += vals.astype(np.float64).sum() if dist == "uniform" else int(vals.sum())
    return total


@pytest.fixture(scope="module")
def k16_u8(fr):
    n = 1 << 16
    a = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    b = torch.empty_like(a)
    return n, a, b


@pytest.mark.parametrize("tuned", [False, 25, True])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("rho", [8, 16, 32])
def test_k16_ca_100_steps(fr, k16_u8, rho, mode, tuned):
    n, a, b = k16_u8
    steps = 100
    synth.device_fill(a.data_ptr(), synth.SYNTH_BERNOULLI_U8, n, SEED)
    plan = fr.fractal_map(16, rho, mode)
    if tuned is True:       # what the benchmark runs: the autotuner's choice
        fr.fractal_plan_autotune(plan, fr.FRACTAL_U8, a, b, 2)
    elif tuned:             # temporal fusion, 25 steps per launch
        fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_U8, tuned)
    out = fr.fractal_step_ca(plan, a, b, steps).view(n, n)
    for (x0, y0, w, h) in windows(n, steps) + seam_windows(n, steps):
        dom, want = oracle_window("ca", n, x0, y0, w, h, steps)
        got = out[y0:y0 + h, x0:x0 + w].cpu().numpy()
        rs, cs = valid_region(n, x0, y0, w, h, steps)
        m = dom.mask[rs, cs]
        assert np.array_equal(got[rs, cs][m], want[rs, cs][m]), (rho, mode, x0, y0)
    # exact count over the whole gasket is consistent between lambda and BB
    alive = fr.fractal_reduce(plan, out, fr.FRACTAL_U8)
    assert 0 < alive < 3 ** 16


def test_k16_member_count_and_sums(fr, k16_u8):
    n, a, _ = k16_u8
    plan = fr.fractal_map(16, 32)
    fr.fractal_map_write(plan, a, fr.FRACTAL_U8, 1)
    assert fr.fractal_reduce(plan, a, fr.FRACTAL_U8) == 3 ** 16
    synth.device_fill(a.data_ptr(), synth.SYNTH_BERNOULLI_U8, n, SEED)
    want = _member_sum(n, "bernoulli", SEED)
    for mode in (0, 1):
        assert fr.fractal_reduce(fr.fractal_map(16, 32, mode), a, fr.FRACTAL_U8) == want


@pytest.fixture(scope="module")
def k16_f32(fr, k16_u8):
    n = 1 << 16
    a = torch.empty(n * n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    return n, a, b


@pytest.mark.parametrize("spl", [1, 8, 32, 50, "tuned"])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("rho", [8, 16, 32])
def test_k16_diffusion_200_steps(fr, k16_f32, rho, mode, spl):
    n, a, b = k16_f32
    steps = 200
    synth.device_fill(a.data_ptr(), synth.SYNTH_UNIFORM_F32, n, SEED)
    plan = fr.fractal_map(16, rho, mode)
    if spl == "tuned":      # what the benchmark runs: the autotuner's choice
        fr.fractal_plan_autotune(plan, fr.FRACTAL_F32, a, b, 2)
    elif spl > 1:
        fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, spl)
    start = fr.fractal_reduce(plan, a, fr.FRACTAL_F32)
    out = fr.fractal_step_diffusion(plan, a, b, 0.2, steps).view(n, n)
    for (x0, y0, w, h) in windows(n, steps, inner=128) + seam_windows(n, steps):
        dom, want = oracle_window("diffusion", n, x0, y0, w, h, steps)
        got = out[y0:y0 + h, x0:x0 + w].cpu().numpy()
        rs, cs = valid_region(n, x0, y0, w, h, steps)
        err, _ = rel_err(got[rs, cs], want[rs, cs], dom.mask[rs, cs])
        assert err <= 1e-4, (rho, mode, x0, y0, err)
    end = fr.fractal_reduce(plan, out, fr.FRACTAL_F32)
    # zero-flux walls conserve heat; FP32 rounding of 200 steps stays far below 1e-4
    assert abs(end - start) <= 1e-4 * start


def test_k16_diffusion_start_sum(fr, k16_f32):
    n, a, _ = k16_f32
    synth.device_fill(a.data_ptr(), synth.SYNTH_UNIFORM_F32, n, SEED)
    want = _member_sum(n, "uniform", SEED)
    for mode in (0, 1):
        got = fr.fractal_reduce(fr.fractal_map(16, 8, mode), a, fr.FRACTAL_F32)
        assert abs(got - want) <= 1e-6 * want


@pytest.mark.parametrize("mode", [0, 1])
def test_k14_diffusion_1000_steps(fr, mode):
    # 16384 x 16384 FP32, a = 0.2, 1000 steps with a reduce every 100 steps
    n, steps = 1 << 14, 1000
    a = torch.empty(n * n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    synth.device_fill(a.data_ptr(), synth.SYNTH_UNIFORM_F32, n, SEED)
    plan = fr.fractal_map(14, 16, mode)
    fr.fractal_plan_autotune(plan, fr.FRACTAL_F32, a, b, 2)
    sums = [fr.fractal_reduce(plan, a, fr.FRACTAL_F32)]
    cur, other = a, b
    for _ in range(10):
        cur = fr.fractal_step_diffusion(plan, cur, other, 0.2, 100)
        other = b if cur is a else a
        sums.append(fr.fractal_reduce(plan, cur, fr.FRACTAL_F32))
    assert max(abs(s - sums[0]) for s in sums) <= 1e-4 * sums[0]
    out = cur.view(n, n)
    for (x0, y0, w, h) in [(0, 0, 1400, 1400), (n - 1400, 0, 1400, 1400)]:
        dom = oracle.Domain.build(n, x0, y0, w, h)
        u0 = synth.uniform_f32(SEED, n, x0, y0, w, h).astype(np.float64)
        want = oracle.diffusion_run(u0, steps, 0.2, dom)
        got = out[y0:y0 + h, x0:x0 + w].cpu().numpy()
        rs, cs = valid_region(n, x0, y0, w, h, steps)
        err, raw = rel_err(got[rs, cs], want[rs, cs], dom.mask[rs, cs])
        assert err <= 1e-4, (mode, x0, y0, err, raw)


@pytest.mark.parametrize("mode", [0, 1])
def test_k10_ca_10_steps_rho16(fr, mode):
    # 1024 x 1024 uint8, B3/S23, 10 steps, rho = 16: whole array, bit-exact
    n = 1 << 10
    s0 = synth.bernoulli_u8(SEED, n)
    a = torch.from_numpy(s0.reshape(-1).copy()).cuda()
    b = torch.zeros_like(a)
    out = fr.fractal_step_ca(fr.fractal_map(10, 16, mode), a, b, 10)
    want = oracle.ca_run(s0, 10)
    mask = oracle.member_mask(n)
    assert np.array_equal(out.cpu().numpy().reshape(n, n)[mask], want[mask])
