"""Batches: many gaskets of uneven levels in one persistent launch.

Every instance of a batch must hold exactly what the single-instance fused
diffusion leaves (the same per-cell arithmetic in the same 8 x 8 blocks), and
so agree with the FP64 oracle within the diffusion tolerance; graphs replay
the same launches; per-instance reduces match the oracle's sums.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fr():
    from paper_2004_13475_gb300 import build as fbuild
    fbuild.build()
    import paper_2004_13475_gb300 as m
    assert torch.cuda.is_available()
    return m


def make_batch(fr, ks, seed0):
    states = [synth.uniform_f32(seed0 + i, 1 << k) for i, k in enumerate(ks)]
    a = [torch.from_numpy(s.reshape(-1).copy()).cuda() for s in states]
    b = [torch.zeros_like(x) for x in a]
    batch = fr.fractal_batch_create(ks)
    fr.fractal_batch_bind(batch, a, b)
    return batch, states, a, b


def reference(fr, k, u0, steps, spl):
    """The single-instance fused path on one instance."""
    n = 1 << k
    plan = fr.fractal_map(k, 8)
    fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, spl)
    a = torch.from_numpy(u0.reshape(-1).copy()).cuda()
    b = torch.zeros_like(a)
    return fr.fractal_step_diffusion(plan, a, b, 0.2, steps).cpu().numpy().reshape(n, n)


@pytest.mark.parametrize("ks_range,T,spl", [((4, 9), 16, 8), ((6, 10), 64, 32), ((7, 11), 128, 16), ((8, 10), 0, 3),
                                             ((8, 11), 256, 50), ((8, 10), 256, 40)])
def test_batch_equals_single_instances_and_oracle(fr, ks_range, T, spl):
    rng = np.random.default_rng(ks_range[0])
    ks = [int(k) for k in rng.integers(ks_range[0], ks_range[1] + 1, size=9)]
    batch, states, a, b = make_batch(fr, ks, 500)
    fr.fractal_batch_configure(batch, T, spl)
    inf = batch.info()
    assert inf["count"] == 9 and inf["steps_per_launch"] == spl and inf["bound"] == 1
    assert inf["members"] == sum(3 ** k for k in ks)
    for steps in (5, 2 * spl + 1):
        fr.fractal_batch_bind(batch, a, b)
        for i, s in enumerate(states):        # restart from the initial states
            a[i].copy_(torch.from_numpy(s.reshape(-1).copy()))
        which = fr.fractal_batch_step_diffusion(batch, 0.2, steps)
        torch.cuda.synchronize()
        for i, k in enumerate(ks):
            n = 1 << k
            got = (b[i] if which else a[i]).cpu().numpy().reshape(n, n)
            same = reference(fr, k, states[i], steps, min(spl, 32))
            dom = oracle.Domain.build(n)
            assert np.array_equal(got[dom.mask], same[dom.mask]), (k, steps)
            want = oracle.diffusion_run(states[i].astype(np.float64), steps, 0.2, dom)
            assert rel_err(got, want, dom.mask)[0] <= 2e-5, (k, steps)


def _windows(n, steps, inner=128):
    """Oracle windows for a large instance: the corners of the bounding
    triangle and inner squares centred on contacts between 256-cell
    super-tiles and between the level-(k-1) replicas."""
    h = inner // 2
    origins = [(0, 0), (n - inner, 0), (0, n - inner), (3 * 256 - h, -h), (-h, 5 * 256 - h),
               (n // 2 + 256 - h, 256 - h), (n // 2 - h, -h), (-h, n // 2 - h)]
    out = []
    for X, Y in origins:
        x0, y0 = max(0, X - steps), max(0, Y - steps)
        x1, y1 = min(n, X + inner + steps), min(n, Y + inner + steps)
        out.append((x0, y0, x1 - x0, y1 - y0))
    return out


def _valid(n, x0, y0, w, h, steps):
    lo_x = 0 if x0 <= 0 else steps
    lo_y = 0 if y0 <= 0 else steps
    hi_x = w if x0 + w >= n else w - steps
    hi_y = h if y0 + h >= n else h - steps
    return slice(lo_y, hi_y), slice(lo_x, hi_x)


@pytest.mark.parametrize("spl", [32, 50])
def test_batch_as_benchmarked_against_oracle(fr, spl):
    """The configurations the benchmark's autotuner chooses between: super-tile
    side 256 with 32 steps per launch (one block per thread) or 50 (four
    warps, 320 block slots), levels drawn from 8..13, 100 steps through the
    captured graph.  One instance of every level is compared with the FP64
    oracle (whole array up to k = 11, windows across super-tile and replica
    seams above)."""
    rng = np.random.default_rng(13)
    ks = [8, 9, 10, 11, 12, 13] + [int(k) for k in rng.integers(8, 14, size=10)]
    seed0, steps = 900, 100
    a = [torch.empty((1 << k) ** 2, dtype=torch.float32, device="cuda") for k in ks]
    b = [torch.empty_like(x) for x in a]
    for i, k in enumerate(ks):
        synth.device_fill(a[i].data_ptr(), synth.SYNTH_UNIFORM_F32, 1 << k, seed0 + i)
    batch = fr.fractal_batch_create(ks)
    fr.fractal_batch_bind(batch, a, b)
    fr.fractal_batch_configure(batch, 256, spl)
    inf = batch.info()
    assert inf["supertile"] == 256 and inf["steps_per_launch"] == spl
    fr.fractal_batch_graph_capture(batch, 0.2, steps)
    fr.fractal_batch_graph_launch(batch)              # 100 steps: result in a (records between launches)
    torch.cuda.synchronize()
    for i, k in enumerate(ks[:6]):
        n = 1 << k
        out = a[i].view(n, n)
        if k <= 11:
            u0 = synth.uniform_f32(seed0 + i, n).astype(np.float64)
            dom = oracle.Domain.build(n)
            want = oracle.diffusion_run(u0, steps, 0.2, dom)
            err, raw = rel_err(out.cpu().numpy(), want, dom.mask)
            assert err <= 1e-4, (k, err, raw)
            continue
        for (x0, y0, w, h) in _windows(n, steps):
            dom = oracle.Domain.build(n, x0, y0, w, h)
            u0 = synth.uniform_f32(seed0 + i, n, x0, y0, w, h).astype(np.float64)
            want = oracle.diffusion_run(u0, steps, 0.2, dom)
            rs, cs = _valid(n, x0, y0, w, h, steps)
            got = out[y0:y0 + h, x0:x0 + w].cpu().numpy()
            err, raw = rel_err(got[rs, cs], want[rs, cs], dom.mask[rs, cs])
            assert err <= 1e-4, (k, x0, y0, err, raw)
    batch.close()


def test_batch_graph_replays_the_steps(fr):
    ks = [6, 9, 7, 8, 6, 10, 8]
    batch, states, a, b = make_batch(fr, ks, 600)
    fr.fractal_batch_configure(batch, 32, 16)
    fr.fractal_batch_graph_capture(batch, 0.2, 20)
    assert batch.info()["graph_steps"] == 20
    fr.fractal_batch_graph_launch(batch)
    fr.fractal_batch_graph_launch(batch)          # 40 steps, result in a
    torch.cuda.synchronize()
    got = [x.cpu().numpy() for x in a]
    for i, s in enumerate(states):
        a[i].copy_(torch.from_numpy(s.reshape(-1).copy()))
    fr.fractal_batch_step_diffusion(batch, 0.2, 40)
    torch.cuda.synchronize()
    for i in range(len(ks)):
        assert np.array_equal(got[i], a[i].cpu().numpy())


def test_batch_reduce_matches_oracle_sums(fr):
    ks = [5, 8, 11, 7, 9, 6]
    batch, states, a, b = make_batch(fr, ks, 700)
    out = torch.full((len(ks) + 1,), -1.0, dtype=torch.float64, device="cuda")
    fr.fractal_batch_reduce(batch, 0, out)
    first = out.cpu().numpy().copy()
    fr.fractal_batch_reduce(batch, 0, out)
    assert np.array_equal(first, out.cpu().numpy())            # deterministic
    assert first[-1] == -1.0                                     # nothing beyond count written
    for i, k in enumerate(ks):
        dom = oracle.Domain.build(1 << k)
        want = oracle.reduce_sum(dom.take(states[i]).astype(np.float64))
        assert abs(first[i] - want) <= 1e-6 * want, (k, first[i], want)
    # after steps, the sums of the b buffers are conserved (zero-flux walls)
    fr.fractal_batch_step_diffusion(batch, 0.2, 9)
    fr.fractal_batch_reduce(batch, 1, out)
    after = out.cpu().numpy()
    assert np.allclose(after[:-1], first[:-1], rtol=1e-5, atol=0)


def test_batch_autotune_keeps_results_exact(fr):
    ks = [8, 9, 10, 8, 9]
    batch, states, a, b = make_batch(fr, ks, 800)
    us = fr.fractal_batch_autotune(batch, 0.2, 2)
    assert us > 0
    inf = batch.info()
    for i, s in enumerate(states):             # autotune only reads a
        assert np.array_equal(a[i].cpu().numpy(), s.reshape(-1))
    fr.fractal_batch_step_diffusion(batch, 0.2, 6)
    torch.cuda.synchronize()
    for i, k in enumerate(ks):
        got = a[i].cpu().numpy().reshape(1 << k, 1 << k)
        same = reference(fr, k, states[i], 6, inf["steps_per_launch"])
        m = oracle.member_mask(1 << k)
        assert np.array_equal(got[m], same[m])


def test_batch_validation(fr):
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_create([3, 8])                 # level below 4
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_create([17])
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_create([])
    batch = fr.fractal_batch_create([6, 7])
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_step_diffusion(batch, 0.2, 3)  # not bound
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_graph_launch(batch)            # no graph
    x = [torch.zeros(64 * 64, device="cuda"), torch.zeros(128 * 128, device="cuda")]
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_bind(batch, x, x)              # a == b
    y = [torch.zeros(64 * 64 + 1, device="cuda")[1:], torch.zeros(128 * 128, device="cuda")]
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_bind(batch, y, [torch.zeros_like(t) for t in x])   # misaligned
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_configure(batch, 128, 8)       # side above 2^k_min
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_configure(batch, 48, 8)        # not a power of two
    with pytest.raises(fr.FractalError):
        fr.fractal_batch_configure(batch, 32, 17)       # margin 24 > T/2
    fr.fractal_batch_configure(batch, 64, 32)
    assert batch.info()["supertile"] == 64
