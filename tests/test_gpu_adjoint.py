"""Diffusion with per-cell conductivity and its adjoint on the GPU.

Forward steps against the FP64 oracle step; gradients through the
checkpointed torch.autograd.Function against the oracle's FP64 adjoint and
FP64 central finite differences; the full-size case (k = 13, 200 steps,
checkpoint every 20) on sampled cells whose gradients a window of the array
gives exactly (no influence travels farther than one cell per step, forward
and backward).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

A = 0.2


@pytest.fixture(scope="module")
def fr():
    from paper_2004_13475_gb300 import build as fbuild
    fbuild.build()
    import paper_2004_13475_gb300 as m
    assert torch.cuda.is_available()
    return m


def fields(k, seed):
    n = 1 << k
    u0 = synth.uniform_f32(seed, n)
    mask = oracle.member_mask(n)
    kappa = np.where(mask, np.float32(0.5) + synth.uniform_f32(seed + 1, n), np.float32(0))
    # the loss runs over members: the target is 0 elsewhere (u0 keeps its
    # non-member noise, which the function must ignore)
    target = np.where(mask, synth.uniform_f32(seed + 2, n), np.float32(0)).astype(np.float32)
    return u0, kappa.astype(np.float32), target


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).cuda()


def block_cover(n):
    nb = n // 8
    by, bx = np.mgrid[0:nb, 0:nb]
    return np.kron((bx & by) == 0, np.ones((8, 8), dtype=bool))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k", [3, 5, 8, 10])
def test_kappa_steps_match_oracle(fr, k, mode):
    n = 1 << k
    u0, kappa, _ = fields(k, 10 + k)
    plan = fr.fractal_map(k, 8 if k >= 3 else n, mode)
    dom = oracle.Domain.build(n)
    for steps in (1, 7):
        a = dev(u0)
        b = torch.full_like(a, -3.0)
        out = fr.fractal_step_diffusion_kappa(plan, a, b, dev(kappa), A, steps)
        got = out.cpu().numpy().reshape(n, n)
        want = oracle.diffusion_run(u0.astype(np.float64), steps, A, dom, kappa.astype(np.float64))
        assert rel_err(got, want, dom.mask)[0] <= 2e-6, steps
        cover = block_cover(n)
        assert np.all(got[cover & ~dom.mask] == 0)
        if steps % 2:
            assert np.all(got[~cover] == -3.0)
        # the float64-state kernel: FP64 arithmetic in another order
        a64 = dev(u0.astype(np.float64))
        b64 = torch.zeros_like(a64)
        got64 = fr.fractal_step_diffusion_kappa_f64(plan, a64, b64, dev(kappa), A, steps).cpu().numpy().reshape(n, n)
        assert rel_err(got64, want, dom.mask)[0] <= 1e-13
        # the double-float kernel: (hi, lo) pairs, about 48 significant bits
        adf = torch.stack([dev(u0), torch.zeros(n * n, device="cuda")], dim=1).reshape(-1).contiguous()
        bdf = torch.zeros_like(adf)
        hl = fr.fractal_step_diffusion_kappa_df(plan, adf, bdf, dev(kappa), A, steps).view(-1, 2).cpu().numpy()
        gotdf = (hl[:, 0].astype(np.float64) + hl[:, 1]).reshape(n, n)
        assert rel_err(gotdf, want, dom.mask)[0] <= 1e-12
        assert np.all(np.abs(hl[:, 1]) <= np.abs(hl[:, 0]) * 2.0 ** -23 + 1e-45)   # normalised pairs


def grads_gpu(fr, k, u0, kappa, target, steps, every, mode=0, state="df"):
    from paper_2004_13475_gb300.autograd import diffusion_kappa
    u = dev(u0).requires_grad_(True)
    kp = dev(kappa).requires_grad_(True)
    uT = diffusion_kappa(u, kp, k, A, steps, every, mode, state)
    loss = ((uT - dev(target)) ** 2).sum()
    loss.backward()
    n = 1 << k
    return (float(loss.detach()), u.grad.cpu().numpy().reshape(n, n), kp.grad.cpu().numpy().reshape(n, n),
            uT.detach().cpu().numpy().reshape(n, n))


@pytest.mark.parametrize("state", ["df", "f64"])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k,steps,every", [(4, 9, 1), (6, 25, 7), (8, 45, 20), (9, 60, 20)])
def test_gradients_match_oracle_adjoint(fr, k, steps, every, mode, state):
    n = 1 << k
    u0, kappa, target = fields(k, 30 + k)
    dom = oracle.Domain.build(n)
    J, gu, gk, uT = grads_gpu(fr, k, u0, kappa, target, steps, every, mode, state)
    Jw, wu, wk = oracle.diffusion_loss_gradients(dom, dom.take(u0).astype(np.float64),
                                                 dom.take(kappa).astype(np.float64),
                                                 dom.take(target).astype(np.float64), steps, A)
    assert J == pytest.approx(Jw, rel=1e-5)
    WU, WK = dom.put(wu, np.float64), dom.put(wk, np.float64)
    assert rel_err(gu, WU, dom.mask)[0] <= 1e-4
    assert rel_err(gk, WK, dom.mask)[0] <= 1e-4
    assert not gu[~dom.mask].any() and not gk[~dom.mask].any()


@pytest.mark.parametrize("k,steps,every", [(6, 25, 7), (9, 60, 20)])
def test_float32_state_gradients(fr, k, steps, every):
    # float32 trajectory: its per-step roundings alone put the gradients a
    # few 1e-4 (of their scale) from the exact ones; bound 1e-3
    n = 1 << k
    u0, kappa, target = fields(k, 50 + k)
    dom = oracle.Domain.build(n)
    _, gu, gk, _ = grads_gpu(fr, k, u0, kappa, target, steps, every, state="f32")
    _, wu, wk = oracle.diffusion_loss_gradients(dom, dom.take(u0).astype(np.float64),
                                                dom.take(kappa).astype(np.float64),
                                                dom.take(target).astype(np.float64), steps, A)
    assert rel_err(gu, dom.put(wu, np.float64), dom.mask)[0] <= 1e-3
    assert rel_err(gk, dom.put(wk, np.float64), dom.mask)[0] <= 1e-3


def test_gradients_match_finite_differences(fr):
    # FP64 central differences of the oracle's loss on sampled cells (1e-3 bound)
    k, steps = 6, 30
    n = 1 << k
    u0, kappa, target = fields(k, 77)
    dom = oracle.Domain.build(n)
    _, gu, gk, _ = grads_gpu(fr, k, u0, kappa, target, steps, 10)
    U, K, G = (dom.take(x).astype(np.float64) for x in (u0, kappa, target))

    def loss(uu, kk):
        for _ in range(steps):
            uu = oracle.diffusion_step(dom, uu, A, kk)
        return float(np.sum((uu - G) ** 2))

    rng = np.random.default_rng(3)
    h = 1e-6
    for c in rng.choice(dom.m, size=6, replace=False):
        e = np.zeros(dom.m)
        e[c] = h
        fdu = (loss(U + e, K) - loss(U - e, K)) / (2 * h)
        fdk = (loss(U, K + e) - loss(U, K - e)) / (2 * h)
        x, y = dom.cx[c], dom.cy[c]
        assert gu[y, x] == pytest.approx(fdu, rel=1e-3, abs=1e-6)
        assert gk[y, x] == pytest.approx(fdk, rel=1e-3, abs=1e-6)


def test_level_13_200_steps_sampled_cells(fr):
    """k = 13 (8192 x 8192), kappa ~ U[0.5, 1.5), 200 steps, checkpoint every 20."""
    k, steps, every = 13, 200, 20
    n = 1 << k
    u0, kappa, target = fields(k, 2024)
    _, gu, gk, _ = grads_gpu(fr, k, u0, kappa, target, steps, every)
    r = 2 * steps + 1
    # sampled member cells: near the corner (window clipped by the array edges) and inside
    for (x, y) in ((3, 400), (1000, 17), (2048 + 600, 1024)):
        assert (x & y) == 0
        x0, y0 = max(0, x - r), max(0, y - r)
        x1, y1 = min(n, x + r + 1), min(n, y + r + 1)
        win = oracle.Domain.build(n, x0, y0, x1 - x0, y1 - y0)
        sl = (slice(y0, y1), slice(x0, x1))
        _, wu, wk = oracle.diffusion_loss_gradients(win, win.take(u0[sl]).astype(np.float64),
                                                    win.take(kappa[sl]).astype(np.float64),
                                                    win.take(target[sl]).astype(np.float64), steps, A)
        WU, WK = win.put(wu, np.float64), win.put(wk, np.float64)
        for G, W in ((gu, WU), (gk, WK)):
            want = W[y - y0, x - x0]
            scale = max(abs(want), 1e-3 * np.abs(W).max())
            assert abs(G[y, x] - want) <= 1e-4 * scale, (x, y, G[y, x], want)


def test_adjoint_validation(fr):
    plan = fr.fractal_map(6, 8)
    x = [torch.zeros(64 * 64, device="cuda") for _ in range(5)]
    with pytest.raises(fr.FractalError):
        fr.fractal_adjoint_diffusion_step(plan, x[0], x[1], x[1], x[3], x[4], A)     # p_in == p_out
    with pytest.raises(fr.FractalError):
        fr.fractal_step_diffusion_kappa(plan, x[0], x[1], x[0], A, 2)              # kappa aliases a
    with pytest.raises(fr.FractalError):
        fr.fractal_step_diffusion_kappa(fr.fractal_map(2, 4), x[0], x[1], x[2], A, 1)   # k < 3
    fr.fractal_adjoint_diffusion_step(plan, x[0], x[1], x[2], x[3], x[4], A)
    y = [torch.zeros(2 * 64 * 64, device="cuda") for _ in range(5)]
    with pytest.raises(fr.FractalError):
        fr.fractal_adjoint_diffusion_step_df(plan, y[0], y[1], y[1], x[3], y[4], A)   # p_in == p_out
    with pytest.raises(fr.FractalError):
        fr.fractal_step_diffusion_kappa_df(plan, y[0], y[0], x[3], A, 1)              # a == b
    fr.fractal_adjoint_diffusion_step_df(plan, y[0], y[1], y[2], x[3], y[4], A)


def _df(x):
    """A float32 field as double-float (hi, lo = 0) pairs on the device."""
    t = dev(x)
    return torch.stack([t, torch.zeros_like(t)], dim=1).reshape(-1).contiguous()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k,steps", [(4, 8), (5, 13), (7, 32), (9, 20)])
def test_fused_trajectory_launch_matches_oracle(fr, k, steps, mode):
    """One fused double-float launch (the gradient path's forward and reverse
    passes) against the FP64 oracle, every cell of every member block written;
    the records it keeps are consistent: the same launch without an output
    records the same states before each step, and its final record equals the
    record of the output state."""
    n = 1 << k
    u0, kappa, _ = fields(k, 60 + k)
    plan = fr.fractal_map(k, 8, mode)
    rf, ms = fr.fractal_kappa_fused_limits(k, mode)
    assert steps <= ms and rf == 3 ** (k - 3) * 56
    kap = dev(kappa)
    a_in = _df(u0)
    out = torch.full_like(a_in, -5.0)
    tr1 = torch.zeros(rf * (steps + 1), device="cuda")
    tr2 = torch.zeros_like(tr1)
    tr3 = torch.zeros(rf * 2, device="cuda")
    fr.fractal_kappa_trajectory_df(plan, a_in, out, tr1, kap, A, steps)
    fr.fractal_kappa_trajectory_df(plan, a_in, None, tr2, kap, A, steps)
    fr.fractal_kappa_trajectory_df(plan, out, None, tr3, kap, A, 1)
    hl = out.view(-1, 2).cpu().numpy()
    got = (hl[:, 0].astype(np.float64) + hl[:, 1]).reshape(n, n)
    dom = oracle.Domain.build(n)
    want = oracle.diffusion_run(u0.astype(np.float64), steps, A, dom, kappa.astype(np.float64))
    assert rel_err(got, want, dom.mask)[0] <= 1e-12
    cover = block_cover(n)
    assert np.all(got[cover & ~dom.mask] == 0) and np.all(got[~cover] == -10.0)
    assert torch.equal(tr1[:rf * steps], tr2[:rf * steps])
    assert torch.equal(tr2[rf * steps:], tr3[:rf])
    assert not torch.equal(tr2[:rf], tr2[rf * steps:])


def test_fused_gradient_path_validation(fr):
    with pytest.raises(fr.FractalError):
        fr.fractal_kappa_fused_limits(3)                                    # below the fused path's levels
    plan = fr.fractal_map(8, 8)
    rf, ms = fr.fractal_kappa_fused_limits(8)
    x = torch.zeros(2 * 256 * 256, device="cuda")
    y = torch.zeros_like(x)
    kap = torch.zeros(256 * 256, device="cuda")
    tr = torch.zeros(rf * (ms + 1), device="cuda")
    with pytest.raises(fr.FractalError):
        fr.fractal_kappa_trajectory_df(plan, x, y, tr, kap, A, ms + 1)      # more steps than one launch takes
    with pytest.raises(fr.FractalError):
        fr.fractal_kappa_trajectory_df(plan, x, x, tr, kap, A, 2)           # in == out
    with pytest.raises(fr.FractalError):
        fr.fractal_kappa_trajectory_df(plan, x, None, None, kap, A, 2)      # nowhere to write
    with pytest.raises(fr.FractalError):
        fr.fractal_kappa_gradient_df(plan, tr, tr, x, A, 2)                 # the two records alias
    fr.fractal_kappa_trajectory_df(plan, x, y, tr, kap, A, ms)


@pytest.mark.parametrize("k,steps,every", [(8, 45, 20), (7, 70, 40)])
def test_fused_and_single_step_gradients_agree(fr, k, steps, every):
    """The fused double-float path (several steps per launch, recorded
    trajectories; every = 40 takes two launches per segment) and the
    single-step path give the same gradients within the double-float
    rounding, both within 1e-4 of the FP64 adjoint."""
    n = 1 << k
    u0, kappa, target = fields(k, 90 + k)
    dom = oracle.Domain.build(n)
    from paper_2004_13475_gb300.autograd import diffusion_kappa
    res = []
    for fused in (True, False):
        u = dev(u0).requires_grad_(True)
        kp = dev(kappa).requires_grad_(True)
        loss = ((diffusion_kappa(u, kp, k, A, steps, every, 0, "df", fused) - dev(target)) ** 2).sum()
        loss.backward()
        res.append((u.grad.cpu().numpy().reshape(n, n), kp.grad.cpu().numpy().reshape(n, n)))
    _, wu, wk = oracle.diffusion_loss_gradients(dom, dom.take(u0).astype(np.float64),
                                                dom.take(kappa).astype(np.float64),
                                                dom.take(target).astype(np.float64), steps, A)
    for gu, gk in res:
        assert rel_err(gu, dom.put(wu, np.float64), dom.mask)[0] <= 1e-4
        assert rel_err(gk, dom.put(wk, np.float64), dom.mask)[0] <= 1e-4
    assert rel_err(res[0][0], res[1][0].astype(np.float64), dom.mask)[0] <= 1e-6
    assert rel_err(res[0][1], res[1][1].astype(np.float64), dom.mask)[0] <= 1e-6


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k,steps", [(5, 13), (9, 20)])
def test_fused_trajectory_float32_formats(fr, k, steps, mode):
    """A float32 input enters as the pairs (x, 0) and a float32 result is
    hi + lo rounded to float: the float32 forms of the fused launch give, bit
    for bit, the double-float launch on the converted input (records
    included) and the float sum of its result; a float32 result writes every
    cell of every member block and nothing else."""
    n = 1 << k
    u0, kappa, _ = fields(k, 70 + k)
    plan = fr.fractal_map(k, 8, mode)
    rf, _ = fr.fractal_kappa_fused_limits(k, mode)
    kap = dev(kappa)
    x32 = dev(u0)
    out_df = torch.zeros(2 * n * n, device="cuda")
    tr_df = torch.zeros(rf * (steps + 1), device="cuda")
    fr.fractal_kappa_trajectory_df(plan, _df(u0), out_df, tr_df, kap, A, steps)
    out_a = torch.zeros_like(out_df)
    tr_a = torch.zeros_like(tr_df)
    fr.fractal_kappa_trajectory_df_io(plan, x32, fr.FRACTAL_F32, out_a, fr.FRACTAL_DF, tr_a, kap, A, steps)
    assert torch.equal(out_a, out_df) and torch.equal(tr_a, tr_df)
    out_b = torch.full((n * n,), -7.0, device="cuda")
    fr.fractal_kappa_trajectory_df_io(plan, x32, fr.FRACTAL_F32, out_b, fr.FRACTAL_F32, None, kap, A, steps)
    hl = out_df.view(-1, 2)
    cover = torch.from_numpy(block_cover(n).reshape(-1)).cuda()
    assert torch.equal(out_b[cover], (hl[:, 0] + hl[:, 1])[cover])
    assert bool((out_b[~cover] == -7.0).all())
    out_c = torch.zeros(n * n, device="cuda")
    fr.fractal_kappa_trajectory_df_io(plan, _df(u0), fr.FRACTAL_DF, out_c, fr.FRACTAL_F32, None, kap, A, steps)
    assert torch.equal(out_c[cover], out_b[cover])
    with pytest.raises(fr.FractalError):
        fr.fractal_kappa_trajectory_df_io(plan, x32, 0, out_c, fr.FRACTAL_F32, None, kap, A, steps)  # uint8 format


@pytest.mark.parametrize("k,steps,every", [(8, 45, 20), (7, 70, 40)])
def test_fused_gradients_float32_and_float64_inputs_agree(fr, k, steps, every):
    """The fused path with float32 u0 and dJ/du_T read and written by the
    kernels as float32 gives the same u_T and gradients, bit for bit after
    rounding to float32, as the same path with float64 inputs (converted to
    double-float pairs around the kernels): the conversions moved into the
    kernels change no value."""
    n = 1 << k
    u0, kappa, target = fields(k, 110 + k)
    from paper_2004_13475_gb300.autograd import diffusion_kappa
    res = []
    g = None
    for dt in (torch.float32, torch.float64):
        u = dev(u0).to(dt).requires_grad_(True)
        kp = dev(kappa).requires_grad_(True)
        uT = diffusion_kappa(u, kp, k, A, steps, every)
        if g is None:  # one float32 dJ/du_T for both runs
            g = dev(target) - uT.detach()
        uT.backward(g.to(dt))
        res.append((uT.detach().float(), u.grad.float(), kp.grad.float()))
    for x32, x64 in zip(res[0], res[1]):
        assert torch.equal(x32, x64)
    mask = torch.from_numpy(oracle.member_mask(n).reshape(-1)).cuda()
    assert bool((res[0][0][~mask] == 0).all()) and bool((res[0][1][~mask] == 0).all())


@pytest.mark.parametrize("mode", [0, 1])
def test_gradient_pass_start_and_float32_result(fr, mode):
    """The dJ/dkappa pass started from 0 (its buffer not read) equals the pass
    added to a cleared buffer, and its float32 result is the float sum hi + lo
    of the double-float one, bit for bit, with every cell of every member
    block written and no other cell."""
    k, steps = 8, 12
    n = 1 << k
    u0, kappa, target = fields(k, 130)
    plan = fr.fractal_map(k, 8, mode)
    rf, _ = fr.fractal_kappa_fused_limits(k, mode)
    kap = dev(kappa)
    ut = torch.zeros(rf * (steps + 1), device="cuda")
    pt = torch.zeros(rf * steps, device="cuda")
    fr.fractal_kappa_trajectory_df(plan, _df(u0), None, ut, kap, A, steps - 1)
    fr.fractal_kappa_trajectory_df(plan, _df(target), None, pt, kap, A, steps - 1)
    g_acc = torch.zeros(2 * n * n, device="cuda")
    fr.fractal_kappa_gradient_df(plan, ut, pt, g_acc, A, steps)
    g_new = torch.full_like(g_acc, float("nan"))
    fr.fractal_kappa_gradient_df_io(plan, ut, pt, g_new, False, None, A, steps)
    cover = torch.from_numpy(block_cover(n).reshape(-1)).cuda()
    cover2 = cover.repeat_interleave(2)
    assert torch.equal(g_new[cover2], g_acc[cover2])
    g32 = torch.full((n * n,), -3.0, device="cuda")
    fr.fractal_kappa_gradient_df_io(plan, ut, pt, None, False, g32, A, steps)
    hl = g_acc.view(-1, 2)
    assert torch.equal(g32[cover], (hl[:, 0] + hl[:, 1])[cover]) and bool((g32[~cover] == -3.0).all())
    g_twice = g_acc.clone()
    fr.fractal_kappa_gradient_df_io(plan, ut, pt, g_twice, True, g32, A, steps)     # 2x the sum, into g32
    assert torch.equal(g_twice, g_acc)                                               # gkappa not written
    with pytest.raises(fr.FractalError):
        fr.fractal_kappa_gradient_df_io(plan, ut, pt, None, True, g32, A, steps)    # nothing to add to
    with pytest.raises(fr.FractalError):
        fr.fractal_kappa_gradient_df_io(plan, ut, pt, None, False, None, A, steps)  # nowhere to write


def test_fused_gradients_float64_kappa(fr):
    """A float64 kappa takes the double-float dJ/dkappa sum through a cleared
    buffer and the torch conversion; rounded to float32 it equals the float32
    kappa's result, which the last gradient pass writes as float32 itself."""
    k, steps, every = 8, 45, 20
    u0, kappa, target = fields(k, 150)
    from paper_2004_13475_gb300.autograd import diffusion_kappa
    res = []
    for dt in (torch.float32, torch.float64):
        u = dev(u0).requires_grad_(True)
        kp = dev(kappa).to(dt).requires_grad_(True)
        loss = ((diffusion_kappa(u, kp, k, A, steps, every) - dev(target)) ** 2).sum()
        loss.backward()
        assert kp.grad.dtype == dt
        res.append((u.grad.clone(), kp.grad.float()))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
