"""Pins for the oracle's diffusion gradients (discrete adjoint).

The adjoint is checked against things it does not use: central finite
differences of the loss in FP64, the step it transposes, and special cases
with a known answer."""
import numpy as np
import pytest

import oracle
import synth


def _problem(k, seed, kappa_lo=0.5):
    n = 1 << k
    dom = oracle.Domain.build(n)
    u0 = dom.take(synth.uniform_f32(seed, n)).astype(np.float64)
    kappa = kappa_lo + dom.take(synth.uniform_f32(seed + 1, n)).astype(np.float64)
    target = dom.take(synth.uniform_f32(seed + 2, n)).astype(np.float64)
    return dom, u0, kappa, target


def _loss(dom, u0, kappa, target, steps, a):
    u = u0.copy()
    for _ in range(steps):
        u = oracle.diffusion_step(dom, u, a, kappa)
    return float(np.sum((u - target) ** 2))


@pytest.mark.parametrize("k,steps", [(3, 1), (4, 6), (5, 11)])
def test_matrix_is_the_step(k, steps):
    dom, u0, kappa, _ = _problem(k, 3)
    A = oracle.diffusion_matrix(dom, 0.2, kappa)
    assert np.allclose(A @ u0, oracle.diffusion_step(dom, u0, 0.2, kappa), rtol=0, atol=1e-15)
    A1 = oracle.diffusion_matrix(dom, 0.2)
    assert np.allclose(A1 @ u0, oracle.diffusion_step(dom, u0, 0.2), rtol=0, atol=1e-15)
    # the conductance (kappa_c + kappa_nb) / 2 is symmetric, so is A; columns sum to 1 (conservation)
    assert abs(A - A.T).max() == 0.0
    assert np.allclose(np.asarray(A.sum(axis=0)).reshape(-1), 1.0, atol=1e-15)


@pytest.mark.parametrize("k,steps,seed", [(4, 5, 11), (5, 9, 12), (6, 4, 13)])
def test_gradients_match_central_differences(k, steps, seed):
    dom, u0, kappa, target = _problem(k, seed)
    a = 0.2
    J, gu, gk = oracle.diffusion_loss_gradients(dom, u0, kappa, target, steps, a)
    assert J == pytest.approx(_loss(dom, u0, kappa, target, steps, a), rel=1e-14)
    rng = np.random.default_rng(seed)
    h = 1e-5
    for c in rng.choice(dom.m, size=8, replace=False):
        e = np.zeros(dom.m)
        e[c] = h
        fd_u = (_loss(dom, u0 + e, kappa, target, steps, a) - _loss(dom, u0 - e, kappa, target, steps, a)) / (2 * h)
        fd_k = (_loss(dom, u0, kappa + e, target, steps, a) - _loss(dom, u0, kappa - e, target, steps, a)) / (2 * h)
        assert gu[c] == pytest.approx(fd_u, rel=1e-6, abs=1e-9)
        assert gk[c] == pytest.approx(fd_k, rel=1e-6, abs=1e-9)


def test_directional_derivative():
    # dJ along a random direction (u0 and kappa together) equals <grad, direction>
    dom, u0, kappa, target = _problem(5, 21)
    a, steps = 0.2, 8
    _, gu, gk = oracle.diffusion_loss_gradients(dom, u0, kappa, target, steps, a)
    rng = np.random.default_rng(5)
    du, dk = rng.standard_normal(dom.m), rng.standard_normal(dom.m)
    h = 1e-6
    fd = (_loss(dom, u0 + h * du, kappa + h * dk, target, steps, a)
          - _loss(dom, u0 - h * du, kappa - h * dk, target, steps, a)) / (2 * h)
    assert float(gu @ du + gk @ dk) == pytest.approx(fd, rel=1e-7)


def test_special_cases():
    dom, u0, kappa, target = _problem(4, 31)
    # no steps: dJ/du0 = 2 (u0 - target), no dependence on kappa
    J, gu, gk = oracle.diffusion_loss_gradients(dom, u0, kappa, target, 0, 0.2)
    assert np.array_equal(gu, 2 * (u0 - target)) and not gk.any()
    # a constant field never moves: no flux, so kappa has no effect (up to the
    # rounding of the diagonal 1 - a * sum g)
    c = np.full(dom.m, 0.7)
    _, gu, gk = oracle.diffusion_loss_gradients(dom, c, kappa, target, 5, 0.2)
    assert np.abs(gk).max() < 1e-15
    # a = 0: the identity, dJ/du0 = 2 (u0 - target)
    _, gu, gk = oracle.diffusion_loss_gradients(dom, u0, kappa, target, 4, 0.0)
    assert np.array_equal(gu, 2 * (u0 - target)) and not gk.any()
    # kappa = 1 everywhere: the same step as the conductivity-free one
    one = np.ones(dom.m)
    assert np.array_equal(oracle.diffusion_step(dom, u0, 0.2, one), oracle.diffusion_step(dom, u0, 0.2))


def test_gradient_of_a_windowed_domain_is_exact_far_from_its_edges():
    # What the full-size GPU test relies on: a window of the array reproduces
    # the whole-array gradient at cells farther than 2 * steps from its edges.
    k, steps = 7, 6
    n = 1 << k
    full = oracle.Domain.build(n)
    U = synth.uniform_f32(41, n).astype(np.float64)
    K = 0.5 + synth.uniform_f32(42, n).astype(np.float64)
    G = synth.uniform_f32(43, n).astype(np.float64)
    _, gu, gk = oracle.diffusion_loss_gradients(full, full.take(U), full.take(K), full.take(G), steps, 0.2)
    GU, GK = full.put(gu, np.float64), full.put(gk, np.float64)
    x0, y0, w = 16, 0, 48
    win = oracle.Domain.build(n, x0, y0, w, w)
    _, wu, wk = oracle.diffusion_loss_gradients(win, win.take(U[y0:y0 + w, x0:x0 + w]),
                                                win.take(K[y0:y0 + w, x0:x0 + w]),
                                                win.take(G[y0:y0 + w, x0:x0 + w]), steps, 0.2)
    WU, WK = win.put(wu, np.float64), win.put(wk, np.float64)
    r = 2 * steps + 1
    sl = (slice(r, w - r), slice(r, w - r))        # y0 = 0 is the array edge, exact too
    assert np.allclose(WU[sl], GU[y0:y0 + w, x0:x0 + w][sl], rtol=1e-12, atol=1e-14)
    assert np.allclose(WK[sl], GK[y0:y0 + w, x0:x0 + w][sl], rtol=1e-12, atol=1e-14)
