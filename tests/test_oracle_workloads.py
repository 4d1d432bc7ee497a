"""Pins for the oracle's workloads: CA (B3/S23), FP64 diffusion, reduce, single write."""
import math

import numpy as np
import pytest
import scipy.signal
import scipy.sparse
import scipy.sparse.csgraph

import oracle
import synth
from conftest import read_golden


def _cells(tok):
    if tok.strip() == "-":
        return set()
    return {tuple(int(v) for v in c.split(",")) for c in tok.split()}


# ---------------------------------------------------------------- CA ----------

def test_ca_hand_cases():
    for line in read_golden("ca_hand_cases.txt"):
        head, before, after = line.split("|")
        _, k, steps = head.split()
        n = 1 << int(k)
        state = np.zeros((n, n), dtype=np.uint8)
        for x, y in _cells(before):
            state[y, x] = 1
        out = oracle.ca_run(state, int(steps))
        got = {(int(x), int(y)) for y, x in zip(*np.nonzero(out))}
        assert got == _cells(after), head


def test_ca_all_dead_stays_dead():
    out = oracle.ca_run(np.zeros((32, 32), dtype=np.uint8), 5)
    assert not out.any()


def _plain_life_masked(state, mask, steps):
    # Special case that reduces to a library routine: because absent cells are
    # always dead, counting live member neighbours equals counting live cells
    # in plain Life (scipy 2-D convolution, zero boundary); the gasket rule is
    # then plain B3/S23 with non-members forced dead.
    kernel = np.ones((3, 3), dtype=np.int64)
    kernel[1, 1] = 0
    s = (state != 0).astype(np.int64) * mask
    for _ in range(steps):
        cnt = scipy.signal.convolve2d(s, kernel, mode="same", boundary="fill", fillvalue=0)
        s = (((cnt == 3) | ((s == 1) & (cnt == 2))) & mask).astype(np.int64)
    return s.astype(np.uint8)


@pytest.mark.parametrize("k,seed", [(4, 0), (5, 1), (6, 2), (7, 3)])
def test_ca_matches_masked_plain_life(k, seed):
    n = 1 << k
    state = synth.bernoulli_u8(seed, n)     # non-members hold noise: must be ignored
    mask = oracle.member_mask(n)
    for steps in (1, 2, 5, 12):
        assert np.array_equal(oracle.ca_run(state, steps), _plain_life_masked(state, mask, steps))


def test_ca_window_light_cone():
    # A window is exact at cells farther than `steps` from its inner edges
    # (information moves one cell per step) — used for full-size sampling.
    n, steps = 256, 6
    state = synth.bernoulli_u8(11, n)
    full = oracle.ca_run(state, steps)
    x0, y0, w, h = 40, 0, 70, 64       # top edge is the array edge
    dom = oracle.Domain.build(n, x0, y0, w, h)
    win = oracle.ca_run(state[y0:y0 + h, x0:x0 + w], steps, dom)
    inner = win[0:h - steps, steps:w - steps]
    assert np.array_equal(inner, full[y0:y0 + h - steps, x0 + steps:x0 + w - steps])


# --------------------------------------------------------- diffusion ---------

def test_diffusion_hand_case_k1():
    rows = [list(map(float, r.split())) for r in read_golden("diffusion_k1.txt")]
    u = np.zeros((2, 2))
    u[0, 0], u[0, 1], u[1, 0] = rows[0][1], rows[0][2], rows[0][3]   # [y, x]
    for step, u00, u10, u01 in rows[1:]:
        out = oracle.diffusion_run(u, int(step), 0.2)
        assert out[0, 0] == pytest.approx(u00, abs=1e-15)
        assert out[0, 1] == pytest.approx(u10, abs=1e-15)
        assert out[1, 0] == pytest.approx(u01, abs=1e-15)
        assert out[1, 1] == 0.0


@pytest.mark.parametrize("k", [3, 6, 8])
def test_diffusion_conserves_heat(k):
    n = 1 << k
    u0 = synth.uniform_f32(5, n).astype(np.float64)
    mask = oracle.member_mask(n)
    out = oracle.diffusion_run(u0, 50, 0.2)
    assert math.isclose(out.sum(), u0[mask].sum(), rel_tol=1e-12)
    assert (out[~mask] == 0).all()
    assert out.min() >= 0.0        # a * max degree (3) < 1 keeps the update positive


def test_diffusion_constant_is_fixed_point():
    n = 64
    mask = oracle.member_mask(n)
    out = oracle.diffusion_run(np.full((n, n), 0.625), 20, 0.2)
    assert np.all(out[mask] == 0.625)


def _laplacian(n):
    # Graph Laplacian of the gasket's 4-neighbour graph, built from brute-force
    # pairs of member cells at Manhattan distance 1 (scipy's csgraph routine).
    mask = oracle.member_mask(n)
    idx = -np.ones((n, n), dtype=np.int64)
    ys, xs = np.nonzero(mask)
    idx[ys, xs] = np.arange(ys.size)
    rows, cols = [], []
    for a, (y, x) in enumerate(zip(ys, xs)):
        for dy, dx in ((0, 1), (1, 0)):
            yy, xx = y + dy, x + dx
            if yy < n and xx < n and mask[yy, xx]:
                rows += [a, idx[yy, xx]]
                cols += [idx[yy, xx], a]
    adj = scipy.sparse.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(ys.size,) * 2)
    return scipy.sparse.csgraph.laplacian(adj.tocsr()).toarray(), ys, xs


@pytest.mark.parametrize("k", [2, 4, 5])
def test_diffusion_equals_graph_laplacian_powers(k):
    n = 1 << k
    L, ys, xs = _laplacian(n)
    u0 = synth.uniform_f32(9, n).astype(np.float64)
    step = np.eye(L.shape[0]) - 0.2 * L
    ref = np.linalg.matrix_power(step, 10) @ u0[ys, xs]
    out = oracle.diffusion_run(u0, 10, 0.2)
    np.testing.assert_allclose(out[ys, xs], ref, rtol=1e-12, atol=1e-14)


def test_diffusion_converges_to_mean():
    # The gasket's 4-neighbour graph is connected, so the explicit scheme
    # (stable for a * max degree < 1) relaxes to the mean of the start field.
    n = 8
    u0 = synth.uniform_f32(4, n).astype(np.float64)
    mask = oracle.member_mask(n)
    out = oracle.diffusion_run(u0, 4000, 0.2)
    np.testing.assert_allclose(out[mask], u0[mask].mean(), rtol=1e-9)


def test_diffusion_operator_is_symmetric():
    n = 32
    dom = oracle.Domain.build(n)
    v = synth.uniform_f32(1, n).astype(np.float64)[dom.cy, dom.cx]
    w = synth.uniform_f32(2, n).astype(np.float64)[dom.cy, dom.cx]
    kap = synth.uniform_f32(3, n, lo=0.5).astype(np.float64)[dom.cy, dom.cx]
    for kappa in (None, kap):
        Sv = oracle.diffusion_step(dom, v, 0.2, kappa)
        Sw = oracle.diffusion_step(dom, w, 0.2, kappa)
        assert math.isclose(v @ Sw, Sv @ w, rel_tol=1e-13)


def test_diffusion_kappa_one_is_plain_and_conserves():
    n = 64
    dom = oracle.Domain.build(n)
    u = synth.uniform_f32(1, n).astype(np.float64)[dom.cy, dom.cx]
    ones = np.ones(dom.m)
    assert np.array_equal(oracle.diffusion_step(dom, u, 0.2, ones), oracle.diffusion_step(dom, u, 0.2))
    kap = synth.uniform_f32(3, n, lo=0.5).astype(np.float64)[dom.cy, dom.cx]
    out = oracle.diffusion_step(dom, u, 0.2, kap)
    assert math.isclose(out.sum(), u.sum(), rel_tol=1e-13)


def test_diffusion_window_light_cone():
    n, steps = 256, 7
    u0 = synth.uniform_f32(13, n).astype(np.float64)
    full = oracle.diffusion_run(u0, steps, 0.2)
    x0, y0, w, h = 0, 100, 50, 60        # left edge is the array edge
    dom = oracle.Domain.build(n, x0, y0, w, h)
    win = oracle.diffusion_run(u0[y0:y0 + h, x0:x0 + w], steps, 0.2, dom)
    np.testing.assert_array_equal(win[steps:h - steps, 0:w - steps],
                                  full[y0 + steps:y0 + h - steps, 0:w - steps])


# ------------------------------------------------------- reduce / SW ---------

@pytest.mark.parametrize("k", [0, 1, 5, 10])
def test_reduce_of_single_write_is_volume(k):
    n = 1 << k
    sw = oracle.sw_write(n, 1.0)
    assert oracle.reduce_sum(sw[oracle.member_mask(n)]) == 3 ** k
    assert sw.sum() == 3 ** k


def test_reduce_matches_exactly_rounded_sum():
    n = 256
    u = synth.uniform_f32(21, n)
    vals = u[oracle.member_mask(n)]
    assert math.isclose(oracle.reduce_sum(vals), math.fsum(vals.astype(np.float64)), rel_tol=1e-14)
