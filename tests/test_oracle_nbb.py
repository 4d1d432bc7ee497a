"""CPU pins of the NBB-family oracle (oracle/nbb.py): membership against the
bottom-up construction of Sec. 3.1 and the counts of Sec. 3.2, the packed
grid of Lemma 2, lambda of Theorem 1 as a bijection onto the member blocks,
and the gasket special case against the gasket oracle."""
import numpy as np
import pytest

import oracle
from oracle import nbb

NAMES = nbb.names()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("r", [0, 1, 2, 3, 4])
def test_membership_digits_match_bottom_up_construction(name, r):
    assert np.array_equal(nbb.member_mask(name, r), nbb.member_mask_recursive(name, r))


@pytest.mark.parametrize("name", NAMES)
def test_member_counts_are_k_to_the_r(name):
    s, k, cells = nbb.FRACTALS[name]
    assert len(set(cells)) == k and all(0 <= x < s and 0 <= y < s for x, y in cells)
    for r in range(5):
        assert int(nbb.member_mask(name, r).sum()) == k ** r          # V = k^r (Sec. 3.1, Lemma 1)


def test_textbook_shapes():
    """Hand-checked features: the carpet's centre hole of side s**(r-1); the
    Vicsek plus holds the whole middle row and column; the X holds both
    diagonals; the H holds its left and right columns and its middle row."""
    r = 3
    c = nbb.member_mask("carpet", r)
    assert not c[9:18, 9:18].any() and c[0, :].all() and c[:, 0].all()
    v = nbb.member_mask("vicsek", r)
    assert v[13, :].all() and v[:, 13].all() and not v[0, 0]
    x = nbb.member_mask("xfractal", r)
    assert all(x[i, i] and x[i, 26 - i] for i in range(27)) and not x[0, 13]
    h = nbb.member_mask("hfractal", r)
    assert h[:, 0].all() and h[:, 26].all() and h[13, :].all() and not h[0, 13]


def test_gasket_case_is_the_gasket():
    for r in range(6):
        n = 1 << r
        assert np.array_equal(nbb.member_mask("gasket", r), oracle.member_mask(n))


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("r", [0, 1, 2, 3, 4, 5])
def test_lambda_is_a_bijection_onto_member_blocks(name, r):
    """Theorem 1: lambda maps the packed grid (Lemma 2: W * H = k^r) one to
    one onto the member blocks (brute force)."""
    s, k, _ = nbb.FRACTALS[name]
    if k ** r > 40000:
        pytest.skip("large case")
    W, H = nbb.grid_dims(k, r)
    assert W * H == k ** r and (W == H or W == k * H)
    tab = nbb.block_table(name, r).reshape(-1, 2)
    pts = {(int(x), int(y)) for x, y in tab}
    assert len(pts) == k ** r
    mask = nbb.member_mask(name, r)
    assert all(mask[y, x] for x, y in pts)


def test_generic_lambda_reproduces_the_gasket_map():
    """With the gasket's step cells in this library's numbering, the generic
    map is the gasket map of the gasket oracle, block for block."""
    for r in range(1, 8):
        W, H = oracle.grid_dims(r)
        for wy in range(H):
            for wx in range(W):
                assert nbb.lam("gasket", r, wx, wy) == oracle.lambda_canonical(wx, wy, r)


def test_single_write_field():
    f = nbb.sw_write("vicsek", 2, 1, 2.5)
    mask = nbb.member_mask("vicsek", 3)
    assert np.all(f[mask] == 2.5)
    assert np.isnan(f).sum() == 27 * 27 - 25 * 9               # outside the 25 member tiles of side 3
    assert np.count_nonzero(f == 0) == 25 * 9 - 125             # non-members of member tiles


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("r", [1, 2, 3])
def test_ca_step_matches_cell_by_cell_loops(name, r):
    s, _, _ = nbb.FRACTALS[name]
    n = s ** r
    rng = np.random.default_rng(7 + r)
    alive = (rng.random((n, n)) < 0.5).astype(np.uint8)
    assert np.array_equal(nbb.ca_step(name, r, alive), nbb.ca_step_loops(name, r, alive))


def test_ca_gasket_case_is_the_gasket_automaton():
    r = 6
    n = 1 << r
    rng = np.random.default_rng(3)
    alive = (rng.random((n, n)) < 0.5).astype(np.uint8)
    a = alive.copy()
    b = alive.copy()
    for _ in range(5):
        a = nbb.ca_step("gasket", r, a)
    b = oracle.ca_run(b, 5)
    assert np.array_equal(a, b.astype(np.uint8))


def test_ca_still_life_and_dead_field():
    """A 2 x 2 block of member cells is a still life (each of its cells has 3
    alive neighbours, no dead cell has 3); an all-dead field stays dead."""
    r = 3
    n = 27
    alive = np.zeros((n, n), dtype=np.uint8)
    alive[0:2, 2:4] = 1                                  # carpet cells (2,0), (3,0), (2,1), (3,1)
    assert nbb.member_mask("carpet", r)[0:2, 2:4].all()
    nxt = alive
    for _ in range(4):
        nxt = nbb.ca_step("carpet", r, nxt)
    assert np.array_equal(nxt, alive)
    assert not nbb.ca_step("vicsek", r, np.zeros((n, n), dtype=np.uint8)).any()


@pytest.mark.parametrize("name", NAMES)
def test_diffusion_conserves_heat_and_keeps_constants(name):
    """Zero-flux walls: the sum over the members is conserved; a constant
    field on the members is a fixed point."""
    s, _, _ = nbb.FRACTALS[name]
    r = 3
    n = s ** r
    mask = nbb.member_mask(name, r)
    rng = np.random.default_rng(5)
    u = rng.random((n, n))
    total = u[mask].sum()
    v = u
    for _ in range(20):
        v = nbb.diffusion_step(name, r, v, 0.2)
    assert abs(v[mask].sum() - total) <= 1e-12 * total
    c = nbb.diffusion_step(name, r, np.full((n, n), 2.5), 0.2)
    assert np.all(c[mask] == 2.5) and np.all(c[~mask] == 0)


def test_diffusion_gasket_case_is_the_gasket_step():
    r = 6
    n = 1 << r
    rng = np.random.default_rng(9)
    u = rng.random((n, n))
    dom = oracle.Domain.build(n)
    a = u
    for _ in range(5):
        a = nbb.diffusion_step("gasket", r, a, 0.2)
    b = oracle.diffusion_run(u, 5, 0.2, dom)
    mask = dom.mask
    assert np.allclose(a[mask], b[mask], rtol=0, atol=1e-14)


def test_diffusion_hand_example_vicsek_level_1():
    """Level 1 of the Vicsek plus: the centre (1,1) has four member neighbours,
    each arm cell one (the centre)."""
    u = np.zeros((3, 3))
    u[1, 1] = 1.0
    v = nbb.diffusion_step("vicsek", 1, u, 0.2)
    assert v[1, 1] == pytest.approx(1.0 - 4 * 0.2)
    for y, x in ((0, 1), (1, 0), (1, 2), (2, 1)):
        assert v[y, x] == pytest.approx(0.2)
    assert v[0, 0] == 0 and v[2, 2] == 0
