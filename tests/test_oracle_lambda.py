"""Pins for the oracle's block-space map lambda(omega) (Sec. 4 Theorem 1, Lemma 2, Sec. 6.1)."""
import math

import numpy as np
import pytest

import oracle
from conftest import read_golden


@pytest.mark.parametrize("r", range(0, 14))
def test_lemma2_grid(r):
    W, H = oracle.grid_dims(r)
    assert W * H == 3 ** r
    # Lemma 2's induction: even r grows the horizontal side, odd r the vertical.
    if r > 0:
        pW, pH = oracle.grid_dims(r - 1)
        if (r - 1) % 2 == 0:
            assert (W, H) == (3 * pW, pH)
        else:
            assert (W, H) == (pW, 3 * pH)


def test_arithmetic_hash_equals_table():
    # Sec. 6.1: the arithmetic hash gives the same replica offsets as H.
    for b in range(3):
        assert oracle.hash_arith(b) == oracle.hash_table(b)


def test_beta_digits():
    # beta_mu is base-3 digit ceil(mu/2)-1 of omega_x (odd mu) or omega_y (even mu).
    wx, wy = 2 + 1 * 3 + 0 * 9 + 2 * 27, 1 + 2 * 3 + 2 * 9
    assert [oracle.beta(mu, wx, wy) for mu in range(1, 8)] == [2, 1, 1, 2, 0, 2, 2]


def test_golden_rb2():
    rows = read_golden("lambda_rb2.txt")
    assert len(rows) == 9
    for line in rows:
        wx, wy, plx, ply, lx, ly = (int(t) for t in line.split())
        assert oracle.lambda_paper(wx, wy, 2) == (plx, ply)
        assert oracle.lambda_canonical(wx, wy, 2) == (lx, ly)


def test_worked_example_n64_rho8():
    # Fig. "thread vs block" caption: n = 64, |B| = 8 x 8 gives n_b = 8, i.e.
    # block level r_b = 3: 27 member blocks packed in a 9 x 3 grid.
    table = oracle.block_table(6, 8)
    assert table.shape == (3, 9, 2)
    blocks = {tuple(v) for v in table.reshape(-1, 2)}
    assert len(blocks) == 27
    assert blocks == {(x, y) for y in range(8) for x in range(8) if x & y == 0}


@pytest.mark.parametrize("k", range(0, 9))
def test_bijection_onto_member_blocks(k):
    # Theorem 1: the packed grid maps one-to-one onto the non-empty blocks.
    # Brute force for every block size rho <= n (k <= 8).
    for lg in range(0, k + 1):
        rho = 1 << lg
        rb = k - lg
        nb = 1 << rb
        table = oracle.block_table(k, rho).reshape(-1, 2)
        assert table.shape[0] == 3 ** rb
        got = {(int(x), int(y)) for x, y in table}
        assert len(got) == 3 ** rb, "lambda must not map two blocks to one"
        expect = {(x, y) for y in range(nb) for x in range(nb) if x & y == 0}
        assert got == expect


@pytest.mark.parametrize("r", range(0, 8))
def test_paper_orientation_lands_on_paper_gasket(r):
    # Without the flip, lambda must land on the paper's gasket, whose blocks
    # satisfy bx & (n_b - 1 - by) == 0 (the in-block test of Sec. 6.1 one level up).
    W, H = oracle.grid_dims(r)
    nb = 1 << r
    seen = set()
    for wy in range(H):
        for wx in range(W):
            bx, by = oracle.lambda_paper(wx, wy, r)
            assert bx & (nb - 1 - by) == 0
            seen.add((bx, by))
    assert len(seen) == 3 ** r


@pytest.mark.parametrize("r", range(1, 12))
def test_theorem2_parallel_space_ratio(r):
    # Theorem 2: bounding-box blocks over lambda blocks = n_b**2 / 3**r_b = (4/3)**r_b,
    # unbounded as n grows.
    W, H = oracle.grid_dims(r)
    assert math.isclose((1 << r) ** 2 / (W * H), (4 / 3) ** r, rel_tol=1e-12)


@pytest.mark.parametrize("r", [6, 7, 8, 9])
def test_packed_rectangles_are_level6_subgaskets(r):
    """The device pack kernel for narrow tiles relies on this: a 27 x 27
    rectangle of the packed grid aligned to multiples of 27 varies the low
    three base-3 digits of omega_x and omega_y, which are the digits of
    mu = 1..6, so (Theorem 1) its blocks are the level-6 gasket in one 64 x 64
    square whose corner is lambda of the high digits at level r - 6, shifted
    by six bits, and the block at (u mod 27, u div 27) of the rectangle is
    that corner plus lambda of (u mod 27, u div 27) at level 6."""
    W, H = oracle.grid_dims(r)
    local = [oracle.lambda_canonical(u % 27, u // 27, 6) for u in range(729)]
    assert sorted(local) == sorted((x, y) for y in range(64) for x in range(64) if (x & y) == 0)
    for gy in range(H // 27):
        for gx in range(W // 27):
            cx, cy = oracle.lambda_canonical(gx, gy, r - 6)
            for u in range(729):
                wx, wy = gx * 27 + u % 27, gy * 27 + u // 27
                lx, ly = local[u]
                assert oracle.lambda_canonical(wx, wy, r) == ((cx << 6) + lx, (cy << 6) + ly), (r, gx, gy, u)
