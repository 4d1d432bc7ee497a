"""Pins for the oracle's gasket membership and volume (Sec. 3.1 Eq. 2, Lemma 1)."""
import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden


@pytest.mark.parametrize("k", range(0, 12))
def test_volume_is_3_pow_k(k):
    # Eq. 2: an NBB fractal of scale level r holds k_replicas**r cells; the
    # gasket has 3 replicas, so level k has 3**k cells.
    assert oracle.n_members(k) == 3 ** k


@pytest.mark.parametrize("k", [3, 6, 9])
def test_hausdorff_volume(k):
    # Lemma 1: V = n**H with H = log2(3); exact in integers as n**log2(3) = 3**k.
    n = 1 << k
    assert round(n ** np.log2(3)) == oracle.n_members(k)


def test_pascal_triangle_mod_2():
    # Independent characterisation (Lucas' theorem): C(x + y, x) is odd iff
    # x & y == 0.  Build Pascal's triangle mod 2 by its additive recurrence and
    # read cell (x, y) from row x + y, column x.
    n = 64
    rows = [np.array([1], dtype=np.uint8)]
    for _ in range(2 * n):
        prev = rows[-1]
        nxt = np.zeros(prev.size + 1, dtype=np.uint8)
        nxt[:-1] ^= prev
        nxt[1:] ^= prev
        rows.append(nxt)
    pascal = np.zeros((n, n), dtype=bool)
    for y in range(n):
        for x in range(n):
            pascal[y, x] = rows[x + y][x] == 1
    assert np.array_equal(pascal, oracle.member_mask(n))


@pytest.mark.parametrize("rho", [1, 2, 4, 8, 16, 32, 64])
def test_block_times_bounding_subbox(rho):
    # Sec. 5.3 / 6.1: a cell lies in the gasket iff its rho-block is a member
    # block and its in-block offset passes the in-block test (in this
    # orientation t_x & t_y == 0).  Brute force on n = 64.
    n = 64
    full = oracle.member_mask(n)
    nb = n // rho
    for by in range(nb):
        for bx in range(nb):
            tile = full[by * rho:(by + 1) * rho, bx * rho:(bx + 1) * rho]
            ty, tx = np.mgrid[0:rho, 0:rho]
            expect = ((bx & by) == 0) & ((tx & ty) == 0)
            assert np.array_equal(tile, expect)


def test_paper_orientation_is_y_flip():
    # The paper's in-block test t_x & (b - 1 - t_y) == 0 (Sec. 6.1) describes
    # the same gasket with y flipped.
    n = 32
    ys, xs = np.mgrid[0:n, 0:n]
    paper = (xs & (n - 1 - ys)) == 0
    assert np.array_equal(paper[::-1, :], oracle.member_mask(n))


def test_windowed_mask_matches_whole():
    n = 128
    full = oracle.member_mask(n)
    win = oracle.member_mask(n, 37, 5, 60, 90)
    assert np.array_equal(win, full[5:95, 37:97])
    # windows may run off the array: those cells are absent
    edge = oracle.member_mask(n, 120, -3, 16, 8)
    assert not edge[:3].any() and not edge[:, 8:].any()
    assert np.array_equal(edge[3:, :8], full[0:5, 120:128])


def test_synth_reference_vectors():
    # Published SplitMix64 outputs (tests/golden/splitmix64.txt).
    for line in read_golden("splitmix64.txt"):
        seed, idx, val = (int(t) for t in line.split())
        got = int(synth.splitmix64(seed, np.array([idx], dtype=np.uint64))[0])
        assert got == val


def test_synth_window_consistency():
    n = 64
    full = synth.uniform_f32(7, n)
    assert np.array_equal(synth.uniform_f32(7, n, 10, 20, 30, 5), full[20:25, 10:40])
    bern = synth.bernoulli_u8(3, n)
    assert set(np.unique(bern)) <= {0, 1}
    assert 0.4 < bern.mean() < 0.6
    assert full.min() >= 0.0 and full.max() < 1.0
