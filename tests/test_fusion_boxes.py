"""The geometric fact behind temporal fusion (several steps per launch).

A CTA that advances its member super-tile (side T, T a power of two) by s
steps needs every gasket cell that can influence it within s steps.  Non-member
cells never change and hold 0, so influence travels only along chains of
member cells: s moves of the step's neighbourhood (4 neighbours for the
diffusion, 8 for the automaton).  Besides its member tiles, a fused kernel
stages four margin boxes of width M >= s (super-tile coordinates):

  diffusion (4 neighbours)
    left   [-M, 0) x [0, M)        top    [0, M) x [-M, 0)
    right  [T, T+M) x [-M, M)      bottom [-M, M) x [T, T+M)
  automaton (8 neighbours): the same, but the right box spans rows [-M, M]
    and the bottom box columns [-M, M] (the corner cells (T-1, 0) and (0, T-1)
    reach one row or column further diagonally)

This file checks, by breadth-first search over member cells from every member
super-tile of small gaskets, that for M <= T/2 every member reached in M moves
outside the super-tile lies in one of the boxes, and that each box is needed.
The kernels fuse s <= M <= T/2 steps.
"""
import numpy as np
import pytest

import oracle


def _boxes(T, M, nb):
    e = 1 if nb == 8 else 0      # the automaton's boxes reach one row / column further
    return [(-M, 0, 0, M), (0, M, -M, 0), (T, T + M, -M, M + e), (-M, M + e, T, T + M)]   # x0, x1, y0, y1


def _moves(nb):
    m = [(0, 1), (0, -1), (1, 0), (-1, 0)]
    return m + [(1, 1), (1, -1), (-1, 1), (-1, -1)] if nb == 8 else m


def _check(k, t, M, nb):
    n = 1 << k
    T = 1 << t
    mem = oracle.member_mask(n)
    g = M + 1                                        # padding: a guard ring beyond the reach
    pad = np.zeros((n + 2 * g, n + 2 * g), dtype=bool)
    pad[g:g + n, g:g + n] = mem
    used = [False] * 4
    for sy in range(n // T):
        for sx in range(n // T):
            if sx & sy:
                continue
            ox, oy = sx * T, sy * T
            win = pad[oy:oy + T + 2 * g, ox:ox + T + 2 * g]
            reach = np.zeros_like(win)
            reach[g:g + T, g:g + T] = win[g:g + T, g:g + T]
            for _ in range(M):                       # M moves along member cells
                nxt = reach.copy()
                for dy, dx in _moves(nb):
                    nxt |= np.roll(np.roll(reach, dy, 0), dx, 1)
                reach = nxt & win
            reach[g:g + T, g:g + T] = False
            ys, xs = np.nonzero(reach)
            for y, x in zip(ys - g, xs - g):         # super-tile coordinates
                hit = [b for b, (x0, x1, y0, y1) in enumerate(_boxes(T, M, nb))
                       if x0 <= x < x1 and y0 <= y < y1]
                assert hit, (k, T, M, nb, sx, sy, x, y)
                for b in hit:
                    used[b] = True
    return used


@pytest.mark.parametrize("nb", [4, 8])
@pytest.mark.parametrize("k,t", [(6, 2), (6, 3), (7, 3), (7, 4), (8, 4), (8, 5), (9, 5), (8, 6)])
def test_margin_boxes_hold_every_reachable_member(k, t, nb):
    T = 1 << t
    used = [False] * 4
    for M in sorted({1, 2, 4, T // 4, T // 2} - {0}):
        if M > T // 2:
            continue
        u = _check(k, t, M, nb)
        used = [a or b for a, b in zip(used, u)]
    assert all(used)     # each box is needed somewhere


@pytest.mark.parametrize("nb", [4, 8])
def test_margin_bound_is_sharp(nb):
    # The kernels fuse at most T/2 steps; the boxes actually hold up to M = T
    # (4 neighbours) or T - 1 (8 neighbours) and no further: one more move
    # reaches the member (-1, -T) of the super-tile above-left.
    T = 8
    for M in range(T // 2, T if nb == 8 else T + 1):
        _check(8, 3, M, nb)
    with pytest.raises(AssertionError):
        _check(8, 3, T if nb == 8 else T + 1, nb)


def test_automaton_needs_the_wider_boxes():
    # The diffusion's boxes are too small for 8 neighbours: the member (T, M)
    # is M diagonal moves from the corner (T-1, 0).
    T, M = 8, 2
    n = 1 << 6
    assert oracle.is_member(n, T, M) and oracle.is_member(n, T - 1, 0)
    assert not any(x0 <= T < x1 and y0 <= M < y1 for x0, x1, y0, y1 in _boxes(T, M, 4))
    assert any(x0 <= T < x1 and y0 <= M < y1 for x0, x1, y0, y1 in _boxes(T, M, 8))


def _active_box_blocks(k, T, M):
    """Member 8 x 8 blocks in the 4-neighbour margin boxes of every member super-tile."""
    nblk = (1 << k) // 8
    s = (1 << k) // T
    sy, sx = np.nonzero((np.arange(s)[None, :] & np.arange(s)[:, None]) == 0)
    OX, OY = sx * (T // 8), sy * (T // 8)
    W, side = M // 8, T // 8
    boxes = [(-W, 0, 0, W), (0, W, -W, 0), (side, side + W, -W, W), (-W, W, side, side + W)]
    cnt = np.zeros(sx.size, dtype=np.int64)
    for x0, x1, y0, y1 in boxes:
        for by in range(y0, y1):
            for bx in range(x0, x1):
                gx, gy = OX + bx, OY + by
                cnt += (gx >= 0) & (gx < nblk) & (gy >= 0) & (gy < nblk) & ((gx & gy) == 0)
    return cnt


@pytest.mark.parametrize("M", [8, 16, 32, 64, 128])
def test_member_blocks_of_the_boxes_are_few(M):
    # The fused diffusion gives a thread only to the member blocks of the
    # margin boxes: at most 3 * 3^log2(M/8) of the 6 (M/8)^2 (a gasket
    # fragment of side M at each of the three contacts).  Every member
    # super-tile position of the largest array is checked.
    W = M // 8
    cap = 3 * 3 ** int(np.log2(W))
    for t in range(4, 10):
        T = 1 << t
        if T < 2 * M:
            continue
        cnt = _active_box_blocks(16, T, M)
        assert cnt.max() <= cap, (T, M, cnt.max())
        assert cnt.max() == cap           # and the bound is reached


@pytest.mark.parametrize("k", range(2, 13))
def test_member_cells_have_at_most_five_member_neighbours(k):
    """The fused automaton sums the nine-cell neighbourhood modulo 4.  That
    decides B3/S23 on the gasket because no member cell has more than five
    member neighbours (non-members hold 0 for ever), so the nine-cell sum is at
    most 6 and its residue mod 4 separates 3 (alive next) and 4 (alive next if
    alive now) from every other value.  Brute-force count of member neighbours
    of every member cell of the level-k gasket; five occurs (from level 3 on),
    six never."""
    n = 1 << k
    m = oracle.member_mask(n).astype(np.int32)
    p = np.pad(m, 1)
    count = sum(p[1 + dy:1 + dy + n, 1 + dx:1 + dx + n]
                for dy in (-1, 0, 1) for dx in (-1, 0, 1) if (dx, dy) != (0, 0))
    assert count[m == 1].max() == (4 if k == 2 else 5)


def test_mod4_rule_matches_b3s23_for_sums_up_to_six():
    """The residue form of the rule, for every neighbour count 0..5 and state:
    alive next iff m == 3, or m == 0 and alive now, m = (count + self) mod 4."""
    for count in range(6):
        for self_ in (0, 1):
            m = (count + self_) % 4
            assert (m == 3 or (m == 0 and self_ == 1)) == (count == 3 or (count == 2 and self_ == 1))


def _automaton_tasks(T, M):
    """The fused automaton's staging layout (word column c, first row y0,
    rows) in super-tile coordinates: every member 32 x 32 word tile of the
    super-tile, then the seven box pieces, with the margin rounded up to a
    multiple of 8 (ME8) and the right box reaching rows [-ME8, ME8 + 8)."""
    ws = T // 32
    tasks = [(tx, 32 * ty, 32) for ty in range(ws) for tx in range(ws) if (tx & ty) == 0]
    ME8 = (M + 7) // 8 * 8
    right = 2 * ME8 + 8
    tasks += [(-1, 0, ME8), (0, -ME8, ME8), (ws, -ME8, min(right, 32)), (ws, -ME8 + 32, min(max(right - 32, 0), 32)),
              (ws, -ME8 + 64, max(right - 64, 0)), (-1, T, ME8), (0, T, ME8)]
    return tasks


@pytest.mark.parametrize("T", [32, 64, 128, 256, 512])
def test_automaton_staging_layout(T):
    """For every margin the fused automaton takes (1 <= M <= 31, 2 M <= T):
    each task starts on a row that is a multiple of 8 and has a multiple of 8
    rows (a lane keeps four rows as one 16-byte group, and lanes pair up
    within 8-row blocks); no word of the bit
    image is staged twice (each has one writer); the staged words hold the
    automaton's margin boxes; and the rows a lane reads (the 16-byte groups
    above and below its four, in its column and the two beside it) stay inside the image's
    word columns [-2, T/32 + 1] and rows [-36, T + 36)."""
    ws = T // 32
    for M in range(1, 32):
        if 2 * M > T:
            break
        staged = set()
        for c, y0, rows in _automaton_tasks(T, M):
            assert y0 % 8 == 0 and rows % 8 == 0 and 0 <= rows <= 32
            for y in range(y0, y0 + rows):
                assert (c, y) not in staged, (T, M, c, y)
                staged.add((c, y))
            if rows:
                assert -2 <= c - 1 and c + 1 <= ws + 1
                assert -36 <= y0 - 4 and y0 + rows + 4 <= T + 36
        for x0, x1, y0, y1 in _boxes(T, M, 8):
            for y in range(y0, y1):
                for x in (x0, x1 - 1):
                    assert (x // 32, y) in staged, (T, M, x, y)


@pytest.mark.parametrize("M", [1, 8, 25, 31])
def test_automaton_nine_cell_rule_on_the_staged_image(M):
    """The fused automaton's arithmetic on the bit image, emulated word by
    word on the host (row sums of three cells by funnel shifts and a full
    adder, the nine-cell sum modulo 4, births masked to members) over the
    staging layout above, for one launch of M steps at level 7 with
    super-tiles of side 64: equal to the oracle's automaton."""
    k, T = 7, 64
    n = 1 << k
    rng = np.random.default_rng(10 + M)
    mem = oracle.member_mask(n)
    state = ((rng.random((n, n)) < 0.5) & mem).astype(np.uint8)
    want = oracle.ca_run(state, M)
    mask32 = (1 << 32) - 1

    def word(a, x0, y):
        return sum(int(a[y, x0 + i]) << i for i in range(32)) if 0 <= y < n and 0 <= x0 < n else 0

    def members(x0, y):
        return word(mem, x0, y)

    def row_sum(l, w, r):
        a = ((w << 1) | (l >> 31)) & mask32
        c = ((w >> 1) | (r << 31)) & mask32
        return a ^ w ^ c, (a & w) | (c & (a ^ w))

    got = np.zeros_like(state)
    for sy in range(n // T):
        for sx in range(n // T):
            if sx & sy:
                continue
            ox, oy = sx * T, sy * T
            img, msk = {}, {}
            for c, y0, rows in _automaton_tasks(T, M):
                for y in range(y0, y0 + rows):
                    img[(c, y)] = word(state, ox + 32 * c, oy + y)
                    msk[(c, y)] = members(ox + 32 * c, oy + y)
            for _ in range(M):
                def at(c, y):
                    return img.get((c, y), 0)
                nxt = {}
                for (c, y), v in img.items():
                    us, uk = row_sum(at(c - 1, y - 1), at(c, y - 1), at(c + 1, y - 1))
                    ms, mk = row_sum(at(c - 1, y), v, at(c + 1, y))
                    ds, dk = row_sum(at(c - 1, y + 1), at(c, y + 1), at(c + 1, y + 1))
                    bit0 = us ^ ms ^ ds
                    k0 = (us & ms) | (ds & (us ^ ms))
                    bit1 = (uk ^ mk ^ dk ^ k0) & msk[(c, y)]
                    nxt[(c, y)] = ((bit0 & bit1) | (~bit0 & ~bit1 & v)) & mask32
                img = nxt
            for (c, y), v in img.items():
                if 0 <= c < T // 32 and 0 <= y < T:
                    got[oy + y, ox + 32 * c:ox + 32 * c + 32] = [(v >> i) & 1 for i in range(32)]
    assert np.array_equal(got, want)


def _box_block_distance(qx, qy, side):
    """Manhattan distance from the nearest cell of 8 x 8 block (qx, qy) to the
    super-tile [0, 8 side)^2 (block coordinates relative to the super-tile)."""
    def gap(q):
        return -8 * q - 7 if q < 0 else 8 * (q - side) + 1 if q >= side else 0
    return gap(qx) + gap(qy)


@pytest.mark.parametrize("T,M,reach", [(64, 32, 8), (64, 32, 9), (64, 32, 17), (64, 32, 20), (64, 32, 32), (128, 64, 50),
                                         (64, 16, 13)])
def test_diffusion_box_blocks_within_reach_suffice(T, M, reach):
    """The fused diffusion stages, besides its super-tile, only the member
    blocks of its margin boxes (width M) whose nearest cell lies within
    `reach` cells of the super-tile, and runs up to `reach` steps.  Emulated
    in float64 on the host: staged member cells take the step with their true
    member degree and read every member neighbour that is not staged as 0 (the
    kernel's zero port slot); after `reach` steps every cell of the super-tile
    equals the oracle's diffusion of the whole gasket."""
    k, a = 9, 0.2
    n = 1 << k
    rng = np.random.default_rng(T + M + reach)
    mem = oracle.member_mask(n)
    u0 = np.where(mem, rng.random((n, n)), 0.0)
    want = oracle.diffusion_run(u0, reach, a)
    side, W = T // 8, M // 8
    pad = 8 * (W + 1)
    big = n + 2 * pad
    memp = np.zeros((big, big), dtype=bool)
    memp[pad:pad + n, pad:pad + n] = mem
    deg = sum(np.roll(np.roll(memp, dy, 0), dx, 1) for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1))) * memp
    for sy in range(n // T):
        for sx in range(n // T):
            if sx & sy:
                continue
            staged = np.zeros((big, big), dtype=bool)
            oy, ox = pad + sy * T, pad + sx * T
            staged[oy:oy + T, ox:ox + T] = True
            for x0, x1, y0, y1 in _boxes(T, M, 4):
                for qy in range(y0 // 8, y1 // 8):
                    for qx in range(x0 // 8, x1 // 8):
                        if _box_block_distance(qx, qy, side) <= reach:
                            staged[oy + 8 * qy:oy + 8 * qy + 8, ox + 8 * qx:ox + 8 * qx + 8] = True
            staged &= memp
            u = np.zeros((big, big))
            u[pad:pad + n, pad:pad + n] = u0
            u = np.where(staged, u, 0.0)
            for _ in range(reach):
                nb = sum(np.roll(np.roll(u, dy, 0), dx, 1) for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1)))
                u = np.where(staged, u + a * (nb - deg * u), 0.0)
            got = u[oy:oy + T, ox:ox + T]
            ref = want[sy * T:(sy + 1) * T, sx * T:(sx + 1) * T]
            assert np.allclose(got, ref, rtol=0, atol=1e-12), (T, M, reach, sx, sy)
