"""Plain CPU oracle for other fractals of the NBB family (test infrastructure).

Test infrastructure only, like the rest of this package: only the tests,
``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may use it, and
it shares no code with the CUDA library.

An NBB fractal (Sec. 3.1) is built bottom-up: the level-(r+1) fractal is k
replicas of the level-r one, placed without overlap on an s x s grid of
cells of side s**r (the "NBB step", Table 1).  Written as the set of the k
cells (dx, dy) of the s x s step that hold a replica, a cell (x, y) of the
level-r fractal (side n = s**r) is a member iff every pair of base-s digits
(x_i, y_i), i < r, is one of those cells.  The lambda map of Theorem 1 takes
block omega = (wx, wy) of the packed k**ceil(r/2) x k**floor(r/2) grid
(Lemma 2) to the member block sum_mu H[beta_mu] * s**(mu - 1), with beta_mu
the base-k digit of Theorem 1's formula and H a numbering of the k step
cells (the paper leaves the numbering free; footnote to Theorem 1).

Fractals (step cells as (dx, dy), numbered in this order):
- gasket: s = 2, k = 3, the (x & y) == 0 orientation, numbered as the gasket
  map of this library (H = (0,1), (0,0), (1,0)), so that the generic map
  reproduces it;
- carpet (Sierpinski carpet): s = 3, k = 8, every cell but the centre;
- vicsek (Vicsek fractal, the "plus" form): s = 3, k = 5, the centre and its
  four edge neighbours;
- xfractal (the diagonal "X" form, Table 1's X-fractal, H = log 5 / log 3):
  s = 3, k = 5, the centre and the four corners;
- hfractal (H-fractal, k = 7, s = 3 as Sec. 3.1 states): the left and right
  columns and the centre.
The step cells of the X- and H-fractal are a reading: Table 1 gives their
pictures only.  Chandelier, Candy and Empty-Bottles are left out: the text
gives no cells for them.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np

Step = Tuple[int, int, Tuple[Tuple[int, int], ...]]  # (s, k, cells)

FRACTALS: Dict[str, Step] = {
    "gasket": (2, 3, ((0, 1), (0, 0), (1, 0))),
    "carpet": (3, 8, tuple((x, y) for y in range(3) for x in range(3) if (x, y) != (1, 1))),
    "vicsek": (3, 5, ((1, 0), (0, 1), (1, 1), (2, 1), (1, 2))),
    "xfractal": (3, 5, ((0, 0), (2, 0), (1, 1), (0, 2), (2, 2))),
    "hfractal": (3, 7, ((0, 0), (2, 0), (0, 1), (1, 1), (2, 1), (0, 2), (2, 2))),
}


def step_mask(s: int, cells: Sequence[Tuple[int, int]]) -> np.ndarray:
    """The s x s NBB step as a boolean array [dy, dx] (Table 1)."""
    m = np.zeros((s, s), dtype=bool)
    for dx, dy in cells:
        m[dy, dx] = True
    return m


def member_mask(name: str, r: int) -> np.ndarray:
    """Members of the level-r fractal as an (s**r, s**r) boolean array [y, x]:
    (x, y) is a member iff each base-s digit pair is a step cell (Sec. 3.1's
    bottom-up construction, level by level)."""
    s, _, cells = FRACTALS[name]
    step = step_mask(s, cells)
    n = s ** r
    ys, xs = np.mgrid[0:n, 0:n]
    ok = np.ones((n, n), dtype=bool)
    for _ in range(r):
        ok &= step[ys % s, xs % s]
        xs //= s
        ys //= s
    return ok


def member_mask_recursive(name: str, r: int) -> np.ndarray:
    """The same set built as Sec. 3.1 defines it: level r + 1 is k copies of
    level r placed at the step cells (times s**r).  An independent
    construction to pin member_mask against."""
    s, _, cells = FRACTALS[name]
    m = np.ones((1, 1), dtype=bool)
    for _ in range(r):
        side = m.shape[0]
        nxt = np.zeros((side * s, side * s), dtype=bool)
        for dx, dy in cells:
            nxt[dy * side:(dy + 1) * side, dx * side:(dx + 1) * side] = m
        m = nxt
    return m


def grid_dims(k: int, r: int) -> Tuple[int, int]:
    """Packed grid of a level-r NBB fractal with k replicas: (k**ceil(r/2), k**floor(r/2)) (Lemma 2)."""
    return k ** ((r + 1) // 2), k ** (r // 2)


def beta(mu: int, wx: int, wy: int, k: int) -> int:
    """Replica index at scale level mu >= 1 (Theorem 1): the base-k digit
    ceil(mu/2) - 1 of wx for odd mu, of wy for even mu."""
    num = wx if mu % 2 == 1 else wy
    return (num // k ** ((mu + 1) // 2 - 1)) % k


def lam(name: str, r: int, wx: int, wy: int) -> Tuple[int, int]:
    """lambda(omega) = sum_{mu=1}^{r} H[beta_mu] * s**(mu - 1) (Theorem 1), H the fractal's step cells."""
    s, k, cells = FRACTALS[name]
    lx = ly = 0
    for mu in range(1, r + 1):
        tx, ty = cells[beta(mu, wx, wy, k)]
        lx += tx * s ** (mu - 1)
        ly += ty * s ** (mu - 1)
    return lx, ly


def block_table(name: str, r: int) -> np.ndarray:
    """Blocks of every omega in row-major order of the packed grid: int32 (H, W, 2) of (x, y)."""
    _, k, _ = FRACTALS[name]
    W, H = grid_dims(k, r)
    out = np.zeros((H, W, 2), dtype=np.int32)
    for wy in range(H):
        for wx in range(W):
            out[wy, wx] = lam(name, r, wx, wy)
    return out


def sw_write(name: str, r_b: int, j: int, value: float) -> np.ndarray:
    """The single write of Sec. 6.2 on the level-(r_b + j) fractal in tiles of
    side s**j: `value` at every member cell, 0 at the non-member cells of
    member tiles, NaN where no member tile lies (cells a launch must not touch)."""
    s, _, _ = FRACTALS[name]
    n = s ** (r_b + j)
    t = s ** j
    cells = member_mask(name, r_b + j)
    tiles = member_mask(name, r_b)
    in_tile = np.kron(tiles, np.ones((t, t), dtype=bool))
    out = np.full((n, n), np.nan)
    out[in_tile] = 0.0
    out[cells] = value
    assert not np.any(cells & ~in_tile)
    return out


def names() -> List[str]:
    return list(FRACTALS)
