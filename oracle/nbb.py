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


def ca_step(name: str, r: int, alive: np.ndarray) -> np.ndarray:
    """One synchronous B3/S23 step on the level-r fractal (Sec. 6.2's CA test,
    the rule read as for the gasket): a cell's count is its alive member
    neighbours in the Moore neighbourhood (cells outside the array count 0);
    a member is alive next if it has 3, or if it is alive and has 2;
    non-members stay 0.  alive: (n, n) array, nonzero = alive, read at members only."""
    mask = member_mask(name, r)
    a = (alive != 0) & mask
    n = a.shape[0]
    p = np.zeros((n + 2, n + 2), dtype=np.int32)
    p[1:-1, 1:-1] = a
    cnt = sum(p[1 + dy:n + 1 + dy, 1 + dx:n + 1 + dx] for dy in (-1, 0, 1) for dx in (-1, 0, 1)
              if (dx, dy) != (0, 0))
    nxt = (cnt == 3) | (a & (cnt == 2))
    return (nxt & mask).astype(np.uint8)


def ca_step_loops(name: str, r: int, alive: np.ndarray) -> np.ndarray:
    """The same step cell by cell with plain loops over the neighbours, for
    small levels: an independent formulation to pin ca_step against."""
    s, _, cells = FRACTALS[name]
    n = s ** r
    allowed = set(cells)

    def member(x, y):
        if not (0 <= x < n and 0 <= y < n):
            return False
        for _ in range(r):
            if (x % s, y % s) not in allowed:
                return False
            x //= s
            y //= s
        return True

    out = np.zeros((n, n), dtype=np.uint8)
    for y in range(n):
        for x in range(n):
            if not member(x, y):
                continue
            c = 0
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if (dx or dy) and member(x + dx, y + dy) and alive[y + dy, x + dx]:
                        c += 1
            me = bool(alive[y, x])
            out[y, x] = 1 if (c == 3 or (me and c == 2)) else 0
    return out


def ca_write(name: str, r_b: int, j: int, alive: np.ndarray) -> np.ndarray:
    """The next state as a tile launch writes it: the step's values in member
    tiles (side s**j), NaN elsewhere (cells the launch must not touch)."""
    s, _, _ = FRACTALS[name]
    t = s ** j
    nxt = ca_step(name, r_b + j, alive).astype(np.float64)
    in_tile = np.kron(member_mask(name, r_b), np.ones((t, t), dtype=bool))
    nxt[~in_tile] = np.nan
    return nxt


def diffusion_step(name: str, r: int, u: np.ndarray, a: float) -> np.ndarray:
    """One explicit heat-diffusion step on the level-r fractal, FP64 (the
    gasket's step, read the same way for the family): at a member c,
    u'_c = u_c + a * sum over its member 4-neighbours nb of (u_nb - u_c);
    non-members (and cells outside the array) carry no flux, so the sum over
    the members is conserved; non-members are returned as 0."""
    mask = member_mask(name, r)
    n = mask.shape[0]
    v = np.where(mask, np.asarray(u, dtype=np.float64), 0.0)
    pv = np.zeros((n + 2, n + 2))
    pm = np.zeros((n + 2, n + 2), dtype=bool)
    pv[1:-1, 1:-1] = v
    pm[1:-1, 1:-1] = mask
    flux = np.zeros((n, n))
    for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        nb = pm[1 + dy:n + 1 + dy, 1 + dx:n + 1 + dx]
        flux += np.where(nb, pv[1 + dy:n + 1 + dy, 1 + dx:n + 1 + dx] - v, 0.0)
    return np.where(mask, v + a * flux, 0.0)
