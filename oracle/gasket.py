"""Plain CPU oracle: gasket membership, the block-space map and the workloads.

Test infrastructure only (see the package docstring): the product path never
imports this module, and this module imports nothing from the product.

Conventions
-----------
* The gasket of level k lives in an n x n array, n = 2**k, row-major with
  index y * n + x.  Cell (x, y) is a member iff 0 <= x, y < n and
  (x & y) == 0.  This is the paper's right-angled gasket (Sec. 6, bottom-up
  construction of Fig. "construction steps") with the y axis flipped; the
  paper's own intra-block test, t_x & (b - 1 - t_y) == 0 (Sec. 6.1), is the
  same set before the flip.
* "Absent" cells (non-members and cells outside the array) take no part in
  any update: they are neither counted as neighbours nor written as members.
* Parity status of each function is stated in its docstring; pins live in
  tests/test_oracle_*.py.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np

# ---------------------------------------------------------------------------
# Membership and volume (Sec. 3.1, Eq. 2; Lemma 1)
# ---------------------------------------------------------------------------


def is_member(n: int, x: int, y: int) -> bool:
    """Cell (x, y) belongs to the gasket embedded in n x n.

    Pinned by: Eq. 2 volume 3**k (count), Pascal's triangle mod 2 (Lucas).
    """
    return 0 <= x < n and 0 <= y < n and (x & y) == 0


def member_mask(n: int, x0: int = 0, y0: int = 0, w: Optional[int] = None,
                h: Optional[int] = None) -> np.ndarray:
    """Boolean (h, w) mask of the members inside the window [x0,x0+w) x [y0,y0+h).

    Brute force: every cell of the window is tested on its own.
    """
    w = n - x0 if w is None else w
    h = n - y0 if h is None else h
    xs = np.arange(x0, x0 + w, dtype=np.int64)
    mask = np.zeros((h, w), dtype=bool)
    inx = (xs >= 0) & (xs < n)
    for r in range(h):
        y = y0 + r
        if 0 <= y < n:
            mask[r] = inx & ((xs & y) == 0)
    return mask


def n_members(k: int) -> int:
    """Number of gasket cells at level k, counted by brute force (Eq. 2: 3**k)."""
    n = 1 << k
    return int(member_mask(n).sum())


# ---------------------------------------------------------------------------
# The block-space map lambda(omega) (Sec. 4, Theorem 1; Sec. 6.1)
# ---------------------------------------------------------------------------


def grid_dims(r: int) -> Tuple[int, int]:
    """Packed orthotope of a level-r gasket, (width, height) = (3**ceil(r/2), 3**floor(r/2)).

    Lemma 2 with k = 3 replicas.  Pinned by: width * height == 3**r and the
    worked example of Sec. 6.1 (n = 64, rho = 8 -> 27 blocks).
    """
    if r < 0:
        raise ValueError("level must be >= 0")
    return 3 ** ((r + 1) // 2), 3 ** (r // 2)


def beta(mu: int, wx: int, wy: int) -> int:
    """Replica index of block omega = (wx, wy) at scale level mu >= 1 (Theorem 1; Sec. 6.1).

    beta_mu = ((wx * (mu mod 2) + wy * ((mu + 1) mod 2)) / 3**(ceil(mu/2) - 1)) mod 3,
    with integer division.  Odd mu reads wx, even mu reads wy (the formula's
    reading; the surrounding prose swaps the words "even" and "odd").
    """
    if mu < 1:
        raise ValueError("scale levels start at mu = 1")
    num = wx * (mu % 2) + wy * ((mu + 1) % 2)
    return (num // 3 ** (math.ceil(mu / 2) - 1)) % 3


def hash_table(b: int) -> Tuple[int, int]:
    """Replica offsets tau = H[beta] of the gasket (Sec. 6.1): H[0]=(0,0), H[1]=(0,1), H[2]=(1,1)."""
    return {0: (0, 0), 1: (0, 1), 2: (1, 1)}[b]


def hash_arith(b: int) -> Tuple[int, int]:
    """Arithmetic replacement of H (Sec. 6.1): h(beta) = (floor(beta/2), beta - floor(beta/2))."""
    return b // 2, b - b // 2


def lambda_paper(wx: int, wy: int, r: int) -> Tuple[int, int]:
    """lambda(omega) in the paper's orientation (Eqs. for Delta and lambda, Sec. 4 and 6.1).

    Delta^mu = tau^mu * 2**(mu - 1), lambda = sum_{mu=1}^{r} Delta^mu.
    """
    lx = 0
    ly = 0
    for mu in range(1, r + 1):
        tx, ty = hash_table(beta(mu, wx, wy))
        lx += tx * 2 ** (mu - 1)
        ly += ty * 2 ** (mu - 1)
    return lx, ly


def lambda_canonical(wx: int, wy: int, r: int) -> Tuple[int, int]:
    """lambda(omega) in the (x & y) == 0 orientation: the paper's map with y flipped.

    The paper's gasket satisfies x & (n_b - 1 - y) == 0; flipping y maps it
    onto x & y == 0, so the block is (lambda_x, n_b - 1 - lambda_y).
    """
    lx, ly = lambda_paper(wx, wy, r)
    return lx, (1 << r) - 1 - ly


def block_table(k: int, rho: int) -> np.ndarray:
    """Canonical block table: for omega in row-major order of the packed grid, lambda(omega).

    Returns an int32 array of shape (H, W, 2) with [wy, wx] = (block_x, block_y)
    in the (x & y) == 0 orientation, for blocks of rho x rho cells
    (block-space level r_b = k - log2(rho), Sec. 3.3 and Theorem 1).
    """
    rb = k - int(round(math.log2(rho)))
    if rb < 0 or (1 << int(round(math.log2(rho)))) != rho:
        raise ValueError("rho must be a power of two <= 2**k")
    W, H = grid_dims(rb)
    out = np.zeros((H, W, 2), dtype=np.int32)
    for wy in range(H):
        for wx in range(W):
            out[wy, wx] = lambda_canonical(wx, wy, rb)
    return out


# ---------------------------------------------------------------------------
# Member-list domain over a window of the embedding
# ---------------------------------------------------------------------------

# Moore neighbourhood (CA) and von Neumann neighbourhood (diffusion) offsets.
_MOORE = [(-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]
_VON_NEUMANN = [(0, -1), (-1, 0), (1, 0), (0, 1)]


@dataclass
class Domain:
    """The member cells of a window of the n x n embedding, with neighbour indices.

    ``cx, cy``: coordinates of the m members (row-major order).
    ``nb8``/``nb4``: (m, 8) / (m, 4) indices of the Moore / von Neumann
    neighbours that are members inside the window, -1 where the neighbour is
    absent (non-member, outside the array, or outside the window).  Cells
    within ``steps`` of a window edge that is not the array edge are only
    exact for fewer than that many steps; callers choose windows accordingly.
    """

    n: int
    x0: int
    y0: int
    w: int
    h: int
    mask: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    nb8: np.ndarray
    nb4: np.ndarray

    @classmethod
    def build(cls, n: int, x0: int = 0, y0: int = 0, w: Optional[int] = None,
              h: Optional[int] = None) -> "Domain":
        w = n - x0 if w is None else w
        h = n - y0 if h is None else h
        mask = member_mask(n, x0, y0, w, h)
        ry, rx = np.nonzero(mask)
        m = ry.size
        index = np.full((h, w), -1, dtype=np.int64)
        index[ry, rx] = np.arange(m, dtype=np.int64)

        def gather(offsets):
            out = np.full((m, len(offsets)), -1, dtype=np.int64)
            for j, (dx, dy) in enumerate(offsets):
                qx = rx + dx
                qy = ry + dy
                ok = (qx >= 0) & (qx < w) & (qy >= 0) & (qy < h)
                out[ok, j] = index[qy[ok], qx[ok]]
            return out

        return cls(n=n, x0=x0, y0=y0, w=w, h=h, mask=mask,
                   cx=rx.astype(np.int64) + x0, cy=ry.astype(np.int64) + y0,
                   nb8=gather(_MOORE), nb4=gather(_VON_NEUMANN))

    @property
    def m(self) -> int:
        return int(self.cx.size)

    def take(self, arr: np.ndarray) -> np.ndarray:
        """Values of the members from an (h, w) window array."""
        return arr[self.cy - self.y0, self.cx - self.x0]

    def put(self, vals: np.ndarray, dtype) -> np.ndarray:
        """An (h, w) window array with ``vals`` at the members and 0 elsewhere."""
        out = np.zeros((self.h, self.w), dtype=dtype)
        out[self.cy - self.y0, self.cx - self.x0] = vals
        return out


# ---------------------------------------------------------------------------
# Workloads (Sec. 6.2 tests SW, RD, CA; FDM time step named in Sec. 1)
# ---------------------------------------------------------------------------


def sw_write(n: int, value) -> np.ndarray:
    """Single-write test (Sec. 6.2, SW): zero n x n matrix with ``value`` at every member.

    Returned as float64; callers cast to the dtype under test.
    """
    out = np.zeros((n, n), dtype=np.float64)
    out[member_mask(n)] = value
    return out


def ca_step(dom: Domain, alive: np.ndarray) -> np.ndarray:
    """One synchronous step of the fractal Life-like automaton (Sec. 6.2, CA), rule B3/S23.

    Neighbours are the Moore neighbourhood restricted to gasket members; absent
    cells count as dead.  ``alive`` is a 0/1 (or nonzero = alive) vector over the
    members; returns the next 0/1 uint8 vector.
    """
    a = (np.asarray(alive) != 0).astype(np.int64)
    padded = np.append(a, 0)              # index -1 reads this trailing 0
    count = padded[dom.nb8].sum(axis=1)
    born = (a == 0) & (count == 3)
    survive = (a == 1) & ((count == 2) | (count == 3))
    return (born | survive).astype(np.uint8)


def diffusion_step(dom: Domain, u: np.ndarray, a: float,
                   kappa: Optional[np.ndarray] = None) -> np.ndarray:
    """One explicit FDM heat-diffusion step on the gasket, FP64.

    u'_c = u_c + a * sum_{nb in N4(c), nb member} g_{c,nb} * (u_nb - u_c),
    with g = 1, or g = (kappa_c + kappa_nb) / 2 when a per-cell conductivity is
    given.  Absent neighbours carry no flux (zero-flux walls), so the sum of u
    over the members is conserved.  The FDM time-step pattern is named in
    Sec. 1; the stencil itself is the usual 5-point update.
    """
    u = np.asarray(u, dtype=np.float64)
    valid = dom.nb4 >= 0
    upad = np.append(u, 0.0)
    diff = np.where(valid, upad[dom.nb4] - u[:, None], 0.0)
    if kappa is None:
        flux = diff.sum(axis=1)
    else:
        kap = np.asarray(kappa, dtype=np.float64)
        kpad = np.append(kap, 0.0)
        g = np.where(valid, 0.5 * (kap[:, None] + kpad[dom.nb4]), 0.0)
        flux = (g * diff).sum(axis=1)
    return u + a * flux


def reduce_sum(values: np.ndarray) -> float:
    """Global measure (Sec. 6.2, RD): the sum over all members, FP64 (numpy pairwise)."""
    return float(np.sum(np.asarray(values, dtype=np.float64)))


# ---------------------------------------------------------------------------
# Whole-array helpers used by the tests
# ---------------------------------------------------------------------------


def embed(n: int, dom: Domain, vals: np.ndarray, dtype) -> np.ndarray:
    """Place member values of a whole-array domain into a zero n x n array."""
    assert dom.w == n and dom.h == n and dom.x0 == 0 and dom.y0 == 0
    return dom.put(vals, dtype)


def ca_run(state: np.ndarray, steps: int, dom: Optional[Domain] = None) -> np.ndarray:
    """Run ``steps`` CA steps on an (h, w) window array (default: the whole array).

    Returns the window array after the steps, members updated, all else 0.
    """
    if dom is None:
        n = state.shape[0]
        dom = Domain.build(n)
    s = dom.take(state)
    for _ in range(steps):
        s = ca_step(dom, s)
    return dom.put(s, np.uint8)


def diffusion_run(u0: np.ndarray, steps: int, a: float, dom: Optional[Domain] = None,
                  kappa: Optional[np.ndarray] = None) -> np.ndarray:
    """Run ``steps`` FP64 diffusion steps on an (h, w) window array; returns float64."""
    if dom is None:
        n = u0.shape[0]
        dom = Domain.build(n)
    u = dom.take(u0).astype(np.float64)
    kap = None if kappa is None else dom.take(kappa).astype(np.float64)
    for _ in range(steps):
        u = diffusion_step(dom, u, a, kap)
    return dom.put(u, np.float64)


# ---------------------------------------------------------------------------
# Differentiation of the diffusion (not in the paper: the gradient of a
# loss through the FDM steps named in Sec. 1, by the discrete adjoint)
# ---------------------------------------------------------------------------


def diffusion_matrix(dom: Domain, a: float, kappa: Optional[np.ndarray] = None):
    """The step as a sparse matrix A over the members: u_{t+1} = A u_t.

    Row c: A_cc = 1 - a * sum_nb g_{c,nb}, A_{c,nb} = a * g_{c,nb} for every
    member neighbour nb in N4(c), g as in ``diffusion_step`` (1, or
    (kappa_c + kappa_nb) / 2).  Pinned against ``diffusion_step``.
    """
    import scipy.sparse as sp
    m = dom.m
    valid = dom.nb4 >= 0
    rows = np.repeat(np.arange(m), 4)[valid.reshape(-1)]
    cols = dom.nb4.reshape(-1)[valid.reshape(-1)]
    if kappa is None:
        g = np.ones(rows.size)
    else:
        kap = np.asarray(kappa, dtype=np.float64)
        g = 0.5 * (kap[rows] + kap[cols])
    off = sp.csr_matrix((a * g, (rows, cols)), shape=(m, m))
    diag = 1.0 - np.asarray(off.sum(axis=1)).reshape(-1)
    return (off + sp.diags(diag)).tocsr()


def diffusion_loss_gradients(dom: Domain, u0: np.ndarray, kappa: np.ndarray, target: np.ndarray,
                             steps: int, a: float):
    """Loss J = sum over members of (u_T - target)^2, u_T after ``steps`` steps
    of ``diffusion_step`` with conductivity ``kappa``, and its gradients, FP64.

    Discrete adjoint, every state kept:
      u_{t+1} = A u_t                      (A = diffusion_matrix(dom, a, kappa))
      p_T = dJ/du_T = 2 (u_T - target)
      p_t = A^T p_{t+1}                    (explicit transpose)
      dJ/du_0 = p_0
      dJ/dkappa_c = sum_{t < T} p_{t+1}^T (d A / d kappa_c) u_t
                  = sum_t sum_{nb in N4(c)} (a / 2) (u_t,nb - u_t,c) (p_{t+1},c - p_{t+1},nb)
    (A u depends on kappa_c through g_{c,nb} = (kappa_c + kappa_nb) / 2 in row
    c and in the rows of c's neighbours).  Member vectors in, member vectors
    out: returns (J, dJ/du_0, dJ/dkappa).  Pinned by finite differences.
    """
    A = diffusion_matrix(dom, a, kappa)
    AT = A.T.tocsr()
    u = [np.asarray(u0, dtype=np.float64)]
    for _ in range(steps):
        u.append(A @ u[-1])
    r = u[-1] - np.asarray(target, dtype=np.float64)
    J = float(np.sum(r * r))
    p = 2.0 * r
    gk = np.zeros(dom.m)
    valid = dom.nb4 >= 0
    for t in range(steps - 1, -1, -1):
        upad = np.append(u[t], 0.0)
        ppad = np.append(p, 0.0)
        du = upad[dom.nb4] - u[t][:, None]
        dp = p[:, None] - ppad[dom.nb4]
        gk += 0.5 * a * np.where(valid, du * dp, 0.0).sum(axis=1)
        p = AT @ p
    return J, p, gk
