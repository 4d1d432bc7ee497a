"""Helpers shared by the GPU parity tests (no tests here)."""
import numpy as np

import oracle

SENTINEL_U8 = 0xA5
SENTINEL_F32 = -7.25


def tile_cover(n, rho):
    """Boolean n x n mask of the cells that lie in a member rho-tile."""
    nb = n // rho
    by, bx = np.mgrid[0:nb, 0:nb]
    blocks = (bx & by) == 0
    return np.kron(blocks, np.ones((rho, rho), dtype=bool)).astype(bool)


def rel_err(got, want, mask):
    """Max over members of |got - want| / max(|want|, 1e-3 * max|want|), and the unfloored max."""
    g = got[mask].astype(np.float64)
    w = want[mask].astype(np.float64)
    scale = np.abs(w).max() if w.size else 1.0
    floor = max(1e-3 * scale, 1e-300)
    d = np.abs(g - w)
    return float((d / np.maximum(np.abs(w), floor)).max()), float((d / np.maximum(np.abs(w), 1e-300)).max())


def check_field_contract(got, want_members, n, rho, sentinel, mask=None):
    """Members equal want; other cells of member tiles are 0; cells outside member tiles untouched."""
    mask = oracle.member_mask(n) if mask is None else mask
    cover = tile_cover(n, rho)
    assert np.array_equal(got[mask], want_members[mask])
    assert np.all(got[cover & ~mask] == 0)
    assert np.all(got[~cover] == sentinel)
