"""Other fractals of the NBB family on the GPU (fractal_nbb_map_blocks,
fractal_nbb_write) against the oracle (oracle/nbb.py): Theorem 1's lambda
block for block, and the single write of Sec. 6.2 by the lambda and the BB
launch cell for cell."""
import numpy as np
import pytest

import oracle
from oracle import nbb

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NAMES = nbb.names()
SENTINEL = -5.0


@pytest.fixture(scope="module")
def fr():
    from paper_2004_13475_gb300 import build as fbuild
    fbuild.build()
    import paper_2004_13475_gb300 as m
    assert torch.cuda.is_available()
    return m


def step(name):
    s, k, cells = nbb.FRACTALS[name]
    return s, list(cells)


@pytest.mark.parametrize("name", NAMES)
def test_map_blocks_match_oracle(fr, name):
    s, cells = step(name)
    k = len(cells)
    for r in range(0, 8):
        if k ** r > 40000:
            break
        out = torch.zeros(2 * k ** r, dtype=torch.int32, device="cuda")
        fr.fractal_nbb_map_blocks(s, cells, r, out)
        want = nbb.block_table(name, r).reshape(-1)
        assert np.array_equal(out.cpu().numpy(), want), (name, r)


def test_generic_map_is_the_gasket_map_at_level_12(fr):
    """The generic kernel with the gasket's step equals this library's
    gasket map (ballot form) over all 3^12 blocks of a level-12 block grid."""
    s, cells = step("gasket")
    out = torch.zeros(2 * 3 ** 12, dtype=torch.int32, device="cuda")
    fr.fractal_nbb_map_blocks(s, cells, 12, out)
    plan = fr.fractal_map(15, 8)                     # r_b = 12
    ref = torch.zeros_like(out)
    fr.fractal_map_blocks(plan, ref)
    assert torch.equal(out, ref)


@pytest.mark.parametrize("name", NAMES)
def test_map_blocks_bijection_large(fr, name):
    """At a larger level: every block is a member block and none repeats."""
    s, cells = step(name)
    k = len(cells)
    r = max(rr for rr in range(1, 20) if k ** rr <= 5_000_000 and s ** rr <= 1 << 15)
    out = torch.zeros(2 * k ** r, dtype=torch.int32, device="cuda")
    fr.fractal_nbb_map_blocks(s, cells, r, out)
    xy = out.view(-1, 2).long()
    n = s ** r
    key = xy[:, 1] * n + xy[:, 0]
    assert torch.unique(key).numel() == k ** r
    # membership by digits, on the device with torch integer ops (independent of the kernel)
    x, y = xy[:, 0].clone(), xy[:, 1].clone()
    mask = torch.from_numpy(nbb.step_mask(s, cells).reshape(-1)).cuda()
    ok = torch.ones_like(x, dtype=torch.bool)
    for _ in range(r):
        ok &= mask[(y % s) * s + (x % s)]
        x //= s
        y //= s
    assert bool(ok.all())


@pytest.mark.parametrize("levels", [0, 1, 2])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("rb,j", [(0, 1), (2, 1), (3, 1), (2, 2), (4, 0)])
def test_single_write_matches_oracle(fr, name, rb, j, mode, levels):
    """Both launches and both CTA shapes (one CTA per tile, or per super-tile
    of s^m x s^m tiles) against the oracle, cells outside member tiles untouched."""
    s, cells = step(name)
    if s ** j > 32 or (s ** (rb + j)) ** 2 > 1 << 22 or levels > rb:
        pytest.skip("size")
    n = s ** (rb + j)
    buf = torch.full((n * n,), SENTINEL, device="cuda")
    fr.fractal_nbb_write(s, cells, rb, j, mode, 1.5, buf, cta_levels=levels)
    got = buf.cpu().numpy().reshape(n, n)
    want = nbb.sw_write(name, rb, j, 1.5)
    untouched = np.isnan(want)
    assert np.all(got[untouched] == SENTINEL)
    assert np.array_equal(got[~untouched], want[~untouched].astype(np.float32))


@pytest.mark.parametrize("name", ["carpet", "vicsek", "hfractal"])
def test_single_write_lambda_and_bb_agree_large(fr, name):
    """Level 8 with tiles of side 9 (n = 6561): both launches write the same
    field; the member count is k^8 cells."""
    s, cells = step(name)
    rb, j = 6, 2
    n = s ** (rb + j)
    a = torch.full((n * n,), SENTINEL, device="cuda")
    b = torch.full_like(a, SENTINEL)
    fr.fractal_nbb_write(s, cells, rb, j, 0, 1.0, a)
    fr.fractal_nbb_write(s, cells, rb, j, 1, 1.0, b)
    assert torch.equal(a, b)
    for mode in (0, 1):                                   # super-tiles of 9 x 9 tiles
        c = torch.full_like(a, SENTINEL)
        fr.fractal_nbb_write(s, cells, rb, j, mode, 1.0, c, cta_levels=2)
        assert torch.equal(a, c)
    assert int((a == 1.0).sum()) == len(cells) ** (rb + j)
    assert int((a != SENTINEL).sum()) == len(cells) ** rb * (s ** j) ** 2


def test_nbb_validation(fr):
    buf = torch.zeros(16, device="cuda")
    xy = torch.zeros(32, dtype=torch.int32, device="cuda")
    bad_steps = [(1, [(0, 0)]), (5, [(0, 0)]), (2, [(0, 0), (0, 0)]), (2, [(2, 0)]), (2, [(0, 0)] * 5)]
    for s, cells in bad_steps:
        with pytest.raises(fr.FractalError):
            fr.fractal_nbb_map_blocks(s, cells, 1, xy)
        with pytest.raises(fr.FractalError):
            fr.fractal_nbb_write(s, cells, 1, 1, 0, 1.0, buf)
    s, cells = step("carpet")
    with pytest.raises(fr.FractalError):
        fr.fractal_nbb_write(s, cells, 1, 4, 0, 1.0, buf)          # tile side 81 > 32
    with pytest.raises(fr.FractalError):
        fr.fractal_nbb_write(s, cells, 1, 1, 2, 1.0, buf)          # mode
    with pytest.raises(fr.FractalError):
        fr.fractal_nbb_write(s, cells, 1, 1, 0, 1.0, buf, cta_levels=2)   # more CTA levels than block levels
    with pytest.raises(fr.FractalError):
        fr.fractal_nbb_write(s, cells, 6, 1, 1, 1.0, buf, cta_levels=5)   # 3^10 BB tiles per super-tile
    with pytest.raises(fr.FractalError):
        fr.fractal_nbb_map_blocks(s, cells, 11, xy)                 # 8^11 blocks > 2^31 - 1
    with pytest.raises(fr.FractalError):
        fr.fractal_nbb_map_blocks(s, cells, -1, xy)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("rb,j,steps", [(2, 1, 1), (3, 1, 4), (1, 2, 3), (4, 0, 2), (2, 2, 5)])
def test_ca_matches_oracle(fr, name, rb, j, steps, mode):
    """The CA test on other NBB fractals, bit for bit against the oracle, both
    launches; non-member cells hold noise that must be ignored, cells outside
    member tiles of the output stay as they were."""
    s, cells = step(name)
    if s ** j > 32 or (s ** (rb + j)) ** 2 > 1 << 22:
        pytest.skip("size")
    n = s ** (rb + j)
    rng = np.random.default_rng(11 + rb + j)
    a0 = (rng.random((n, n)) < 0.5).astype(np.uint8)
    a0[~nbb.member_mask(name, rb + j)] = 9                  # noise off the fractal
    a = torch.from_numpy(a0.reshape(-1)).cuda()
    b = torch.full_like(a, 7)
    res = fr.fractal_nbb_step_ca(s, cells, rb, j, mode, a, b, steps)
    got = res.cpu().numpy().reshape(n, n)
    want = a0.copy()
    for _ in range(steps):
        want = nbb.ca_step(name, rb + j, want)
    in_tile = np.kron(nbb.member_mask(name, rb), np.ones((s ** j, s ** j), dtype=bool))
    assert np.array_equal(got[in_tile], want[in_tile])
    outside = a0 if steps % 2 == 0 else np.full((n, n), 7, dtype=np.uint8)
    assert np.array_equal(got[~in_tile], outside[~in_tile])


@pytest.mark.parametrize("name", ["carpet", "vicsek"])
def test_ca_lambda_and_bb_agree_large(fr, name):
    s, cells = step(name)
    rb, j = 6, 2
    n = s ** (rb + j)
    g = torch.Generator(device="cuda").manual_seed(5)
    a0 = (torch.rand(n * n, device="cuda", generator=g) < 0.5).to(torch.uint8)
    outs = []
    for mode in (0, 1):
        a = a0.clone()
        b = torch.zeros_like(a)
        outs.append(fr.fractal_nbb_step_ca(s, cells, rb, j, mode, a, b, 10).clone())
    assert torch.equal(outs[0], outs[1])
    assert int(outs[0].sum()) > 0


def test_ca_validation(fr):
    s, cells = step("carpet")
    a = torch.zeros(81 * 81, dtype=torch.uint8, device="cuda")
    with pytest.raises(fr.FractalError):
        fr.fractal_nbb_step_ca(s, cells, 2, 2, 0, a, a, 1)         # same buffer
    with pytest.raises(fr.FractalError):
        fr.fractal_nbb_step_ca(s, cells, 2, 4, 0, a, torch.zeros_like(a), 1)   # tile side 81
    with pytest.raises(fr.FractalError):
        fr.fractal_nbb_step_ca(s, cells, 2, 2, 0, a, torch.zeros_like(a), -1)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("rb,j", [(2, 1), (3, 2), (4, 0), (5, 1)])
def test_reduce_matches_oracle(fr, name, rb, j, mode):
    """The sum over the members (FP64) against the oracle's FP64 sum, with NaN
    off the fractal that must not be read; the same result on a second call;
    a partials array too short for the launch is refused."""
    s, cells = step(name)
    if s ** j > 32 or (s ** (rb + j)) ** 2 > 1 << 22:
        pytest.skip("size")
    k = len(cells)
    n = s ** (rb + j)
    rng = np.random.default_rng(21 + rb)
    x = rng.random((n, n)).astype(np.float32)
    mask = nbb.member_mask(name, rb + j)
    x[~mask] = np.nan
    buf = torch.from_numpy(x.reshape(-1)).cuda()
    parts = torch.zeros(k ** rb if mode == 0 else s ** (2 * rb), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    fr.fractal_nbb_reduce(s, cells, rb, j, mode, buf, parts, out)
    got = out.item()
    want = oracle.reduce_sum(x[mask].astype(np.float64))
    assert abs(got - want) <= 1e-12 * max(1.0, abs(want))
    fr.fractal_nbb_reduce(s, cells, rb, j, mode, buf, parts, out)
    assert out.item() == got
    short = torch.zeros(parts.numel() - 1, dtype=torch.float64, device="cuda")
    if short.numel() > 0:
        with pytest.raises(fr.FractalError):
            fr.fractal_nbb_reduce(s, cells, rb, j, mode, buf, short, out)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("rb,j,steps", [(2, 1, 1), (3, 1, 6), (1, 2, 3), (4, 0, 2), (2, 2, 25)])
def test_diffusion_matches_oracle(fr, name, rb, j, steps, mode):
    """FP32 diffusion on other NBB fractals against the FP64 oracle (relative
    to the field's scale, 2e-6 + 1e-7 per step), NaN off the fractal ignored,
    cells outside member tiles of the output untouched, heat conserved."""
    s, cells = step(name)
    if s ** j > 32 or (s ** (rb + j)) ** 2 > 1 << 22:
        pytest.skip("size")
    n = s ** (rb + j)
    mask = nbb.member_mask(name, rb + j)
    rng = np.random.default_rng(31 + rb + j)
    u0 = rng.random((n, n)).astype(np.float32)
    u0[~mask] = np.nan
    a = torch.from_numpy(u0.reshape(-1)).cuda()
    b = torch.full_like(a, SENTINEL)
    res = fr.fractal_nbb_step_diffusion(s, cells, rb, j, mode, a, b, 0.2, steps)
    got = res.cpu().numpy().reshape(n, n)
    want = u0.astype(np.float64)
    for _ in range(steps):
        want = nbb.diffusion_step(name, rb + j, want, 0.2)
    in_tile = np.kron(nbb.member_mask(name, rb), np.ones((s ** j, s ** j), dtype=bool))
    assert np.all(got[in_tile & ~mask] == 0)
    err = np.abs(got[mask].astype(np.float64) - want[mask]).max()
    assert err <= (2e-6 + 1e-7 * steps) * max(1.0, np.abs(want[mask]).max())
    outside = u0 if steps % 2 == 0 else np.full((n, n), SENTINEL, dtype=np.float32)
    assert np.array_equal(got[~in_tile], outside[~in_tile], equal_nan=True)
    assert abs(got[mask].astype(np.float64).sum() - u0[mask].astype(np.float64).sum()) <= 1e-5 * mask.sum()


def test_diffusion_lambda_and_bb_agree_bit_for_bit(fr):
    s, cells = step("vicsek")
    rb, j = 6, 2
    n = s ** (rb + j)
    g = torch.Generator(device="cuda").manual_seed(3)
    u0 = torch.rand(n * n, device="cuda", generator=g)
    outs = []
    for mode in (0, 1):
        a = u0.clone()
        b = torch.zeros_like(a)
        outs.append(fr.fractal_nbb_step_diffusion(s, cells, rb, j, mode, a, b, 0.2, 10).clone())
    assert torch.equal(outs[0], outs[1])
