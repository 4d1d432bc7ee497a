"""Compact storage through the block-space map: fractal_pack / fractal_unpack
against the oracle's lambda table (Theorem 1), byte for byte."""
import numpy as np
import pytest

import oracle
from gpu_util import SENTINEL_F32, SENTINEL_U8, tile_cover

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fr():
    from paper_2004_13475_gb300 import build as fbuild
    fbuild.build()
    import paper_2004_13475_gb300 as m
    assert torch.cuda.is_available()
    return m


def expected_packed(arr, k, rho):
    """Member tiles of arr in lambda order, from the oracle's block table."""
    table = oracle.block_table(k, rho).reshape(-1, 2)
    return np.stack([arr[by * rho:(by + 1) * rho, bx * rho:(bx + 1) * rho] for bx, by in table])


def field(k, dtype, seed):
    n = 1 << k
    if dtype == np.uint8:
        return np.random.default_rng(seed).integers(0, 256, (n, n), dtype=np.uint8)
    return np.random.default_rng(seed).standard_normal((n, n)).astype(np.float32)


CASES = [(k, r) for k in (0, 1, 2, 3, 5, 8, 10) for r in (1, 2, 4, 8, 16, 32) if r <= (1 << k)]


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("dt", ["u8", "f32"])
@pytest.mark.parametrize("k,rho", CASES)
def test_pack_unpack_bit_exact(fr, k, rho, dt, mode):
    n = 1 << k
    npdt, code, sentinel = ((np.uint8, fr.FRACTAL_U8, SENTINEL_U8) if dt == "u8"
                            else (np.float32, fr.FRACTAL_F32, SENTINEL_F32))
    plan = fr.fractal_map(k, rho, mode)
    tiles = plan.info()["member_tiles"]
    assert tiles == 3 ** (k - int(np.log2(rho)))
    arr = field(k, npdt, 1000 + k * 7 + rho)
    src = torch.from_numpy(arr.reshape(-1)).cuda()
    packed = torch.full((tiles * rho * rho,), sentinel, dtype=src.dtype, device="cuda")
    fr.fractal_pack(plan, src, code, packed)
    want = expected_packed(arr, k, rho)
    got = packed.cpu().numpy().reshape(tiles, rho, rho)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8))
    # back: member tiles written whole, every other cell untouched
    out = torch.full((n * n,), sentinel, dtype=src.dtype, device="cuda")
    fr.fractal_unpack(plan, packed, code, out)
    back = out.cpu().numpy().reshape(n, n)
    cover = tile_cover(n, rho)
    assert np.array_equal(back[cover].view(np.uint8), arr[cover].view(np.uint8))
    assert np.all(back[~cover] == np.array(sentinel, dtype=npdt))


def test_pack_level_16_sampled(fr):
    """Full-size array (n = 65536), one byte per member: sampled packed tiles
    against the oracle's lambda, and the unpack of the packed members."""
    k, rho = 16, 1
    n = 1 << k
    plan = fr.fractal_map(k, rho)
    info = plan.info()
    m = info["member_tiles"]
    assert m == 3 ** 16
    # cell value = (x * 131 + y * 7) mod 256, a function of position
    i = torch.arange(n, device="cuda", dtype=torch.int32)
    x8 = ((i * 131) & 255).to(torch.uint8).view(1, n)
    y8 = ((i * 7) & 255).to(torch.uint8).view(n, 1)
    arr = (x8 + y8).reshape(-1)  # uint8 addition wraps mod 256
    packed = torch.empty(m, dtype=torch.uint8, device="cuda")
    fr.fractal_pack(plan, arr, fr.FRACTAL_U8, packed)
    W = info["grid_w"]
    rng = np.random.default_rng(16)
    js = [0, 1, W - 1, W, m - 1] + rng.integers(0, m, 200).tolist()
    got = packed[torch.tensor(js, device="cuda")].cpu().numpy()
    for j, g in zip(js, got):
        bx, by = oracle.lambda_canonical(j % W, j // W, 16)
        assert bx & by == 0
        assert g == (bx * 131 + by * 7) & 255
    out = torch.zeros(n * n, dtype=torch.uint8, device="cuda")
    fr.fractal_unpack(plan, packed, fr.FRACTAL_U8, out)
    # members hold their values, every other cell stays 0
    assert int(out.sum(dtype=torch.int64)) == int(packed.sum(dtype=torch.int64))
    for x0, y0 in [(0, 0), (n - 512, 0), (0, n - 512), (32768, 16384)]:
        win = out.view(n, n)[y0:y0 + 512, x0:x0 + 512]
        ref = arr.view(n, n)[y0:y0 + 512, x0:x0 + 512]
        sub = torch.from_numpy(oracle.member_mask(n, x0, y0, 512, 512)).cuda()
        assert bool(torch.equal(win, torch.where(sub, ref, torch.zeros_like(ref))))


@pytest.mark.parametrize("dt", ["u8", "f32"])
def test_pack_through_pinned_host_memory(fr, dt):
    """The packed side may be pinned host memory: the same bytes as through
    a device buffer, both ways."""
    k, rho = 9, 2
    n = 1 << k
    npdt, code = (np.uint8, fr.FRACTAL_U8) if dt == "u8" else (np.float32, fr.FRACTAL_F32)
    plan = fr.fractal_map(k, rho)
    cells = plan.info()["member_tiles"] * rho * rho
    arr = field(k, npdt, 77)
    src = torch.from_numpy(arr.reshape(-1)).cuda()
    dev = torch.zeros(cells, dtype=src.dtype, device="cuda")
    host = torch.zeros(cells, dtype=src.dtype).pin_memory()
    fr.fractal_pack(plan, src, code, dev)
    fr.fractal_pack(plan, src, code, host)
    torch.cuda.synchronize()
    assert torch.equal(dev.cpu(), host)
    out = torch.zeros(n * n, dtype=src.dtype, device="cuda")
    fr.fractal_unpack(plan, host, code, out)
    cover = tile_cover(n, rho)
    back = out.cpu().numpy().reshape(n, n)
    assert np.array_equal(back[cover].view(np.uint8), arr[cover].view(np.uint8))
    assert np.all(back[~cover] == 0)


def test_pack_rejects_pageable_host_memory(fr):
    """Pageable memory is refused by the host-side pointer check, before any launch."""
    plan = fr.fractal_map(6, 8)
    a = torch.zeros(64 * 64, dtype=torch.float32, device="cuda")
    pageable = torch.zeros(27 * 64, dtype=torch.float32)
    assert not pageable.is_pinned()
    with pytest.raises(Exception):
        fr.fractal_pack(plan, a, fr.FRACTAL_F32, pageable)
    with pytest.raises(Exception):
        fr.fractal_unpack(plan, pageable, fr.FRACTAL_F32, a)


def test_pack_rejects_bad_arguments(fr):
    plan = fr.fractal_map(6, 8)
    a = torch.zeros(64 * 64 + 4, dtype=torch.float32, device="cuda")
    b = torch.zeros(27 * 64 + 4, dtype=torch.float32, device="cuda")
    with pytest.raises(Exception):
        fr.fractal_pack(plan, a, fr.FRACTAL_F32, a)          # same buffer
    with pytest.raises(Exception):
        fr.fractal_pack(plan, a[1:], fr.FRACTAL_F32, b)      # unaligned
    with pytest.raises(Exception):
        fr.fractal_unpack(plan, b, 7, a)                     # unknown dtype
