"""fractal_reduce_noalloc: the sum over the gasket without any allocation.

Some callers cannot allocate device memory when they reduce: their memory is
owned by another allocator (a framework's caching allocator or a fixed pool),
or they run in a latency-bound loop that must not pay for, or wait on, an
allocation.  For them the library keeps the reduce's per-CTA partial sums in a
fixed device array built into it.  These tests call that entry point through
the C ABI and compare it with the oracle's sum over the members and with the
plan-based reduce, twice in a row (the array is shared by all calls and keeps
the previous call's contents)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fr():
    from paper_2004_13475_gb300 import build as fbuild
    fbuild.build()
    import paper_2004_13475_gb300 as m
    assert torch.cuda.is_available()
    return m


def _state(dtype, n, seed):
    """The seeded state (host array) and its device copy."""
    host = synth.bernoulli_u8(seed, n) if dtype == 0 else synth.uniform_f32(seed, n)
    return host, torch.from_numpy(host.reshape(-1).copy()).cuda()


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("k,rho", [(10, 16), (12, 8), (14, 32), (13, 4), (11, 2), (12, 1)])
def test_noalloc_matches_oracle_and_plan_reduce_twice(fr, k, rho, dtype):
    n = 1 << k
    plan = fr.fractal_map(k, rho)
    mask = oracle.member_mask(n)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for seed in (11, 12):                       # two calls in a row, different data
        host, buf = _state(dtype, n, seed)
        want = oracle.reduce_sum(host[mask])
        same = fr.fractal_reduce(plan, buf, dtype)
        fr.fractal_reduce_noalloc(k, rho, buf, dtype, out[1:])
        torch.cuda.synchronize()
        got = out[1].item()
        if dtype == 0:
            assert got == want == same          # exact counts
        else:
            # FP32 partials summed in FP64: within 1e-6 of the FP64 sum
            assert abs(got - want) <= 1e-6 * want, (got, want)
            if rho >= 4:                        # the default plan's 8 x 8-block kernel
                assert got == same
            else:
                assert abs(got - same) <= 1e-6 * want
        assert out[0].item() == -1.0            # nothing outside the output word is written


def test_noalloc_full_size_count(fr):
    k, n = 16, 1 << 16
    buf = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    plan = fr.fractal_map(k, 32)
    fr.fractal_map_write(plan, buf, fr.FRACTAL_U8, 1)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        fr.fractal_reduce_noalloc(k, 32, buf, fr.FRACTAL_U8, out)
        torch.cuda.synchronize()
        assert out.item() == 3 ** 16


def test_noalloc_rejects_bad_and_oversized_calls(fr):
    buf = torch.zeros(64 * 64, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(fr.FractalError) as ei:
        fr.fractal_reduce_noalloc(16, 1, buf, fr.FRACTAL_F32, out)   # needs more partials than the array
    assert ei.value.status == fr.FRACTAL_ETOOBIG
    with pytest.raises(fr.FractalError):
        fr.fractal_reduce_noalloc(6, 8, buf, 7, out)                 # unknown dtype
    with pytest.raises(fr.FractalError):
        fr.fractal_reduce_noalloc(6, 8, buf[1:], fr.FRACTAL_F32, out)   # misaligned
    with pytest.raises(fr.FractalError):
        fr.fractal_reduce_noalloc(6, 128, buf, fr.FRACTAL_F32, out)  # bad rho
    host = np.zeros(64 * 64, dtype=np.float32)                       # pageable host memory
    with pytest.raises(fr.FractalError) as ei:
        fr.fractal_reduce_noalloc(6, 8, host.ctypes.data, fr.FRACTAL_F32, out)
    assert ei.value.status == fr.FRACTAL_EINVAL
