"""The record form: a state held as the compact records the fused launches
keep between them, converted from and to the embedded array, and advanced
record to record.  Results equal those of the embedded-array calls bit for
bit (the same kernels and arithmetic) and so the oracle's."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err, tile_cover

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fr():
    from paper_2004_13475_gb300 import build as fbuild
    fbuild.build()
    import paper_2004_13475_gb300 as m
    assert torch.cuda.is_available()
    return m


def block_cover(n):
    return tile_cover(n, 8)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k,rho,spl", [(9, 8, 50), (10, 8, 16), (10, 16, 25)])
def test_diffusion_records_equal_the_array_calls(fr, k, rho, spl, mode):
    n = 1 << k
    plan = fr.fractal_map(k, rho, mode)
    fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, spl)
    nbytes = fr.fractal_plan_records_bytes(plan, fr.FRACTAL_F32)
    assert nbytes == 3 ** (k - 3) * 112
    u0 = synth.uniform_f32(7 + k, n)
    steps, every = 120, 60
    # the embedded-array call
    a = torch.from_numpy(u0.reshape(-1).copy()).cuda()
    b = torch.zeros_like(a)
    sa = torch.zeros(2, dtype=torch.float64, device="cuda")
    want_dev = fr.fractal_step_diffusion_sums(plan, a, b, 0.2, steps, every, sa)
    # the same in record form
    src = torch.from_numpy(u0.reshape(-1).copy()).cuda()
    r0 = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    r1 = torch.empty_like(r0)
    sb = torch.zeros(2, dtype=torch.float64, device="cuda")
    fr.fractal_records_from_array(plan, fr.FRACTAL_F32, src, r0)
    fr.fractal_step_diffusion_records(plan, r0, r1, 0.2, steps, every, sb)
    out = torch.full_like(src, -9.0)
    fr.fractal_records_to_array(plan, fr.FRACTAL_F32, r1, out)
    got = out.cpu().numpy().reshape(n, n)
    want = want_dev.cpu().numpy().reshape(n, n)
    mask = oracle.member_mask(n)
    assert np.array_equal(got[mask], want[mask])
    assert torch.equal(sa, sb)
    cover = tile_cover(n, rho)
    assert np.all(got[cover & ~mask] == 0) and np.all(got[~cover] == -9.0)
    dom = oracle.Domain.build(n)
    ref = oracle.diffusion_run(u0.astype(np.float64), steps, 0.2, dom)
    assert rel_err(got, ref, dom.mask)[0] <= 1e-4


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("k,rho,spl", [(9, 32, 25), (11, 16, 31)])
def test_ca_records_equal_the_array_calls(fr, k, rho, spl, mode):
    n = 1 << k
    plan = fr.fractal_map(k, rho, mode)
    fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_U8, spl)
    nbytes = fr.fractal_plan_records_bytes(plan, fr.FRACTAL_U8)
    assert nbytes == 3 ** (k - 5) * 128
    s0 = synth.bernoulli_u8(5 + k, n)
    steps = 70
    a = torch.from_numpy(s0.reshape(-1).copy()).cuda()
    b = torch.zeros_like(a)
    ca = torch.zeros(1, dtype=torch.float64, device="cuda")
    want_dev = fr.fractal_step_ca_count(plan, a, b, steps, ca)
    src = torch.from_numpy(s0.reshape(-1).copy()).cuda()
    r0 = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    r1 = torch.empty_like(r0)
    cb = torch.zeros(1, dtype=torch.float64, device="cuda")
    fr.fractal_records_from_array(plan, fr.FRACTAL_U8, src, r0)
    fr.fractal_step_ca_records(plan, r0, r1, steps, cb)
    out = torch.zeros_like(src)
    fr.fractal_records_to_array(plan, fr.FRACTAL_U8, r1, out)
    mask = oracle.member_mask(n)
    got = out.cpu().numpy().reshape(n, n)
    assert np.array_equal(got[mask], want_dev.cpu().numpy().reshape(n, n)[mask])
    assert np.array_equal(got[mask], oracle.ca_run(s0, steps)[mask])
    assert cb.item() == ca.item() == int(got[mask].sum())


def test_records_round_trip_and_validation(fr):
    k, n = 9, 512
    plan = fr.fractal_map(k, 8)
    x = torch.zeros(n * n, device="cuda")
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_records_bytes(plan, fr.FRACTAL_F32)          # no fused configuration yet
    fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, 8)
    r = torch.empty(fr.fractal_plan_records_bytes(plan, fr.FRACTAL_F32) // 4, device="cuda")
    u0 = synth.uniform_f32(3, n)
    src = torch.from_numpy(u0.reshape(-1).copy()).cuda()
    fr.fractal_records_from_array(plan, fr.FRACTAL_F32, src, r)
    fr.fractal_records_to_array(plan, fr.FRACTAL_F32, r, x)
    mask = oracle.member_mask(n)
    assert np.array_equal(x.cpu().numpy().reshape(n, n)[mask], u0[mask])
    with pytest.raises(fr.FractalError):
        fr.fractal_step_diffusion_records(plan, r, r, 0.2, 4)          # in place
    with pytest.raises(fr.FractalError):
        fr.fractal_step_diffusion_records(plan, r, x, 0.2, 0)          # no steps
