"""Failure handling, exercised without faulting the GPU (the paper has none).

* A bounded device wait that runs out: the self-test kernel arms an mbarrier
  that nothing completes and waits with the step kernels' bounded wait; the
  wait gives up, the plan's status word reads 1, and the context stays usable
  (a run afterwards still matches the oracle).
* An allocation that fails: the library's device allocations can be made to
  fail one at a time (as if the device were full); each call that meets one
  returns FRACTAL_ENOMEM, writes nothing into the caller's buffers, and leaves
  the plan (or batch) in its previous, working configuration.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fr():
    from paper_2004_13475_gb300 import build as fbuild
    fbuild.build()
    import paper_2004_13475_gb300 as m
    assert torch.cuda.is_available()
    yield m
    m.fractal_debug_fail_allocs(-1)


def _diffusion_matches(fr, plan, k, steps, seed):
    n = 1 << k
    u0 = synth.uniform_f32(seed, n)
    a = torch.from_numpy(u0.reshape(-1).copy()).cuda()
    b = torch.zeros_like(a)
    out = fr.fractal_step_diffusion(plan, a, b, 0.2, steps).cpu().numpy().reshape(n, n)
    dom = oracle.Domain.build(n)
    want = oracle.diffusion_run(u0.astype(np.float64), steps, 0.2, dom)
    return rel_err(out, want, dom.mask)[0] <= 1e-4


def test_bounded_wait_runs_out_and_the_context_survives(fr):
    plan = fr.fractal_map(7, 8)
    assert fr.fractal_plan_device_status(plan) == 0
    fr.fractal_plan_selftest_wait(plan, 1 << 12)
    assert fr.fractal_plan_device_status(plan) == 1       # the wait's timeout code
    fr.fractal_plan_selftest_wait(plan, 1 << 10)
    assert fr.fractal_plan_device_status(plan) == 1       # first code wins
    assert _diffusion_matches(fr, plan, 7, 12, 3)         # kernels still run correctly
    other = fr.fractal_map(7, 8)
    assert fr.fractal_plan_device_status(other) == 0      # the word is per plan
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_selftest_wait(plan, 0)            # spin limit out of range


def test_failed_allocation_in_map(fr):
    fr.fractal_debug_fail_allocs(0)
    with pytest.raises(fr.FractalError) as ei:
        fr.fractal_map(8, 8)
    assert ei.value.status == fr.FRACTAL_ENOMEM
    plan = fr.fractal_map(8, 8)                           # injection is off again
    assert _diffusion_matches(fr, plan, 8, 5, 4)


@pytest.mark.parametrize("dtype,spl", [(1, 50), (1, 16), (0, 25)])
def test_failed_allocation_in_steps_per_launch_keeps_the_plan(fr, dtype, spl):
    k, n = 8, 1 << 8
    failures = 0
    for after in range(6):
        plan = fr.fractal_map(k, 8)
        fr.fractal_debug_fail_allocs(after)
        try:
            fr.fractal_plan_set_steps_per_launch(plan, dtype, spl)
            fr.fractal_debug_fail_allocs(-1)
            assert plan.info()["steps_per_launch"][dtype] == spl
        except fr.FractalError as e:
            fr.fractal_debug_fail_allocs(-1)
            assert e.status == fr.FRACTAL_ENOMEM
            failures += 1
            assert plan.info()["steps_per_launch"][dtype] == 1    # the previous configuration
        # whatever happened, the plan computes the right result
        if dtype == 1:
            assert _diffusion_matches(fr, plan, k, 2 * spl + 1, 5 + after)
        else:
            s0 = synth.bernoulli_u8(6 + after, n)
            a = torch.from_numpy(s0.reshape(-1).copy()).cuda()
            b = torch.zeros_like(a)
            got = fr.fractal_step_ca(plan, a, b, 2 * spl + 1).cpu().numpy().reshape(n, n)
            m = oracle.member_mask(n)
            assert np.array_equal(got[m], oracle.ca_run(s0, 2 * spl + 1)[m])
    assert failures >= 2       # the records (two buffers) and, for float32, the descriptors


def test_failed_allocation_in_batches(fr):
    ks = [6, 7, 8]
    states = [synth.uniform_f32(40 + i, 1 << k) for i, k in enumerate(ks)]
    a = [torch.from_numpy(s.reshape(-1).copy()).cuda() for s in states]
    b = [torch.full_like(x, -3.0) for x in a]
    fr.fractal_debug_fail_allocs(0)
    with pytest.raises(fr.FractalError) as ei:
        fr.fractal_batch_create(ks)
    assert ei.value.status == fr.FRACTAL_ENOMEM
    batch = fr.fractal_batch_create(ks)
    fr.fractal_debug_fail_allocs(0)                       # the bind's block records
    with pytest.raises(fr.FractalError) as ei:
        fr.fractal_batch_bind(batch, a, b)
    fr.fractal_debug_fail_allocs(-1)
    assert ei.value.status == fr.FRACTAL_ENOMEM
    for i, s in enumerate(states):                        # caller's buffers untouched
        assert np.array_equal(a[i].cpu().numpy(), s.reshape(-1))
        assert bool((b[i] == -3.0).all())
    fr.fractal_batch_bind(batch, a, b)                    # and the batch still works
    fr.fractal_batch_step_diffusion(batch, 0.2, 6)
    torch.cuda.synchronize()
    for i, k in enumerate(ks):
        n = 1 << k
        dom = oracle.Domain.build(n)
        want = oracle.diffusion_run(states[i].astype(np.float64), 6, 0.2, dom)
        assert rel_err(a[i].cpu().numpy().reshape(n, n), want, dom.mask)[0] <= 1e-4
