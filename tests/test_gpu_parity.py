"""Element-by-element parity of the CUDA path against the CPU oracle, through
the C ABI, on sizes the oracle finishes in seconds.  Maps, the single write
and the automaton are bit-exact; FP32 diffusion is held to the FP64 oracle."""
import functools

import numpy as np
import pytest

import oracle
import synth
from gpu_util import SENTINEL_F32, SENTINEL_U8, check_field_contract, rel_err, tile_cover

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def fr():
    from paper_2004_13475_gb300 import build as fbuild
    fbuild.build()
    import paper_2004_13475_gb300 as m
    assert torch.cuda.is_available()
    return m


@functools.lru_cache(maxsize=None)
def domain(k):
    return oracle.Domain.build(1 << k)


def cases(ks, rhos=(1, 2, 4, 8, 16, 32)):
    return [(k, r) for k in ks for r in rhos if r <= (1 << k)]


MODES = [0, 1]   # FRACTAL_LAMBDA, FRACTAL_BB
SCHEDS = [0, 1]  # FRACTAL_SCHED_AUTO (TMA where it applies), FRACTAL_SCHED_STAGED


def make_plan(fr, k, rho, mode, sched=0):
    plan = fr.fractal_map(k, rho, mode)
    fr.fractal_plan_set_schedule(plan, sched)
    return plan


def dev_u8(arr):
    return torch.from_numpy(np.ascontiguousarray(arr).reshape(-1)).cuda()


def dev_f32(arr):
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float32).reshape(-1)).cuda()


# ------------------------------------------------------------------ map ----

@pytest.mark.parametrize("k,rho", cases(range(0, 11)))
def test_map_blocks_bit_exact(fr, k, rho):
    plan = fr.fractal_map(k, rho)
    info = plan.info()
    xy = torch.full((2 * info["member_tiles"],), -1, dtype=torch.int32, device="cuda")
    fr.fractal_map_blocks(plan, xy)
    assert np.array_equal(xy.cpu().numpy(), oracle.block_table(k, rho).reshape(-1))


@pytest.mark.parametrize("method", [1, 2])     # per thread, tensor-core MMA
@pytest.mark.parametrize("k,rho", cases(range(0, 12)))
def test_map_blocks_methods_bit_exact(fr, k, rho, method):
    plan = fr.fractal_map(k, rho)
    info = plan.info()
    xy = torch.full((2 * info["member_tiles"] + 2,), -7, dtype=torch.int32, device="cuda")
    fr.fractal_map_blocks_method(plan, xy, method)
    got = xy.cpu().numpy()
    assert np.array_equal(got[:-2], oracle.block_table(k, rho).reshape(-1))
    assert got[-2] == -7 and got[-1] == -7           # nothing past the table


@pytest.mark.parametrize("method", [0, 1, 2])
def test_map_blocks_methods_level16(fr, method):
    # 16 levels (k = 16, rho = 1): both MMA halves; the three forms agree everywhere
    plan = fr.fractal_map(16, 1)
    m = plan.info()["member_tiles"]
    ref = torch.empty(2 * m, dtype=torch.int32, device="cuda")
    fr.fractal_map_blocks(plan, ref)
    xy = torch.full((2 * m,), -1, dtype=torch.int32, device="cuda")
    fr.fractal_map_blocks_method(plan, xy, method)
    assert torch.equal(xy, ref)
    W = plan.info()["grid_w"]
    for wx, wy in [(0, 0), (W - 1, 0), (5, 7), (W - 1, plan.info()["grid_h"] - 1), (1234, 321)]:
        assert tuple(xy[2 * (wy * W + wx):2 * (wy * W + wx) + 2].tolist()) == oracle.lambda_canonical(wx, wy, 16)


def test_map_blocks_level16(fr):
    # full-size block level r_b = 13 (k = 16, rho = 8): bijection onto member blocks
    plan = fr.fractal_map(16, 8)
    info = plan.info()
    xy = torch.empty((info["member_tiles"], 2), dtype=torch.int32, device="cuda")
    fr.fractal_map_blocks(plan, xy)
    bx, by = xy[:, 0].long(), xy[:, 1].long()
    assert int(((bx & by) != 0).sum()) == 0
    assert int(bx.max()) < 8192 and int(by.max()) < 8192
    key = torch.unique(by * 8192 + bx)
    assert key.numel() == 3 ** 13
    # spot rows against the oracle's formula
    W = info["grid_w"]
    for wx, wy in [(0, 0), (W - 1, 0), (5, 7), (W - 1, info["grid_h"] - 1), (1234, 321)]:
        assert tuple(xy[wy * W + wx].tolist()) == oracle.lambda_canonical(wx, wy, 13)


# ------------------------------------------------------------------- SW ----

@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k,rho", cases([0, 1, 2, 3, 5, 8, 10]))
def test_single_write(fr, k, rho, mode):
    n = 1 << k
    plan = fr.fractal_map(k, rho, mode)
    mask = oracle.member_mask(n)
    b8 = torch.full((n * n,), SENTINEL_U8, dtype=torch.uint8, device="cuda")
    fr.fractal_map_write(plan, b8, fr.FRACTAL_U8, 3)
    check_field_contract(b8.cpu().numpy().reshape(n, n), (oracle.sw_write(n, 3)).astype(np.uint8), n, rho,
                         SENTINEL_U8, mask)
    bf = torch.full((n * n,), SENTINEL_F32, dtype=torch.float32, device="cuda")
    fr.fractal_map_write(plan, bf, fr.FRACTAL_F32, 1.5)
    check_field_contract(bf.cpu().numpy().reshape(n, n), oracle.sw_write(n, 1.5).astype(np.float32), n, rho,
                         SENTINEL_F32, mask)


# ------------------------------------------------------------------- CA ----

def run_ca(fr, plan, s0, steps, sentinel=SENTINEL_U8):
    n = s0.shape[0]
    a = dev_u8(s0)
    b = torch.full_like(a, sentinel)
    out = fr.fractal_step_ca(plan, a, b, steps)
    return out.cpu().numpy().reshape(n, n), a, b


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k,rho", cases([1, 2, 3, 4, 6, 8, 10]))
def test_ca_bit_exact(fr, k, rho, mode, sched):
    n = 1 << k
    plan = make_plan(fr, k, rho, mode, sched)
    s0 = synth.bernoulli_u8(k, n)          # non-member cells hold noise and must be ignored
    want = oracle.ca_run(s0, 6, domain(k))
    # 6 steps: result in a; b holds step 5.  Cells outside member tiles keep
    # their starting contents (a: noise, b: sentinel).
    a = dev_u8(s0)
    b = torch.full_like(a, SENTINEL_U8)
    out = fr.fractal_step_ca(plan, a, b, 6)
    got = out.cpu().numpy().reshape(n, n)
    mask = domain(k).mask
    cover = tile_cover(n, rho)
    assert np.array_equal(got[mask], want[mask])
    assert np.all(got[cover & ~mask] == 0)
    assert np.array_equal(got[~cover], s0[~cover])
    odd = b.cpu().numpy().reshape(n, n)
    assert np.array_equal(odd[mask], oracle.ca_run(s0, 5, domain(k))[mask])
    assert np.all(odd[~cover] == SENTINEL_U8)
    assert fr.fractal_plan_device_status(plan) == 0


@pytest.mark.parametrize("k,rho", [(9, 8), (9, 16), (9, 32), (10, 32)])
@pytest.mark.parametrize("sched", SCHEDS)
def test_ca_every_cta_level(fr, k, rho, sched):
    n = 1 << k
    s0 = synth.bernoulli_u8(100 + k, n)
    want = oracle.ca_run(s0, 3, domain(k))
    mask = domain(k).mask
    for mode in MODES:
        plan = make_plan(fr, k, rho, mode, sched)
        rb = k - int(np.log2(rho))
        for m in range(0, min(rb, 5) + 1):
            try:
                fr.fractal_plan_set_cta_levels(plan, fr.FRACTAL_U8, m)
            except fr.FractalError:
                continue     # super-tile too large for shared memory
            got, _, _ = run_ca(fr, plan, s0, 3)
            assert np.array_equal(got[mask], want[mask]), (mode, m)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("spl", [2, 3, 8, 16, 25, 31])
@pytest.mark.parametrize("k,rho", [(6, 8), (7, 16), (8, 32), (9, 4), (10, 8), (10, 32), (11, 16)])
def test_ca_fused_bit_exact(fr, k, rho, mode, spl):
    # several automaton steps per launch on the bit image: members equal the
    # oracle bit for bit; the launch writes whole 32-cell row segments of
    # member word tiles (non-members there become 0) and nothing else
    n = 1 << k
    plan = fr.fractal_map(k, rho, mode)
    fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_U8, spl)
    assert plan.info()["steps_per_launch"][0] == spl
    s0 = synth.bernoulli_u8(40 + k, n)      # noise on non-members too: ignored
    mask = domain(k).mask
    cover = tile_cover(n, 32) if n >= 32 else np.ones((n, n), dtype=bool)
    for steps in (1, 5, spl, 2 * spl + 1, 40):
        want = oracle.ca_run(s0, steps, domain(k))
        a = dev_u8(s0)
        b = torch.full_like(a, SENTINEL_U8)
        out = fr.fractal_step_ca(plan, a, b, steps)
        assert out is (a if steps % 2 == 0 else b)
        got = out.cpu().numpy().reshape(n, n)
        assert np.array_equal(got[mask], want[mask]), steps
        assert np.all(got[cover & ~mask] == 0)
        if steps % 2:
            assert np.all(got[~cover] == SENTINEL_U8)
        else:
            assert np.array_equal(got[~cover], s0[~cover])
    assert fr.fractal_plan_device_status(plan) == 0


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k,rho", [(10, 32), (12, 8)])
def test_ca_fused_every_cta_level(fr, k, rho, mode):
    n = 1 << k
    s0 = synth.bernoulli_u8(7 * k, n)
    want = oracle.ca_run(s0, 30, domain(k))
    mask = domain(k).mask
    rb = k - int(np.log2(rho))
    done = 0
    for m in range(0, min(rb, 5) + 1):
        plan = fr.fractal_map(k, rho, mode)
        try:
            fr.fractal_plan_set_cta_levels(plan, fr.FRACTAL_U8, m)
            fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_U8, 12)
        except fr.FractalError:
            continue     # super-tile below 32 or 24 cells, or above 512
        got, _, _ = run_ca(fr, plan, s0, 30)
        assert np.array_equal(got[mask], want[mask]), m
        done += 1
    assert done >= 2


def test_ca_fused_100_steps_level_12(fr):
    k, n = 12, 4096
    s0 = synth.bernoulli_u8(5, n)
    want = oracle.ca_run(s0, 100, domain(k))
    for mode in MODES:
        plan = fr.fractal_map(k, 32, mode)
        fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_U8, 25)
        got, _, _ = run_ca(fr, plan, s0, 100)
        assert np.array_equal(got[domain(k).mask], want[domain(k).mask]), mode


def test_ca_fused_needs_room(fr):
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_set_steps_per_launch(fr.fractal_map(4, 4), fr.FRACTAL_U8, 2)    # n = 16 < 32
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_set_steps_per_launch(fr.fractal_map(10, 8), fr.FRACTAL_U8, 32)
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_set_steps_per_launch(fr.fractal_map(5, 8), fr.FRACTAL_U8, 17)   # T = 32 < 2 * 17
    p = fr.fractal_map(5, 8)
    fr.fractal_plan_set_steps_per_launch(p, fr.FRACTAL_U8, 16)
    assert p.info()["steps_per_launch"] == [16, 1]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("spl", [1, 25])
def test_ca_count_fused_into_the_steps(fr, mode, spl):
    k, n = 10, 1024
    plan = fr.fractal_map(k, 32, mode)
    if spl > 1:
        fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_U8, spl)
    s0 = synth.bernoulli_u8(61, n)
    mask = domain(k).mask
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for steps in (0, 1, 7, 40):
        a = dev_u8(s0)
        b = torch.zeros_like(a)
        res = fr.fractal_step_ca_count(plan, a, b, steps, out[1:])
        want = oracle.ca_run(s0, steps, domain(k))
        assert out[1].item() == int(want[mask].sum()) == fr.fractal_reduce(plan, res, fr.FRACTAL_U8)
        assert out[0].item() == -1.0


def test_ca_zero_steps_and_states(fr):
    k, n = 6, 64
    plan = fr.fractal_map(k, 16)
    s0 = synth.bernoulli_u8(1, n)
    a = dev_u8(s0)
    b = torch.zeros_like(a)
    assert fr.fractal_step_ca(plan, a, b, 0) is a
    assert np.array_equal(a.cpu().numpy().reshape(n, n), s0)
    # any nonzero byte is alive
    s2 = s0 * np.uint8(77)
    got, _, _ = run_ca(fr, plan, s2, 4)
    want = oracle.ca_run(s0, 4, domain(k))
    assert np.array_equal(got[domain(k).mask], want[domain(k).mask])


def test_ca_hand_cases_on_gpu(fr):
    from conftest import read_golden
    for line in read_golden("ca_hand_cases.txt"):
        head, before, after = line.split("|")
        _, k, steps = head.split()
        n = 1 << int(k)
        s = np.zeros((n, n), dtype=np.uint8)
        for tok in before.split():
            x, y = map(int, tok.split(","))
            s[y, x] = 1
        for rho in (1, 2, 4, 8):
            got, _, _ = run_ca(fr, fr.fractal_map(int(k), rho), s, int(steps), 0)
            cells = {(int(x), int(y)) for y, x in zip(*np.nonzero(got))}
            want = set() if after.strip() == "-" else {tuple(map(int, t.split(","))) for t in after.split()}
            assert cells == want, (head, rho)


# ------------------------------------------------------------ diffusion ----

def run_diffusion(fr, plan, u0, steps, a=0.2, sentinel=SENTINEL_F32):
    n = u0.shape[0]
    ua = dev_f32(u0)
    ub = torch.full_like(ua, sentinel)
    out = fr.fractal_step_diffusion(plan, ua, ub, a, steps)
    return out.cpu().numpy().reshape(n, n)


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k,rho", cases([1, 2, 3, 4, 6, 8, 10]))
def test_diffusion_parity(fr, k, rho, mode, sched):
    n = 1 << k
    plan = make_plan(fr, k, rho, mode, sched)
    u0 = synth.uniform_f32(k, n)
    want = oracle.diffusion_run(u0.astype(np.float64), 7, 0.2, domain(k))
    got = run_diffusion(fr, plan, u0, 7)
    mask = domain(k).mask
    err, _ = rel_err(got, want, mask)
    assert err <= 2e-6, err
    cover = tile_cover(n, rho)
    assert np.all(got[cover & ~mask] == 0)
    assert np.array_equal(got[~cover], np.full_like(got[~cover], SENTINEL_F32))
    assert fr.fractal_plan_device_status(plan) == 0


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("spl", [2, 3, 4, 8, 16, 32, 50, 100])
@pytest.mark.parametrize("k,rho", [(5, 4), (6, 8), (8, 4), (8, 8), (9, 16), (10, 32), (10, 8), (11, 16)])
def test_diffusion_fused_parity(fr, k, rho, mode, spl):
    # several steps per launch: same field as the oracle, same result buffer,
    # cells outside member tiles untouched
    n = 1 << k
    plan = fr.fractal_map(k, rho, mode)
    margin = 8
    while margin < spl:
        margin *= 2
    if min(1 << k, rho << 5) < 2 * margin:     # super-tile side: at most rho * 2^5 and n
        with pytest.raises(fr.FractalError):       # no super-tile of side >= 2 * margin
            fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, spl)
        return
    fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, spl)
    assert plan.info()["steps_per_launch"][1] == spl
    u0 = synth.uniform_f32(70 + k, n)
    mask = domain(k).mask
    cover = tile_cover(n, rho)
    for steps in (1, 5, 8, 13, 2 * spl + 1):
        want = oracle.diffusion_run(u0.astype(np.float64), steps, 0.2, domain(k))
        got = run_diffusion(fr, plan, u0, steps)
        # FP32 rounding grows with the steps (1e-4 after 1000, the bound of the workload)
        bound = 2e-6 + 1e-7 * steps
        assert rel_err(got, want, mask)[0] <= bound, (steps, rel_err(got, want, mask))
        assert np.all(got[cover & ~mask] == 0)
        if steps % 2:
            assert np.all(got[~cover] == SENTINEL_F32)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("spl", [8, 32, 100])
def test_diffusion_fused_1000_steps(fr, mode, spl):
    k, n = 10, 1024
    u0 = synth.uniform_f32(3, n)
    want = oracle.diffusion_run(u0.astype(np.float64), 1000, 0.2, domain(k))
    plan = fr.fractal_map(k, 8, mode)
    fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, spl)
    got = run_diffusion(fr, plan, u0, 1000)
    err, raw = rel_err(got, want, domain(k).mask)
    assert err <= 1e-4, (err, raw)


@pytest.mark.parametrize("spl", [1, 4, 8])
def test_diffusion_zero_coefficient_is_identity(fr, spl):
    k, n = 9, 512
    plan = fr.fractal_map(k, 8)
    if spl > 1:
        fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, spl)
    u0 = synth.uniform_f32(4, n)
    got = run_diffusion(fr, plan, u0, 10, a=0.0)
    mask = domain(k).mask
    assert np.array_equal(got[mask], u0[mask])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("spl", [1, 8, 32])
def test_diffusion_sum_fused_into_the_steps(fr, mode, spl):
    k, n = 10, 1024
    plan = fr.fractal_map(k, 8, mode)
    if spl > 1:
        fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, spl)
    u0 = synth.uniform_f32(62, n)
    dom = domain(k)
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    for steps in (0, 1, 7, 40):
        a = dev_f32(u0)
        b = torch.zeros_like(a)
        res = fr.fractal_step_diffusion_sum(plan, a, b, 0.2, steps, out[1:])
        got = out[1].item()
        assert got == pytest.approx(fr.fractal_reduce(plan, res, fr.FRACTAL_F32), rel=1e-6)
        host = res.cpu().numpy().reshape(n, n)
        assert got == pytest.approx(oracle.reduce_sum(dom.take(host).astype(np.float64)), rel=1e-6)
        assert out[0].item() == -1.0


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("spl", [1, 8, 25, 50])
def test_diffusion_sums_every(fr, mode, spl):
    """A sum every `every` steps in one call (the state kept in records across
    the sums): each sum and the result against the oracle run segment by
    segment, the same sums as separate calls."""
    k, n = 10, 1024
    plan = fr.fractal_map(k, 8, mode)
    if spl > 1:
        fr.fractal_plan_set_steps_per_launch(plan, fr.FRACTAL_F32, spl)
    u0 = synth.uniform_f32(63, n)
    dom = domain(k)
    for steps, every in ((60, 20), (50, 25), (9, 3), (7, 7)):
        a = dev_f32(u0)
        b = torch.full_like(a, SENTINEL_F32)
        sums = torch.full((steps // every + 1,), -1.0, dtype=torch.float64, device="cuda")
        res = fr.fractal_step_diffusion_sums(plan, a, b, 0.2, steps, every, sums)
        assert sums[-1].item() == -1.0                      # nothing beyond steps / every sums
        v = dom.take(u0).astype(np.float64)
        for j in range(steps // every):
            for _ in range(every):
                v = oracle.diffusion_step(dom, v, 0.2)
            assert sums[j].item() == pytest.approx(oracle.reduce_sum(v), rel=1e-5), (steps, every, j)
        got = res.cpu().numpy().reshape(n, n)
        want = dom.put(v, np.float64)
        assert rel_err(got, want, dom.mask)[0] <= 2e-6 + 1e-7 * steps
        # the same sums as one call per segment
        a2 = dev_f32(u0)
        b2 = torch.zeros_like(a2)
        one = torch.zeros(1, dtype=torch.float64, device="cuda")
        cur, oth = a2, b2
        for j in range(steps // every):
            cur = fr.fractal_step_diffusion_sum(plan, cur, oth, 0.2, every, one)
            oth = b2 if cur is a2 else a2
            assert one.item() == pytest.approx(sums[j].item(), rel=1e-6)
    a = dev_f32(u0)
    b = torch.zeros_like(a)
    sums = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(fr.FractalError):
        fr.fractal_step_diffusion_sums(plan, a, b, 0.2, 10, 3, sums)        # not a multiple
    with pytest.raises(fr.FractalError):
        fr.fractal_step_diffusion_sums(plan, a, b, 0.2, 10, 0, sums)        # every < 1
    fr.fractal_step_diffusion_sums(plan, a, b, 0.2, 0, 5, sums)             # no steps: nothing written
    assert sums[0].item() == -1.0


def test_fused_needs_room(fr):
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_set_steps_per_launch(fr.fractal_map(3, 4), fr.FRACTAL_F32, 8)   # super-tile < 16
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_set_steps_per_launch(fr.fractal_map(10, 8), fr.FRACTAL_F32, 129)
    p = fr.fractal_map(10, 8)
    fr.fractal_plan_set_steps_per_launch(p, fr.FRACTAL_F32, 1)
    assert p.info()["steps_per_launch"] == [1, 1]


@pytest.mark.parametrize("k,rho", [(9, 4), (9, 8), (10, 16), (10, 32)])
@pytest.mark.parametrize("sched", SCHEDS)
def test_diffusion_every_cta_level(fr, k, rho, sched):
    n = 1 << k
    u0 = synth.uniform_f32(50 + k, n)
    want = oracle.diffusion_run(u0.astype(np.float64), 3, 0.2, domain(k))
    mask = domain(k).mask
    for mode in MODES:
        plan = make_plan(fr, k, rho, mode, sched)
        rb = k - int(np.log2(rho))
        for m in range(0, min(rb, 5) + 1):
            try:
                fr.fractal_plan_set_cta_levels(plan, fr.FRACTAL_F32, m)
            except fr.FractalError:
                continue
            got = run_diffusion(fr, plan, u0, 3)
            assert rel_err(got, want, mask)[0] <= 1e-6, (mode, m)


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("mode", MODES)
def test_diffusion_1000_steps(fr, mode, sched):
    # the accuracy bound at the step count of the k = 14 workload, on k = 10
    k, n = 10, 1024
    u0 = synth.uniform_f32(3, n)
    want = oracle.diffusion_run(u0.astype(np.float64), 1000, 0.2, domain(k))
    got = run_diffusion(fr, make_plan(fr, k, 8, mode, sched), u0, 1000)
    err, raw = rel_err(got, want, domain(k).mask)
    assert err <= 1e-4, (err, raw)


def test_diffusion_conserves_and_ignores_nonmembers(fr):
    k, n = 8, 256
    plan = fr.fractal_map(k, 8)
    u0 = synth.uniform_f32(2, n)
    noisy = u0.copy()
    noisy[~domain(k).mask] = np.float32(np.nan)
    got = run_diffusion(fr, plan, noisy, 40)
    clean = run_diffusion(fr, plan, u0, 40)
    mask = domain(k).mask
    assert np.array_equal(got[mask], clean[mask])
    s0 = u0[mask].astype(np.float64).sum()
    assert abs(got[mask].astype(np.float64).sum() - s0) <= 1e-5 * s0


# --------------------------------------------------------------- reduce ----

@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("k,rho", cases([0, 1, 3, 5, 8, 10]))
def test_reduce(fr, k, rho, mode):
    n = 1 << k
    plan = fr.fractal_map(k, rho, mode)
    mask = oracle.member_mask(n)
    s = synth.bernoulli_u8(7, n)
    assert fr.fractal_reduce(plan, dev_u8(s), fr.FRACTAL_U8) == int(s[mask].sum())
    u = synth.uniform_f32(7, n)
    want = oracle.reduce_sum(u[mask])
    got = fr.fractal_reduce(plan, dev_f32(u), fr.FRACTAL_F32)
    assert abs(got - want) <= 1e-6 * max(want, 1.0)
    # deterministic
    assert fr.fractal_reduce(plan, dev_f32(u), fr.FRACTAL_F32) == got
    # reduce of the single write is the volume 3^k (Eq. 2)
    b = torch.zeros(n * n, dtype=torch.float32, device="cuda")
    fr.fractal_map_write(plan, b, fr.FRACTAL_F32, 1.0)
    assert fr.fractal_reduce(plan, b, fr.FRACTAL_F32) == 3 ** k


def test_reduce_async_device_output(fr):
    k, n = 9, 512
    plan = fr.fractal_map(k, 16)
    s = synth.bernoulli_u8(5, n)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    fr.fractal_reduce_async(plan, dev_u8(s), fr.FRACTAL_U8, out[1:])
    torch.cuda.synchronize()
    assert out[1].item() == int(s[oracle.member_mask(n)].sum())
    assert out[0].item() == 0.0


# ------------------------------------------------------------ generator ----

@pytest.mark.parametrize("n", [1, 64, 1000])
def test_device_generator_matches_host(fr, n):
    b = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    synth.device_fill(b.data_ptr(), synth.SYNTH_BERNOULLI_U8, n, 42)
    f = torch.empty(n * n, dtype=torch.float32, device="cuda")
    synth.device_fill(f.data_ptr(), synth.SYNTH_UNIFORM_F32, n, 42, lo=0.5, width=1.0)
    torch.cuda.synchronize()
    assert np.array_equal(b.cpu().numpy().reshape(n, n), synth.bernoulli_u8(42, n))
    assert np.array_equal(f.cpu().numpy().reshape(n, n), synth.uniform_f32(42, n, lo=0.5))


# -------------------------------------------------------------- errors -----

def test_l2_fetch_granularity_hint(fr):
    old = fr.fractal_get_l2_fetch_granularity()
    for v in (32, 64, 128):
        fr.fractal_set_l2_fetch_granularity(v)
        assert fr.fractal_get_l2_fetch_granularity() == v
    with pytest.raises(fr.FractalError):
        fr.fractal_set_l2_fetch_granularity(48)
    fr.fractal_set_l2_fetch_granularity(old if old in (32, 64, 128) else 64)


def test_runtime_validation(fr):
    plan = fr.fractal_map(6, 8)
    a = torch.zeros(64 * 64 + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(fr.FractalError):
        fr.fractal_step_ca(plan, a, a, 1)                 # same buffer
    with pytest.raises(fr.FractalError):
        fr.fractal_step_ca(plan, a[1:], a[16:], 1)        # misaligned
    with pytest.raises(fr.FractalError):
        fr.fractal_step_ca(plan, a[:4096], a[16:], -1)    # negative steps
    f = torch.zeros(2 * 64 * 64, dtype=torch.float32, device="cuda")
    with pytest.raises(fr.FractalError):
        fr.fractal_step_diffusion(plan, f[:4096], f[4096:], float("nan"), 1)
    with pytest.raises(fr.FractalError):
        fr.fractal_map_write(plan, f, 5, 1.0)
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_set_cta_levels(plan, 0, 9)
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_set_schedule(plan, 7)
    tiny = fr.fractal_map(2, 1)        # rows of 1 element: no TMA kernel applies
    with pytest.raises(fr.FractalError):
        fr.fractal_plan_set_schedule(tiny, fr.FRACTAL_SCHED_TMA)


@pytest.mark.parametrize("dtype", [0, 1])
def test_autotune_keeps_results_exact(fr, dtype):
    k, n = 12, 4096
    plan = fr.fractal_map(k, 16)
    if dtype == 0:
        s0 = synth.bernoulli_u8(9, n)
        src, scratch = dev_u8(s0), torch.zeros(n * n, dtype=torch.uint8, device="cuda")
    else:
        s0 = synth.uniform_f32(9, n)
        src, scratch = dev_f32(s0), torch.zeros(n * n, dtype=torch.float32, device="cuda")
    keep = src.clone()
    us = fr.fractal_plan_autotune(plan, dtype, src, scratch, 3)
    assert us > 0
    assert torch.equal(src, keep)                      # the input is only read
    mask = domain(k).mask
    if dtype == 0:
        got, _, _ = run_ca(fr, plan, s0, 3)
        assert np.array_equal(got[mask], oracle.ca_run(s0, 3, domain(k))[mask])
    else:
        got = run_diffusion(fr, plan, s0, 3)
        want = oracle.diffusion_run(s0.astype(np.float64), 3, 0.2, domain(k))
        assert rel_err(got, want, mask)[0] <= 1e-6
    assert fr.fractal_plan_device_status(plan) == 0


def test_plan_reports_tma(fr):
    inf = fr.fractal_map(16, 8).info()
    assert inf["tma"] == [0, 1]          # uint8 rho = 8 stages by vector loads; float32 by TMA
    inf = fr.fractal_map(16, 32).info()
    assert inf["tma"] == [1, 1]
    p = fr.fractal_map(16, 32)
    fr.fractal_plan_set_schedule(p, fr.FRACTAL_SCHED_STAGED)
    assert p.info()["tma"] == [0, 0]
