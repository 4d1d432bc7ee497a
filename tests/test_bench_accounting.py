"""The benchmark's roofline accounting on CPU: the algorithmic flops and bytes
it divides by, pinned to the oracle's member graph and to hand counts."""
import oracle

import bench


def test_diffusion_flops_count_the_member_links():
    # 2 deg + 1 flops per member update; the links of the level-k gasket are
    # 3^k - 1 (three copies joined by two links per level)
    for k in range(1, 8):
        dom = oracle.Domain.build(1 << k)
        deg = (dom.nb4 >= 0).sum(axis=1)
        assert int(deg.sum()) // 2 == 3 ** k - 1
        assert bench.diffusion_flops_per_step(k) == int((2 * deg + 1).sum())


def test_launch_kinds_follow_the_step_driver():
    # ceil(steps / spl) launches per segment (two for a one-launch call of an
    # even number of steps); records between the launches of one call
    assert bench.fused_launch_kinds(100, 50) == ["ER", "RE"]
    assert bench.fused_launch_kinds(100, 25) == ["ER", "RR", "RR", "RE"]
    assert bench.fused_launch_kinds(100, 100) == ["ER", "RE"]
    assert bench.fused_launch_kinds(25, 25) == ["EE"]
    assert bench.fused_launch_kinds(26, 26) == ["ER", "RE"]
    assert bench.fused_launch_kinds(3, 3) == ["EE"]
    assert bench.kernel_launches(50, 100) == 2 and bench.kernel_launches(25, 100) == 4
    assert bench.kernel_launches(50, 75) == 2                      # no parity launch: records decouple
    assert bench.fused_launch_kinds(200, 25, 100) == ["ER"] + ["RR"] * 6 + ["RE"]
    assert bench.kernel_launches(50, 200, 100) == 4 and bench.kernel_launches(100, 200, 100) == 2


def test_launch_bytes_by_hand():
    # k = 5: 9 member 8 x 8 blocks (256 B embedded, 112 B records), 1 word tile
    assert bench.fused_launch_bytes("diffusion", "EE", 5, 0) == 9 * 512
    assert bench.fused_launch_bytes("diffusion", "ER", 5, 2) == 11 * 256 + 9 * 112
    assert bench.fused_launch_bytes("diffusion", "RR", 5, 2) == 11 * 112 + 9 * 112
    assert bench.fused_launch_bytes("diffusion", "RE", 5, 2) == 11 * 112 + 9 * 256
    assert bench.fused_launch_bytes("ca", "ER", 5, 3) == 1024 + 3 * 32 + 128
    assert bench.fused_launch_bytes("ca", "RE", 5, 3) == 128 + 3 * 4 + 1024


def test_box_blocks_within_reach_agree_with_the_library():
    """The algorithmic bytes count the margin-box blocks a launch stages: at
    reach = margin all member blocks of the boxes, fewer for a shorter reach,
    and never more per super-tile than the library gives thread slots to
    (fractal_fused_box_blocks, the most any super-tile has)."""
    from paper_2004_13475_gb300 import build as fbuild
    import paper_2004_13475_gb300 as fr
    fbuild.build()
    k, T, M = 12, 256, 64
    supertiles = 3 ** (k - 8)
    full = bench.diffusion_box_member_blocks(k, T, M)
    assert bench.diffusion_box_member_blocks(k, T, M, M) == full
    prev = full
    for reach in (50, 40, 25, 9, 1):
        c = bench.diffusion_box_member_blocks(k, T, M, reach)
        assert c <= prev
        assert c <= supertiles * fr.fractal_fused_box_blocks(T, M, reach)
        prev = c
    assert bench.diffusion_box_member_blocks(k, T, M, 50) < full


def test_automaton_words_are_the_member_holding_row_segments():
    """The automaton's ALU accounting counts one 32-cell word per row of every
    member 32 x 32 word tile: exactly the 32-aligned row segments of the
    array that hold at least one gasket member (brute force over the
    oracle's membership)."""
    import numpy as np
    for k in range(5, 11):
        n = 1 << k
        mask = oracle.member_mask(n)
        holding = mask.reshape(n, n // 32, 32).any(axis=2)
        assert int(np.count_nonzero(holding)) == bench.ca_words_per_step(k)


def test_automaton_ops_per_word_by_hand():
    # per word and step: the row's three-cell sum (2 funnel shifts, sum bit,
    # carry bit) and the rule modulo 4 (5 three-input logic operations)
    assert bench.CA_OPS_PER_WORD_STEP == 4 + 5
    assert abs(bench.ALU_PEAK_TOPS - 152 * 64 * 2.07e-3) < 1e-9


def test_committed_profile_tables_parse():
    """profiles/traffic.txt and profiles/stalls.txt name kernels whose sources
    the bench can hash, with well-formed values (the bench reports them only
    while the hashes match)."""
    import os
    for path, ncol in ((bench.TRAFFIC_FILE, 4), (bench.STALLS_FILE, 4)):
        assert os.path.exists(path)
        rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
        assert rows
        for r in rows:
            assert len(r) >= ncol and r[0] in bench.KERNEL_SOURCES
            assert len(bench.sources_hash(r[0])) == 16
    for r in (ln.split() for ln in open(bench.STALLS_FILE) if ln.strip() and not ln.startswith("#")):
        assert all(float(kv.split("=")[1]) >= 0 for kv in r[3:])


def test_bench_nbb_steps_match_the_oracle():
    """The NBB steps bench.py measures are the oracle's (same cells, same order)."""
    from oracle import nbb
    for name, (s, cells) in bench.NBB_STEPS.items():
        s2, k2, cells2 = nbb.FRACTALS[name]
        assert s == s2 and len(cells) == k2 and [tuple(c) for c in cells] == list(cells2)
