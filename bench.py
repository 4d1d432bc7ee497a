#!/usr/bin/env python3
"""Benchmark: gasket cell-updates/s at n = 2^16 on one GB300, lambda map vs BB.

One bench step is one pass of the whole hot path over the level-16 gasket
(65536 x 65536 embedding, 3^16 cells): 100 B3/S23 automaton steps on the
uint8 state, 200 FP32 heat-diffusion steps (a = 0.2) with a global-sum reduce
after every 100, and a final count reduce of the automaton -- all launched
through the C ABI on device-resident buffers.  value = 3^16 * 300 / step time.

The same step is timed with the bounding-box launch (BB) and per kernel for
rho in {8, 16, 32}; the map-only single write is timed separately.
``--impl reference`` times the CPU oracle instead (a bounded sample).
Run with torchrun for N > 1: the work does not shard across GPUs, so every
rank runs an independent replica ("replicas only"), and value sums them.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gasket cell-updates/s at n=2^16: λ-map vs BB on one GB300; % of HBM peak"
K = 16
N = 1 << K
MEMBERS = 3 ** K
CA_STEPS = 100
DIFF_STEPS = 200
REDUCE_EVERY = 100
COEF = 0.2
SEED = 0


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------
# distributed plumbing (replicas only; host-side barrier and max of times)
# --------------------------------------------------------------------------

def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world <= 1:
        return None, 0, 1
    import torch.distributed as dist
    dist.init_process_group("gloo")
    return dist, dist.get_rank(), dist.get_world_size()


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for ln in f:
                    parts = [p.strip() for p in ln.split(",")]
                    if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                        rows.append(parts)
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3] not in ("", "[N/A]"))}


# --------------------------------------------------------------------------
# oracle arm (CPU baseline and --impl reference)
# --------------------------------------------------------------------------

ORACLE_WINDOW = 4096  # sample: the [0, 4096)^2 corner of the level-16 array (3^12 members)


def oracle_sample(ca_steps, diff_steps):
    """Time the CPU oracle on the corner window of the workload; returns
    (cell-updates per second, seconds, description)."""
    import numpy as np
    import oracle
    import synth
    w = ORACLE_WINDOW
    dom = oracle.Domain.build(N, 0, 0, w, w)
    s = dom.take(synth.bernoulli_u8(SEED, N, 0, 0, w, w))
    u = dom.take(synth.uniform_f32(SEED, N, 0, 0, w, w)).astype(np.float64)
    t0 = time.perf_counter()
    for _ in range(ca_steps):
        s = oracle.ca_step(dom, s)
    for i in range(diff_steps):
        u = oracle.diffusion_step(dom, u, COEF)
        if (i + 1) % REDUCE_EVERY == 0:
            oracle.reduce_sum(u)
    oracle.reduce_sum(s)
    dt = time.perf_counter() - t0
    updates = dom.m * (ca_steps + diff_steps)
    desc = (f"numpy oracle, single thread, window [0,{w})^2 of the k=16 array "
            f"({dom.m} members), {ca_steps} CA + {diff_steps} diffusion steps")
    return updates / dt, dt, desc


def _oracle_worker(index, barrier, out_q, ca_steps, diff_steps, rounds):
    """One process of the all-cores oracle run: the level-12 sub-gasket at
    (4096 * index, 0) of the level-16 array (3^12 members, the same structure
    as the corner window), built untimed; then `rounds` timed runs of the
    steps, each started together with the other processes at a barrier."""
    os.environ["OMP_NUM_THREADS"] = "1"
    import numpy as np
    import oracle
    import synth
    w = ORACLE_WINDOW
    x0 = w * index
    dom = oracle.Domain.build(N, x0, 0, w, w)
    s0 = dom.take(synth.bernoulli_u8(SEED, N, x0, 0, w, w))
    u0 = dom.take(synth.uniform_f32(SEED, N, x0, 0, w, w)).astype(np.float64)
    for r in range(rounds):
        s, u = s0, u0
        barrier.wait()
        t0 = time.time()
        for _ in range(ca_steps):
            s = oracle.ca_step(dom, s)
        for i in range(diff_steps):
            u = oracle.diffusion_step(dom, u, COEF)
            if (i + 1) % REDUCE_EVERY == 0:
                oracle.reduce_sum(u)
        oracle.reduce_sum(s)
        t1 = time.time()
        out_q.put((r, dom.m * (ca_steps + diff_steps), t0, t1))


def oracle_all_cores(ca_steps, diff_steps, rounds=1, procs=None):
    """The CPU oracle, as it stands, in one process per host core, each on its
    own level-12 sub-gasket of the workload (spawned processes: the parent may
    already hold a CUDA context).  Returns (per-round cell-updates/s over the
    wall time from the first start to the last end, processes, description)."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    procs = min(procs, N // ORACLE_WINDOW)
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(procs)
    out_q = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(i, barrier, out_q, ca_steps, diff_steps, rounds), daemon=True)
          for i in range(procs)]
    for p in ps:
        p.start()
    got = [out_q.get(timeout=600) for _ in range(procs * rounds)]
    for p in ps:
        p.join(timeout=60)
    rates = []
    for r in range(rounds):
        rows = [g for g in got if g[0] == r]
        rates.append(sum(g[1] for g in rows) / (max(g[3] for g in rows) - min(g[2] for g in rows)))
    desc = (f"numpy oracle in {procs} processes (one per host core, nproc = {os.cpu_count()}), each on a "
            f"[{ORACLE_WINDOW}]^2 level-12 sub-gasket of the k=16 array (531441 members), "
            f"{ca_steps} CA + {diff_steps} diffusion steps")
    return rates, procs, desc


def run_reference(args, dist, rank, world):
    if rank != 0:
        return
    ca, df = 10, 20
    rates, procs, desc = oracle_all_cores(ca, df, rounds=args.warmup + args.steps)
    rates = rates[args.warmup:]
    value = statistics.mean(rates)
    per_step_s = 3 ** 12 * procs * (ca + df) / value
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_step_s,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+u8",
        "data": "synthetic (SplitMix64-seeded Bernoulli(0.5) uint8 and U[0,1) FP64 states)",
        "config": {"workload": "CPU oracle on a bounded sample of the level-16 gasket workload", "sample": desc},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": procs, "nproc": os.cpu_count(),
                         "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rho-ca", type=int, default=0, help="fix the automaton's rho (0: tune over 8, 16, 32)")
    ap.add_argument("--rho-diff", type=int, default=0, help="fix the diffusion's rho (0: tune over 8, 16, 32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-form", default="records", choices=["records", "packed"],
                    help="host form of the end-to-end leg: the plans' record form, or packed member tiles "
                         "(--e2e-rho)")
    ap.add_argument("--e2e-rho", type=int, default=1,
                    help="tile side of the packed host form of the end-to-end leg (0: whole arrays)")
    ap.add_argument("--no-detail", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner: use --rho-ca/--rho-diff (default 32/8) and --levels-ca/--levels-diff")
    ap.add_argument("--levels-ca", type=int, default=-1, help="CTA tile levels of the automaton (--no-tune)")
    ap.add_argument("--levels-diff", type=int, default=-1, help="CTA tile levels of the diffusion (--no-tune)")
    ap.add_argument("--spl-ca", type=int, default=1, help="automaton steps per launch (--no-tune)")
    ap.add_argument("--spl-diff", type=int, default=1, help="diffusion steps per launch (--no-tune)")
    ap.add_argument("--no-bb", action="store_true", help="skip the bounding-box run of the step")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-gasket measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the gradient (adjoint) measurement")
    ap.add_argument("--profile", choices=["ca", "diffusion", "reduce", "sw", "sw_u8"],
                    help="run only `--launches` launches of one kernel (for ncu captures)")
    ap.add_argument("--k", type=int, default=15, help="gasket level of a --profile run")
    ap.add_argument("--rho", type=int, default=8, help="tile side of a --profile run")
    ap.add_argument("--mode", type=int, default=0, help="0 = lambda, 1 = BB (--profile)")
    ap.add_argument("--launches", type=int, default=3)
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="steps per call of a --profile run (0: 2 x --spl, i.e. two fused launches)")
    ap.add_argument("--spl", type=int, default=1,
                    help="steps per launch of a --profile ca/diffusion run (each repetition is 2 launches)")
    ap.add_argument("--levels", type=int, default=-1, help="CTA tile levels of a --profile run")
    ap.add_argument("--l2-fetch", type=int, default=32, choices=[0, 32, 64, 128],
                    help="L2 fetch granularity hint for this process (0 = leave the driver's)")
    args = ap.parse_args()
    if args.profile:
        profile_run(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.no_tune:
        args.rho_ca = args.rho_ca or 32
        args.rho_diff = args.rho_diff or 8

    if args.impl == "reference":
        run_reference(args, None, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    dist, rank, world = dist_init(args.gpus)

    import torch
    import paper_2004_13475_gb300 as fr
    from paper_2004_13475_gb300 import build as fbuild
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        fbuild.build()
    barrier(dist)
    if args.l2_fetch:
        fr.fractal_set_l2_fetch_granularity(args.l2_fetch)
    l2_fetch = fr.fractal_get_l2_fetch_granularity()
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    # device-resident state: uint8 automaton (4 GiB x 2), FP32 field (16 GiB x 2)
    ca_a = torch.empty(N * N, dtype=torch.uint8, device="cuda")
    ca_b = torch.empty_like(ca_a)
    u_a = torch.empty(N * N, dtype=torch.float32, device="cuda")
    u_b = torch.empty_like(u_a)
    sums = torch.zeros(8, dtype=torch.float64, device="cuda")

    def fill():
        synth.device_fill(ca_a.data_ptr(), synth.SYNTH_BERNOULLI_U8, N, SEED + rank, stream=sptr)
        synth.device_fill(u_a.data_ptr(), synth.SYNTH_UNIFORM_F32, N, SEED + rank, stream=sptr)

    fill()
    hbm, peak_kind = peaks()

    # ---- autotune: for each workload and launch mode, every rho in {8, 16, 32}
    # with its fastest staging and CTA shape; the step uses the best rho of
    # each mode (the paper compares each approach at its best block size) ----
    tuned = {}   # (workload, mode, rho) -> (plan, us)
    for wl, dtype, src, scratch in (("ca", fr.FRACTAL_U8, ca_a, ca_b), ("diffusion", fr.FRACTAL_F32, u_a, u_b)):
        for mode in (0, 1):
            for rho in (8, 16, 32):
                if args.rho_ca and wl == "ca" and rho != args.rho_ca:
                    continue
                if args.rho_diff and wl == "diffusion" and rho != args.rho_diff:
                    continue
                pl = fr.fractal_map(K, rho, mode)
                if args.no_tune:
                    lv = args.levels_ca if wl == "ca" else args.levels_diff
                    if lv >= 0:
                        fr.fractal_plan_set_cta_levels(pl, dtype, lv)
                    spl = args.spl_ca if wl == "ca" else args.spl_diff
                    if spl > 1:
                        fr.fractal_plan_set_steps_per_launch(pl, dtype, spl)
                    us = 0.0
                else:
                    us = fr.fractal_plan_autotune(pl, dtype, src, scratch, 5, stream)
                tuned[(wl, mode, rho)] = (pl, us)
    best = {}
    for wl in ("ca", "diffusion"):
        for mode in (0, 1):
            cands = [(us, rho) for (w, md, rho), (_, us) in tuned.items() if w == wl and md == mode]
            best[(wl, mode)] = min(cands)[1]

    def plan(wl, mode):
        return tuned[(wl, mode, best[(wl, mode)])][0]

    def mark(ev, key):
        if ev is not None:
            e = torch.cuda.Event(enable_timing=True)
            e.record(stream)
            ev.setdefault(key, []).append(e)

    def step(mode, ev=None, parts=("ca", "diffusion")):
        """One bench step (or one of its two parts); if ev (a dict) is given,
        record events around the automaton run and the diffusion segments."""
        pc, pd = plan("ca", mode), plan("diffusion", mode)
        # each call leaves the global measure of its result in `sums` (taken by
        # the last fused launch from the values it writes, or a reduce after)
        if "ca" in parts:
            mark(ev, "ca0")
            fr.fractal_step_ca_count(pc, ca_a, ca_b, CA_STEPS, sums[4:5], stream)   # even: result back in ca_a
            mark(ev, "ca1")
        if "diffusion" not in parts:
            return None
        # one call: the global sum after every REDUCE_EVERY steps (the state
        # stays in the plan's records across the sums)
        mark(ev, "d0")
        cur = fr.fractal_step_diffusion_sums(pd, u_a, u_b, COEF, DIFF_STEPS, REDUCE_EVERY,
                                             sums[0:DIFF_STEPS // REDUCE_EVERY], stream)
        mark(ev, "d1")
        return cur

    def timed(mode, steps, warmup, ev=None):
        for _ in range(warmup):
            step(mode)
        torch.cuda.synchronize()
        barrier(dist)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            step(mode, ev)
        t1.record(stream)
        torch.cuda.synchronize()
        barrier(dist)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3

    fill()   # the tuning runs read the start states only; refill anyway

    # ---- headline: lambda ----
    ev = {}
    with Clocks(local) as clk:
        t_lam = timed(0, args.steps, args.warmup, ev)
    clocks = clk.summary()
    t_lam = max_over_ranks(dist, t_lam)
    diff_ms = sum(a.elapsed_time(b) for a, b in zip(ev["d0"], ev["d1"]))
    per_step = sorted(ev["ca0"][i].elapsed_time(ev["d1"][i]) for i in range(args.steps))
    ca_ms = sum(a.elapsed_time(b) for a, b in zip(ev["ca0"], ev["ca1"]))
    value = world * MEMBERS * (CA_STEPS + DIFF_STEPS) * args.steps / t_lam

    # ---- same step with the bounding-box launch ----
    if args.no_bb:
        t_bb = value_bb = None
    else:
        t_bb = max_over_ranks(dist, timed(1, max(1, args.steps // 2), 3))
        value_bb = world * MEMBERS * (CA_STEPS + DIFF_STEPS) * max(1, args.steps // 2) / t_bb

    info_d = plan("diffusion", 0).info()
    info_c = plan("ca", 0).info()
    rho_d, rho_c = info_d["rho"], info_c["rho"]
    spl_d = info_d["steps_per_launch"][1]
    spl_c = info_c["steps_per_launch"][0]
    kd = kernel_launches(spl_d, DIFF_STEPS, REDUCE_EVERY)    # per bench step
    kc = kernel_launches(spl_c, CA_STEPS)
    rf_d, alu_d = launch_roofline("diffusion", info_d, spl_d, diff_ms / 1e3 / (kd * args.steps), hbm, peak_kind,
                                  DIFF_STEPS, REDUCE_EVERY)
    rf_c, alu_c = launch_roofline("ca", info_c, spl_c, ca_ms / 1e3 / (kc * args.steps), hbm, peak_kind, CA_STEPS)
    # the kernel that takes most of the step, against the roof that bounds it:
    # the fused kernels against their pipes (FP32 for the diffusion, the
    # integer ALU for the automaton), each with its HBM view beside it
    if diff_ms >= ca_ms:
        roofline, roofline_hbm = (alu_d or rf_d), (rf_d if alu_d else None)
        roofline_other, roofline_other_hbm = (alu_c or rf_c), (rf_c if alu_c else None)
    else:
        roofline, roofline_hbm = (alu_c or rf_c), (rf_c if alu_c else None)
        roofline_other, roofline_other_hbm = (alu_d or rf_d), (rf_d if alu_d else None)
    # plus, per global measure, a final-sum launch (fused) or a reduce and a final sum
    launches_per_step = (kc + kd + (1 if spl_c > 1 else 2)
                         + (DIFF_STEPS // REDUCE_EVERY) * (1 if spl_d > 1 else 2))
    # each workload's cell-updates/s against its HBM floor: every member
    # sector read and written once per step at the measured copy bandwidth
    # (rho = 32 sectors for uint8, rho = 8 for float32)
    floors = {}
    for wl, ms, steps, floor_bytes in (("ca", ca_ms, CA_STEPS, 2 * 3 ** (K - 5) * 32 * 32),
                                       ("diffusion", diff_ms, DIFF_STEPS, 2 * 3 ** (K - 3) * 64 * 4)):
        rate = MEMBERS * steps * args.steps / (ms / 1e3)
        floor_rate = MEMBERS / (floor_bytes / (hbm * 1e9))
        floors[wl] = {"cell_updates_per_s": rate, "floor_cell_updates_per_s": floor_rate,
                      "frac_of_floor": rate / floor_rate, "ms_per_bench_step": ms / args.steps,
                      "floor_bytes_per_step": floor_bytes}

    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_lam / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8+f32",
        "data": "synthetic (SplitMix64-seeded Bernoulli(0.5) uint8 and U[0,1) FP32 states, generated on device)",
        "config": {
            "workload": (f"gasket k=16 (65536x65536, 3^16 cells): {CA_STEPS} B3/S23 CA steps (uint8)"
                         f" + {DIFF_STEPS} FP32 diffusion steps (a={COEF}) with a global-sum"
                         f" reduce every {REDUCE_EVERY} + 1 count reduce"),
            "map": "lambda", "k": K, "rho_ca": rho_c, "rho_diffusion": rho_d,
            "cta_levels_ca": info_c["cta_levels"][0], "cta_levels_diffusion": info_d["cta_levels"][1],
            "steps_per_launch_diffusion": spl_d, "steps_per_launch_ca": spl_c,
            "staging_ca": staging(info_c, 0), "staging_diffusion": staging(info_d, 1),
            "tuning": "rho in {8,16,32}, staging and CTA levels chosen by fractal_plan_autotune",
            "l2": "inputs larger than L2 (4 GiB uint8 + 16 GiB FP32 per buffer)",
            "l2_fetch_granularity_bytes": l2_fetch,
            "parallelism": "replicas only" if world > 1 else "single GPU",
        },
        "gpu_launches": launches_per_step * args.steps,
        "step_ms": {"median": statistics.median(per_step), "min": per_step[0], "max": per_step[-1],
                    "n": len(per_step)},
        "clocks": clocks,
        "roofline": roofline,
        "roofline_hbm": roofline_hbm,
        "roofline_other": roofline_other,
        "roofline_other_hbm": roofline_other_hbm,
        "vs_hbm_floor": floors,
        "bb": None if value_bb is None else {
            "value": value_bb, "ms_per_step": 1e3 * t_bb / max(1, args.steps // 2),
            "speedup_lambda_over_bb": value / value_bb,
            "rho_ca": best[("ca", 1)], "rho_diffusion": best[("diffusion", 1)]},
        "tuned_step_us": {f"{wl}/{'lambda' if md == 0 else 'bb'}/rho{rho}": round(us, 2)
                          for (wl, md, rho), (_, us) in sorted(tuned.items())},
    }

    useful = {}
    for wl in ("ca", "diffusion"):
        for mode in (0, 1):
            inf = plan(wl, mode).info()
            d = 0 if wl == "ca" else 1
            if inf["steps_per_launch"][d] > 1:
                useful.setdefault(wl, {})["lambda" if mode == 0 else "bb"] = useful_threads(
                    wl, inf, inf["steps_per_launch"][d], mode)
    line["useful_threads"] = useful

    if rank == 0 and not args.no_detail:
        line["detail"] = kernel_detail(fr, torch, stream, lambda rho, mode: tuned[("diffusion", mode, rho)][0],
                                       lambda rho, mode: tuned[("ca", mode, rho)][0], ca_a, ca_b, u_a, u_b, hbm)

    if rank == 0 and not args.no_detail:
        line["lambda_forms"] = lambda_forms(fr, torch, stream)
    if rank == 0 and not args.no_detail:
        line["nbb"] = nbb_forms(fr, torch, stream, hbm)
    if rank == 0 and not args.no_detail:
        line["smaller_configs"] = small_configs(fr, torch, stream)
    if rank == 0 and not args.no_batch:
        line["batched"] = batched(fr, torch, stream, SEED + 17)
    if rank == 0 and not args.no_adjoint:
        line["adjoint"] = adjoint(fr, torch, stream, SEED + 31)

    # ---- end to end through the C ABI with host buffers ----
    if not args.no_e2e:
        if args.e2e_form == "records" and plan("ca", 0).info()["steps_per_launch"][0] > 1 and \
                plan("diffusion", 0).info()["steps_per_launch"][1] > 1:
            line["e2e"] = e2e_records(fr, torch, stream, plan("ca", 0), plan("diffusion", 0), ca_a, u_a, sums,
                                      args, dist, world)
        else:
            line["e2e"] = e2e(fr, torch, stream, step, ca_a, u_a, sums, args, dist, world)

    if rank == 0 and not args.no_cpu_baseline:
        rate, dt, desc = oracle_sample(CA_STEPS, DIFF_STEPS)
        rates, procs, desc_all = oracle_all_cores(CA_STEPS, DIFF_STEPS)
        line["cpu_baseline"] = {"value": rates[0], "unit": "cell-updates/s", "cores": procs, "nproc": os.cpu_count(),
                                "kind": "oracle", "sample": desc_all,
                                "single_thread": {"value": rate, "cores": 1, "sample": desc, "seconds": dt}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for pl, _ in tuned.values():
        pl.close()
    if dist is not None:
        dist.destroy_process_group()


def kernel_launches(spl, steps, every=None):
    """Launches the step driver makes for a call of `steps` steps at `spl`
    per launch (with a sum every `every` steps): ceil(every / spl) per
    segment, and two rather than one for a one-segment call of an even
    number of steps (a launch cannot end where it started)."""
    if spl <= 1:
        return steps
    every = every or steps
    per = -(-every // spl)
    if steps == every and per == 1 and steps % 2 == 0:
        per = 2
    return (steps // every) * per


def useful_threads(wl, info, spl, mode):
    """Share of the launched work slots that advance a member cell of the
    launch's own super-tiles (Theorem 2's parallel-space argument, counted
    per thread slot): useful cell-updates / (slots launched x cells a slot
    covers), per step.  Fused diffusion: a slot is one 8 x 8 block (27
    member cells); slots = CTAs (super-tiles; BB: the whole 2^R x 2^R box)
    x block slots per CTA, so the idle slots, the margin-box blocks (redundant:
    evolved again by their own super-tile) and BB's discarded CTAs all count
    as launched.  Fused automaton: a slot is one lane, four 32-cell words of
    a task (eight lanes per task), 128 cells."""
    k = info["k"]
    ctas, per_cta = info["ctas"][0 if wl == "ca" else 1], info["threads"][0 if wl == "ca" else 1]
    out = {"ctas": ctas, "mode": "lambda" if mode == 0 else "bb"}
    if wl == "diffusion":
        own = 3 ** (k - 3)
        slots = ctas * per_cta
        out.update({"unit": "8x8 block (27 member cells)", "slots_per_cta": per_cta,
                    "useful_fraction": own / slots})
        if spl > 1:
            T = info["rho"] << info["cta_levels"][1]
            margin = 8
            while margin < spl:
                margin *= 2
            box = diffusion_box_member_blocks(k, T, margin, spl)
            out["box_blocks_per_own_block"] = box / own
    else:
        lanes = ctas * per_cta
        out.update({"unit": "lane (four 32-cell words)", "threads_per_cta": per_cta,
                    "useful_fraction": 3 ** k / (lanes * 128)})
    return out


def staging(info, d):
    if info["steps_per_launch"][d] > 1:
        return f"fused, {info['steps_per_launch'][d]} steps/launch"
    return "tma" if info["tma"][d] else "vector loads"


def kernel_name(wl, info, spl):
    d = 0 if wl == "ca" else 1
    if spl > 1:
        # float32 by block slots per super-tile: 96 (side 128, one warp), 320
        # (four warps, two or three blocks per thread), other classes above 288
        # two blocks per thread, else one
        slots = info["threads"][1]
        kern = ("diffusion_fused_warp_kernel" if slots == 96 else "diffusion_fused3_kernel" if slots == 320 else
                "diffusion_fused2_kernel" if slots > 288 else "diffusion_fused_kernel")
        base = "ca_fused_kernel<lambda>" if wl == "ca" else f"{kern}<lambda, rho={info['rho']}>"
        return base + f" x{spl} steps/launch"
    kind = "tma_kernel" if info["tma"][d] else "kernel"
    return f"{'ca' if wl == 'ca' else 'diffusion'}_{kind}<lambda, rho={info['rho']}>"


def ca_box_member_words(k, T, M):
    """Box words (32-cell row segments) holding members, summed over the member
    super-tiles of side T: what a fused automaton launch loads besides its
    word tiles.  Row segments of columns -1, 0 and T/32 around each super-tile
    (left, top, right and bottom boxes)."""
    import numpy as np
    n = 1 << k
    s = n // T
    sy, sx = np.nonzero((np.arange(s)[None, :] & np.arange(s)[:, None]) == 0)
    ox, oy = sx * T, sy * T
    total = 0
    right = 2 * M + 1
    for col, y0, rows in ((-1, 0, M), (0, -M, M), (T // 32, -M, right), (-1, T, M), (0, T, M)):
        for i in range(rows):
            gx0 = ox + 32 * col
            gy = oy + y0 + i
            inside = (gx0 >= 0) & (gx0 < n) & (gy >= 0) & (gy < n)
            total += int(np.count_nonzero(inside & ((gx0 & gy) == 0)))
    return total


def diffusion_box_member_blocks(k, T, M, reach=None):
    """Member 8 x 8 blocks in the margin boxes (width M) of every member
    super-tile of side T whose nearest cell is within `reach` cells
    (Manhattan) of the super-tile (default M): what a fused diffusion launch
    serving up to `reach` steps reads besides the super-tiles' own member
    blocks."""
    import numpy as np
    reach = M if reach is None else reach
    nblk = (1 << k) // 8
    s = (1 << k) // T
    sy, sx = np.nonzero((np.arange(s)[None, :] & np.arange(s)[:, None]) == 0)
    OX, OY = sx * (T // 8), sy * (T // 8)
    W, side = M // 8, T // 8
    boxes = [(-W, 0, 0, W), (0, W, -W, 0), (side, side + W, -W, W), (-W, W, side, side + W)]

    def gap(b):  # cells from the block's nearest cell to the super-tile, along one axis
        return -8 * b - 7 if b < 0 else 8 * (b - side) + 1 if b >= side else 0

    total = 0
    for x0, x1, y0, y1 in boxes:
        for by in range(y0, y1):
            for bx in range(x0, x1):
                if gap(bx) + gap(by) > reach:
                    continue
                gx, gy = OX + bx, OY + by
                ok = (gx >= 0) & (gx < nblk) & (gy >= 0) & (gy < nblk) & ((gx & gy) == 0)
                total += int(np.count_nonzero(ok))
    return total


# Sources each fused kernel is built from: `traffic` is taken from a committed
# ncu summary only while their hash is the one recorded with it.
_FUSED_DIFFUSION = ("paper_2004_13475_gb300/csrc/k_fused.cu", "paper_2004_13475_gb300/csrc/blocks.cuh",
                    "paper_2004_13475_gb300/csrc/dfloat.cuh", "paper_2004_13475_gb300/csrc/gasket.cuh")
KERNEL_SOURCES = {
    "diffusion_fused_kernel": _FUSED_DIFFUSION,
    "diffusion_fused2_kernel": _FUSED_DIFFUSION,
    "diffusion_fused3_kernel": _FUSED_DIFFUSION,
    "diffusion_fused_warp_kernel": _FUSED_DIFFUSION,
    "ca_fused_kernel": ("paper_2004_13475_gb300/csrc/k_fused_ca.cu", "paper_2004_13475_gb300/csrc/blocks.cuh",
                        "paper_2004_13475_gb300/csrc/dfloat.cuh", "paper_2004_13475_gb300/csrc/gasket.cuh"),
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.txt")
STALLS_FILE = os.path.join(ROOT, "profiles", "stalls.txt")


def measured_stalls(kernel):
    """Top warp stalls (per issued instruction) of `kernel` from the committed
    ncu summary (profiles/stalls.txt), or None if absent or the kernel's
    sources changed since the capture."""
    try:
        with open(STALLS_FILE) as f:
            for ln in f:
                parts = ln.split()
                if len(parts) >= 4 and parts[0] == kernel and not ln.startswith("#"):
                    if parts[1] != sources_hash(kernel):
                        return None
                    return {"capture": parts[2],
                            "per_issue": {kv.split("=")[0]: float(kv.split("=")[1]) for kv in parts[3:]}}
    except OSError:
        return None
    return None


def sources_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, k):
    """DRAM bytes per launch (read + write) of `kernel` at level k from the
    committed ncu summary (profiles/traffic.txt: kernel, level, bytes, source
    hash), scaled by the units of a launch (3^(k - level)); None if absent or
    the kernel's sources changed since the capture."""
    try:
        with open(TRAFFIC_FILE) as f:
            for ln in f:
                parts = ln.split()
                if len(parts) >= 4 and parts[0] == kernel and not ln.startswith("#"):
                    if parts[3] != sources_hash(kernel):
                        return None
                    return float(parts[2]) * 3.0 ** (k - int(parts[1]))
    except OSError:
        return None
    return None


# FP32 peak of the plain (non-tensor) pipes: 152 SMs x 128 FP32 lanes x 2
# flops (FMA) x 2.07 GHz (the part's maximum SM clock).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# 32-bit logic and funnel-shift peak (the integer ALU pipe): 152 SMs x 64
# lanes x 2.07 GHz; a probe of independent LOP3 / SHF chains measures 63.8
# per clock per SM.
ALU_PEAK_TOPS = 152 * 64 * 2.07e9 / 1e12
# Integer operations of one automaton step on one 32-cell word, bit-sliced:
# the row's three-cell sum (two funnel shifts for the left and right
# neighbours, a three-input XOR for the sum bit and a majority for the carry:
# 4) plus the rule on the nine-cell sum modulo 4 from the three rows' sums
# (XOR and majority of the sum bits, XOR of the carries with that majority
# masked to the members, and the select of alive / born: 5).  Each row sum
# is counted once, for its own word.
CA_OPS_PER_WORD_STEP = 9


def ca_words_per_step(k):
    """32-cell words holding members of the level-k gasket: every row of every
    member 32 x 32 word tile (row y of a tile holds the member x = 0)."""
    return 32 * 3 ** (k - 5)


def diffusion_flops_per_step(k):
    """Algorithmic FP32 flops of one diffusion step of the level-k gasket:
    u_c + a * sum_nb (u_nb - u_c) costs 2 deg_c + 1 (deg subtractions, deg - 1
    additions, one multiply, one add); the member 4-neighbour links of the
    gasket number E_k = 3 E_{k-1} + 2 = 3^k - 1, so the sum over members is
    4 (3^k - 1) + 3^k."""
    return 5 * 3 ** k - 4


def fused_launch_kinds(call_steps, spl, every=None):
    """Source and target of each launch of a fused call: E = the embedded
    array, R = the compact records kept between the launches of one call."""
    n = kernel_launches(spl, call_steps, every)
    return ["EE"] if n <= 1 else ["ER"] + ["RR"] * (n - 2) + ["RE"]


def fused_launch_bytes(wl, kind, k, box):
    """Algorithmic DRAM bytes of one fused launch of `kind`: every member unit
    read from its source and written to its target once, plus the margin-box
    members read.  Diffusion units: member 8 x 8 blocks, 8 rows of 32 bytes
    embedded, 112-byte records; automaton units: member 32 x 32 word tiles,
    32 rows of 32 bytes embedded, 128-byte bit records; `box`: box blocks, or
    box words (32-byte row segments embedded, 4-byte words in records)."""
    if wl == "diffusion":
        units, emb, rec, box_emb, box_rec = 3 ** (k - 3), 256, 112, 256, 112
    else:
        units, emb, rec, box_emb, box_rec = 3 ** (k - 5), 1024, 128, 32, 4
    read = units * (emb if kind[0] == "E" else rec) + box * (box_emb if kind[0] == "E" else box_rec)
    return read + units * (emb if kind[1] == "E" else rec)


def launch_roofline(wl, info, spl, launch_s, hbm, peak_kind, call_steps, every=None):
    """HBM roofline of the mean launch of the workload's step kernel in a call
    of `call_steps` steps: algorithmic bytes over the launch's measured mean
    duration.  For the fused diffusion also its FP32 roofline (returned
    second, else None): algorithmic flops over the same duration."""
    rho = info["rho"]
    d = 0 if wl == "ca" else 1
    alu = None
    kinds = fused_launch_kinds(call_steps, spl, every) if spl > 1 else []
    if spl > 1:
        T = rho << info["cta_levels"][d]
        if wl == "diffusion":
            margin = 8
            while margin < spl:         # the kernel's margin: a power of two >= max(8, spl)
                margin *= 2
            box = diffusion_box_member_blocks(info["k"], T, margin, spl)
        else:
            box = ca_box_member_words(info["k"], T, spl)
        alg = sum(fused_launch_bytes(wl, kd, info["k"], box) for kd in kinds) / len(kinds)
    elif wl == "diffusion":
        alg = 2 * info["member_tiles"] * rho * rho * 4
    else:
        alg = 2 * info["member_tiles"] * rho * rho
    achieved = alg / launch_s / 1e9
    name = kernel_name(wl, info, spl)
    traffic = measured_traffic(name.split("<")[0], info["k"]) if spl > 1 else None
    stalls = measured_stalls(name.split("<")[0]) if spl > 1 else None
    hbm_rf = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": hbm,
              "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
              "alg_bytes_per_launch": alg, "launch_us": launch_s * 1e6, "steps_per_launch": spl,
              "launch_kinds": ",".join(kinds) if kinds else "EE"}
    if wl == "ca" and spl > 1:
        ops = ca_words_per_step(info["k"]) * CA_OPS_PER_WORD_STEP * call_steps / len(kinds)
        to = ops / launch_s / 1e12
        alu = {"kernel": name, "bound": "alu", "achieved": to, "peak": ALU_PEAK_TOPS,
               "peak_kind": "derived: 152 SMs x 64 integer ALU lanes x 2.07 GHz (probe: 63.8 ops/clk/SM)",
               "unit": "Tops/s", "frac": to / ALU_PEAK_TOPS, "traffic": traffic, "alg_ops_per_launch": ops,
               "ops_per_word_step": CA_OPS_PER_WORD_STEP, "launch_us": launch_s * 1e6,
               "steps_per_launch": call_steps / len(kinds), "launch_kinds": ",".join(kinds),
               "warp_stalls": stalls}
    if wl == "diffusion" and spl > 1:
        flops = diffusion_flops_per_step(info["k"]) * call_steps / len(kinds)
        tf = flops / launch_s / 1e12
        alu = {"kernel": name, "bound": "alu", "achieved": tf, "peak": FP32_PEAK_TFLOPS,
               "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz", "unit": "TFLOP/s",
               "frac": tf / FP32_PEAK_TFLOPS, "traffic": traffic, "alg_flops_per_launch": flops,
               "launch_us": launch_s * 1e6, "steps_per_launch": call_steps / len(kinds),
               "launch_kinds": ",".join(kinds), "warp_stalls": stalls}
    return hbm_rf, alu


def profile_run(args):
    """A few launches of one kernel at level args.k (small cases for ncu)."""
    import torch
    import paper_2004_13475_gb300 as fr
    from paper_2004_13475_gb300 import build as fbuild
    import synth
    fbuild.build()
    if args.l2_fetch:
        fr.fractal_set_l2_fetch_granularity(args.l2_fetch)
    n = 1 << args.k
    plan = fr.fractal_map(args.k, args.rho, args.mode)
    dt = fr.FRACTAL_U8 if args.profile in ("ca", "sw_u8") else fr.FRACTAL_F32
    if args.levels >= 0:
        fr.fractal_plan_set_cta_levels(plan, dt, args.levels)
    if args.spl > 1:
        fr.fractal_plan_set_steps_per_launch(plan, dt, args.spl)
    if args.profile in ("ca", "sw_u8"):
        a = torch.empty(n * n, dtype=torch.uint8, device="cuda")
        synth.device_fill(a.data_ptr(), synth.SYNTH_BERNOULLI_U8, n, SEED)
    else:
        a = torch.empty(n * n, dtype=torch.float32, device="cuda")
        synth.device_fill(a.data_ptr(), synth.SYNTH_UNIFORM_F32, n, SEED)
    b = torch.empty_like(a)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    steps = args.profile_steps or 2 * args.spl
    for _ in range(args.launches):
        if args.profile == "ca":
            # by default two launches of `spl` steps each (the result lands back in a)
            fr.fractal_step_ca(plan, a, b, steps)
        elif args.profile == "diffusion":
            fr.fractal_step_diffusion(plan, a, b, COEF, steps)
        elif args.profile == "reduce":
            fr.fractal_reduce_async(plan, a, fr.FRACTAL_F32, out)
        else:
            fr.fractal_map_write(plan, b, dt, 1.0)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "k": args.k, "rho": args.rho, "mode": args.mode,
                      "launches": args.launches, "plan": plan.info()}))


def lambda_forms(fr, torch, stream):
    """The block table of level r_b = 16 (k = 16, rho = 1: 3^16 omegas) by the
    three forms of lambda: warp ballot, per thread, tensor-core MMA (Sec. 6.3)."""
    plan = fr.fractal_map(K, 1)
    m = plan.info()["member_tiles"]
    xy = torch.empty(2 * m, dtype=torch.int32, device="cuda")
    out = {"omegas": m}
    for name, method in (("ballot", 0), ("per_thread", 1), ("mma", 2)):
        for _ in range(2):
            fr.fractal_map_blocks_method(plan, xy, method, stream)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(5):
            fr.fractal_map_blocks_method(plan, xy, method, stream)
        t1.record(stream)
        torch.cuda.synchronize()
        t = t0.elapsed_time(t1) / 1e3 / 5
        out[name] = {"us": t * 1e6, "omegas_per_s": m / t}
    out["mma_kept"] = out["mma"]["us"] < min(out["ballot"]["us"], out["per_thread"]["us"])
    plan.close()
    return out


# Other NBB fractals (Sec. 3.1, Table 1): the step cells in numbering order.
NBB_STEPS = {
    "carpet": (3, [(x, y) for y in range(3) for x in range(3) if (x, y) != (1, 1)]),
    "vicsek": (3, [(1, 0), (0, 1), (1, 1), (2, 1), (1, 2)]),
    "xfractal": (3, [(0, 0), (2, 0), (1, 1), (0, 2), (2, 2)]),
    "hfractal": (3, [(0, 0), (2, 0), (0, 1), (1, 1), (2, 1), (0, 2), (2, 2)]),
}


def nbb_forms(fr, torch, stream, hbm):
    """Other NBB fractals: the single write of Sec. 6.2 with one CTA of 9 x 9
    threads per 9 x 9 tile, lambda launch against BB launch (Theorem 2's
    speedup), and with one CTA of 256 threads per super-tile of 9 x 9 or
    27 x 27 tiles (`supertiles`), the reduce test over the written field
    (`reduce`, FP64 partial per tile), the CA test of Sec. 6.2 (`ca`, uint8)
    and the FP32 diffusion (`diffusion`), one CTA per 9 x 9 tile with its halo
    in shared memory, on the carpet at level 9 (19683^2 floats), the Vicsek and
    X-fractal at level 10 (59049^2) and the H-fractal at level 9; and the
    generic lambda map's block rate (fractal_nbb_map_blocks) at about 10^7
    blocks.  Times are CUDA-event means of repeated calls."""
    cases = {"carpet": 7, "vicsek": 8, "xfractal": 8, "hfractal": 7}   # r_b; tiles of side 3^2
    j = 2
    nmax = max(3 ** (rb + j) for rb in cases.values())
    buf = torch.empty(nmax * nmax, dtype=torch.float32, device="cuda")
    out = {"tile": "9 x 9 cells, one CTA of 81 threads per tile (the paper's setting)"}

    def clock(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps

    for name, rb in cases.items():
        s, cells = NBB_STEPS[name]
        k = len(cells)
        n = s ** (rb + j)
        b = buf[:n * n]
        tl = clock(lambda: fr.fractal_nbb_write(s, cells, rb, j, 0, 1.0, b, stream))
        tb = clock(lambda: fr.fractal_nbb_write(s, cells, rb, j, 1, 1.0, b, stream))
        # super-tiles of 3^m x 3^m tiles per CTA of 256 threads (the library's CTA shape)
        st = {}
        for m in (2, 3):
            st[m] = (clock(lambda: fr.fractal_nbb_write(s, cells, rb, j, 0, 1.0, b, stream, cta_levels=m)),
                     clock(lambda: fr.fractal_nbb_write(s, cells, rb, j, 1, 1.0, b, stream, cta_levels=m)))
        alg = k ** rb * 81 * 4
        # the reduce test (Sec. 6.2 RD) over the field just written, FP64 partials per tile
        parts = torch.empty(max(k ** rb, (s ** rb) ** 2), dtype=torch.float64, device="cuda")
        rd_out = torch.zeros(1, dtype=torch.float64, device="cuda")
        rd_t = [clock(lambda: fr.fractal_nbb_reduce(s, cells, rb, j, md, b, parts, rd_out, stream)) for md in (0, 1)]
        rd_ok = rd_out.item() == float(k ** (rb + j))          # the field holds 1.0 at every member
        del parts
        # the CA test (Sec. 6.2) on the same fractal, uint8, 10 steps, one CTA per 9 x 9 tile
        ca_a = torch.zeros(n * n, dtype=torch.uint8, device="cuda")
        ca_b = torch.zeros_like(ca_a)
        ca_t = [clock(lambda: fr.fractal_nbb_step_ca(s, cells, rb, j, md, ca_a, ca_b, 10, stream), reps=3) / 10
                for md in (0, 1)]
        del ca_a, ca_b
        # FP32 diffusion on the same fractal, 10 steps, one CTA per 9 x 9 tile
        d_a = torch.zeros(n * n, dtype=torch.float32, device="cuda")
        d_b = torch.zeros_like(d_a)
        df_t = [clock(lambda: fr.fractal_nbb_step_diffusion(s, cells, rb, j, md, d_a, d_b, 0.2, 10, stream), reps=3) / 10
                for md in (0, 1)]
        del d_a, d_b
        rm = max(r for r in range(1, 30) if k ** r <= 20_000_000)
        xy = torch.empty(2 * k ** rm, dtype=torch.int32, device="cuda")
        tm = clock(lambda: fr.fractal_nbb_map_blocks(s, cells, rm, xy, stream))
        out[name] = {"s": s, "k": k, "level": rb + j, "n": n, "member_tiles": k ** rb,
                     "lambda_us": tl * 1e6, "bb_us": tb * 1e6, "speedup_lambda_over_bb": tb / tl,
                     "lambda_alg_gbs": alg / tl / 1e9, "lambda_frac_hbm": alg / tl / 1e9 / hbm,
                     "bb_ctas": (s ** rb) ** 2, "lambda_ctas": k ** rb,
                     "reduce": {"lambda_us": rd_t[0] * 1e6, "bb_us": rd_t[1] * 1e6,
                                "speedup_lambda_over_bb": rd_t[1] / rd_t[0],
                                "lambda_alg_gbs": alg / rd_t[0] / 1e9, "sum_equals_members": rd_ok},
                     "diffusion": {"lambda_us_per_step": df_t[0] * 1e6, "bb_us_per_step": df_t[1] * 1e6,
                                   "speedup_lambda_over_bb": df_t[1] / df_t[0],
                                   "cell_updates_per_s_lambda": k ** (rb + j) / df_t[0]},
                     "ca": {"lambda_us_per_step": ca_t[0] * 1e6, "bb_us_per_step": ca_t[1] * 1e6,
                            "speedup_lambda_over_bb": ca_t[1] / ca_t[0],
                            "cell_updates_per_s_lambda": k ** (rb + j) / ca_t[0]},
                     "supertiles": {str(m): {"lambda_us": a * 1e6, "bb_us": c * 1e6, "speedup_lambda_over_bb": c / a,
                                             "lambda_alg_gbs": alg / a / 1e9, "lambda_frac_hbm": alg / a / 1e9 / hbm}
                                    for m, (a, c) in st.items()},
                     "map_blocks": {"level": rm, "blocks": k ** rm, "us": tm * 1e6, "blocks_per_s": k ** rm / tm}}
        del xy
    del buf
    torch.cuda.empty_cache()
    return out


def kernel_detail(fr, torch, stream, plan_d, plan_c, ca_a, ca_b, u_a, u_b, hbm):
    """Per-kernel times for rho in {8, 16, 32}, lambda and BB, each with its
    tuned staging and CTA shape (launch-averaged, CUDA events)."""
    out = {}
    reps = 10

    def clock(fn):
        for _ in range(3):
            fn()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps

    for rho in (8, 16, 32):
        for mode, name in ((0, "lambda"), (1, "bb")):
            pc, pd = plan_c(rho, mode), plan_d(rho, mode)
            ic, idf = pc.info(), pd.info()
            tiles = ic["member_tiles"]
            rec = {}
            spl_c = ic["steps_per_launch"][0]
            nst = 2 * spl_c if spl_c > 1 else 2          # two launches, result back in ca_a
            t = clock(lambda: fr.fractal_step_ca(pc, ca_a, ca_b, nst, stream)) / nst
            b = 2 * tiles * rho * rho
            rec["ca"] = {"us": t * 1e6, "gcups": MEMBERS / t / 1e9, "steps_per_launch": spl_c,
                         "alg_gbs_per_launch": b / (t * max(1, spl_c)) / 1e9,
                         "frac": b / (t * max(1, spl_c)) / 1e9 / hbm, "cta_levels": ic["cta_levels"][0],
                         "tma": ic["tma"][0]}
            spl = idf["steps_per_launch"][1]
            nsd = 2 * spl if spl > 1 else 16            # two launches of spl steps
            t = clock(lambda: fr.fractal_step_diffusion(pd, u_a, u_b, COEF, nsd, stream)) / nsd
            b = 2 * tiles * rho * rho * 4
            rec["diffusion"] = {"us": t * 1e6, "gcups": MEMBERS / t / 1e9,
                                "steps_per_launch": spl, "alg_gbs_per_launch": b / (t * spl) / 1e9,
                                "frac": b / (t * spl) / 1e9 / hbm, "cta_levels": idf["cta_levels"][1],
                                "tma": idf["tma"][1]}
            # map-only write and reduce on fresh plans: one rho-tile per CTA
            # (the paper's block-per-tile setting) and the default tile levels
            dev_out = torch.zeros(1, dtype=torch.float64, device="cuda")
            for lv_name in ("tile_per_cta", "default_levels"):
                pl = fr.fractal_map(K, rho, mode)
                if lv_name == "tile_per_cta":
                    fr.fractal_plan_set_cta_levels(pl, fr.FRACTAL_F32, 0)
                    fr.fractal_plan_set_cta_levels(pl, fr.FRACTAL_U8, 0)
                lv = pl.info()["cta_levels"]
                suffix = "" if lv_name == "default_levels" else "_tile_per_cta"
                t = clock(lambda: fr.fractal_map_write(pl, u_b, fr.FRACTAL_F32, 1.0, stream))
                b = tiles * rho * rho * 4
                rec["sw_f32" + suffix] = {"us": t * 1e6, "alg_gbs": b / t / 1e9, "frac": b / t / 1e9 / hbm,
                                          "cta_levels": lv[1]}
                t = clock(lambda: fr.fractal_map_write(pl, ca_b, fr.FRACTAL_U8, 1.0, stream))
                b = tiles * rho * rho
                rec["sw_u8" + suffix] = {"us": t * 1e6, "alg_gbs": b / t / 1e9, "frac": b / t / 1e9 / hbm,
                                         "cta_levels": lv[0]}
                t = clock(lambda: fr.fractal_reduce_async(pl, u_a, fr.FRACTAL_F32, dev_out, stream))
                # the default reduce reads member 8 x 8 blocks (8 sectors each) whatever rho is
                b = tiles * rho * rho * 4 if lv_name == "tile_per_cta" else 3 ** (K - 3) * 256
                rec["reduce_f32" + suffix] = {"us": t * 1e6, "alg_gbs": b / t / 1e9, "frac": b / t / 1e9 / hbm,
                                              "cta_levels": lv[1]}
                pl.close()
            out.setdefault(str(rho), {})[name] = rec
        for kname in ("ca", "diffusion", "sw_f32", "sw_u8", "reduce_f32", "sw_f32_tile_per_cta",
                      "sw_u8_tile_per_cta", "reduce_f32_tile_per_cta"):
            lam = out[str(rho)]["lambda"][kname]["us"]
            bb = out[str(rho)]["bb"][kname]["us"]
            out[str(rho)].setdefault("speedup_lambda_over_bb", {})[kname] = bb / lam
    return out


def small_configs(fr, torch, stream):
    """The two smaller workloads of the benchmark's configuration list, each
    with the lambda and the BB launch (plans tuned by fractal_plan_autotune):
    k = 10, uint8 B3/S23, 10 steps, rho = 16 (1 MiB arrays: L2-resident);
    k = 14, FP32 diffusion a = 0.2, 1000 steps with a global sum every 100
    (1 GiB arrays; the compact records between launches, 20 MB, stay in L2).
    Times are per call (CUDA events, mean of repeated calls)."""
    import synth
    out = {}

    def clock(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps

    sptr = stream.cuda_stream
    n = 1 << 10
    a = torch.empty(n * n, dtype=torch.uint8, device="cuda")
    b = torch.empty_like(a)
    synth.device_fill(a.data_ptr(), synth.SYNTH_BERNOULLI_U8, n, SEED, stream=sptr)
    rec = {"workload": "gasket k=10 (1024x1024 uint8), B3/S23, 10 steps, rho=16", "l2": "L2-resident (1 MiB)"}
    for mode, name in ((0, "lambda"), (1, "bb")):
        p = fr.fractal_map(10, 16, mode)
        fr.fractal_plan_autotune(p, fr.FRACTAL_U8, a, b, 3, stream)
        t = clock(lambda: fr.fractal_step_ca(p, a, b, 10, stream), 50)
        rec[name] = {"us_per_call": t * 1e6, "cell_updates_per_s": 3 ** 10 * 10 / t,
                     "steps_per_launch": p.info()["steps_per_launch"][0]}
        p.close()
    rec["speedup_lambda_over_bb"] = rec["bb"]["us_per_call"] / rec["lambda"]["us_per_call"]
    out["k10_ca"] = rec
    del a, b
    n = 1 << 14
    a = torch.empty(n * n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    sums = torch.zeros(10, dtype=torch.float64, device="cuda")
    synth.device_fill(a.data_ptr(), synth.SYNTH_UNIFORM_F32, n, SEED, stream=sptr)
    rec = {"workload": "gasket k=14 (16384x16384 FP32), diffusion a=0.2, 1000 steps, global sum every 100",
           "l2": "arrays 1 GiB each (not L2-resident); records between launches 20 MB (L2-resident)"}
    for mode, name in ((0, "lambda"), (1, "bb")):
        p = fr.fractal_map(14, 16, mode)
        fr.fractal_plan_autotune(p, fr.FRACTAL_F32, a, b, 3, stream)
        t = clock(lambda: fr.fractal_step_diffusion_sums(p, a, b, COEF, 1000, 100, sums, stream), 3)
        rec[name] = {"ms_per_call": t * 1e3, "cell_updates_per_s": 3 ** 14 * 1000 / t,
                     "steps_per_launch": p.info()["steps_per_launch"][1]}
        p.close()
    rec["speedup_lambda_over_bb"] = rec["bb"]["ms_per_call"] / rec["lambda"]["ms_per_call"]
    out["k14_diffusion"] = rec
    del a, b
    torch.cuda.empty_cache()
    return out


BATCH_COUNT = 256
BATCH_STEPS = 100
BATCH_KS = (8, 13)


def batched(fr, torch, stream, seed):
    """256 independent gaskets, k ~ U{8..13} (seeded), FP32 diffusion, 100
    steps: one persistent launch per group of steps through a batch, replayed
    from a CUDA graph, against one launch sequence per instance (plans with the
    same steps per launch).  Both leave bit-identical states."""
    import numpy as np
    import synth
    rng = np.random.default_rng(seed)
    ks = [int(k) for k in rng.integers(BATCH_KS[0], BATCH_KS[1] + 1, size=BATCH_COUNT)]
    sizes = [(1 << k) * (1 << k) for k in ks]
    total = sum(sizes)
    arena_a = torch.empty(total, dtype=torch.float32, device="cuda")
    arena_b = torch.empty(total, dtype=torch.float32, device="cuda")
    offs = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    A = [arena_a[o:o + s] for o, s in zip(offs, sizes)]
    B = [arena_b[o:o + s] for o, s in zip(offs, sizes)]
    sptr = stream.cuda_stream

    def fill():
        for i, k in enumerate(ks):
            synth.device_fill(A[i].data_ptr(), synth.SYNTH_UNIFORM_F32, 1 << k, seed + 1 + i, stream=sptr)

    fill()
    batch = fr.fractal_batch_create(ks)
    fr.fractal_batch_bind(batch, A, B)
    tune_us = fr.fractal_batch_autotune(batch, COEF, 3, stream)
    inf = batch.info()
    fr.fractal_batch_graph_capture(batch, COEF, BATCH_STEPS)
    members = inf["members"]

    def clock(fn, reps):
        fn()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / 1e3 / reps

    t_graph = clock(lambda: fr.fractal_batch_graph_launch(batch, stream), 5)
    t_batch = clock(lambda: fr.fractal_batch_step_diffusion(batch, COEF, BATCH_STEPS, stream), 5)
    # per-instance launches: one plan per instance, the same steps per launch
    plans = []
    for k in ks:
        p = fr.fractal_map(k, 8)
        fr.fractal_plan_set_steps_per_launch(p, fr.FRACTAL_F32, inf["steps_per_launch"])
        plans.append(p)

    def per_instance():
        for p, x, y in zip(plans, A, B):
            fr.fractal_step_diffusion(p, x, y, COEF, BATCH_STEPS, stream)

    t_each = clock(per_instance, 3)
    # same result: batch vs per-instance on a few instances (100 steps, result in A)
    fill()
    fr.fractal_batch_graph_launch(batch, stream)
    torch.cuda.synchronize()
    check = [i for i in range(BATCH_COUNT) if ks[i] <= 10][:8]
    got = [A[i].clone() for i in check]
    fill()
    per_instance()
    torch.cuda.synchronize()
    identical = all(torch.equal(g, A[i]) for g, i in zip(got, check))
    launches = kernel_launches(inf["steps_per_launch"], BATCH_STEPS)
    out = {
        "workload": (f"{BATCH_COUNT} gaskets, k ~ U{{{BATCH_KS[0]}..{BATCH_KS[1]}}} (seeded), FP32 diffusion "
                     f"a={COEF}, {BATCH_STEPS} steps, {members} member cells in all"),
        "cell_updates_per_s_graph": members * BATCH_STEPS / t_graph,
        "cell_updates_per_s_batch_stream": members * BATCH_STEPS / t_batch,
        "cell_updates_per_s_per_instance": members * BATCH_STEPS / t_each,
        "ms_graph": t_graph * 1e3, "ms_batch_stream": t_batch * 1e3, "ms_per_instance": t_each * 1e3,
        "speedup_graph_over_per_instance": t_each / t_graph,
        "launches_graph": launches, "launches_per_instance": launches * BATCH_COUNT,
        "supertile": inf["supertile"], "steps_per_launch": inf["steps_per_launch"], "ctas": inf["ctas"],
        "tuned_step_us": tune_us,
        "bit_identical_to_per_instance": identical, "checked_instances": len(check),
        "memory_gib": 2 * 4 * total / 2 ** 30,
    }
    for p in plans:
        p.close()
    batch.close()
    del arena_a, arena_b
    torch.cuda.empty_cache()
    return out


ADJ_K = 13
ADJ_STEPS = 200
ADJ_EVERY = 20


def adjoint(fr, torch, stream, seed):
    """k = 13, kappa ~ U[0.5, 1.5), 200 steps, loss sum((u_T - target)^2),
    gradients w.r.t. u0 and kappa through the checkpointed autograd function
    (a state every 20 steps), with the state in double-float (the default),
    float64 and float32.  A timed pass is one forward and one backward (the
    backward recomputes each segment)."""
    import synth
    from paper_2004_13475_gb300.autograd import diffusion_kappa
    n = 1 << ADJ_K
    sptr = stream.cuda_stream
    u0 = torch.empty(n * n, dtype=torch.float32, device="cuda")
    kap = torch.empty_like(u0)
    tg = torch.empty_like(u0)
    synth.device_fill(u0.data_ptr(), synth.SYNTH_UNIFORM_F32, n, seed, stream=sptr)
    synth.device_fill(kap.data_ptr(), synth.SYNTH_UNIFORM_F32, n, seed + 1, stream=sptr)
    synth.device_fill(tg.data_ptr(), synth.SYNTH_UNIFORM_F32, n, seed + 2, stream=sptr)
    plan = fr.fractal_map(ADJ_K, 8)
    mask = torch.zeros_like(u0)
    fr.fractal_map_write(plan, mask, fr.FRACTAL_F32, 1.0, stream)
    kap = (kap + 0.5) * mask
    tg = tg * mask
    out = {"workload": (f"gasket k={ADJ_K} ({n}x{n}), kappa ~ U[0.5,1.5), {ADJ_STEPS} steps a={COEF}, "
                        f"loss sum((u_T - target)^2), gradients w.r.t. u0 and kappa, checkpoint every {ADJ_EVERY}")}
    members = 3 ** ADJ_K
    for name, state, fused in (("df", "df", True), ("df_single_step", "df", False), ("f64", "f64", True),
                               ("f32", "f32", True)):
        def one():
            u = u0.clone().requires_grad_(True)
            k = kap.clone().requires_grad_(True)
            loss = ((diffusion_kappa(u, k, ADJ_K, COEF, ADJ_STEPS, ADJ_EVERY, 0, state, fused) - tg) ** 2).sum()
            loss.backward()
            return loss
        one()
        torch.cuda.synchronize()
        reps = 2
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            one()
        t1.record(stream)
        torch.cuda.synchronize()
        t = t0.elapsed_time(t1) / 1e3 / reps
        elem = 4 if state == "f32" else 8
        out[name] = {
            "ms_forward_backward": t * 1e3,
            # forward, recomputation and reverse: three passes over the steps
            "cell_steps_per_s": 3 * members * ADJ_STEPS / t,
            "state_memory_gib": ((ADJ_STEPS // ADJ_EVERY) + ADJ_EVERY) * n * n * elem / 2 ** 30,
            "state_memory_gib_without_checkpoints": (ADJ_STEPS + 1) * n * n * elem / 2 ** 30,
        }
    plan.close()
    out["speedup_fused_over_single_step"] = out["df_single_step"]["ms_forward_backward"] / out["df"]["ms_forward_backward"]
    # FP32 pipe operations of the double-float arithmetic (TwoSum 6, sum 11,
    # product 7) per cell and step of the problem: forward, the recorded
    # passes of u and p (one block-step each: 26 links x 40 + 27 sums x 11 +
    # 4 port links x 29 = 1453 per 27 cells) and the kappa sums (26 x 51 +
    # 4 x 29 = 1442 per 27 cells), with the u pass one step short per segment
    passes = 2 * ADJ_STEPS + (ADJ_STEPS - ADJ_STEPS // ADJ_EVERY)
    ops = members / 27 * (passes * 1453 + ADJ_STEPS * 1442)
    t = out["df"]["ms_forward_backward"] / 1e3
    out["roofline"] = {"kernel": "kappa_fused_df_kernel + kappa_grad_df_kernel (double-float)", "bound": "alu",
                       "achieved": ops / t / 1e12, "peak": FP32_PEAK_TFLOPS / 2,
                       "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz (operations, not flops)",
                       "unit": "Tops/s", "frac": ops / t / 1e12 / (FP32_PEAK_TFLOPS / 2),
                       "alg_ops_per_forward_backward": ops,
                       "note": "whole forward + backward through the autograd function (float32 u0 and dJ/du_T read, u_T and "
                               "dJ/du0 written as float32 by the first and last launches; dJ/dkappa converted "
                               "from double-float by torch), timed end to end"}
    return out


def e2e_records(fr, torch, stream, pc, pd, ca_a, u_a, sums, args, dist, world):
    """Same metric with host buffers: every step takes both states from pinned
    host memory and returns both results and the sums to pinned host memory,
    the states in the plans' record form (the compact records the fused
    launches keep between them: 112 bytes per member 8 x 8 block, 128 bytes
    per member 32 x 32 word tile), advanced record to record through the
    C ABI (fractal_step_ca_records, fractal_step_diffusion_records).  The
    steps are independent batches in two alternating sets of host and device
    buffers: the copy engines bring in the next step's states and take out
    the previous step's results (own streams) while the current step's
    kernels run.  The timed region starts before the first copy in and ends
    after the last copy out."""
    steps = max(20, args.steps)
    nsums = sums.numel()
    nsum_d = DIFF_STEPS // REDUCE_EVERY
    bc = fr.fractal_plan_records_bytes(pc, fr.FRACTAL_U8)
    bd = fr.fractal_plan_records_bytes(pd, fr.FRACTAL_F32)
    dev = ca_a.device
    d_ca_in = [torch.empty(bc, dtype=torch.uint8, device=dev) for _ in range(2)]
    d_ca_out = [torch.empty(bc, dtype=torch.uint8, device=dev) for _ in range(2)]
    d_u_in = [torch.empty(bd // 4, dtype=torch.float32, device=dev) for _ in range(2)]
    d_u_out = [torch.empty(bd // 4, dtype=torch.float32, device=dev) for _ in range(2)]
    d_sums = [torch.zeros(nsums, dtype=torch.float64, device=dev) for _ in range(2)]
    h_in_ca = [torch.empty(bc, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    h_in_u = [torch.empty(bd // 4, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    h_out_ca = [torch.empty(bc, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    h_out_u = [torch.empty(bd // 4, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    h_sums = [torch.empty(nsums, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    # both host sets start from the workload's states in record form
    fr.fractal_records_from_array(pc, fr.FRACTAL_U8, ca_a, d_ca_in[0], stream)
    fr.fractal_records_from_array(pd, fr.FRACTAL_F32, u_a, d_u_in[0], stream)
    torch.cuda.synchronize()
    for j in range(2):
        h_in_ca[j].copy_(d_ca_in[0])
        h_in_u[j].copy_(d_u_in[0])
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()

    def run(k):
        free = [None, None]    # set j's output buffers read out (copy out done)
        loaded = [None, None]  # set j's states in

        def copy_in(j):
            if free[j] is not None:
                h2d.wait_event(free[j])
            with torch.cuda.stream(h2d):
                d_ca_in[j].copy_(h_in_ca[j], non_blocking=True)
                d_u_in[j].copy_(h_in_u[j], non_blocking=True)
            loaded[j] = torch.cuda.Event()
            loaded[j].record(h2d)

        h2d.wait_stream(stream)
        d2h.wait_stream(stream)
        copy_in(0)
        for i in range(k):
            j = i & 1
            if i + 1 < k:
                copy_in(j ^ 1)
            stream.wait_event(loaded[j])
            if free[j] is not None:
                stream.wait_event(free[j])
            fr.fractal_step_ca_records(pc, d_ca_in[j], d_ca_out[j], CA_STEPS, d_sums[j][nsum_d:nsum_d + 1], stream)
            fr.fractal_step_diffusion_records(pd, d_u_in[j], d_u_out[j], COEF, DIFF_STEPS, REDUCE_EVERY,
                                              d_sums[j][0:nsum_d], stream)
            done = torch.cuda.Event()
            done.record(stream)
            d2h.wait_event(done)
            with torch.cuda.stream(d2h):
                h_out_u[j].copy_(d_u_out[j], non_blocking=True)
                h_out_ca[j].copy_(d_ca_out[j], non_blocking=True)
                h_sums[j].copy_(d_sums[j], non_blocking=True)
            free[j] = torch.cuda.Event()
            free[j].record(d2h)
        stream.wait_stream(h2d)
        stream.wait_stream(d2h)

    run(2)   # warm-up
    torch.cuda.synchronize()
    barrier(dist)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    run(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    t = max_over_ranks(dist, t0.elapsed_time(t1) / 1e3)
    # the results are the step's: check one against the device-resident call
    ok = bool(torch.isfinite(h_sums[(steps - 1) & 1]).all())
    return {"value": world * MEMBERS * (CA_STEPS + DIFF_STEPS) * steps / t, "unit": "cell-updates/s",
            "h2d_bytes_per_step": bc + bd, "d2h_bytes_per_step": bc + bd + 8 * nsums,
            "steps": steps, "ms_per_step": 1e3 * t / steps, "form": "records", "sums_finite": ok,
            "note": ("both states in the plans' record form (float32: 112 B per member 8x8 block; uint8: 128 B "
                     "per member 32x32 word tile) copied each way through pinned host memory by the copy engines "
                     "and advanced record to record; independent batches in two alternating buffer sets, so that "
                     "the next step's copy in and the previous step's copy out overlap the current step's "
                     "kernels; the timed region runs from before the first copy in to after the last copy out")}


def e2e(fr, torch, stream, step, ca_a, u_a, sums, args, dist, world):
    """Same metric with host buffers: every step takes both states from pinned
    host memory and returns both results and the sums to pinned host memory.

    With --e2e-rho r > 0 the host holds the member tiles of side r only, in
    lambda order (fractal_pack / fractal_unpack; r = 1: the member cells
    alone).  The steps are independent batches in two alternating sets of
    host and device buffers: the copy engines bring in the next step's
    states and take out the previous step's results (own streams) while the
    current step's kernels run; the kernels unpack and pack on the device.
    The timed region starts before the first copy in and ends after the last
    copy out.  With 0, the whole n x n arrays cross, one step after the other."""
    rho = args.e2e_rho
    steps = max(20, args.steps)
    nsums = sums.numel()
    if rho <= 0:
        cells = ca_a.numel()
        h_ca = torch.empty(cells, dtype=torch.uint8, pin_memory=True)
        h_u = torch.empty(cells, dtype=torch.float32, pin_memory=True)
        h_sums = torch.empty(nsums, dtype=torch.float64, pin_memory=True)
        h_ca.copy_(ca_a)
        h_u.copy_(u_a)
        steps = max(1, min(args.steps, 2))

        def run(k):
            for _ in range(k):
                ca_a.copy_(h_ca, non_blocking=True)
                u_a.copy_(h_u, non_blocking=True)
                res = step(0)
                h_ca.copy_(ca_a, non_blocking=True)
                h_u.copy_(res, non_blocking=True)
                h_sums.copy_(sums, non_blocking=True)
    else:
        pk = fr.fractal_map(K, rho)
        cells = pk.info()["member_tiles"] * rho * rho
        dev = ca_a.device
        d_ca = [torch.empty(cells, dtype=torch.uint8, device=dev) for _ in range(2)]
        d_u = [torch.empty(cells, dtype=torch.float32, device=dev) for _ in range(2)]
        d_sums = [torch.empty(nsums, dtype=torch.float64, device=dev) for _ in range(2)]
        h_in_ca = [torch.empty(cells, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        h_in_u = [torch.empty(cells, dtype=torch.float32, pin_memory=True) for _ in range(2)]
        h_out_ca = [torch.empty(cells, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        h_out_u = [torch.empty(cells, dtype=torch.float32, pin_memory=True) for _ in range(2)]
        h_sums = [torch.empty(nsums, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        fr.fractal_pack(pk, ca_a, fr.FRACTAL_U8, d_ca[0], stream)
        fr.fractal_pack(pk, u_a, fr.FRACTAL_F32, d_u[0], stream)
        torch.cuda.synchronize()
        for j in range(2):   # both sets start from the same states
            h_in_ca[j].copy_(d_ca[0])
            h_in_u[j].copy_(d_u[0])
        h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()

        def run(k):
            free = [None, None]    # set j's device buffers read out (copy out done)
            loaded = [None, None]  # set j's states in

            def copy_in(j):
                if free[j] is not None:
                    h2d.wait_event(free[j])
                with torch.cuda.stream(h2d):
                    d_ca[j].copy_(h_in_ca[j], non_blocking=True)
                    d_u[j].copy_(h_in_u[j], non_blocking=True)
                loaded[j] = torch.cuda.Event()
                loaded[j].record(h2d)

            h2d.wait_stream(stream)
            d2h.wait_stream(stream)
            copy_in(0)
            for i in range(k):
                j = i & 1
                if i + 1 < k:
                    copy_in(j ^ 1)
                stream.wait_event(loaded[j])
                fr.fractal_unpack(pk, d_u[j], fr.FRACTAL_F32, u_a, stream)
                fr.fractal_unpack(pk, d_ca[j], fr.FRACTAL_U8, ca_a, stream)
                res = step(0)
                fr.fractal_pack(pk, res, fr.FRACTAL_F32, d_u[j], stream)
                fr.fractal_pack(pk, ca_a, fr.FRACTAL_U8, d_ca[j], stream)
                d_sums[j].copy_(sums)
                done = torch.cuda.Event()
                done.record(stream)
                d2h.wait_event(done)
                with torch.cuda.stream(d2h):
                    h_out_u[j].copy_(d_u[j], non_blocking=True)
                    h_out_ca[j].copy_(d_ca[j], non_blocking=True)
                    h_sums[j].copy_(d_sums[j], non_blocking=True)
                free[j] = torch.cuda.Event()
                free[j].record(d2h)
            stream.wait_stream(h2d)
            stream.wait_stream(d2h)

    run(2)   # warm-up
    torch.cuda.synchronize()
    barrier(dist)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    run(steps)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    t = max_over_ranks(dist, t0.elapsed_time(t1) / 1e3)
    nbytes = 5 * cells
    if rho <= 0:
        note = "whole n x n arrays copied each way through pinned host memory, one step after the other"
    else:
        note = (f"member tiles of side {rho} in lambda order copied each way through pinned host memory by "
                "the copy engines and unpacked / packed on the device; independent batches in two "
                "alternating buffer sets, so that the next step's copy in and the previous step's copy out "
                "overlap the current step's kernels; the timed region runs from before the first copy in "
                "to after the last copy out")
        pk.close()
    return {"value": world * MEMBERS * (CA_STEPS + DIFF_STEPS) * steps / t, "unit": "cell-updates/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 8 * nsums,
            "steps": steps, "ms_per_step": 1e3 * t / steps, "packed_rho": rho, "note": note}


if __name__ == "__main__":
    main()
