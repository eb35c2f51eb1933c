#!/usr/bin/env python3
"""Benchmark of the parallel-tempering Edwards-Anderson simulator on GB300.

Workload (one step): the L=8 ensemble -- 512 sites, 2048 realizations (64 words
per site), 24 temperatures geometric in [0.9, 2.0] x 2 copies -- run for 10^5
checkerboard sweeps with a replica-exchange pass after every sweep (energies of
every slot computed every sweep for it).  Metric: ps per spin-flip attempt
(Eq. tsf of the paper, copies counted), with measurements discarded as in the
paper's own figure (Sec. 3):
    t = T / (sweeps * N * NT * C * realizations).
The same workload with the energy / overlap-q histogram measurement after every
sweep of the second half is reported beside it ("with_measurement"), and at
N = 1 samples of the L=16 / L=32 ensembles ("large"), the batched mixed-size
form and the served trace ("batched", "served").

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch under torch.distributed.run: the N ranks hold the word-groups
of one ensemble of N x 2048 realizations, 64 groups each with their global
group index (weak scaling, no data exchange), and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "ps per spin-flip attempt at 1 GPU, % of INT/HBM roofline; served p50/p99 latency"
UNIT = "ps/flip"
# Algorithmic integer operations of one site-word update (32 flip attempts):
# 6 LOP3 bond XORs + 8 adder-tree LOP3 + 3 compares + 3 selects + 3 LOP
# mask terms + 1 flip = 24, plus a quarter of a Philox4x32-10 call
# (10 rounds x (2 IMAD.WIDE + 2 LOP3) / 4 = 10) minus the two constant-key
# XORs folded into the LOP3s = 32.
ALG_OPS_PER_SITE_WORD = 32
ALU_LANES_PER_CLK_PER_SM = 64     # integer ALU pipe (LOP3/IADD3/ISETP/SEL) of one SM


WORKLOADS = {
    # name: (instance, sweeps per step, swap every, measurement over the second half)
    "scale": (W.SCALE, W.SCALE_SWEEPS, W.SCALE_SWAP_EVERY, False),
    "scale_measured": (W.SCALE, W.SCALE_SWEEPS, W.SCALE_SWAP_EVERY, True),
    "small": (W.SMALL, W.SMALL_SWEEPS, W.SMALL_SWAP_EVERY, False),
    "large16": (W.LARGE16, W.LARGE_SWEEPS, W.LARGE_SWAP_EVERY, False),
    "large32": (W.LARGE32, W.LARGE_SWEEPS, W.LARGE_SWAP_EVERY, False),
}


def workload(name="scale", sweeps=None):
    inst, n, swap_every, meas = WORKLOADS[name]
    if sweeps:
        n = sweeps
    text = (f"EA +-J L={inst.L} ({inst.N} sites), {32 * inst.G} realizations "
            f"({inst.G} words/site), {inst.NT} temperatures geometric in "
            f"[{inst.tmin},{inst.tmax}] x {inst.C} copies, {n} sweeps, PT swap every "
            f"{'sweep' if swap_every == 1 else f'{swap_every} sweeps'}"
            + (", energy + overlap-q histograms over the second half" if meas else ""))
    return {
        "key": name, "inst": inst, "sweeps": n, "swap_every": swap_every,
        "measure_from": n // 2 if meas else 0, "measure_every": 1 if meas else 0,
        "flips": n * inst.N * inst.NT * inst.C * 32 * inst.G, "name": text,
    }


# Sources each workload's dominant kernel is compiled from (its traffic record
# goes stale when one of them changes).
KERNEL_SOURCES = {
    "scale": ["ea_unit_wave.cu", "ea_wave.cuh", "ea_fast.cuh", "ea_device.cuh", "ea_internal.h"],
    "scale_measured": ["ea_unit_wave.cu", "ea_wave.cuh", "ea_fast.cuh", "ea_device.cuh", "ea_internal.h"],
    "small": ["ea_kernels.cu", "ea_bodies.cuh", "ea_device.cuh", "ea_internal.h"],
    "large16": ["ea_kernels.cu", "ea_bodies.cuh", "ea_device.cuh", "ea_internal.h"],
    "large32": ["ea_kernels.cu", "ea_bodies.cuh", "ea_device.cuh", "ea_internal.h"],
}


def kernel_source_hash(workload_key: str = "scale") -> str:
    """SHA-256 over the sources of the workload's dominant kernel: a traffic
    figure measured on other sources is stale."""
    import hashlib
    d = os.path.join(ROOT, "paper_1311_5582_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[workload_key]:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_key: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary
    (profiles/*.md line 'traffic-record: <workload> <bytes per launch> <source hash>'),
    or None when absent or taken on different kernel sources."""
    import glob
    want = kernel_source_hash(workload_key)
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(path) as f:
            for line in f:
                parts = line.strip().strip("`").split()
                if len(parts) == 4 and parts[0] == "traffic-record:" and parts[1] == workload_key:
                    if parts[3] == want:
                        return float(parts[2])
    return None


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_instance(inst, world):
    """Weak scaling over one ensemble: N ranks simulate one ensemble of N times
    the workload's word-groups (same Philox key, disorder drawn for all of them);
    at N = 1 it is the workload itself."""
    if world <= 1:
        return inst
    return W.Instance(L=inst.L, G=inst.G * world, NT=inst.NT, C=inst.C, seed=inst.seed,
                      tmin=inst.tmin, tmax=inst.tmax, input_seed=inst.input_seed)


def rank_groups(G_total, rank, world):
    """Word-groups [g0, g1) of the job's ensemble that rank `rank` holds.  Groups
    are independent and their random numbers carry the global group index
    (group_base = g0), so the shards together follow exactly the trajectory of
    the whole ensemble on one device; nothing is exchanged."""
    return G_total * rank // world, G_total * (rank + 1) // world


def rank_inputs(inst, rank, world):
    """(job instance, this rank's (g0, g1), its bonds / spins and the ladder)."""
    job = job_instance(inst, world)
    inp = W.draw_inputs(job)
    g0, g1 = rank_groups(job.G, rank, world)
    return job, (g0, g1), {"bonds": inp["bonds"][g0:g1], "spins": inp["spins"][g0:g1],
                           "betas": inp["betas"]}


def aggregate(times_s, flips_per_rank):
    """Job value: slowest rank's time over all ranks' flips (ps per flip)."""
    t = max(times_s)
    return t / (flips_per_rank * len(times_s)) * 1e12, t


def reduce_max(x: float, world: int) -> float:
    """Largest value of x over the ranks (the only cross-rank traffic of the
    bench besides barriers): a CUDA tensor under NCCL, a CPU one under gloo."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def cpu_baseline(wl, budget_s=15.0, threads=None, single_thread_s=3.0):
    """The oracle as it stands, on this host's cores, on a bounded sample of the
    workload: the first `threads` word-groups for as many sweeps (from sweep 0,
    same schedule and measurement) as fit the time budget; beside it the oracle
    on one core and one word-group."""
    import oracle
    inst = wl["inst"]
    threads = threads or max(1, min(os.cpu_count() or 1, inst.G))
    inp = W.draw_inputs(inst)
    g = threads
    metro = oracle.metro_table(inp["betas"])
    swapt = oracle.swap_table_trimmed(inp["betas"], inst.N)

    def run(n):
        sim = oracle.OracleSim(inst.L, g, inst.NT, inst.C, inst.seed, inp["bonds"][:g],
                               inp["spins"][:g], metro, swapt)
        qh = np.zeros((inst.NT, inst.N + 1), np.uint64)
        es = np.zeros(inst.NT, np.int64)
        t0 = time.perf_counter()
        me = wl["measure_every"]
        sim.sweep(n, wl["swap_every"], qhist=qh if me else None, esum=es if me else None,
                  measure_from=n // 2 if me else 0, measure_every=me, threads=threads)
        return time.perf_counter() - t0

    t_probe = run(10)
    n = max(10, int(10 * budget_s / max(t_probe, 1e-3)))
    t = run(n)
    flips = n * inst.N * inst.NT * inst.C * 32 * g
    out = {"value": t / flips * 1e12, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{g} of {inst.G} word-groups ({32 * g} realizations), {n} sweeps "
                     f"with the same swap and measurement schedule, {t:.1f} s"}
    # one core, one word-group: the figure comparable to a single-thread CPU code
    g, threads = 1, 1
    t1 = run(10)
    n1 = max(10, int(10 * single_thread_s / max(t1, 1e-3)))
    t1 = run(n1)
    out["single_thread"] = {"value": t1 / (n1 * inst.N * inst.NT * inst.C * 32) * 1e12, "unit": UNIT,
                            "cores": 1, "sample": f"1 word-group (32 realizations), {n1} sweeps, {t1:.1f} s"}
    return out


def _flips(inst, sweeps):
    return sweeps * inst.N * inst.NT * inst.C * 32 * inst.G


def _alu_peak_tops(torch):
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * ALU_LANES_PER_CLK_PER_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def bench_batched(ea, torch, sweeps=W.BATCH_SWEEPS, swap_every=W.BATCH_SWAP_EVERY, autotune=True):
    """The mixed ensemble (L in {4..16}, uneven sizes and ladders) advanced by one
    persistent batched launch, against the same instances launched one after
    another; both sides autotuned, both timed from warm state with L2 flushed."""
    insts = W.batch_instances()
    ens, twins = [], []          # plain launches / the batch, from the same inputs
    for inst in insts:
        inp = W.draw_inputs(inst)
        metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
        for dst in (ens, twins):
            dst.append(ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"],
                                   inp["spins"], metro, swapt))
    flips = sum(_flips(i, sweeps) for i in insts)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def timed(fn):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / 1e3

    if autotune:
        for e in ens:
            e.autotune(probe_sweeps=200, swap_every=swap_every)

    def plain():
        for e in ens:
            e.sweep(sweeps, swap_every)

    l0 = sum(e.launches for e in ens)
    timed(plain)                                 # warm
    l1 = sum(e.launches for e in ens)
    t_plain = timed(plain)
    plain_launches = sum(e.launches for e in ens) - l1
    batch = ea.Batch(twins)
    if autotune:
        batch.autotune(probe_sweeps=200, swap_every=swap_every)

    def batched():
        batch.sweep(sweeps, swap_every)
        batch.sync()

    timed(batched)                               # warm
    b0 = batch.launches
    t_batch = timed(batched)
    del l0
    plans = [batch.plans(i)[batch.plan(i)] for i in range(len(insts))]
    # both sides ran the same sweeps from the same state: identical results
    same = all(np.array_equal(a.read_spins_host(), b.read_spins_host())
               and np.array_equal(a.measure()[0].cpu().numpy(), b.measure()[0].cpu().numpy())
               and a.counters == b.counters for a, b in zip(ens, twins))
    if not same:
        raise AssertionError("batched results differ from the per-instance launches")
    return {
        "workload": "EA +-J batched mix: " + ", ".join(
            f"L={i.L} {32 * i.G} realizations x {i.NT} temps" for i in insts)
            + f" (C=2, ladders geometric in [0.8,2.0]), {sweeps} sweeps, swap every {swap_every}",
        "value": t_batch / flips * 1e12, "unit": UNIT, "plain_value": t_plain / flips * 1e12,
        "roofline_frac": flips / 32 * ALG_OPS_PER_SITE_WORD / t_batch / 1e12 / _alu_peak_tops(torch),
        "speedup_vs_plain": t_plain / t_batch, "gpu_launches": batch.launches - b0,
        "plain_gpu_launches": plain_launches, "flips": flips, "identical_to_plain": bool(same),
        "plans": [f"{p['form']} t{p['threads']} g{p['group_threads']} u{p['units_per_cta']}"
                  for p in plans],
    }


def bench_large(ea, torch, peak_tops, sweeps=None):
    """The L=16 and L=32 ensembles of the largest configuration (10^5 sweeps each,
    swap every 10), each under the plan its autotuner picks, timed over the whole
    run (or `sweeps` sweeps) after a short warm-up with L2 flushed, with the
    integer-ALU roofline fraction of the whole run."""
    out = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    for key in ("large16", "large32"):
        wl = workload(key, sweeps)
        inst = wl["inst"]
        inp = W.draw_inputs(inst)
        metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
        ens = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                          metro, swapt)
        ens.autotune(probe_sweeps=60, swap_every=wl["swap_every"])
        ens.sweep(100, wl["swap_every"])                      # warm
        flush.fill_(2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ens.launches
        a.record()
        ens.sweep(wl["sweeps"], wl["swap_every"])
        b.record()
        b.synchronize()
        t = a.elapsed_time(b) / 1e3
        site_words = wl["sweeps"] * inst.N * inst.NT * inst.C * inst.G
        achieved = site_words * ALG_OPS_PER_SITE_WORD / t / 1e12
        plan = ens.plans()[ens.plan]
        out[key] = {"workload": wl["name"] + (" (sample)" if sweeps else " (whole run)"),
                    "value": t / wl["flips"] * 1e12, "unit": UNIT,
                    "roofline_frac": achieved / peak_tops, "achieved_tops": achieved,
                    "gpu_launches": ens.launches - l0,
                    "plan": f"{plan['form']} t{plan['threads']} g{plan['group_threads']} "
                            f"n{plan['lattices_per_cta']}"}
        ens.close()
        del ens
    return out


def bench_field(ea, torch, peak_tops, sweeps=200, h=(1, 2)):
    """The headline ensemble in the external field h = h_num / h_den (Eq. 1 with
    h != 0; generic unit and chunked kernels), autotuned and timed like the
    headline from warm state with L2 flushed, beside the same ensemble at h = 0
    restricted to the same generic plans (the cost of the field itself)."""
    wl = workload("scale", sweeps)
    inst = wl["inst"]
    inp = W.draw_inputs(inst)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def timed(ens):
        ens.sweep(wl["sweeps"], wl["swap_every"])            # warm
        flush.fill_(3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ens.launches
        a.record()
        ens.sweep(wl["sweeps"], wl["swap_every"])
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / 1e3 / wl["flips"] * 1e12, ens.launches - l0

    def plan_text(ens):
        p = ens.plans()[ens.plan]
        return f"{p['form']} t{p['threads']} g{p['group_threads']} n{p['lattices_per_cta']}"

    mf, sw = ea.ea_build_tables_field(inp["betas"], inst.N, *h)
    ens = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], None, sw,
                      field=(h[0], h[1], mf))
    ens.autotune(probe_sweeps=60, swap_every=wl["swap_every"])
    v_field, launches = timed(ens)
    # achieved on the field-free algorithmic count (the field adds its own tests on top)
    achieved = ALG_OPS_PER_SITE_WORD / 32 / (v_field * 1e-12) / 1e12
    out = {"workload": wl["name"] + f", field h = {h[0]}/{h[1]}", "value": v_field, "unit": UNIT,
           "roofline_frac": achieved / peak_tops, "achieved_tops": achieved,
           "alg_ops_basis": f"{ALG_OPS_PER_SITE_WORD} per site-word (field-free count)",
           "plan": plan_text(ens), "gpu_launches": launches}
    ens_form = ens.plans()[ens.plan]["form"]
    ens.close()
    field_form = ens_form
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    ens = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    best = None
    for i, p in enumerate(ens.plans()):
        if p["form"] != field_form:                     # the same kernel form at h = 0
            continue
        ens.select_plan(i)
        v, _ = timed(ens)
        if best is None or v < best[0]:
            best = (v, plan_text(ens))
    ens.close()
    if best is not None:
        out["h0_same_kernel_family"] = {"value": best[0], "unit": UNIT, "plan": best[1]}
        out["field_cost"] = v_field / best[0]
    return out


def bench_field_plain(ea, torch, sweeps=200, h=(1, 2)):
    """The headline ensemble in the field h under its default plan (the field
    wavefront kernel for 0 < |h| < 2): one warm-up call, then one timed call."""
    wl = workload("scale", sweeps)
    inst = wl["inst"]
    inp = W.draw_inputs(inst)
    mf, sw = ea.ea_build_tables_field(inp["betas"], inst.N, *h)
    ens = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], None, sw,
                      field=(h[0], h[1], mf))
    ens.sweep(wl["sweeps"], wl["swap_every"])
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    ens.sweep(wl["sweeps"], wl["swap_every"])
    b.record()
    b.synchronize()
    plan = ens.plans()[ens.plan]["form"]
    ens.close()
    return {"workload": wl["name"] + f", field h = {h[0]}/{h[1]}", "plan": plan,
            "value": a.elapsed_time(b) / 1e3 / wl["flips"] * 1e12, "unit": UNIT}


# Algorithmic integer ops of the temperature-packed form per flip attempt: a
# quarter Philox4x32-10 call (one uniform per attempt: 10), three threshold
# tests and three mask-bit ORs, plus the 24-op bit-sliced update of the site
# word shared by its NT slots.
TP_ALG_OPS_PER_FLIP = 16


def bench_tpack(ea, torch, peak_tops, sweeps=200):
    """The temperature-packed form on its workload (few realizations, 32
    temperatures, one uniform per flip attempt), timed from warm state with L2
    flushed, beside the realization-packed form computing the same trajectories
    (realization r as bit 0 of word-group r) per flip of those realizations."""
    inst = W.TPACK
    wl = {"sweeps": sweeps, "swap_every": W.TPACK_SWAP_EVERY,
          "name": (f"EA +-J L={inst.L} ({inst.N} sites), {inst.G} realizations temperature-packed "
                   f"(one word per realization, copy and site), {inst.NT} temperatures geometric in "
                   f"[{inst.tmin},{inst.tmax}] x {inst.C} copies, {sweeps} of {W.TPACK_SWEEPS} sweeps "
                   f"(sample), PT swap every {W.TPACK_SWAP_EVERY} sweeps")}
    inp = W.draw_tp_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")

    def timed(ens):
        ens.sweep(wl["sweeps"], wl["swap_every"])            # warm
        flush.fill_(4)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = ens.launches
        a.record()
        ens.sweep(wl["sweeps"], wl["swap_every"])
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / 1e3, ens.launches - l0

    tp = ea.TPEnsemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    t_tp, launches = timed(tp)
    tp.close()
    flips = wl["sweeps"] * inst.N * inst.NT * inst.C * inst.G
    ops = flips * (TP_ALG_OPS_PER_FLIP + 24 / inst.NT)
    out = {"workload": wl["name"], "value": t_tp / flips * 1e12, "unit": UNIT,
           "roofline_frac": ops / t_tp / 1e12 / peak_tops, "achieved_tops": ops / t_tp / 1e12,
           "alg_ops_basis": f"{TP_ALG_OPS_PER_FLIP} per flip attempt + 24 per site-word",
           "gpu_launches": launches}
    b, s = W.tp_as_groups(inp["bonds"], inp["spins"], inst.NT)
    rp = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, b, s, metro, swapt)
    rp.autotune(probe_sweeps=20, swap_every=wl["swap_every"])
    t_rp, _ = timed(rp)
    rp.close()
    out["packed_form_same_trajectories"] = {"value": t_rp / flips * 1e12, "unit": UNIT,
                                            "note": "per flip of the same realizations (bit 0 of each group)"}
    out["speedup_vs_packed_form"] = t_rp / t_tp
    # few realizations: 8 x 2 units, each split into slot groups, against one CTA per unit
    few = W.Instance(L=inst.L, G=8, NT=inst.NT, C=inst.C, seed=7, tmin=inst.tmin, tmax=inst.tmax,
                     input_seed=107)
    fi = W.draw_tp_inputs(few)
    tp = ea.TPEnsemble(few.L, few.G, few.NT, few.C, few.seed, fi["bonds"], fi["spins"], metro, swapt)
    k = tp.split
    t_split, l_split = timed(tp)
    tp.set_split(1)
    t_one, _ = timed(tp)
    tp.close()
    f_few = wl["sweeps"] * few.N * few.NT * few.C * few.G
    out["few_realizations"] = {"realizations": few.G, "value": t_split / f_few * 1e12, "unit": UNIT,
                               "slot_groups": k, "gpu_launches": l_split,
                               "one_cta_per_unit": t_one / f_few * 1e12, "speedup": t_one / t_split}
    return out


def bench_served(ea, n_requests=32, round_ms=20, load=None, rate_flips_s=None):
    """Poisson-arriving requests (200/s) replayed in real time through the server,
    against serving them one at a time with plain launches (arrival order); the
    results of the two are compared bit for bit.  With `load`, arrival times are
    stretched so that the offered work is that fraction of `rate_flips_s`."""
    trace = W.served_trace(n_requests)
    scale = 1.0
    if load:
        work = sum(_flips(r["inst"], r["sweeps"]) for r in trace)
        scale = work / rate_flips_s / load / max(trace[-1]["arrival_s"], 1e-9)
        trace = [dict(r, arrival_s=r["arrival_s"] * scale) for r in trace]
    data = []
    for r in trace:
        inst = r["inst"]
        inp = W.draw_inputs(inst)
        metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
        data.append((inst, inp, metro, swapt))
    flips = sum(_flips(d[0], r["sweeps"]) for d, r in zip(data, trace))
    srv = ea.Server(round_ms=round_ms)
    start = time.monotonic()
    tickets = []
    for r, (inst, inp, metro, swapt) in zip(trace, data):
        wait = r["arrival_s"] - (time.monotonic() - start)
        if wait > 0:
            time.sleep(wait)
        tickets.append(srv.submit(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"],
                                  inp["spins"], metro, swapt, r["sweeps"], r["swap_every"]))
    outs = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.close()
    lat, same = [], True
    plain_busy = 0.0
    start = time.monotonic()
    for r, (inst, inp, metro, swapt), o in zip(trace, data, outs):
        wait = r["arrival_s"] - (time.monotonic() - start)
        if wait > 0:
            time.sleep(wait)
        t_req = time.monotonic()
        e = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                        metro, swapt)
        e.sweep(r["sweeps"], r["swap_every"])
        sp = e.read_spins_host()
        en = e.measure()[0].cpu().numpy()
        plain_busy += time.monotonic() - t_req
        lat.append((time.monotonic() - start - r["arrival_s"]) * 1e3)
        same = same and np.array_equal(sp, o["spins"]) and np.array_equal(en, o["energies"])
        e.close()
    span = time.monotonic() - start - trace[0]["arrival_s"]
    lat.sort()
    rank = lambda q: lat[max(0, int(np.ceil(q * len(lat))) - 1)]
    return {
        "workload": f"first {n_requests} requests of the served trace: Poisson arrivals at "
                    f"{200.0 / scale:.3g}/s" + (f" (offered load {load:.0%} of the served rate)" if load else "")
                    + ", L in {6..16}, 32-2048 realizations, 16-32 temps in [0.8,2.0], 10^3-10^5 "
                    "sweeps log-uniform, swap every 10",
        "value": st["span_s"] / st["flip_attempts"] * 1e12, "unit": UNIT,
        "roofline_frac": (st["flip_attempts"] / 32 * ALG_OPS_PER_SITE_WORD / st["span_s"] / 1e12
                          / _alu_peak_tops(__import__("torch"))),
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "rounds": st["rounds"],
        "peak_bytes": st["peak_bytes"], "round_ms": round_ms,
        "plain_value": span / flips * 1e12, "plain_p50_ms": rank(0.5), "plain_p99_ms": rank(0.99),
        # per flip of busy time (at least one request resident / being served): the
        # efficiency of the device work itself, free of the idle gaps of the arrival process
        "busy_value": st["busy_s"] / st["flip_attempts"] * 1e12, "plain_busy_value": plain_busy / flips * 1e12,
        "identical_to_plain": bool(same), "flips": flips,
    }


def run_reference(args, wl):
    """Reference arm: the CPU oracle, timed as it stands on the host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    inst = wl["inst"]
    per_step_budget = max(2.0, 120.0 / max(1, args.steps + args.warmup))
    import oracle
    threads = max(1, min(os.cpu_count() or 1, inst.G))
    inp = W.draw_inputs(inst)
    metro = oracle.metro_table(inp["betas"])
    swapt = oracle.swap_table_trimmed(inp["betas"], inst.N)
    g = threads

    def step(n):
        sim = oracle.OracleSim(inst.L, g, inst.NT, inst.C, inst.seed, inp["bonds"][:g],
                               inp["spins"][:g], metro, swapt)
        qh = np.zeros((inst.NT, inst.N + 1), np.uint64)
        es = np.zeros(inst.NT, np.int64)
        t0 = time.perf_counter()
        me = wl["measure_every"]
        sim.sweep(n, wl["swap_every"], qhist=qh if me else None, esum=es if me else None,
                  measure_from=n // 2 if me else 0, measure_every=me, threads=threads)
        return time.perf_counter() - t0

    t_probe = step(10)
    n = max(10, int(10 * per_step_budget / max(t_probe, 1e-3)))
    for _ in range(args.warmup):
        step(n)
    ts = [step(n) for _ in range(args.steps)]
    flips = n * inst.N * inst.NT * inst.C * 32 * g
    val = sum(ts) / len(ts) / flips * 1e12
    sample = (f"{g} of {inst.G} word-groups, {n} sweeps per step, swap every "
              f"{wl['swap_every']}" + (", measurement over the second half" if wl["measure_every"] else ""))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / len(ts),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": wl["name"], "sample": sample},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="scale", choices=sorted(WORKLOADS),
                    help="scale (default): the L=8 ensemble of the headline metric")
    ap.add_argument("--sweeps", type=int, default=None,
                    help="sweeps per step (default: the workload's full run)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched-mix and served-trace measurements (N=1 only)")
    ap.add_argument("--served-requests", type=int, default=32)
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched mix with default plans (--sweeps sweeps) and print its object")
    ap.add_argument("--tpack-only", action="store_true",
                    help="run only the temperature-packed workload (--sweeps sweeps) and print its object")
    ap.add_argument("--field-only", action="store_true",
                    help="run only the headline ensemble in the field h = 1/2 under its default plan "
                         "(one warm-up and one timed call of --sweeps sweeps) and print its object")
    args = ap.parse_args()
    if args.field_only:
        import torch
        import paper_1311_5582_gb300 as ea
        print(json.dumps(bench_field_plain(ea, torch, sweeps=args.sweeps or 200)))
        return 0
    if args.tpack_only:
        import torch
        import paper_1311_5582_gb300 as ea
        print(json.dumps(bench_tpack(ea, torch, _alu_peak_tops(torch), sweeps=args.sweeps or 200)))
        return 0
    if args.batched_only:
        import torch
        import paper_1311_5582_gb300 as ea
        print(json.dumps(bench_batched(ea, torch, sweeps=args.sweeps or W.BATCH_SWEEPS, autotune=False)))
        return 0
    wl = workload(args.workload, args.sweeps)
    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    import paper_1311_5582_gb300 as ea

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    job, (g0, g1), inp = rank_inputs(wl["inst"], rank, world)
    inst = W.Instance(L=job.L, G=g1 - g0, NT=job.NT, C=job.C, seed=job.seed, tmin=job.tmin,
                      tmax=job.tmax, input_seed=job.input_seed)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    stream = torch.cuda.Stream()
    ens = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                      metro, swapt, stream=stream, group_base=g0)
    qh = torch.zeros((inst.NT, inst.N + 1), dtype=torch.int64, device="cuda")
    es = torch.zeros(inst.NT, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")  # > L2 (129 MB)

    def step():
        s0 = ens.sweep_index
        ens.sweep(wl["sweeps"], wl["swap_every"], qhist=qh, esum=es,
                  measure_from=s0 + wl["measure_from"], measure_every=wl["measure_every"])

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        l0 = ens.launches
        with ClockSampler(dev) as clk:
            for i in range(args.steps):
                flush.fill_(i)        # evict the ensemble from L2 between steps
                ev[i][0].record(stream)
                step()
                ev[i][1].record(stream)
            barrier()
        launches = ens.launches - l0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = reduce_max(sum(step_ms) / 1e3, world)
    value = t_total / (wl["flips"] * args.steps * world) * 1e12
    clocks = clk.summary()

    # the same workload with the energy / overlap-q measurement after every sweep
    # of the second half (the paper measures every few thousand sweeps and
    # quotes its speed without measurements, Sec. 3): reported beside the value
    with_meas = None
    wm_key = args.workload + "_measured"
    if world == 1 and not args.no_extras and wm_key in WORKLOADS:
        wm = workload(wm_key, args.sweeps)

        def mstep():
            s0 = ens.sweep_index
            ens.sweep(wm["sweeps"], wm["swap_every"], qhist=qh, esum=es,
                      measure_from=s0 + wm["measure_from"], measure_every=wm["measure_every"])

        with torch.cuda.stream(stream):
            mstep()
            mt = []
            for i in range(2):
                flush.fill_(i)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                mstep()
                b.record(stream)
                b.synchronize()
                mt.append(a.elapsed_time(b))
        v_meas = statistics.mean(mt) / 1e3 / wm["flips"] * 1e12
        with_meas = {"workload": wm["name"], "value": v_meas, "unit": UNIT, "steps": 2,
                     "measurement_share": 1.0 - value / v_meas}

    # roofline of the dominant kernel (the fused sweep kernel: one launch per step)
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = peaks.get("sm_max_mhz", 2070.0)
    peak_tops = sms * ALU_LANES_PER_CLK_PER_SM * mhz * 1e6 / 1e12
    site_words = wl["sweeps"] * inst.N * inst.NT * inst.C * inst.G
    # the dominant kernel's launches per step (1 for the unit form; the chunked form
    # launches a sweep kernel per swap interval, timed here as the whole step)
    launch_s = statistics.mean(step_ms) / 1e3
    achieved = site_words * ALG_OPS_PER_SITE_WORD / launch_s / 1e12

    # end to end through the host-buffer entry point (pinned host memory both ways)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    h_in = {k: pin(v) for k, v in (("bonds", inp["bonds"]), ("spins", inp["spins"]),
                                   ("metro", metro), ("swapt", swapt))}
    h_out = {"energies": pin(np.zeros((inst.G, inst.NT, inst.C, 32), np.int32)),
             "spins": pin(np.zeros((inst.G, inst.NT, inst.C, inst.N), np.uint32)),
             "qhist": pin(np.zeros((inst.NT, inst.N + 1), np.uint64)),
             "esum": pin(np.zeros(inst.NT, np.int64))}
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ea.ea_run(inst.L, inst.G, inst.NT, inst.C, inst.seed, h_in["bonds"], h_in["spins"],
                  h_in["metro"], h_in["swapt"], wl["sweeps"], wl["swap_every"],
                  measure_from=wl["measure_from"], measure_every=wl["measure_every"],
                  want_spins=True, want_qhist=True, want_esum=True, host_out=h_out, stream=stream,
                  group_base=g0)
    t_e2e = reduce_max((time.perf_counter() - t0) / e2e_steps, world)
    h2d = sum(v.nbytes for v in h_in.values())
    d2h = sum(v.nbytes for v in h_out.values())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(step_ms),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": wl["name"], "l2_flush": True, "L": inst.L,
                       "realizations": 32 * job.G, "temps": inst.NT, "copies": inst.C,
                       "parallelism": (f"{world} ranks x {inst.G} word-groups of one ensemble "
                                       "(group_base = rank x groups), no data exchange"
                                       if world > 1 else "1 GPU"),
                       "sweeps_per_step": wl["sweeps"], "swap_every": wl["swap_every"],
                       "kernel_launches_per_step": launches / args.steps},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                         "frac": achieved / peak_tops, "traffic": recorded_traffic(wl["key"]),
                         "traffic_source_hash": kernel_source_hash(wl["key"]),
                         "peak_basis": f"{sms} SMs x {ALU_LANES_PER_CLK_PER_SM} int-ALU lanes/clk x "
                                       f"{mhz:.0f} MHz (max SM clock of measured peaks file)",
                         "alg_ops_per_site_word": ALG_OPS_PER_SITE_WORD},
            "e2e": {"value": t_e2e / (wl["flips"] * world) * 1e12, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "flips_per_step": wl["flips"] * world,
        }
        if with_meas is not None:
            line["with_measurement"] = with_meas
        if world == 1 and not args.no_extras:
            line["large"] = bench_large(ea, torch, peak_tops)
            line["field"] = bench_field(ea, torch, peak_tops)
            line["tpack"] = bench_tpack(ea, torch, peak_tops)
            line["batched"] = bench_batched(ea, torch)
            line["served"] = bench_served(ea, args.served_requests)
            line["served_load70"] = bench_served(ea, 128, load=0.7,
                                                 rate_flips_s=1e12 / line["served"]["value"])
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
