"""Batched form: one persistent launch advancing several ensembles of mixed
shapes must leave each exactly where its own sweeps would (bit for bit), and
where the oracle does.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts too; every test here needs a device
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1311_5582_gb300 as ea  # noqa: E402

# (L, G, NT, C): unit form (L 4, 6, 10), the L % 8 == 0 unit kernel (L 8, L 16 with
# few slots) and chunked units (L 12 and 16 with 32 slots)
MIX = [(4, 3, 16, 2), (6, 2, 7, 1), (8, 3, 24, 2), (10, 2, 9, 2), (12, 1, 32, 2),
       (16, 2, 32, 2), (16, 1, 5, 2)]


def instances(mix=MIX, base_seed=500):
    return [W.Instance(L=L, G=G, NT=NT, C=C, seed=base_seed + i, tmin=0.9, tmax=2.0,
                       input_seed=base_seed + 17 * i) for i, (L, G, NT, C) in enumerate(mix)]


def make(inst: W.Instance):
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    gpu = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                      metro, swapt)
    return gpu, inp, metro, swapt


def state(gpu):
    torch.cuda.synchronize()
    sp = gpu.read_spins().cpu().numpy().view(np.uint32).copy()
    en = gpu.measure()[0].cpu().numpy().copy()
    return sp, en, gpu.counters


def run_alone(inst, schedule):
    gpu, *_ = make(inst)
    for n, k in schedule:
        gpu.sweep(n, k)
    return state(gpu)


def test_mixed_batch_matches_each_member_alone_and_the_oracle():
    insts = instances()
    members = [make(i) for i in insts]
    batch = ea.Batch([m[0] for m in members])
    schedule = [(37, 3), (25, 10), (6, 0), (11, 1)]
    for n, k in schedule:
        batch.sweep(n, k)
    batch.sync()
    total = sum(n for n, _ in schedule)
    for inst, (gpu, inp, metro, swapt) in zip(insts, members):
        sp, en, ctr = state(gpu)
        sp_a, en_a, ctr_a = run_alone(inst, schedule)
        tag = f"L={inst.L} G={inst.G} NT={inst.NT} C={inst.C}"
        assert ctr == ctr_a and ctr[0] == total, tag
        np.testing.assert_array_equal(sp, sp_a, err_msg=f"spins vs alone, {tag}")
        np.testing.assert_array_equal(en, en_a, err_msg=f"energies vs alone, {tag}")
        sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"],
                               inp["spins"], metro, swapt)
        for n, k in schedule:
            sim.sweep(n, k, threads=8)
        np.testing.assert_array_equal(sp, sim.spins(), err_msg=f"spins vs oracle, {tag}")
        np.testing.assert_array_equal(en, sim.energies(), err_msg=f"energies vs oracle, {tag}")
        assert ctr == (sim.sweep_index, sim.pass_index), tag


@pytest.mark.parametrize("segment", [1, 5000, 1 << 24])
def test_segment_length_does_not_change_results(segment):
    """Unit pieces of 8 sweeps up to whole calls: the same trajectories."""
    insts = instances([(4, 2, 16, 2), (8, 2, 24, 2), (10, 1, 9, 2), (16, 1, 32, 2)], 900)
    members = [make(i) for i in insts]
    batch = ea.Batch([m[0] for m in members])
    batch.set_segment(segment)
    schedule = [(53, 10), (19, 4)]
    for n, k in schedule:
        batch.sweep(n, k)
    batch.sync()
    for inst, (gpu, *_rest) in zip(insts, members):
        sp, en, ctr = state(gpu)
        sp_a, en_a, ctr_a = run_alone(inst, schedule)
        np.testing.assert_array_equal(sp, sp_a, err_msg=f"L={inst.L} segment={segment}")
        np.testing.assert_array_equal(en, en_a)
        assert ctr == ctr_a


@pytest.mark.parametrize("L,G,NT,C", [(8, 2, 24, 2), (4, 3, 16, 2), (6, 2, 20, 2), (10, 2, 28, 1),
                                       (16, 1, 32, 2)])
def test_every_batch_plan_gives_the_same_result(L, G, NT, C):
    """Each plan of the member's batch list (lockstep multi-unit bodies, the
    specialised kernel, balanced chunks) at both kernel widths."""
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=77 + L, tmin=0.9, tmax=2.0, input_seed=78 + L)
    ref = run_alone(inst, [(30, 3)])
    probe, *_ = make(inst)
    plans = ea.Batch([probe]).plans(0)
    assert len(plans) >= 2
    forms = set()
    for idx, p in enumerate(plans):
        for width in (384, 512):
            if p["threads"] > width:
                continue
            gpu, *_ = make(inst)
            batch = ea.Batch([gpu])
            batch.set_width(width)
            batch.set_plan(0, idx)
            assert batch.plan(0) == idx
            batch.sweep(30, 3)
            batch.sync()
            sp, en, ctr = state(gpu)
            np.testing.assert_array_equal(sp, ref[0], err_msg=f"plan {idx} width {width}: {p}")
            np.testing.assert_array_equal(en, ref[1])
            assert ctr == ref[2]
            forms.add((p["form"], p["units_per_cta"] > 1))
    if L == 4:
        assert ("unit", True) in forms        # several units per CTA were exercised


def test_autotune_keeps_state_and_results():
    insts = instances([(4, 4, 16, 2), (8, 2, 24, 2), (12, 1, 32, 2)], 1500)
    members = [make(i) for i in insts]
    batch = ea.Batch([m[0] for m in members])
    batch.sweep(7, 3)
    batch.sync()
    before = [state(m[0]) for m in members]
    ms = batch.autotune(probe_sweeps=20, swap_every=5)
    assert ms > 0
    for m, b in zip(members, before):
        s = state(m[0])
        np.testing.assert_array_equal(s[0], b[0])
        np.testing.assert_array_equal(s[1], b[1])
        assert s[2] == b[2]
    batch.sweep(26, 5)
    batch.sync()
    for inst, (gpu, *_rest) in zip(insts, members):
        sp, en, ctr = state(gpu)
        sp_a, en_a, ctr_a = run_alone(inst, [(7, 3), (26, 5)])
        np.testing.assert_array_equal(sp, sp_a, err_msg=f"L={inst.L}")
        np.testing.assert_array_equal(en, en_a)
        assert ctr == ctr_a


def test_graph_replay_over_repeated_calls():
    """Same-shape calls replay the captured launch; the state keeps advancing correctly."""
    insts = instances([(6, 2, 8, 2), (16, 1, 32, 1)], 1300)
    members = [make(i) for i in insts]
    batch = ea.Batch([m[0] for m in members])
    for _ in range(5):
        batch.sweep(10, 10)
    batch.sync()
    assert batch.launches == 10
    for inst, (gpu, *_rest) in zip(insts, members):
        sp, en, ctr = state(gpu)
        sp_a, en_a, ctr_a = run_alone(inst, [(10, 10)] * 5)
        np.testing.assert_array_equal(sp, sp_a)
        np.testing.assert_array_equal(en, en_a)
        assert ctr == ctr_a == (50, 5)


def test_members_interleave_with_their_own_sweeps_and_rejoin():
    inst_a, inst_b = instances([(8, 1, 24, 2), (12, 1, 32, 2)], 1700)
    (a, *_), (b, *_) = make(inst_a), make(inst_b)
    batch = ea.Batch([a, b])
    batch.sweep(12, 5)
    batch.sync()
    a.sweep(7, 5)          # alone, between batched calls (counters continue)
    batch.clear()
    batch.add(b)
    batch.sweep(9, 5)
    batch.add(a)
    batch.sweep(4, 2)
    batch.sync()
    sa = state(a)
    sb = state(b)
    ra = run_alone(inst_a, [(12, 5), (7, 5), (4, 2)])
    rb = run_alone(inst_b, [(12, 5), (9, 5), (4, 2)])
    for s, r in ((sa, ra), (sb, rb)):
        np.testing.assert_array_equal(s[0], r[0])
        np.testing.assert_array_equal(s[1], r[1])
        assert s[2] == r[2]


def test_empty_batch_and_zero_sweeps_are_no_ops():
    batch = ea.Batch()
    batch.sweep(10, 1)
    batch.sync()
    inst = instances([(4, 1, 4, 2)], 2100)[0]
    gpu, inp, *_ = make(inst)
    batch.add(gpu)
    batch.sweep(0, 1)
    batch.sync()
    assert gpu.counters == (0, 0)
    np.testing.assert_array_equal(gpu.read_spins().cpu().numpy().view(np.uint32), inp["spins"])
    assert batch.launches == 0


def test_large_lattices_in_a_batch():
    """Chunked members of the largest sizes (L = 20, 24, 32) beside small unit members."""
    insts = instances([(20, 1, 6, 2), (24, 1, 4, 1), (32, 1, 3, 2), (4, 2, 8, 2), (14, 1, 12, 2)], 2500)
    members = [make(i) for i in insts]
    batch = ea.Batch([m[0] for m in members])
    schedule = [(7, 2), (5, 3)]
    for n, k in schedule:
        batch.sweep(n, k)
    batch.sync()
    for inst, (gpu, inp, metro, swapt) in zip(insts, members):
        sp, en, ctr = state(gpu)
        sp_a, en_a, ctr_a = run_alone(inst, schedule)
        tag = f"L={inst.L} NT={inst.NT} C={inst.C}"
        np.testing.assert_array_equal(sp, sp_a, err_msg=tag)
        np.testing.assert_array_equal(en, en_a, err_msg=tag)
        assert ctr == ctr_a, tag
        if inst.L <= 24:
            sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"],
                                   inp["spins"], metro, swapt)
            for n, k in schedule:
                sim.sweep(n, k, threads=8)
            np.testing.assert_array_equal(sp, sim.spins(), err_msg="oracle " + tag)


def test_per_member_sweeps_and_schedules():
    """ea_batch_sweep_each: members advance by their own counts and swap periods (0: not this call)."""
    insts = instances([(6, 2, 8, 2), (8, 1, 24, 2), (16, 1, 32, 1)], 2700)
    members = [make(i) for i in insts]
    batch = ea.Batch([m[0] for m in members])
    calls = [([13, 0, 9], [3, 1, 10]), ([4, 21, 17], [1, 5, 4]), ([0, 6, 0], [2, 2, 2])]
    for n, k in calls:
        batch.sweep_each(n, k)
    batch.sync()
    for i, (inst, (gpu, *_rest)) in enumerate(zip(insts, members)):
        sp, en, ctr = state(gpu)
        sched = [(n[i], k[i]) for n, k in calls if n[i] > 0]
        sp_a, en_a, ctr_a = run_alone(inst, sched)
        np.testing.assert_array_equal(sp, sp_a, err_msg=f"member {i}")
        np.testing.assert_array_equal(en, en_a)
        assert ctr == ctr_a


def test_a_wait_that_runs_out_reports_timeout_and_the_batch_recovers():
    """Failure path without a fault: one queued task is never published, the CTA
    waiting for it gives up after a short limit, every CTA returns, ea_batch_sync
    reports EA_ETIMEOUT, and the same batch object then runs correctly."""
    insts = instances([(4, 1, 4, 2), (8, 1, 8, 2)], 3100)
    members = [make(i) for i in insts]
    batch = ea.Batch([m[0] for m in members])
    batch.set_wait_limit(4096)                  # ~1 ms of naps
    batch.inject_stall()
    batch.sweep(20, 5)
    with pytest.raises(ea.EAError) as ei:
        batch.sync()
    assert ei.value.code == -4                  # EA_ETIMEOUT
    torch.cuda.synchronize()                    # the context is healthy
    # fresh members through the same batch object, default wait limit
    batch.set_wait_limit(0)
    batch.clear()
    fresh = [make(i) for i in insts]
    for m in fresh:
        batch.add(m[0])
    batch.sweep(20, 5)
    batch.sync()
    for inst, (gpu, *_rest) in zip(insts, fresh):
        sp, en, ctr = state(gpu)
        sp_a, en_a, ctr_a = run_alone(inst, [(20, 5)])
        np.testing.assert_array_equal(sp, sp_a)
        np.testing.assert_array_equal(en, en_a)
        assert ctr == ctr_a
