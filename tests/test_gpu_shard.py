"""Exact sharding of one ensemble's word-groups (group_base / real_base).

Word-groups are independent (Sec. 3.3: realizations map to independent jobs)
and every random number carries its group's global index, so contexts holding
groups [b, b + G') of an ensemble -- on one device or on several -- must
reproduce bit for bit what those groups do inside the whole ensemble: spins,
energies, swap masks and per-sweep energies, in every kernel form (the
L % 8 == 0 unit kernel, the generic unit body, the chunked form, the field
kernels), in batches, through the server and the host-buffer entry point, and
in the temperature-packed form with real_base.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1311_5582_gb300 as ea  # noqa: E402


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def run(inst, inp, metro, swapt, groups, n, k, group_base=0, plan=None, field=None):
    g0, g1 = groups
    e = ea.Ensemble(inst.L, g1 - g0, inst.NT, inst.C, inst.seed, inp["bonds"][g0:g1],
                    inp["spins"][g0:g1], metro, swapt, group_base=group_base, field=field)
    if plan is not None:
        e.select_plan(plan)
    out = e.sweep(n, k, energy_log=True, swap_log=True)
    return {"spins": u32(e.read_spins()), "energies": e.measure()[0].cpu().numpy(),
            "elog": out["energy_log"].cpu().numpy(), "slog": u32(out["swap_log"]),
            "plans": e.plans(), "plan": e.plan}


def assert_shards_equal_whole(whole, shards, bounds):
    for (g0, g1), s in zip(bounds, shards):
        np.testing.assert_array_equal(s["spins"], whole["spins"][g0:g1])
        np.testing.assert_array_equal(s["energies"], whole["energies"][g0:g1])
        np.testing.assert_array_equal(s["elog"], whole["elog"][:, g0:g1])
        np.testing.assert_array_equal(s["slog"], whole["slog"][:, g0:g1])


@pytest.mark.parametrize("L,G,NT,C,k,n", [(8, 6, 24, 2, 1, 30), (6, 5, 9, 2, 2, 20),
                                          (16, 4, 32, 2, 10, 25), (12, 3, 7, 1, 3, 12)])
def test_halves_reproduce_the_whole_ensemble_in_every_plan(L, G, NT, C, k, n):
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=31 + L, tmin=0.9, tmax=2.0, input_seed=300 + L)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    whole = run(inst, inp, metro, swapt, (0, G), n, k)
    cut = G // 2
    bounds = [(0, cut), (cut, G)]
    for p in range(len(whole["plans"])):
        shards = [run(inst, inp, metro, swapt, b, n, k, group_base=b[0], plan=p) for b in bounds]
        assert_shards_equal_whole(whole, shards, bounds)
    # without the base the second half draws group 0's numbers: a different trajectory
    wrong = run(inst, inp, metro, swapt, (cut, G), n, k, group_base=0)
    assert not np.array_equal(wrong["spins"], whole["spins"][cut:])


def test_single_group_with_base_equals_the_oracle():
    inst = W.Instance(L=8, G=1, NT=12, C=2, seed=77, tmin=0.9, tmax=2.0, input_seed=5)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    base = 4_000_000_000          # near the top of the 32-bit counter word
    got = run(inst, inp, metro, swapt, (0, 1), 15, 1, group_base=base)
    sim = oracle.OracleSim(inst.L, 1, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                           metro, swapt, group_base=base)
    ref = sim.sweep(15, 1, energy_log=True, swap_log=True)
    np.testing.assert_array_equal(got["elog"], ref["energy_log"])
    np.testing.assert_array_equal(got["slog"], ref["swap_log"])
    np.testing.assert_array_equal(got["spins"], sim.spins())


def test_field_shards():
    inst = W.Instance(L=8, G=4, NT=10, C=2, seed=12, tmin=0.9, tmax=2.0, input_seed=61)
    inp = W.draw_inputs(inst)
    mf, sw = ea.ea_build_tables_field(inp["betas"], inst.N, 1, 2)
    fld = (1, 2, mf)
    whole = run(inst, inp, None, sw, (0, 4), 12, 2, field=fld)
    bounds = [(0, 1), (1, 4)]
    shards = [run(inst, inp, None, sw, b, 12, 2, group_base=b[0], field=fld) for b in bounds]
    assert_shards_equal_whole(whole, shards, bounds)


def test_batch_server_and_host_entry_point_honour_the_base():
    inst = W.Instance(L=10, G=4, NT=16, C=2, seed=91, tmin=0.9, tmax=2.0, input_seed=71)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    n, k = 40, 10
    whole = run(inst, inp, metro, swapt, (0, 4), n, k)
    # batch of the two halves
    halves = [ea.Ensemble(inst.L, 2, inst.NT, inst.C, inst.seed, inp["bonds"][b:b + 2],
                          inp["spins"][b:b + 2], metro, swapt, group_base=b) for b in (0, 2)]
    batch = ea.Batch(halves)
    batch.sweep(n, k)
    batch.sync()
    for b, h in zip((0, 2), halves):
        np.testing.assert_array_equal(u32(h.read_spins()), whole["spins"][b:b + 2])
        np.testing.assert_array_equal(h.measure()[0].cpu().numpy(), whole["energies"][b:b + 2])
    # server
    srv = ea.Server()
    t = srv.submit(inst.L, 2, inst.NT, inst.C, inst.seed, inp["bonds"][2:], inp["spins"][2:], metro,
                   swapt, n, k, group_base=2)
    out = srv.wait(t)
    srv.close()
    np.testing.assert_array_equal(out["spins"], whole["spins"][2:])
    np.testing.assert_array_equal(out["energies"], whole["energies"][2:])
    # host-buffer entry point
    h = ea.ea_run(inst.L, 1, inst.NT, inst.C, inst.seed, inp["bonds"][3:], inp["spins"][3:], metro,
                  swapt, n, k, group_base=3)
    np.testing.assert_array_equal(h["spins"], whole["spins"][3:])
    np.testing.assert_array_equal(h["energies"], whole["energies"][3:])


@pytest.mark.parametrize("split", [1, 4])
def test_temperature_packed_shards(split):
    inst = W.Instance(L=8, G=6, NT=20, C=2, seed=23, tmin=0.8, tmax=2.0, input_seed=41)
    inp = W.draw_tp_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)

    def tp_run(r0, r1, base):
        tp = ea.TPEnsemble(inst.L, r1 - r0, inst.NT, inst.C, inst.seed, inp["bonds"][r0:r1],
                           inp["spins"][r0:r1], metro, swapt, real_base=base)
        tp.set_split(split)
        out = tp.sweep(30, 3, energy_log=True, swap_log=True)
        sp, en = tp.read()
        return (u32(sp), en.cpu().numpy(), out["energy_log"].cpu().numpy(), u32(out["swap_log"]))

    whole = tp_run(0, 6, 0)
    for r0, r1 in ((0, 2), (2, 6)):
        part = tp_run(r0, r1, r0)
        np.testing.assert_array_equal(part[0], whole[0][r0:r1])
        np.testing.assert_array_equal(part[1], whole[1][r0:r1])
        np.testing.assert_array_equal(part[2], whole[2][:, r0:r1])
        np.testing.assert_array_equal(part[3], whole[3][:, r0:r1])
