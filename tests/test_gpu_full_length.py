"""Full-length parity of the five workloads against the oracle's digests.

tests/golden/make_digests.py ran the oracle (and only the oracle) on sampled
word-groups of every workload at its stated shape and length, with
group_base = g so that each equals group g of the whole ensemble, and stored
SHA-256 digests of the spins, energies, swap masks and per-sweep energies
after each chunk of sweeps (plus the L=8 workload's q histogram).  Here the
GPU path runs the WHOLE ensembles -- once in the launch configuration the
benchmark times (one call, no logs) and once in chunks with logs -- and the
same digests are taken of the sampled groups' slices.  Bit-exact: the
trajectory is a deterministic function of the inputs (tolerance 0).
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1311_5582_gb300 as ea  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_length.json")


def digest(a: np.ndarray) -> str:
    a = np.ascontiguousarray(a)
    return hashlib.sha256(a.astype(a.dtype.newbyteorder("<")).tobytes()).hexdigest()


def golden(name):
    if not os.path.exists(GOLDEN):
        pytest.skip("tests/golden/full_length.json not written yet")
    with open(GOLDEN) as f:
        doc = json.load(f)["workloads"]
    if name not in doc:
        pytest.skip(f"no oracle digests for {name}")
    return doc[name]


def instance(ent) -> W.Instance:
    i = ent["inst"]
    return W.Instance(L=i["L"], G=i["G"], NT=i["NT"], C=i["C"], seed=i["seed"], tmin=i["tmin"],
                      tmax=i["tmax"], input_seed=i["input_seed"])


def make(inst, group_base=0, groups=None):
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    g0, g1 = groups if groups else (0, inst.G)
    e = ea.Ensemble(inst.L, g1 - g0, inst.NT, inst.C, inst.seed, inp["bonds"][g0:g1], inp["spins"][g0:g1],
                    metro, swapt, group_base=group_base)
    return e, inp, metro, swapt


def check_tables(ent, inst):
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    assert digest(metro) == ent["metro_table"] and digest(swapt) == ent["swap_table"]


def final_state(e):
    torch.cuda.synchronize()
    return e.read_spins().cpu().numpy().view(np.uint32), e.measure()[0].cpu().numpy()


def check_final(ent, spins, energies, offset=0):
    last = lambda g: ent["groups"][g]["chunks"][-1]
    for g in ent["groups"]:
        gi = int(g) - offset
        assert digest(spins[gi]) == last(g)["spins"], f"final spins of group {g}"
        assert digest(energies[gi]) == last(g)["energies"], f"final energies of group {g}"


def check_chunks(ent, e):
    """Runs the whole ensemble chunk by chunk with logs and compares every
    chunk's digests of the sampled groups."""
    done = 0
    k = 0
    while done < ent["sweeps"]:
        n = min(ent["chunk"], ent["sweeps"] - done)
        out = e.sweep(n, ent["swap_every"], energy_log=ent["energy_log"], swap_log=True)
        done += n
        spins, energies = final_state(e)
        sl = out["swap_log"]
        for g, rec in ent["groups"].items():
            want = rec["chunks"][k]
            assert want["end_sweep"] == done
            gi = int(g)
            assert digest(spins[gi]) == want["spins"], f"spins of group {g} after sweep {done}"
            assert digest(energies[gi]) == want["energies"], f"energies of group {g} after sweep {done}"
            assert digest(sl[:, gi].cpu().numpy().view(np.uint32)) == want["swap_log"], \
                f"swap masks of group {g}, sweeps {done - n}..{done}"
            if ent["energy_log"]:
                assert digest(out["energy_log"][:, gi].cpu().numpy()) == want["energy_log"], \
                    f"energy log of group {g}, sweeps {done - n}..{done}"
        del out
        k += 1


@pytest.mark.parametrize("name", ["scale", "large16", "large32"])
def test_whole_ensemble_in_the_benchmarked_call(name):
    """One call of the full run, no logs: the kernel and plan the benchmark times."""
    ent = golden(name)
    inst = instance(ent)
    check_tables(ent, inst)
    e, *_ = make(inst)
    e.sweep(ent["sweeps"], ent["swap_every"])
    check_final(ent, *final_state(e))


@pytest.mark.parametrize("name", ["scale", "large16", "large32"])
def test_whole_ensemble_chunk_by_chunk_with_logs(name):
    ent = golden(name)
    e, *_ = make(instance(ent))
    check_chunks(ent, e)


def test_scale_overlap_histogram_per_group():
    """The q histogram and energy sums of the measurement after every sweep of
    the second half, for each sampled group alone (group_base = g)."""
    ent = golden("scale")
    inst = instance(ent)
    mf, me = ent["measure"]
    for g, rec in ent["groups"].items():
        gi = int(g)
        e, *_ = make(inst, group_base=gi, groups=(gi, gi + 1))
        qh = torch.zeros((inst.NT, inst.N + 1), dtype=torch.int64, device="cuda")
        es = torch.zeros(inst.NT, dtype=torch.int64, device="cuda")
        e.sweep(ent["sweeps"], ent["swap_every"], qhist=qh, esum=es, measure_from=mf, measure_every=me)
        q = qh.cpu().numpy().view(np.uint64)
        assert int(q.sum()) == rec["qhist_total"]
        assert digest(q) == rec["qhist"], f"q histogram of group {g}"
        assert [int(x) for x in es.cpu().numpy()] == rec["esum"], f"energy sums of group {g}"
        spins, energies = final_state(e)
        assert digest(spins[0]) == rec["chunks"][-1]["spins"]
        assert digest(energies[0]) == rec["chunks"][-1]["energies"]


def test_batched_mix_in_one_persistent_launch():
    """The six members of the batched form at their full sizes, 10^4 sweeps in
    one persistent launch (as benchmarked), then each member alone with logs."""
    ents = [golden(f"batch_L{L}") for L, _, _ in W.BATCH_MIX]
    made = [make(instance(ent)) for ent in ents]
    batch = ea.Batch([m[0] for m in made])
    batch.sweep(ents[0]["sweeps"], ents[0]["swap_every"])
    batch.sync()
    for ent, m in zip(ents, made):
        check_final(ent, *final_state(m[0]))
    batch.close()
    for ent in ents:
        e, *_ = make(instance(ent))
        check_chunks(ent, e)
        e.close()


def test_served_trace_requests():
    """Requests of the served trace through the server (submitted in arrival
    order, batched across requests), each compared on its sampled group.  The
    digests cover the first sixteen requests that the oracle runs within its
    cost bound; the name carries the request's index in the trace."""
    if not os.path.exists(GOLDEN):
        pytest.skip("tests/golden/full_length.json not written yet")
    with open(GOLDEN) as f:
        names = sorted(n for n in json.load(f)["workloads"] if n.startswith("served_"))
    if not names:
        pytest.skip("no oracle digests for the served trace")
    ents = [golden(n) for n in names]
    full = W.served_trace()
    trace = [full[int(n.split("_")[1])] for n in names]
    srv = ea.Server()
    tickets = []
    for ent, req in zip(ents, trace):
        inst = instance(ent)
        assert inst == req["inst"] and ent["sweeps"] == req["sweeps"]
        inp = W.draw_inputs(inst)
        metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
        tickets.append(srv.submit(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                                  metro, swapt, req["sweeps"], req["swap_every"]))
    for ent, t in zip(ents, tickets):
        out = srv.wait(t)
        check_final(ent, out["spins"], out["energies"])
    srv.close()


def test_temperature_packed_form_over_its_whole_run():
    """The temperature-packed workload (76 realizations, 32 temperatures x 2
    copies, L = 16) over its whole run in chunks with swap logs: realization r
    is bit 0 of word-group r of the oracle run with group_base = r, so its slot
    bits, energies and accepted pairs match the oracle's digests."""
    ent = golden("tpack")
    inst = instance(ent)
    inp = W.draw_tp_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    assert digest(metro) == ent["metro_table"] and digest(swapt) == ent["swap_table"]
    tp = ea.TPEnsemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    shifts = np.arange(inst.NT, dtype=np.uint32)[:, None, None]
    done = k = 0
    while done < ent["sweeps"]:
        n = min(ent["chunk"], ent["sweeps"] - done)
        out = tp.sweep(n, ent["swap_every"], swap_log=True)
        done += n
        torch.cuda.synchronize()
        sp, en = tp.read()
        sp = sp.cpu().numpy().view(np.uint32)                   # [R][C][N], bit t = slot t
        en = en.cpu().numpy()                                    # [R][NT][C]
        sl = out["swap_log"].cpu().numpy().view(np.uint32)      # [passes][R][C], bit p = pair p
        for g, rec in ent["groups"].items():
            want = rec["chunks"][k]
            assert want["end_sweep"] == done
            r = int(g)
            bits = ((sp[r][None, :, :] >> shifts) & np.uint32(1)).astype(np.uint8)   # [NT][C][N]
            assert digest(bits) == want["spins"], f"slot bits of realization {r} after sweep {done}"
            assert digest(np.ascontiguousarray(en[r])) == want["energies"], \
                f"energies of realization {r} after sweep {done}"
            assert digest(np.ascontiguousarray(sl[:, r])) == want["swap_log"], \
                f"accepted pairs of realization {r}, sweeps {done - n}..{done}"
        k += 1
    tp.close()
