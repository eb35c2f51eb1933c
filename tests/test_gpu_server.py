"""Serving loop: requests arriving while others run are admitted by device
memory, batched with the resident ones, and each result is bit-identical to
the same request run alone (and to the oracle)."""
from __future__ import annotations

import threading
import time

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts too; every test here needs a device
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1311_5582_gb300 as ea  # noqa: E402


def request_set(n, seed):
    """Seeded requests of the served mix, scaled down: L in {4..16}, G 1..3, NT 2..32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs = []
    for r in range(n):
        L = int(rng.choice([4, 6, 8, 10, 12, 14, 16]))
        NT = int(rng.integers(2, 33))
        inst = W.Instance(L=L, G=int(rng.integers(1, 4)), NT=NT, C=int(rng.integers(1, 3)),
                          seed=int(rng.integers(1, 2**40)), tmin=0.8, tmax=2.0,
                          input_seed=int(rng.integers(1, 2**31)))
        reqs.append({"inst": inst, "n": int(rng.integers(0, 120)) if r else 0,
                     "k": int(rng.integers(0, 12)), "delay": float(rng.exponential(0.004))})
    return reqs


def tables(inst):
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    return inp, metro, swapt


def alone(inst, inp, metro, swapt, n, k):
    gpu = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                      metro, swapt)
    gpu.sweep(n, k)
    torch.cuda.synchronize()
    return (gpu.read_spins().cpu().numpy().view(np.uint32), gpu.measure()[0].cpu().numpy())


def submit(server, inst, inp, metro, swapt, n, k):
    return server.submit(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                         metro, swapt, n, k)


def approx_bytes(inst):
    words = inst.G * inst.NT * inst.C * inst.N
    return 4 * (3 * words + 2 * inst.G * 3 * inst.N) + 4 * inst.G * inst.C * (64 + 32 * inst.NT) * 2


def test_served_requests_match_alone_and_oracle():
    reqs = request_set(14, 11)
    prepared = [tables(r["inst"]) for r in reqs]
    # a budget that holds only a few requests at once: admission waits for memory
    budget = 3 * max(approx_bytes(r["inst"]) for r in reqs)
    server = ea.Server(mem_budget=budget, round_ms=2)
    tickets = []
    for r, (inp, metro, swapt) in zip(reqs, prepared):
        time.sleep(r["delay"])
        tickets.append(submit(server, r["inst"], inp, metro, swapt, r["n"], r["k"]))
    outs = [server.wait(t) for t in tickets]
    st = server.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_bytes"] <= st["mem_budget"] == budget
    assert st["rounds"] >= 2 and st["live"] == 0 and st["queued"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    flips = sum(r["inst"].N * r["inst"].NT * r["inst"].C * r["inst"].G * 32 * r["n"] for r in reqs)
    assert st["flip_attempts"] == flips
    server.close()
    for r, (inp, metro, swapt), out in zip(reqs, prepared, outs):
        inst = r["inst"]
        sp, en = alone(inst, inp, metro, swapt, r["n"], r["k"])
        tag = f"L={inst.L} G={inst.G} NT={inst.NT} C={inst.C} n={r['n']} k={r['k']}"
        np.testing.assert_array_equal(out["spins"], sp, err_msg=tag)
        np.testing.assert_array_equal(out["energies"], en, err_msg=tag)
        if inst.N * inst.NT * inst.C * inst.G * max(r["n"], 1) <= 4_000_000:
            sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"],
                                   inp["spins"], metro, swapt)
            sim.sweep(r["n"], r["k"], threads=8)
            np.testing.assert_array_equal(out["spins"], sim.spins(), err_msg="oracle " + tag)
            np.testing.assert_array_equal(out["energies"], sim.energies(), err_msg="oracle " + tag)


def test_submissions_from_several_threads():
    reqs = request_set(8, 12)
    prepared = [tables(r["inst"]) for r in reqs]
    server = ea.Server(round_ms=2)
    tickets = [None] * len(reqs)

    def client(idx):
        for i in idx:
            r = reqs[i]
            tickets[i] = submit(server, r["inst"], *prepared[i], r["n"], r["k"])
            time.sleep(r["delay"])

    th = [threading.Thread(target=client, args=(range(j, len(reqs), 2),)) for j in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    outs = [server.wait(t) for t in tickets]
    server.close()
    for r, (inp, metro, swapt), out in zip(reqs, prepared, outs):
        sp, en = alone(r["inst"], inp, metro, swapt, r["n"], r["k"])
        np.testing.assert_array_equal(out["spins"], sp)
        np.testing.assert_array_equal(out["energies"], en)


def test_request_errors():
    server = ea.Server(mem_budget=1 << 20)
    inst = W.Instance(L=8, G=1, NT=4, C=2, seed=3, tmin=1.0, tmax=2.0, input_seed=3)
    inp, metro, swapt = tables(inst)
    # odd L is rejected at submission
    bad = ea._Config(5, 1, 4, 2, 3, None, None, None, None, 0)
    req = ea._Request(10, 1, None, None)
    t = ea.ctypes.c_uint64(0)
    assert server.lib.ea_submit(server.s, ea.ctypes.byref(bad), ea.ctypes.byref(req),
                                ea.ctypes.byref(t)) == -1
    # larger than the whole budget: the ticket finishes with EA_ENOMEM
    big = W.Instance(L=16, G=8, NT=32, C=2, seed=4, tmin=1.0, tmax=2.0, input_seed=4)
    tb = submit(server, big, *tables(big), 10, 1)
    with pytest.raises(ea.EAError) as ei:
        server.wait(tb)
    assert ei.value.code == -2
    # a fitting request still runs; its ticket retires after the first poll
    ts = submit(server, inst, inp, metro, swapt, 5, 1)
    out = server.wait(ts)
    sp, en = alone(inst, inp, metro, swapt, 5, 1)
    np.testing.assert_array_equal(out["spins"], sp)
    assert server.lib.ea_poll(server.s, ts, 0) == -1
    assert server.lib.ea_poll(server.s, 987654, 0) == -1
    st = server.stats()
    assert st["completed"] == 1 and st["failed"] == 1
    server.close()


def tp_alone(inst, inp, metro, swapt, n, k):
    tp = ea.TPEnsemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    tp.sweep(n, k)
    torch.cuda.synchronize()
    sp, en = tp.read()
    out = sp.cpu().numpy().view(np.uint32), en.cpu().numpy()
    tp.close()
    return out


def test_temperature_packed_requests_match_alone():
    """Temperature-packed requests (ea_submit_tp) served together with
    realization-packed ones, some arriving while others run: each result equals
    the same temperature-packed ensemble run alone (TPEnsemble), whatever the
    rounds it was split into; two words per site for NT > 32 included."""
    rng = np.random.Generator(np.random.PCG64(77))
    tps = []
    for j, (L, R, NT, C, n, k) in enumerate([(8, 5, 24, 2, 300, 10), (4, 40, 32, 1, 137, 1),
                                             (12, 3, 40, 2, 90, 7), (6, 150, 16, 2, 500, 10),
                                             (16, 2, 33, 1, 45, 5), (10, 9, 1, 2, 60, 3)]):
        inst = W.Instance(L=L, G=R, NT=NT, C=C, seed=int(rng.integers(1, 2**40)), tmin=0.9, tmax=2.0,
                          input_seed=int(rng.integers(1, 2**31)))
        inp = W.draw_tp_inputs(inst)
        metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
        tps.append((inst, inp, metro, swapt, n, k))
    packed = [r for r in request_set(6, 78)]
    srv = ea.Server(round_ms=5)
    tickets = []
    for j in range(max(len(tps), len(packed))):
        if j < len(tps):
            inst, inp, metro, swapt, n, k = tps[j]
            tickets.append(("tp", j, srv.submit_tp(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"],
                                                   inp["spins"], metro, swapt, n, k)))
        if j < len(packed):
            r = packed[j]
            inp, metro, swapt = tables(r["inst"])
            tickets.append(("packed", j, submit(srv, r["inst"], inp, metro, swapt, r["n"], r["k"])))
        time.sleep(0.003)
    for kind, j, t in tickets:
        out = srv.wait(t)
        if kind == "tp":
            sp, en = tp_alone(*tps[j])
            assert np.array_equal(out["spins"], sp), f"temperature-packed request {j}: spins"
            assert np.array_equal(out["energies"], en), f"temperature-packed request {j}: energies"
        else:
            r = packed[j]
            inp, metro, swapt = tables(r["inst"])
            sp, en = alone(r["inst"], inp, metro, swapt, r["n"], r["k"])
            assert np.array_equal(out["spins"], sp) and np.array_equal(out["energies"], en), f"request {j}"
    st = srv.stats()
    assert st["completed"] == len(tickets) and st["failed"] == 0
    srv.close()


def test_temperature_packed_request_errors():
    srv = ea.Server()
    inst = W.Instance(L=8, G=2, NT=8, C=2, seed=5, tmin=0.9, tmax=2.0, input_seed=9)
    inp = W.draw_tp_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    with pytest.raises(ea.EAError) as ei:    # odd L is rejected at once
        srv.submit_tp(7, 2, 8, 2, 5, np.zeros((2, 3, 343), np.uint8), np.zeros((2, 2, 343), np.uint32),
                      metro, swapt, 10, 1)
    assert ei.value.code == -1
    bad = metro.copy()
    bad[0, 0], bad[0, 1] = bad[0, 1] + 1, bad[0, 0]   # not non-decreasing: fails at admission
    t = srv.submit_tp(8, 2, 8, 2, 5, inp["bonds"], inp["spins"], bad, swapt, 10, 1)
    with pytest.raises(ea.EAError) as ei:
        srv.wait(t)
    assert ei.value.code == -1
    st = srv.stats()
    assert st["failed"] == 1
    srv.close()
