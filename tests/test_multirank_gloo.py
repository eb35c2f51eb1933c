"""The N > 1 host path on CPU: two gloo ranks, each simulating its own
ensemble (weak scaling, nothing exchanged but the timing reduction), as the
benchmark's ranks do on GPUs.  The per-rank step here is the oracle."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

import bench
import oracle
import workloads as W

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_step(inst, n, k):
    inp = W.draw_inputs(inst)
    metro = oracle.metro_table(inp["betas"])
    swapt = oracle.swap_table_trimmed(inp["betas"], inst.N)
    sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                           metro, swapt)
    sim.sweep(n, k)
    return sim.energies(), sim.spins()


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        inst = bench.rank_instance(W.SMALL, r)
        energies, spins = _rank_step(inst, 25, 1)
        t_local = 0.25 * (r + 1)                  # a stand-in step time per rank
        t_max = bench.reduce_max(t_local, w)
        flips = 25 * inst.N * inst.NT * inst.C * 32 * inst.G
        value, _ = bench.aggregate([t_max] * w, flips)
        q.put({"rank": r, "world": w, "local": local, "seed": inst.seed,
               "input_seed": inst.input_seed, "energies": energies, "spins": spins,
               "t_max": t_max, "value": value, "flips": flips})
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_exchange():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda d: d["rank"])
    assert [d["rank"] for d in res] == [0, 1] and all(d["world"] == 2 for d in res)
    # each rank has its own disorder and Philox key
    assert res[0]["seed"] != res[1]["seed"] and res[0]["input_seed"] != res[1]["input_seed"]
    # the slowest rank's time sets the job value, the same on every rank
    assert res[0]["t_max"] == res[1]["t_max"] == 0.5
    assert res[0]["value"] == res[1]["value"] == pytest.approx(0.5 / (2 * res[0]["flips"]) * 1e12)
    # a rank's result depends on its own ensemble only: equal to running it here alone
    for d in res:
        e, s = _rank_step(bench.rank_instance(W.SMALL, d["rank"]), 25, 1)
        np.testing.assert_array_equal(d["energies"], e)
        np.testing.assert_array_equal(d["spins"], s)
    assert not np.array_equal(res[0]["spins"], res[1]["spins"])


def test_single_rank_reduction_is_identity():
    assert bench.reduce_max(1.25, 1) == 1.25
    v, t = bench.aggregate([0.5], 1000)
    assert t == 0.5 and v == pytest.approx(0.5 / 1000 * 1e12)
