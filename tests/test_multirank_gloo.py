"""The N > 1 host path on CPU: two gloo ranks holding the word-groups of one
ensemble (bench.rank_groups / rank_inputs, group_base = the shard's first global
group), nothing exchanged but the timing reduction, as the benchmark's ranks do
on GPUs.  The per-rank step here is the oracle; the shards together must equal
the whole ensemble run in one piece."""
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


def _shard_step(inst, groups, inp, n, k):
    g0, g1 = groups
    metro = oracle.metro_table(inp["betas"])
    swapt = oracle.swap_table_trimmed(inp["betas"], inst.N)
    sim = oracle.OracleSim(inst.L, g1 - g0, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                           metro, swapt, group_base=g0)
    out = sim.sweep(n, k, swap_log=True)
    return sim.energies(), sim.spins(), out["swap_log"]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        job, groups, inp = bench.rank_inputs(W.SMALL, r, w)
        energies, spins, slog = _shard_step(job, groups, inp, 25, 1)
        t_local = 0.25 * (r + 1)                  # a stand-in step time per rank
        t_max = bench.reduce_max(t_local, w)
        flips = 25 * job.N * job.NT * job.C * 32 * (groups[1] - groups[0])
        value, _ = bench.aggregate([t_max] * w, flips)
        q.put({"rank": r, "world": w, "local": local, "groups": groups, "job_G": job.G,
               "energies": energies, "spins": spins, "swap_log": slog,
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
    # the two ranks hold disjoint halves of one ensemble of twice the workload's groups
    assert res[0]["job_G"] == res[1]["job_G"] == 2 * W.SMALL.G
    assert res[0]["groups"] == (0, W.SMALL.G) and res[1]["groups"] == (W.SMALL.G, 2 * W.SMALL.G)
    # the slowest rank's time sets the job value, the same on every rank
    assert res[0]["t_max"] == res[1]["t_max"] == 0.5
    assert res[0]["value"] == res[1]["value"] == pytest.approx(0.5 / (2 * res[0]["flips"]) * 1e12)
    # the shards together are exactly the whole ensemble run in one piece
    job = bench.job_instance(W.SMALL, 2)
    inp = W.draw_inputs(job)
    e, s, sl = _shard_step(job, (0, job.G), inp, 25, 1)
    for d in res:
        g0, g1 = d["groups"]
        np.testing.assert_array_equal(d["energies"], e[g0:g1])
        np.testing.assert_array_equal(d["spins"], s[g0:g1])
        np.testing.assert_array_equal(d["swap_log"], sl[:, g0:g1])
    assert not np.array_equal(res[0]["spins"], res[1]["spins"])


def test_rank_groups_partition_the_ensemble():
    for G in (1, 7, 64, 256):
        for world in (1, 2, 3, 8):
            cuts = [bench.rank_groups(G, r, world) for r in range(world)]
            assert cuts[0][0] == 0 and cuts[-1][1] == G
            assert all(a[1] == b[0] for a, b in zip(cuts, cuts[1:]))
    assert bench.job_instance(W.SCALE, 1) == W.SCALE
    assert bench.job_instance(W.SCALE, 4).G == 4 * W.SCALE.G


def test_single_rank_reduction_is_identity():
    assert bench.reduce_max(1.25, 1) == 1.25
    v, t = bench.aggregate([0.5], 1000)
    assert t == 0.5 and v == pytest.approx(0.5 / 1000 * 1e12)
