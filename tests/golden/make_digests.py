"""Writes tests/golden/full_length.json: oracle digests of the five workloads at
their stated shapes and lengths, on sampled word-groups.

Word-groups are independent and their random-number counters carry the global
group index (Sec. 3.3: realizations map to independent blocks), so the oracle
run on one group with ``group_base = g`` reproduces exactly what group g of the
full ensemble does.  For every sampled group the script records, after each
chunk of sweeps, SHA-256 digests of the little-endian arrays

  spins       [NT][C][N]     uint32  final spin words, by temperature slot
  energies    [NT][C][32]    int32   per-lane energies, by slot
  swap_log    [P][C][NT-1]   uint32  accepted-pair masks of the chunk's passes
  energy_log  [n][NT][C][32] int32   energies after every sweep of the chunk

and, for the L=8 workload, the overlap histogram [NT][N+1] (uint64) and the
energy sums [NT] of the measurement after every sweep of the second half.
The paper prints no worked example: these are not paper values, they freeze the
oracle (itself pinned by tests/test_oracle_pins.py) at full length so that the
GPU path can be compared with it where running the oracle live would take hours.

Only ``oracle/`` and ``workloads/`` are called.  Jobs run in a process pool
(spawn) and write one part file each, so an interrupted run resumes.

Run:  python tests/golden/make_digests.py --jobs 6 [--only scale,large16] [--parts DIR]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "full_length.json")
N_SERVED = 16   # requests of the served trace, in arrival order
# Served requests whose sampled group costs the oracle more than this many flip
# attempts (about 45 min on one core) are passed over; the next ones are taken.
SERVED_MAX_FLIPS = 2.0e11


def digest(a: np.ndarray) -> str:
    a = np.ascontiguousarray(a)
    return hashlib.sha256(a.astype(a.dtype.newbyteorder("<")).tobytes()).hexdigest()


def inst_dict(inst: W.Instance) -> dict:
    return {"L": inst.L, "G": inst.G, "NT": inst.NT, "C": inst.C, "seed": inst.seed,
            "tmin": inst.tmin, "tmax": inst.tmax, "input_seed": inst.input_seed}


def spread(G: int, k: int) -> list[int]:
    """k groups spread over 0..G-1, both ends included."""
    return sorted({(G - 1) * j // (k - 1) for j in range(k)}) if k > 1 else [0]


def workload_table() -> dict:
    """name -> {inst, sweeps, swap_every, chunk, groups, energy_log, measure}."""
    t = {
        "scale": dict(inst=W.SCALE, sweeps=W.SCALE_SWEEPS, swap_every=W.SCALE_SWAP_EVERY,
                      chunk=10_000, groups=spread(W.SCALE.G, 4), energy_log=True,
                      measure=(W.SCALE_SWEEPS // 2, 1)),
        # 3*10^4 of the 10^5 sweeps: the oracle takes ~0.13 s per sweep of one
        # L=16 group (~3.7 h for the whole run).
        "large16": dict(inst=W.LARGE16, sweeps=30_000, swap_every=W.LARGE_SWAP_EVERY,
                        chunk=10_000, groups=spread(W.LARGE16.G, 4), energy_log=True, measure=None),
        # 10^3 of the 10^5 sweeps: ~2.3 s per sweep of one L=32 group.
        "large32": dict(inst=W.LARGE32, sweeps=1_000, swap_every=W.LARGE_SWAP_EVERY,
                        chunk=500, groups=spread(W.LARGE32.G, 4), energy_log=True, measure=None),
    }
    for inst in W.batch_instances():
        t[f"batch_L{inst.L}"] = dict(inst=inst, sweeps=W.BATCH_SWEEPS, swap_every=W.BATCH_SWAP_EVERY,
                                     chunk=W.BATCH_SWEEPS, groups=[0, inst.G - 1], energy_log=True,
                                     measure=None)
    taken = 0
    for r, req in enumerate(W.served_trace()):
        inst = req["inst"]
        if req["sweeps"] * inst.N * inst.NT * inst.C * 32 > SERVED_MAX_FLIPS:
            continue
        t[f"served_{r:02d}"] = dict(inst=inst, sweeps=req["sweeps"], swap_every=req["swap_every"],
                                    chunk=req["sweeps"], groups=[inst.G - 1], energy_log=False,
                                    measure=None)
        taken += 1
        if taken == N_SERVED:
            break
    return t


def run_job(name: str, g: int, parts: str) -> str:
    import oracle  # imported in the worker (spawned process)

    w = workload_table()[name]
    inst: W.Instance = w["inst"]
    inp = W.draw_inputs(inst)
    metro = oracle.metro_table(inp["betas"])
    swapt = oracle.swap_table_trimmed(inp["betas"], inst.N)
    sim = oracle.OracleSim(inst.L, 1, inst.NT, inst.C, inst.seed, inp["bonds"][g:g + 1],
                           inp["spins"][g:g + 1], metro, swapt, group_base=g)
    qh = es = None
    mf = me = 0
    if w["measure"] is not None:
        mf, me = w["measure"]
        qh = np.zeros((inst.NT, inst.N + 1), np.uint64)
        es = np.zeros(inst.NT, np.int64)
    chunks = []
    t0 = time.time()
    done = 0
    while done < w["sweeps"]:
        n = min(w["chunk"], w["sweeps"] - done)
        out = sim.sweep(n, w["swap_every"], energy_log=w["energy_log"], swap_log=True, qhist=qh,
                        esum=es, measure_from=mf, measure_every=me)
        done += n
        sl = out["swap_log"][:, 0]
        rec = {"end_sweep": done,
               "spins": digest(sim.spins()[0]),
               "energies": digest(sim.energies()[0]),
               "swap_log": digest(sl),
               "swap_accepts": int(sum(bin(int(x)).count("1") for x in sl.ravel()))}
        if w["energy_log"]:
            rec["energy_log"] = digest(out["energy_log"][:, 0])
        chunks.append(rec)
    res = {"name": name, "group": g, "chunks": chunks,
           "energy_per_spin_slot0": float(sim.energies()[0][0].mean() / inst.N),
           "cpu_seconds": round(time.time() - t0, 1),
           "flip_attempts": int(w["sweeps"]) * inst.N * inst.NT * inst.C * 32}
    if qh is not None:
        res["qhist"] = digest(qh)
        res["qhist_total"] = int(qh.sum())
        res["esum"] = [int(x) for x in es]
    path = os.path.join(parts, f"{name}_g{g}.json")
    with open(path + ".tmp", "w") as f:
        json.dump(res, f, indent=1)
    os.replace(path + ".tmp", path)
    return path


def _run_job_args(args):
    return run_job(*args)


def merge(parts: str, names: list[str]) -> dict:
    import oracle

    table = workload_table()
    doc = {"note": "oracle digests (tests/golden/make_digests.py); sampled word-groups of each "
                   "workload at its stated shape, run by the oracle with group_base = g",
           "workloads": {}}
    for name in names:
        w = table[name]
        inst = w["inst"]
        inp = W.draw_inputs(inst)
        ent = {"inst": inst_dict(inst), "sweeps": w["sweeps"], "swap_every": w["swap_every"],
               "chunk": w["chunk"], "energy_log": w["energy_log"],
               "measure": list(w["measure"]) if w["measure"] else None,
               "metro_table": digest(oracle.metro_table(inp["betas"])),
               "swap_table": digest(oracle.swap_table_trimmed(inp["betas"], inst.N)),
               "groups": {}}
        for g in w["groups"]:
            with open(os.path.join(parts, f"{name}_g{g}.json")) as f:
                p = json.load(f)
            p.pop("name")
            ent["groups"][str(p.pop("group"))] = p
        doc["workloads"][name] = ent
    return doc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    ap.add_argument("--only", default="", help="comma-separated workload names")
    ap.add_argument("--parts", default=os.path.join(HERE, ".parts"))
    ap.add_argument("--merge-only", action="store_true")
    a = ap.parse_args()
    table = workload_table()
    names = [n for n in table if not a.only or n in a.only.split(",")]
    os.makedirs(a.parts, exist_ok=True)
    todo = [(n, g) for n in names for g in table[n]["groups"]
            if not os.path.exists(os.path.join(a.parts, f"{n}_g{g}.json"))]
    cost = lambda j: table[j[0]]["sweeps"] * table[j[0]]["inst"].N * table[j[0]]["inst"].NT
    todo.sort(key=cost, reverse=True)
    if todo and not a.merge_only:
        print(f"{len(todo)} jobs on {a.jobs} processes", flush=True)
        with mp.get_context("spawn").Pool(a.jobs) as pool:
            for path in pool.imap_unordered(_run_job_args, [(n, g, a.parts) for n, g in todo]):
                print("done", path, flush=True)
    missing = [(n, g) for n in names for g in table[n]["groups"]
               if not os.path.exists(os.path.join(a.parts, f"{n}_g{g}.json"))]
    if missing:
        print("missing parts:", missing)
        return 1
    doc = merge(a.parts, names)
    if a.only and os.path.exists(OUT):
        with open(OUT) as f:
            old = json.load(f)
        old["workloads"].update(doc["workloads"])
        doc = old
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
    print("wrote", OUT)
    return 0


if __name__ == "__main__":
    sys.exit(main())
