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

(for the temperature-packed workload, realization r = bit 0 of group r: spins
[NT][C][N] uint8, energies [NT][C] int32, swap_log [P][C] uint32 with bit p =
pair p)
and, for the L=8 workload, the overlap histogram [NT][N+1] (uint64) and the
energy sums [NT] of the measurement after every sweep of the second half.
The paper prints no worked example: these are not paper values, they freeze the
oracle (itself pinned by tests/test_oracle_pins.py) at full length so that the
GPU path can be compared with it where running the oracle live would take hours.

Only ``oracle/`` and ``workloads/`` are called.  Jobs run in a process pool
(spawn); each rewrites its part file after every chunk, so a long run cut short
still gives its completed chunks (the merge keeps the chunks every sampled
group has finished and records that prefix as the workload's length), and a
restarted run redoes only the jobs that had not finished.

Run:  python tests/golden/make_digests.py --jobs 6 [--only scale,large16] [--parts DIR]
      python tests/golden/make_digests.py --merge-only --parts DIR   (records so far)
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
        # the whole 10^5 sweeps (~0.13 s per sweep of one L=16 group on one core,
        # ~3.7 h a group); records after every 10^4
        "large16": dict(inst=W.LARGE16, sweeps=W.LARGE_SWEEPS, swap_every=W.LARGE_SWAP_EVERY,
                        chunk=10_000, groups=spread(W.LARGE16.G, 4), energy_log=True, measure=None),
        # 2*10^3 of the 10^5 sweeps: ~2.3 s per sweep of one L=32 group (the whole
        # run would take ~63 h a group); records after every 500
        "large32": dict(inst=W.LARGE32, sweeps=2_000, swap_every=W.LARGE_SWAP_EVERY,
                        chunk=500, groups=spread(W.LARGE32.G, 4), energy_log=True, measure=None),
    }
    for inst in W.batch_instances():
        t[f"batch_L{inst.L}"] = dict(inst=inst, sweeps=W.BATCH_SWEEPS, swap_every=W.BATCH_SWAP_EVERY,
                                     chunk=W.BATCH_SWEEPS, groups=[0, inst.G - 1], energy_log=True,
                                     measure=None)
    # temperature-packed form: realization r is bit 0 of word-group r of the
    # realization-packed oracle run (group_base = r); sampled realizations
    t["tpack"] = dict(inst=W.TPACK, sweeps=W.TPACK_SWEEPS, swap_every=W.TPACK_SWAP_EVERY, chunk=500,
                      groups=spread(W.TPACK.G, 4), energy_log=False, measure=None, tpack=True)
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
    tp = w.get("tpack", False)
    if tp:
        inp = W.draw_tp_inputs(inst)
        bonds, spins = W.tp_as_groups(inp["bonds"], inp["spins"], inst.NT)
    else:
        inp = W.draw_inputs(inst)
        bonds, spins = inp["bonds"], inp["spins"]
    metro = oracle.metro_table(inp["betas"])
    swapt = oracle.swap_table_trimmed(inp["betas"], inst.N)
    sim = oracle.OracleSim(inst.L, 1, inst.NT, inst.C, inst.seed, bonds[g:g + 1], spins[g:g + 1], metro,
                           swapt, group_base=g)
    qh = es = None
    mf = me = 0
    if w["measure"] is not None:
        mf, me = w["measure"]
        qh = np.zeros((inst.NT, inst.N + 1), np.uint64)
        es = np.zeros(inst.NT, np.int64)
    chunks = []
    t0 = time.time()
    done = 0
    path = os.path.join(parts, f"{name}_g{g}.json")

    def save(complete: bool):
        # the record so far: a run cut short still gives its completed chunks
        res = {"name": name, "group": g, "chunks": chunks, "complete": complete,
               "energy_per_spin_slot0": float(sim.energies()[0][0].mean() / inst.N),
               "cpu_seconds": round(time.time() - t0, 1),
               "flip_attempts": int(done) * inst.N * inst.NT * inst.C * 32}
        if qh is not None and complete:
            res["qhist"] = digest(qh)
            res["qhist_total"] = int(qh.sum())
            res["esum"] = [int(x) for x in es]
        with open(path + ".tmp", "w") as f:
            json.dump(res, f, indent=1)
        os.replace(path + ".tmp", path)

    while done < w["sweeps"]:
        n = min(w["chunk"], w["sweeps"] - done)
        out = sim.sweep(n, w["swap_every"], energy_log=w["energy_log"], swap_log=True, qhist=qh,
                        esum=es, measure_from=mf, measure_every=me)
        done += n
        sl = out["swap_log"][:, 0]
        if tp:
            # realization g alone (bit 0): spins [NT][C][N] uint8, energies [NT][C],
            # accepted pairs per pass and copy as one word (bit p = pair p)
            sl = (sl & np.uint32(1)).astype(np.uint64)
            sl = (sl << np.arange(inst.NT - 1, dtype=np.uint64)).sum(axis=-1).astype(np.uint32)
            rec = {"end_sweep": done,
                   "spins": digest((sim.spins()[0] & np.uint32(1)).astype(np.uint8)),
                   "energies": digest(np.ascontiguousarray(sim.energies()[0][:, :, 0])),
                   "swap_log": digest(sl),
                   "swap_accepts": int(sum(bin(int(x)).count("1") for x in sl.ravel()))}
        else:
            rec = {"end_sweep": done,
                   "spins": digest(sim.spins()[0]),
                   "energies": digest(sim.energies()[0]),
                   "swap_log": digest(sl),
                   "swap_accepts": int(sum(bin(int(x)).count("1") for x in sl.ravel()))}
        if w["energy_log"]:
            rec["energy_log"] = digest(out["energy_log"][:, 0])
        chunks.append(rec)
        save(done >= w["sweeps"])
    return path


def _run_job_args(args):
    return run_job(*args)


def merge(parts: str, names: list[str]) -> dict:
    """Digests of the named workloads whose sampled groups all have a record,
    each cut to the chunks that every group has completed."""
    import oracle

    table = workload_table()
    doc = {"note": "oracle digests (tests/golden/make_digests.py); sampled word-groups of each "
                   "workload at its stated shape, run by the oracle with group_base = g",
           "workloads": {}}
    for name in names:
        w = table[name]
        recs = {}
        for g in w["groups"]:
            path = os.path.join(parts, f"{name}_g{g}.json")
            if os.path.exists(path):
                with open(path) as f:
                    recs[g] = json.load(f)
        if len(recs) < len(w["groups"]) or min(len(r["chunks"]) for r in recs.values()) == 0:
            print("not merged (groups still running or not started):", name)
            continue
        m = min(len(r["chunks"]) for r in recs.values())
        complete = all(r.get("complete", True) for r in recs.values())
        inst = w["inst"]
        inp = W.draw_tp_inputs(inst) if w.get("tpack") else W.draw_inputs(inst)
        ent = {"inst": inst_dict(inst), "tpack": bool(w.get("tpack", False)), "sweeps": recs[w["groups"][0]]["chunks"][m - 1]["end_sweep"],
               "planned_sweeps": w["sweeps"], "swap_every": w["swap_every"],
               "chunk": w["chunk"], "energy_log": w["energy_log"],
               "measure": list(w["measure"]) if (w["measure"] and complete) else None,
               "metro_table": digest(oracle.metro_table(inp["betas"])),
               "swap_table": digest(oracle.swap_table_trimmed(inp["betas"], inst.N)),
               "groups": {}}
        for g, r in recs.items():
            r = dict(r)
            r.pop("name")
            r.pop("group")
            r.pop("complete", None)
            r["chunks"] = r["chunks"][:m]
            if not complete:
                for k in ("qhist", "qhist_total", "esum"):
                    r.pop(k, None)
            ent["groups"][str(g)] = r
        doc["workloads"][name] = ent
    return doc


def _done(parts: str, name: str, g: int) -> bool:
    path = os.path.join(parts, f"{name}_g{g}.json")
    if not os.path.exists(path):
        return False
    with open(path) as f:
        return json.load(f).get("complete", True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 2))
    ap.add_argument("--only", default="", help="comma-separated workload names")
    ap.add_argument("--parts", default=os.path.join(HERE, ".parts"))
    ap.add_argument("--merge-only", action="store_true",
                    help="merge the records written so far (complete chunks only) and exit")
    a = ap.parse_args()
    table = workload_table()
    names = [n for n in table if not a.only or n in a.only.split(",")]
    os.makedirs(a.parts, exist_ok=True)
    todo = [(n, g) for n in names for g in table[n]["groups"] if not _done(a.parts, n, g)]
    # the longest full-length runs start first; the L=32 prefix runs go last,
    # after the short jobs, since any completed prefix of theirs is usable
    cost = lambda j: table[j[0]]["sweeps"] * table[j[0]]["inst"].N * table[j[0]]["inst"].NT
    todo.sort(key=lambda j: (j[0] == "large32", -cost(j)))
    if todo and not a.merge_only:
        print(f"{len(todo)} jobs on {a.jobs} processes", flush=True)
        with mp.get_context("spawn").Pool(a.jobs) as pool:
            for path in pool.imap_unordered(_run_job_args, [(n, g, a.parts) for n, g in todo], chunksize=1):
                print("done", path, flush=True)
    doc = merge(a.parts, names)
    if os.path.exists(OUT):
        with open(OUT) as f:
            old = json.load(f)
        old["workloads"].update(doc["workloads"])
        doc = old
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
    print("wrote", OUT, "with", sorted(doc["workloads"]))
    return 0


if __name__ == "__main__":
    sys.exit(main())
