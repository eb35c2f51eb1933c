"""Writes tests/golden/small_run.json from the CPU oracle alone.

The paper prints no worked example, so this fixture is not a paper value: it
freezes the oracle's output on the small workload (L=4, 32 realizations,
16 temperatures x 2 copies, 2000 sweeps, a swap pass after every sweep) as
SHA-256 digests of its little-endian arrays, so that any later change of the
oracle's arithmetic shows up as a failing regression test.

Run:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<")).tobytes()).hexdigest()


def small_run():
    inst = W.SMALL
    inp = W.draw_inputs(inst)
    metro = oracle.metro_table(inp["betas"])
    swapt = oracle.swap_table_trimmed(inp["betas"], inst.N)
    sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                           metro, swapt)
    out = sim.sweep(W.SMALL_SWEEPS, W.SMALL_SWAP_EVERY, energy_log=True, swap_log=True)
    return {
        "workload": "L=4, G=1 (32 realizations), NT=16 in [0.8,2.0], C=2, seed=1, input_seed=101",
        "sweeps": W.SMALL_SWEEPS,
        "swap_every": W.SMALL_SWAP_EVERY,
        "metro_table": digest(metro),
        "swap_table": digest(swapt),
        "swap_len": int(swapt.shape[1]),
        "energy_log": digest(out["energy_log"]),
        "swap_log": digest(out["swap_log"]),
        "final_spins": digest(sim.spins()),
        "final_energy_mean_per_spin_slot0": float(out["energy_log"][-1, :, 0].mean() / inst.N),
    }


if __name__ == "__main__":
    res = small_run()
    with open(os.path.join(HERE, "small_run.json"), "w") as f:
        json.dump(res, f, indent=1, sort_keys=True)
    print(json.dumps(res, indent=1, sort_keys=True))
