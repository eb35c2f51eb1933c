"""The stored full-length oracle digests (tests/golden/full_length.json) on the CPU:
their shapes are the workloads' own, their chunks are consistent prefixes, the
merge of partial records keeps the common prefix, and the cheapest records are
re-derived here from the oracle alone (a stale file -- one written by an
earlier oracle -- fails)."""
import json
import os

import numpy as np
import pytest

import golden_path  # noqa: F401  (adds tests/golden to sys.path)
import make_digests as MD
import workloads as W

GOLDEN = os.path.join(os.path.dirname(MD.__file__), "full_length.json")


def golden():
    if not os.path.exists(GOLDEN):
        pytest.skip("full_length.json not written yet")
    with open(GOLDEN) as f:
        return json.load(f)["workloads"]


def test_stored_digests_describe_the_workloads():
    table = MD.workload_table()
    for name, ent in golden().items():
        assert name in table, name
        w = table[name]
        assert ent["inst"] == MD.inst_dict(w["inst"]), name
        assert ent["swap_every"] == w["swap_every"] and ent["chunk"] == w["chunk"], name
        assert 0 < ent["sweeps"] <= w["sweeps"], name
        assert sorted(int(g) for g in ent["groups"]) == sorted(w["groups"]), name
        for g, rec in ent["groups"].items():
            ends = [c["end_sweep"] for c in rec["chunks"]]
            want = list(range(w["chunk"], ent["sweeps"], w["chunk"])) + [ent["sweeps"]]
            assert ends == want, (name, g)
            if ent["measure"] is not None:
                inst = w["inst"]
                mf, me = ent["measure"]
                # one histogram entry per (slot, lane, measured sweep) -- the
                # group's 32 lanes x 2 copies count once per copy pair
                n_meas = len(range(mf, ent["sweeps"], me))
                assert rec["qhist_total"] == n_meas * inst.NT * 32, (name, g)
    names = golden()
    assert "scale" in names and names["scale"]["sweeps"] == W.SCALE_SWEEPS


def test_merge_keeps_the_common_prefix(tmp_path):
    """Records of different lengths merge to the chunks every group finished;
    an incomplete workload drops its end-of-run histogram."""
    table = MD.workload_table()
    w = table["scale"]
    for i, g in enumerate(w["groups"]):
        n = 3 + i                                      # 3, 4, 5, 6 chunks
        chunks = [{"end_sweep": (k + 1) * w["chunk"], "spins": f"s{g}{k}", "energies": "e", "swap_log": "l",
                   "swap_accepts": 0} for k in range(n)]
        rec = {"name": "scale", "group": g, "chunks": chunks, "complete": False, "qhist": "q"}
        with open(tmp_path / f"scale_g{g}.json", "w") as f:
            json.dump(rec, f)
    doc = MD.merge(str(tmp_path), ["scale"])["workloads"]["scale"]
    assert doc["sweeps"] == 3 * w["chunk"] and doc["planned_sweeps"] == w["sweeps"]
    assert doc["measure"] is None
    for g, rec in doc["groups"].items():
        assert len(rec["chunks"]) == 3 and "qhist" not in rec
    # a workload with a group not started is left out
    os.remove(tmp_path / f"scale_g{w['groups'][-1]}.json")
    assert MD.merge(str(tmp_path), ["scale"])["workloads"] == {}


@pytest.mark.parametrize("name", ["batch_L4", "served_08"])
def test_cheapest_records_rederived_from_the_oracle(name, tmp_path):
    """Re-runs the oracle for the cheapest stored records (a few seconds each)
    and compares every digest."""
    ent = golden().get(name)
    if ent is None:
        pytest.skip(f"no digests for {name}")
    for g, rec in ent["groups"].items():
        MD.run_job(name, int(g), str(tmp_path))
        with open(tmp_path / f"{name}_g{g}.json") as f:
            got = json.load(f)
        assert got["complete"]
        assert got["chunks"] == rec["chunks"], (name, g)
