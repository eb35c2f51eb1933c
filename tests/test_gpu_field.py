"""GPU parity in an external field (Eq. 1 with h != 0): the field kernels
through the C ABI against the oracle, bit for bit.  Flip and swap decisions
are integer compares of Et = h_den E - h_num M against tables both sides
receive, so spins, energies, magnetisations, energy logs and swap masks must
be equal (tolerance 0)."""
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


def field_pair(inst, h_num, h_den, tmin=None, tmax=None):
    inp = W.draw_inputs(inst)
    mf, sw = ea.ea_build_tables_field(inp["betas"], inst.N, h_num, h_den)
    gpu = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], None, sw,
                      field=(h_num, h_den, mf))
    sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                           oracle.metro_table(inp["betas"]), sw, field=(h_num, h_den, mf))
    return gpu, sim


def plan_indices(gpu, form):
    return [i for i, p in enumerate(gpu.plans()) if p["form"] == form]


def compare(gpu, sim, n, swap_every, tag):
    out = gpu.sweep(n, swap_every, energy_log=True, swap_log=True)
    o = sim.sweep(n, swap_every, energy_log=True, swap_log=True, threads=8)
    np.testing.assert_array_equal(out["energy_log"].cpu().numpy(), o["energy_log"], err_msg="elog " + tag)
    np.testing.assert_array_equal(out["swap_log"].cpu().numpy().view(np.uint32), o["swap_log"],
                                  err_msg="swap log " + tag)
    np.testing.assert_array_equal(gpu.read_spins().cpu().numpy().view(np.uint32), sim.spins(),
                                  err_msg="spins " + tag)
    np.testing.assert_array_equal(gpu.measure()[0].cpu().numpy(), sim.energies(), err_msg="E " + tag)
    np.testing.assert_array_equal(gpu.magnetisations().cpu().numpy(), sim.magnetisations(),
                                  err_msg="M " + tag)


@pytest.mark.parametrize("L,G,NT,C,h_num,h_den,swap_every", [
    (4, 2, 8, 2, 1, 2, 1), (6, 1, 7, 2, -5, 3, 2), (8, 2, 12, 2, 3, 1, 1), (10, 1, 5, 1, 1, 4, 3),
    (12, 1, 6, 2, -1, 2, 1), (16, 1, 4, 2, 2, 5, 2),
])
@pytest.mark.parametrize("form", ["unit", "chunked"])
def test_field_matches_oracle(L, G, NT, C, h_num, h_den, swap_every, form):
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=500 + L, tmin=0.8, tmax=2.0, input_seed=L + 7)
    gpu, sim = field_pair(inst, h_num, h_den)
    idx = plan_indices(gpu, form)
    assert idx, f"no {form} plan"
    assert all(p["form"] != "unit-fast" for p in gpu.plans())
    gpu.select_plan(idx[0])
    tag = f"{form} L={L} NT={NT} h={h_num}/{h_den}"
    compare(gpu, sim, 9, swap_every, tag)
    compare(gpu, sim, 7, swap_every, tag + " (continued)")


def test_field_large_lattice_chunked():
    """L = 32 (chunked form only), a field that favours up spins from a random start."""
    inst = W.Instance(L=32, G=1, NT=4, C=2, seed=77, tmin=0.9, tmax=1.6, input_seed=78)
    gpu, sim = field_pair(inst, 1, 2)
    compare(gpu, sim, 6, 2, "L=32")


def test_every_field_plan_agrees():
    inst = W.Instance(L=8, G=1, NT=16, C=2, seed=91, tmin=0.8, tmax=2.0, input_seed=92)
    outs = []
    for i in range(len(field_pair(inst, 3, 2)[0].plans())):
        gpu, _ = field_pair(inst, 3, 2)
        gpu.select_plan(i)
        gpu.sweep(12, 1)
        outs.append((gpu.read_spins().cpu().numpy(), gpu.measure()[0].cpu().numpy()))
    for sp, en in outs[1:]:
        np.testing.assert_array_equal(sp, outs[0][0])
        np.testing.assert_array_equal(en, outs[0][1])


@pytest.mark.parametrize("h_den", [1, 4])
def test_zero_field_is_the_field_free_path(h_den):
    """h_num = 0 through the field entry point runs the field-free kernels (fast
    plans included) and gives the field-free trajectory."""
    inst = W.Instance(L=8, G=1, NT=8, C=2, seed=5, tmin=0.8, tmax=2.0, input_seed=6)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    mf, sw = ea.ea_build_tables_field(inp["betas"], inst.N, 0, h_den)
    np.testing.assert_array_equal(sw, swapt)
    a = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    b = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], None, sw,
                    field=(0, h_den, mf))
    assert [p["form"] for p in a.plans()] == [p["form"] for p in b.plans()]
    a.sweep(20, 1)
    b.sweep(20, 1)
    np.testing.assert_array_equal(a.read_spins().cpu().numpy(), b.read_spins().cpu().numpy())


def test_magnetisations_of_known_states():
    inst = W.Instance(L=6, G=1, NT=3, C=2, seed=1, tmin=1.0, tmax=2.0, input_seed=2)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    spins = np.zeros_like(inp["spins"])
    spins[0, 1] = 0xFFFFFFFF                       # slot 1 all up in both copies
    spins[0, 2, 0, :10] = 0x0000FFFF               # slot 2, copy 0: ten sites up in lanes 0..15
    gpu = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], spins, metro, swapt)
    M = gpu.magnetisations().cpu().numpy()
    N = inst.N
    assert np.all(M[0, 0] == -N) and np.all(M[0, 1] == N)
    assert np.all(M[0, 2, 0, :16] == 20 - N) and np.all(M[0, 2, 0, 16:] == -N)
    assert np.all(M[0, 2, 1] == -N)


def test_batch_keeps_field_and_field_free_members_apart():
    """One call runs one kernel: a batch takes members all in a field or all without."""
    inst = W.Instance(L=4, G=1, NT=4, C=2, seed=3, tmin=1.0, tmax=2.0, input_seed=4)
    gpu, _ = field_pair(inst, 1, 2)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    plain = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    b = ea.Batch([gpu])
    with pytest.raises(ea.EAError):
        b.add(plain)
    b.clear()
    b.add(plain)
    with pytest.raises(ea.EAError):
        b.add(gpu)


FIELD_MIX = [  # (L, G, NT, C, h_num, h_den): wavefront (L = 8), generic unit, chunked (L = 16 x 32)
    (8, 2, 24, 2, 1, 2), (8, 1, 9, 2, -3, 4), (6, 2, 7, 2, 2, 1), (10, 1, 12, 1, 1, 3), (16, 1, 32, 2, 1, 2),
]


def test_field_batch_matches_members_alone_and_oracle():
    """Ensembles in different fields advanced by one persistent launch of the
    field batch kernel: each member exactly as ea_sweep alone, and as the oracle."""
    made = []
    for i, (L, G, NT, C, hn, hd) in enumerate(FIELD_MIX):
        inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=900 + i, tmin=0.8, tmax=2.0, input_seed=40 + i)
        made.append((inst, hn, hd, field_pair(inst, hn, hd), field_pair(inst, hn, hd)[0]))
    batch = ea.Batch([m[3][0] for m in made])
    forms = [batch.plans(i)[batch.plan(i)]["form"] for i in range(len(made))]
    assert forms[0] == "unit-wave" and "chunked" in forms
    schedule = [(23, 1), (17, 3), (10, 10)]
    for n, k in schedule:
        batch.sweep(n, k)
    batch.sync()
    for inst, hn, hd, (gpu, sim), alone in made:
        for n, k in schedule:
            alone.sweep(n, k)
            sim.sweep(n, k, threads=8)
        tag = f"L={inst.L} h={hn}/{hd}"
        sp = gpu.read_spins().cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(sp, alone.read_spins().cpu().numpy().view(np.uint32), err_msg=tag)
        np.testing.assert_array_equal(sp, sim.spins(), err_msg=tag)
        np.testing.assert_array_equal(gpu.measure()[0].cpu().numpy(), sim.energies(), err_msg=tag)
        np.testing.assert_array_equal(gpu.magnetisations().cpu().numpy(), sim.magnetisations(), err_msg=tag)
        assert gpu.counters == alone.counters


@pytest.mark.parametrize("NT,C,h_num,h_den,swap_every", [
    (12, 2, 1, 2, 1), (7, 2, -1, 2, 1), (24, 2, 3, 2, 1), (5, 1, -5, 4, 3), (2, 2, 1, 3, 1), (31, 2, 19, 10, 2),
])
def test_field_wavefront_kernel_matches_oracle(NT, C, h_num, h_den, swap_every):
    """L = 8 fields with always-accept boundaries u >= 3 / u >= 4 for the two spin
    values (0 < |h| < 2) run the wavefront kernel by default: energies,
    magnetisations, swap masks and spins equal to the oracle's, calls continued."""
    inst = W.Instance(L=8, G=2, NT=NT, C=C, seed=700 + NT, tmin=0.8, tmax=2.0, input_seed=NT + 11)
    gpu, sim = field_pair(inst, h_num, h_den)
    assert gpu.plans()[gpu.plan]["form"] == "unit-wave"
    tag = f"wave NT={NT} h={h_num}/{h_den}"
    compare(gpu, sim, 9, swap_every, tag)
    compare(gpu, sim, 7, swap_every, tag + " (continued)")
    # a field outside that range keeps to the generic forms
    other, _ = field_pair(W.Instance(L=8, G=1, NT=4, C=2, seed=1, tmin=0.8, tmax=2.0, input_seed=2), 2, 1)
    assert all(p["form"] != "unit-wave" for p in other.plans())


def test_server_serves_field_and_field_free_requests_together():
    """Requests in fields and without share the server's rounds (a field batch and
    a field-free batch per round); each result equals the request run alone."""
    srv = ea.Server(round_ms=2)
    reqs = []
    for i, (L, G, NT, C, hn, hd) in enumerate(FIELD_MIX[:4] + [(8, 2, 10, 2, 0, 1), (12, 1, 6, 2, 0, 1)]):
        inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=950 + i, tmin=0.8, tmax=2.0, input_seed=60 + i)
        inp = W.draw_inputs(inst)
        n, k = 30 + 7 * i, 1 + i % 3
        if hn:
            mf, sw = ea.ea_build_tables_field(inp["betas"], inst.N, hn, hd)
            t = srv.submit(L, G, NT, C, inst.seed, inp["bonds"], inp["spins"], None, sw, n, k, field=(hn, hd, mf))
            alone = ea.Ensemble(L, G, NT, C, inst.seed, inp["bonds"], inp["spins"], None, sw, field=(hn, hd, mf))
        else:
            metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
            t = srv.submit(L, G, NT, C, inst.seed, inp["bonds"], inp["spins"], metro, swapt, n, k)
            alone = ea.Ensemble(L, G, NT, C, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
        alone.sweep(n, k)
        reqs.append((t, alone, hn))
    for t, alone, hn in reqs:
        out = srv.wait(t)
        np.testing.assert_array_equal(out["spins"], alone.read_spins_host())
        np.testing.assert_array_equal(out["energies"], alone.measure()[0].cpu().numpy())
        if hn:
            np.testing.assert_array_equal(out["magnetisations"], alone.magnetisations().cpu().numpy())
    srv.close()
