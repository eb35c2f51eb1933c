"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit for bit.

Every Metropolis and swap decision is an integer compare against tables both
sides receive as inputs, so the whole trajectory is a deterministic function
of the inputs: spins, energies, swap masks and q histograms must be equal
(tolerance 0).  Inputs are seeded synthetic ensembles of the paper's shapes.
"""
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


def u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


def i32(t):
    return t.detach().cpu().numpy()


def pair(inst: W.Instance, groups=None, inputs=None):
    """(GPU ensemble, oracle on `groups` (default all), inputs, tables)."""
    inp = W.draw_inputs(inst) if inputs is None else inputs
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    gpu = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], metro,
                      swapt)
    sims = []
    for g in (range(inst.G) if groups is None else groups):
        sims.append((g, oracle.OracleSim(inst.L, 1, inst.NT, inst.C, inst.seed,
                                         inp["bonds"][g:g + 1], inp["spins"][g:g + 1], metro, swapt,
                                         group_base=g)))
    return gpu, sims, inp


def compare(gpu, sims, n, swap_every, threads=8):
    out = gpu.sweep(n, swap_every, energy_log=True, swap_log=True)
    el, sl = i32(out["energy_log"]), u32(out["swap_log"])
    sp = u32(gpu.read_spins())
    e_fin = i32(gpu.measure()[0])
    for g, sim in sims:
        o = sim.sweep(n, swap_every, energy_log=True, swap_log=True, threads=threads)
        np.testing.assert_array_equal(el[:, g], o["energy_log"][:, 0], err_msg=f"energy log g={g}")
        np.testing.assert_array_equal(sl[:, g], o["swap_log"][:, 0], err_msg=f"swap log g={g}")
        np.testing.assert_array_equal(sp[g], sim.spins()[0], err_msg=f"spins g={g}")
        np.testing.assert_array_equal(e_fin[g], sim.energies()[0], err_msg=f"energies g={g}")


def test_small_workload_full_length():
    """L=4, 32 realizations, 16 temperatures x 2 copies, 2000 sweeps, swap every sweep."""
    inst = W.SMALL
    gpu, sims, _ = pair(inst)
    compare(gpu, sims, W.SMALL_SWEEPS, W.SMALL_SWAP_EVERY)
    s, p = gpu.counters
    assert s == 2000 and p == 2000


@pytest.mark.parametrize("L,G,NT,C,swap_every", [
    (4, 3, 5, 1, 1), (6, 2, 7, 2, 3), (8, 3, 24, 2, 1), (10, 2, 9, 2, 2), (12, 2, 6, 2, 1),
    (14, 1, 4, 2, 5), (16, 2, 5, 2, 1), (20, 1, 3, 1, 2), (24, 1, 2, 2, 1),
])
def test_sizes_unit_form(L, G, NT, C, swap_every):
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=1000 + L, tmin=0.9, tmax=2.0, input_seed=L)
    gpu, sims, _ = pair(inst)
    compare(gpu, sims, 24, swap_every)


@pytest.mark.parametrize("L,G,NT,C,swap_every,n", [
    (16, 2, 32, 2, 10, 25), (12, 1, 32, 2, 3, 10), (32, 1, 3, 2, 2, 5),
])
def test_sizes_chunked_form(L, G, NT, C, swap_every, n):
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=2000 + L, tmin=0.95, tmax=2.0, input_seed=L + 50)
    gpu, sims, _ = pair(inst)
    compare(gpu, sims, n, swap_every)


def test_edge_cases_single_temperature_and_no_swaps():
    for (NT, C, se) in [(1, 1, 1), (1, 2, 0), (2, 1, 0), (3, 2, 7)]:
        inst = W.Instance(L=4, G=2, NT=NT, C=C, seed=7, tmin=1.0, tmax=1.5, input_seed=NT * 10 + C)
        gpu, sims, _ = pair(inst)
        compare(gpu, sims, 15, se)


def test_zero_sweeps_is_a_no_op():
    inst = W.Instance(L=8, G=1, NT=3, C=2, seed=3, tmin=1.0, tmax=2.0, input_seed=3)
    gpu, sims, inp = pair(inst)
    gpu.sweep(0, 1)
    np.testing.assert_array_equal(u32(gpu.read_spins()), inp["spins"])
    assert gpu.counters == (0, 0)


def test_measurement_qhist_and_energy_sums():
    """L=8 ensemble with per-sweep measurement in the second half (overlap q histogram)."""
    inst = W.Instance(L=8, G=6, NT=24, C=2, seed=2, tmin=0.9, tmax=2.0, input_seed=102)
    gpu, sims, _ = pair(inst)
    n = 60
    qh = torch.zeros((inst.NT, inst.N + 1), dtype=torch.int64, device="cuda")
    es = torch.zeros(inst.NT, dtype=torch.int64, device="cuda")
    gpu.sweep(n, 1, qhist=qh, esum=es, measure_from=n // 2, measure_every=1)
    qh_o = np.zeros((inst.NT, inst.N + 1), np.uint64)
    es_o = np.zeros(inst.NT, np.int64)
    for g, sim in sims:
        sim.sweep(n, 1, qhist=qh_o, esum=es_o, measure_from=n // 2, measure_every=1, threads=8)
    np.testing.assert_array_equal(qh.cpu().numpy().view(np.uint64), qh_o)
    np.testing.assert_array_equal(es.cpu().numpy(), es_o)
    assert int(qh_o.sum()) == (n // 2) * inst.G * 32 * inst.NT


def test_measurement_chunked_form():
    inst = W.Instance(L=16, G=1, NT=32, C=2, seed=5, tmin=0.95, tmax=2.0, input_seed=9)
    gpu, sims, _ = pair(inst)
    qh = torch.zeros((inst.NT, inst.N + 1), dtype=torch.int64, device="cuda")
    es = torch.zeros(inst.NT, dtype=torch.int64, device="cuda")
    gpu.sweep(12, 5, qhist=qh, esum=es, measure_from=3, measure_every=4)
    qh_o = np.zeros((inst.NT, inst.N + 1), np.uint64)
    es_o = np.zeros(inst.NT, np.int64)
    sims[0][1].sweep(12, 5, qhist=qh_o, esum=es_o, measure_from=3, measure_every=4, threads=8)
    np.testing.assert_array_equal(qh.cpu().numpy().view(np.uint64), qh_o)
    np.testing.assert_array_equal(es.cpu().numpy(), es_o)


def test_pt_swap_measure_and_overlaps():
    inst = W.Instance(L=6, G=2, NT=8, C=2, seed=11, tmin=1.2, tmax=2.0, input_seed=4)
    gpu, sims, _ = pair(inst)
    gpu.sweep(5, 0)
    for _, sim in sims:
        sim.sweep(5, 0)
    masks = u32(gpu.pt_swap())
    e, nd = gpu.measure(energies=True, ndiff=True)
    for g, sim in sims:
        np.testing.assert_array_equal(masks[g], sim.pt_swap()[0])
        np.testing.assert_array_equal(i32(e)[g], sim.energies()[0])
        np.testing.assert_array_equal(u32(nd)[g], sim.overlaps()[0])
    assert gpu.counters == (5, 1)


def test_chunking_checkpoint_and_host_path():
    """sweep(2n) == sweep(n) + sweep(n); write_spins restores a checkpoint exactly;
    the host-buffer entry point gives the same final state."""
    inst = W.Instance(L=8, G=2, NT=6, C=2, seed=21, tmin=1.0, tmax=2.0, input_seed=5)
    a, _, inp = pair(inst, groups=[])
    b, _, _ = pair(inst, groups=[])
    a.sweep(40, 3)
    b.sweep(17, 3)
    ck = b.read_spins().clone()
    s, p = b.counters
    b.sweep(23, 3)
    np.testing.assert_array_equal(u32(a.read_spins()), u32(b.read_spins()))
    b.write_spins(ck, s, p)
    b.sweep(23, 3)
    np.testing.assert_array_equal(u32(a.read_spins()), u32(b.read_spins()))
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    h = ea.ea_run(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"], metro,
                  swapt, 40, 3)
    np.testing.assert_array_equal(h["spins"], u32(a.read_spins()))
    np.testing.assert_array_equal(h["energies"], i32(a.measure()[0]))


def test_fused_energies_equal_recomputation():
    inst = W.Instance(L=8, G=4, NT=10, C=2, seed=31, tmin=0.9, tmax=2.0, input_seed=6)
    gpu, _, _ = pair(inst, groups=[])
    out = gpu.sweep(9, 4, energy_log=True)
    fused = i32(out["energy_log"])[-1]
    recomputed = i32(gpu.measure()[0])
    np.testing.assert_array_equal(fused, recomputed)


# ---------------------------------------------------------------- full-size sampled parity

@pytest.mark.parametrize("name,inst,n,swap_every,groups", [
    ("L8 2048 realizations x 24 temps", W.SCALE, 30, 1, [0, 37, 63]),
    ("L16 8192 realizations x 32 temps", W.LARGE16, 20, 10, [0, 200]),
    ("L32 1024 realizations x 32 temps", W.LARGE32, 10, 10, [31]),
])
def test_full_size_sampled_groups(name, inst, n, swap_every, groups):
    """The full ensembles in the launch configuration the benchmark times, checked
    on sampled word-groups (groups are independent, counters use global indices)."""
    gpu, sims, _ = pair(inst, groups=groups)
    compare(gpu, sims, n, swap_every, threads=16)


@pytest.mark.parametrize("L,G,NT,C", [(8, 3, 24, 2), (16, 2, 6, 2), (4, 2, 16, 2), (12, 1, 28, 2),
                                      (16, 1, 32, 2), (8, 2, 40, 1)])
def test_every_plan_is_bit_identical(L, G, NT, C):
    """All kernel plans (unit, specialised unit, chunked; several CTA shapes)
    give the oracle's trajectory, including swap logs and the q histogram."""
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=77 + L, tmin=0.9, tmax=2.0, input_seed=NT + L)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    probe = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                        metro, swapt)
    plans = probe.plans()
    assert len(plans) >= 2
    sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                           metro, swapt)
    n, se = 12, 2
    qh_o = np.zeros((NT, inst.N + 1), np.uint64) if C == 2 else None
    ref = sim.sweep(n, se, energy_log=True, swap_log=True, qhist=qh_o, measure_from=4,
                    measure_every=3 if C == 2 else 0)
    ref_spins = sim.spins()
    for i, p in enumerate(plans):
        gpu = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                          metro, swapt)
        gpu.select_plan(i)
        qh = torch.zeros((NT, inst.N + 1), dtype=torch.int64, device="cuda") if C == 2 else None
        out = gpu.sweep(n, se, energy_log=True, swap_log=True, qhist=qh, measure_from=4,
                        measure_every=3 if C == 2 else 0)
        msg = f"plan {i}: {p}"
        np.testing.assert_array_equal(i32(out["energy_log"]), ref["energy_log"], err_msg=msg)
        np.testing.assert_array_equal(u32(out["swap_log"]), ref["swap_log"], err_msg=msg)
        np.testing.assert_array_equal(u32(gpu.read_spins()), ref_spins, err_msg=msg)
        if C == 2:
            np.testing.assert_array_equal(qh.cpu().numpy().view(np.uint64), qh_o, err_msg=msg)


def test_autotune_keeps_state_and_picks_a_plan():
    inst = W.Instance(L=8, G=4, NT=24, C=2, seed=5, tmin=0.9, tmax=2.0, input_seed=55)
    gpu, sims, _ = pair(inst, groups=[0, 3])
    gpu.sweep(3, 1)
    for _, sim in sims:
        sim.sweep(3, 1)
    ms = gpu.autotune(probe_sweeps=20, swap_every=1)
    assert len(ms) == len(gpu.plans()) and all(m > 0 for m in ms)
    assert gpu.plan == int(np.argmin(ms))
    assert gpu.counters == (3, 3)
    compare(gpu, sims, 10, 1)


def _plan_index(gpu, form):
    for i, p in enumerate(gpu.plans()):
        if p["form"] == form:
            return i
    return None


@pytest.mark.parametrize("NT,C,swap_every", [(1, 2, 1), (2, 2, 1), (3, 1, 1), (5, 2, 2), (6, 2, 1),
                                             (7, 2, 3), (24, 2, 1), (24, 1, 0), (31, 2, 1), (32, 2, 5)])
def test_wavefront_plan_edge_cases(NT, C, swap_every):
    """The L = 8 wavefront unit kernel (one warp per two slots, the pass run
    pair by pair across warps): odd and even slot counts, one and two copies,
    with and without passes, calls split at arbitrary sweeps; every log equal
    to the oracle's."""
    inst = W.Instance(L=8, G=2, NT=NT, C=C, seed=900 + NT, tmin=0.9, tmax=2.0, input_seed=NT * 7 + C)
    gpu, sims, _ = pair(inst)
    i = _plan_index(gpu, "unit-wave")
    assert i is not None and gpu.plan == i         # the default plan at L = 8, NT <= 32
    for n in (7, 1, 12):
        compare(gpu, sims, n, swap_every)


def test_wavefront_plan_measured_calls_continue_the_chain():
    """Calls that measure (q histogram, energy sums) run the measuring
    instantiation of the wavefront kernel (copy pairs as 2-CTA clusters); before
    and after them the plain one continues the same chain."""
    inst = W.Instance(L=8, G=3, NT=12, C=2, seed=4, tmin=0.9, tmax=2.0, input_seed=77)
    gpu, sims, _ = pair(inst)
    compare(gpu, sims, 5, 1)
    qh = torch.zeros((inst.NT, inst.N + 1), dtype=torch.int64, device="cuda")
    es = torch.zeros(inst.NT, dtype=torch.int64, device="cuda")
    gpu.sweep(10, 1, qhist=qh, esum=es, measure_from=gpu.sweep_index + 3, measure_every=2)
    qh_o = np.zeros((inst.NT, inst.N + 1), np.uint64)
    es_o = np.zeros(inst.NT, np.int64)
    for _, sim in sims:
        sim.sweep(10, 1, qhist=qh_o, esum=es_o, measure_from=sim.sweep_index + 3, measure_every=2)
    np.testing.assert_array_equal(qh.cpu().numpy().view(np.uint64), qh_o)
    np.testing.assert_array_equal(es.cpu().numpy(), es_o)
    compare(gpu, sims, 6, 1)


@pytest.mark.parametrize("G,NT,C,n,swap_every,mfrom,mevery,want_q,want_e", [
    (2, 13, 2, 17, 2, 3, 3, True, True),      # odd NT: the last warp holds one slot
    (3, 24, 2, 12, 1, 0, 1, True, False),     # histogram only, from the first sweep
    (2, 24, 2, 10, 1, 4, 2, False, True),     # energy sums only (no cluster)
    (2, 9, 1, 14, 3, 5, 1, False, True),      # one copy: energy sums
    (1, 32, 2, 8, 1, 2, 1, True, True),       # 32 slots, 512 threads
    (2, 2, 2, 9, 1, 1, 4, True, True),        # one pair
])
def test_wavefront_measurement_matches_oracle(G, NT, C, n, swap_every, mfrom, mevery, want_q, want_e):
    """The measuring wavefront kernel: per-slot energy sums and overlap histograms
    of the measured sweeps, bit-exact against the oracle, and the chain that
    continues after the call."""
    inst = W.Instance(L=8, G=G, NT=NT, C=C, seed=31 + NT, tmin=0.9, tmax=2.0, input_seed=500 + NT)
    gpu, sims, _ = pair(inst)
    assert gpu.plans()[gpu.plan]["form"] == "unit-wave"
    qh = torch.zeros((NT, inst.N + 1), dtype=torch.int64, device="cuda") if want_q else None
    es = torch.zeros(NT, dtype=torch.int64, device="cuda") if want_e else None
    gpu.sweep(n, swap_every, qhist=qh, esum=es, measure_from=mfrom, measure_every=mevery)
    qh_o = np.zeros((NT, inst.N + 1), np.uint64) if want_q else None
    es_o = np.zeros(NT, np.int64) if want_e else None
    for _, sim in sims:
        sim.sweep(n, swap_every, qhist=qh_o, esum=es_o, measure_from=mfrom, measure_every=mevery, threads=8)
    if want_q:
        np.testing.assert_array_equal(qh.cpu().numpy().view(np.uint64), qh_o)
        assert int(qh_o.sum()) > 0
    if want_e:
        np.testing.assert_array_equal(es.cpu().numpy(), es_o)
    compare(gpu, sims, 5, swap_every)


@pytest.mark.parametrize("tmin,tmax,NT", [(1.5, 1.5, 6), (0.2, 50.0, 5), (0.9, 0.95, 24), (0.3, 3.0, 2)])
def test_wavefront_plan_degenerate_ladders(tmin, tmax, NT):
    """Acceptance counts at the ends of the table range: equal temperatures (every
    entry 2^32 - 1, the count is the whole row), widely spaced ones (rows of zeros
    or a few entries), a dense ladder, and a single pair."""
    inst = W.Instance(L=8, G=2, NT=NT, C=2, seed=int(tmax * 10) + NT, tmin=tmin, tmax=tmax,
                      input_seed=NT + 3)
    gpu, sims, _ = pair(inst)
    assert gpu.plans()[gpu.plan]["form"] == "unit-wave"
    compare(gpu, sims, 20, 1)
