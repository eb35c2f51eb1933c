"""Pins of the CPU oracle against what the paper and the mathematics fix.

The paper prints no worked example, so the oracle is pinned by:
  * its Philox4x32-10 against PyTorch's independent header implementation;
  * its FP64 threshold tables against high-precision decimal exponentials;
  * closed forms (ferromagnet / staggered antiferromagnet ground state -3N);
  * exact symmetries of the dynamics (gauge covariance, global spin flip);
  * energy bookkeeping (incremental dE == recomputation by Eq. 1);
  * brute-force restatements of one sweep and one swap pass (numpy + PyTorch Philox);
  * the stationary distribution on a 2x2x2 lattice against exact enumeration.
Mutation tests at the end plant plausible mistakes in a copy of the oracle and
check that one of these pins fails.
"""
from __future__ import annotations

import decimal
import math
import os

import numpy as np
import pytest

import oracle
import refimpl
import workloads as W


def make_sim(L, G, NT, C, seed, input_seed, tmin=0.8, tmax=2.0, bonds=None, spins=None,
             metro=None, lib=None, table_betas_scale=1.0):
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=seed, tmin=tmin, tmax=tmax, input_seed=input_seed)
    inp = W.draw_inputs(inst)
    if bonds is not None:
        inp["bonds"] = bonds
    if spins is not None:
        inp["spins"] = spins
    tb = inp["betas"] * table_betas_scale
    m = oracle.metro_table(tb) if metro is None else metro
    sw = oracle.swap_table_trimmed(tb, inst.N)
    sim = oracle.OracleSim(L, G, NT, C, seed, inp["bonds"], inp["spins"], m, sw)
    if lib is not None:
        sim.lib.or_destroy(sim.h)
        sim.lib = lib
        sim.h = lib.or_create(L, G, NT, C, seed, sim.bonds, np.ascontiguousarray(inp["spins"]),
                              sim.metro, sim.swapt.ctypes.data if sim.swapt.size else None,
                              sim.swap_len, 0)
    return sim, inp


# ------------------------------------------------------------------ Philox

def test_philox_matches_pytorch_engine():
    rng = np.random.default_rng(7)
    ctrs = rng.integers(0, 2**32, size=(3000, 4), dtype=np.uint64)
    keys = rng.integers(0, 2**32, size=(3000, 2), dtype=np.uint64)
    edge = np.array([[0, 0, 0, 0], [2**32 - 1] * 4, [1, 0, 0, 0], [0, 0, 0, 1]], np.uint64)
    ctrs = np.concatenate([edge, edge, ctrs])
    keys = np.concatenate([np.zeros((4, 2), np.uint64), np.full((4, 2), 2**32 - 1, np.uint64), keys])
    ref = refimpl.torch_philox(ctrs, keys)
    ours = np.stack([oracle.philox4x32_10(c, k) for c, k in zip(ctrs, keys)])
    np.testing.assert_array_equal(ours, ref)


def test_philox_outputs_are_uniform():
    # 2^16 outputs: every byte value equally likely (loose chi-square).
    out = np.concatenate([oracle.philox4x32_10([j, 3, 5, 7], [11, 13]) for j in range(16384)])
    counts = np.bincount((out & 0xFF).astype(np.int64), minlength=256)
    exp = out.size / 256
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 400  # 255 dof; mean 255, sd ~22.6


# ------------------------------------------------------------------ tables

decimal.getcontext().prec = 60


def exact_threshold(x: float) -> int:
    """floor(exp(-x) * 2^32) computed with 60-digit decimals."""
    v = (decimal.Decimal(-x).exp() * (2 ** 32)).to_integral_value(rounding=decimal.ROUND_FLOOR)
    return min(int(v), 2**32 - 1)


@pytest.mark.parametrize("nt,tmin,tmax", [(16, 0.8, 2.0), (24, 0.9, 2.0), (32, 0.95, 2.0)])
def test_metro_table_against_decimal_exp(nt, tmin, tmax):
    betas = W.geometric_ladder(nt, tmin, tmax)
    tab = oracle.metro_table(betas)
    for t in range(nt):
        for u in range(3):
            ex = exact_threshold(float(betas[t]) * (12 - 4 * u))
            assert abs(int(tab[t, u]) - ex) <= 1
    # exactly representable case: beta * dE = 0 gives probability one.
    assert (oracle.metro_table(np.zeros(3)) == 2**32 - 1).all()
    # monotone in u (uphill size 12 > 8 > 4) and in beta
    assert (np.diff(tab.astype(np.int64), axis=1) >= 0).all()
    assert (np.diff(tab.astype(np.int64), axis=0) >= 0).all()


def test_swap_table_against_decimal_exp():
    betas = W.geometric_ladder(24, 0.9, 2.0)
    tab = oracle.swap_table(betas, 64)
    for p in (0, 7, 22):
        for k in (1, 2, 5, 17, 64):
            ex = exact_threshold(float(betas[p] - betas[p + 1]) * 4 * k)
            assert abs(int(tab[p, k - 1]) - ex) <= 1
    assert (np.diff(tab.astype(np.int64), axis=1) <= 0).all()
    assert (oracle.swap_table(np.array([1.0, 1.0]), 5) == 2**32 - 1).all()
    with pytest.raises(ValueError):
        oracle.swap_table(np.array([0.5, 1.0]), 5)


def test_swap_table_trim_keeps_every_nonzero_entry():
    betas = W.geometric_ladder(16, 0.8, 2.0)
    N = 64
    full = oracle.swap_table(betas, 3 * N // 2)
    trim = oracle.swap_table_trimmed(betas, N)
    assert trim.shape[1] <= full.shape[1]
    assert (full[:, trim.shape[1]:] == 0).all()
    np.testing.assert_array_equal(full[:, :trim.shape[1]], trim)


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("L", [2, 4, 6])
def test_ferromagnet_ground_state_energy(L):
    N = L ** 3
    G, NT, C = 1, 3, 2
    bonds = np.zeros((G, 3, N), np.uint32)               # all J = +1
    spins = np.full((G, NT, C, N), 0xFFFFFFFF, np.uint32)  # all up
    quench = np.zeros((NT, 3), np.uint32)                 # never accept uphill moves
    sim, _ = make_sim(L, G, NT, C, 9, 1, bonds=bonds, spins=spins, metro=quench)
    assert (sim.energies() == -3 * N).all()
    out = sim.sweep(20, 1, energy_log=True, swap_log=True, check=True)
    assert (out["energy_log"] == -3 * N).all()
    np.testing.assert_array_equal(sim.spins(), spins)
    # equal energies always swap (delta = 0)
    assert (out["swap_log"] == 0xFFFFFFFF).all()


def test_staggered_antiferromagnet_ground_state_energy():
    L = 4
    N = L ** 3
    i = np.arange(N)
    col = ((i % L) + (i // L) % L + i // (L * L)) & 1
    bonds = np.full((1, 3, N), 0xFFFFFFFF, np.uint32)    # all J = -1
    spins = np.where(col == 0, 0xFFFFFFFF, 0).astype(np.uint32)[None, None, None, :]
    spins = np.broadcast_to(spins, (1, 2, 1, N)).copy()
    sim, _ = make_sim(L, 1, 2, 1, 9, 1, bonds=bonds, spins=spins, metro=np.zeros((2, 3), np.uint32))
    assert (sim.energies() == -3 * N).all()
    sim.sweep(5, 0, check=True)
    assert (sim.energies() == -3 * N).all()


def test_energy_matches_numpy_eq1_and_recomputation():
    sim, inp = make_sim(6, 2, 5, 2, 21, 4)
    out = sim.sweep(30, 3, energy_log=True, check=True)
    spins = sim.spins()
    for g in range(2):
        J = refimpl.couplings(inp["bonds"][g], 6)
        for t in range(5):
            for c in range(2):
                E = refimpl.energy_pm(refimpl.unpack_lanes(spins[g, t, c], 6), J)
                np.testing.assert_array_equal(E, out["energy_log"][-1, g, t, c])
    np.testing.assert_array_equal(sim.energies(), sim.energies_recomputed())


# ------------------------------------------------------------------ brute force

def test_one_sweep_matches_brute_force():
    L, G, NT, C, seed = 4, 2, 3, 2, 0x1234_5678_9ABC
    sim, inp = make_sim(L, G, NT, C, seed, 5)
    sim.sweep(2, 0)  # move to global sweep index 2
    before = sim.spins()
    sim.sweep(1, 0)
    after = sim.spins()
    metro = oracle.metro_table(inp["betas"])
    for g in range(G):
        J = refimpl.couplings(inp["bonds"][g], L)
        for t in range(NT):
            for c in range(C):
                sig = refimpl.unpack_lanes(before[g, t, c], L)
                refimpl.brute_sweep(sig, J, metro[t], seed, L, g, t, c, 2)
                np.testing.assert_array_equal(refimpl.pack_lanes(sig), after[g, t, c])


def test_one_swap_pass_matches_brute_force():
    L, G, NT, C, seed = 4, 2, 6, 2, 77
    sim, inp = make_sim(L, G, NT, C, seed, 6, tmin=1.5, tmax=2.0)
    sim.sweep(3, 0)
    E0 = sim.energies()
    sp0 = sim.spins()
    P = sim.pass_index
    masks = sim.pt_swap()
    sp1 = sim.spins()
    swapt = oracle.swap_table_trimmed(inp["betas"], L ** 3)
    for g in range(G):
        for c in range(C):
            rn = refimpl.swap_rn(seed, g, c, P, NT)
            perm, m = refimpl.brute_swap(E0[g, :, c, :], swapt, rn)
            np.testing.assert_array_equal(masks[g, c], m)
            for t in range(NT):
                for b in range(32):
                    src = perm[t, b]
                    np.testing.assert_array_equal((sp1[g, t, c] >> b) & 1, (sp0[g, src, c] >> b) & 1)
    assert sim.pass_index == P + 1


def test_swap_decision_edge_cases():
    # Two slots whose energies differ by exactly -4k: accepted iff r < table[k-1].
    L, N = 4, 64
    bonds = np.zeros((1, 3, N), np.uint32)
    up = np.full(N, 0xFFFFFFFF, np.uint32)
    one_down = up.copy()
    one_down[0] = 0  # every lane: one flipped spin in a ferromagnet, E = -3N + 12
    spins = np.stack([up, one_down])[None, :, None, :]
    rn = refimpl.swap_rn(5, 0, 0, 0, 2)[0]
    for table_val, expect in [(0, 0), (2**32 - 1, None)]:
        tab = np.full((1, 3), table_val, np.uint32)
        sim = oracle.OracleSim(L, 1, 2, 1, 5, bonds, spins, np.zeros((2, 3), np.uint32), tab)
        # slot 0 (E=-192) vs slot 1 (E=-180): delta = -12 -> k = 3
        m = sim.pt_swap()[0, 0, 0]
        if expect == 0:
            assert m == 0
        else:
            want = sum(1 << b for b in range(32) if rn[b] < 2**32 - 1)
            assert m == want
    # thresholds at the RN itself: r < r is false, r < r + 1 is true
    for off, want_bit in [(0, 0), (1, 1)]:
        tab = np.zeros((1, 3), np.uint32)
        tab[0, 2] = min(int(rn[0]) + off, 2**32 - 1)
        sim = oracle.OracleSim(L, 1, 2, 1, 5, bonds, spins, np.zeros((2, 3), np.uint32), tab)
        assert (int(sim.pt_swap()[0, 0, 0]) & 1) == want_bit
    # k beyond the table length is rejected
    tab = np.full((1, 2), 2**32 - 1, np.uint32)
    sim = oracle.OracleSim(L, 1, 2, 1, 5, bonds, spins, np.zeros((2, 3), np.uint32), tab)
    assert sim.pt_swap()[0, 0, 0] == 0
    # higher energy in the colder slot always swaps
    spins_rev = spins[:, ::-1].copy()
    sim = oracle.OracleSim(L, 1, 2, 1, 5, bonds, spins_rev, np.zeros((2, 3), np.uint32),
                           np.zeros((1, 3), np.uint32))
    assert sim.pt_swap()[0, 0, 0] == 0xFFFFFFFF


# ------------------------------------------------------------------ symmetries

def _run(sim, n, se):
    out = sim.sweep(n, se, energy_log=True, swap_log=True)
    return out, sim.spins()


def test_gauge_covariance():
    """J'_ij = e_i J_ij e_j, S' = e S leaves every local field product invariant,
    so the same random numbers give the same decisions: the trajectory maps exactly."""
    L, G, NT, C, seed = 4, 2, 6, 2, 99
    sim, inp = make_sim(L, G, NT, C, seed, 8)
    rng = np.random.default_rng(3)
    eps = rng.integers(0, 2**32, size=(G, L ** 3), dtype=np.uint64).astype(np.uint32)
    e3 = eps.reshape(G, L, L, L)
    bonds2 = np.empty_like(inp["bonds"])
    for d, ax in ((0, 3), (1, 2), (2, 1)):
        nb = np.roll(e3, -1, axis=ax).reshape(G, -1)
        bonds2[:, d] = inp["bonds"][:, d] ^ eps ^ nb
    spins2 = inp["spins"] ^ eps[:, None, None, :]
    sim2, _ = make_sim(L, G, NT, C, seed, 8, bonds=bonds2, spins=spins2)
    o1, s1 = _run(sim, 40, 2)
    o2, s2 = _run(sim2, 40, 2)
    np.testing.assert_array_equal(o1["energy_log"], o2["energy_log"])
    np.testing.assert_array_equal(o1["swap_log"], o2["swap_log"])
    np.testing.assert_array_equal(s1 ^ eps[:, None, None, :], s2)


def test_global_spin_flip():
    L, G, NT, C, seed = 4, 1, 5, 2, 5
    sim, inp = make_sim(L, G, NT, C, seed, 9)
    sim2, _ = make_sim(L, G, NT, C, seed, 9, spins=~inp["spins"])
    o1, s1 = _run(sim, 30, 1)
    o2, s2 = _run(sim2, 30, 1)
    np.testing.assert_array_equal(o1["energy_log"], o2["energy_log"])
    np.testing.assert_array_equal(o1["swap_log"], o2["swap_log"])
    np.testing.assert_array_equal(~s1, s2)


def test_chunking_and_thread_invariance():
    sim_a, _ = make_sim(4, 3, 4, 2, 12, 10)
    sim_b, _ = make_sim(4, 3, 4, 2, 12, 10)
    oa = sim_a.sweep(40, 4, energy_log=True, swap_log=True, threads=3)
    ob1 = sim_b.sweep(17, 4, energy_log=True, swap_log=True)
    ob2 = sim_b.sweep(23, 4, energy_log=True, swap_log=True)
    np.testing.assert_array_equal(oa["energy_log"],
                                  np.concatenate([ob1["energy_log"], ob2["energy_log"]]))
    np.testing.assert_array_equal(oa["swap_log"], np.concatenate([ob1["swap_log"], ob2["swap_log"]]))
    np.testing.assert_array_equal(sim_a.spins(), sim_b.spins())
    assert sim_a.sweep_index == sim_b.sweep_index == 40
    assert sim_a.pass_index == sim_b.pass_index == 10


def test_overlap_histogram_counts():
    L, G, NT = 4, 2, 3
    sim, _ = make_sim(L, G, NT, 2, 31, 11)
    qh = np.zeros((NT, L ** 3 + 1), np.uint64)
    es = np.zeros(NT, np.int64)
    sim.sweep(10, 1, qhist=qh, esum=es, measure_from=4, measure_every=2)
    # sweeps 4, 6, 8 (global indices) are measured: 3 x G x 32 entries per slot
    assert (qh.sum(axis=1) == 3 * G * 32).all()
    ov = sim.overlaps()
    qh2 = np.zeros_like(qh)
    sim.sweep(1, 1, qhist=qh2, measure_from=10, measure_every=1)
    ov = sim.overlaps()
    for t in range(NT):
        np.testing.assert_array_equal(qh2[t], np.bincount(ov[:, t].ravel(), minlength=L ** 3 + 1))


# ------------------------------------------------------------------ enumeration

def _exact_distribution(J, beta):
    """Boltzmann weights of all 256 states of a 2x2x2 lattice for each lane."""
    L = 2
    states = np.arange(256)
    bits = (states[:, None] >> np.arange(8)) & 1
    sig = (bits * 2 - 1).astype(np.int8).reshape(256, 1, L, L, L)
    sig = np.broadcast_to(sig, (256, 32, L, L, L))
    E = refimpl.energy_pm(sig, J)                     # [256][32]
    w = np.exp(-beta * (E - E.min(axis=0)))
    return w / w.sum(axis=0), E


def _state_index(words, b):
    return sum((((words[i] >> b) & 1).astype(np.int64) << i) for i in range(8))


def doubled_bond_cube(G, seed):
    """Bond words for L = 2 in which both bonds of every neighbour pair are equal.

    With L = 2 the two bonds along +d and -d join the same pair of sites.  When
    they have opposite signs the pair is decoupled, and a site whose three pairs
    all cancel has zero local field whatever its neighbours do: it flips
    deterministically every sweep (dE = 0 is always accepted), and two such
    sites keep their relative orientation forever, so the chain is not ergodic
    and cannot be compared with the Boltzmann distribution.  Equal bonds give a
    frustrated cube with couplings +-2 on all 12 edges and no zero fields."""
    rng = np.random.default_rng(seed)
    b = rng.integers(0, 2**32, size=(G, 3, 2, 2, 2), dtype=np.uint64).astype(np.uint32)
    b[:, 0, :, :, 1] = b[:, 0, :, :, 0]
    b[:, 1, :, 1, :] = b[:, 1, :, 0, :]
    b[:, 2, 1, :, :] = b[:, 2, 0, :, :]
    return b.reshape(G, 3, 8)


def enumeration_statistic(lib=None, n_samples=6000, thin=3, beta_scale=1.0):
    """Max over (lane, copy, slot) of chi-square per degree of freedom between the
    sampled 2x2x2 state histogram and the exact Boltzmann distribution.

    Histograms are folded over the global spin flip (an exact symmetry at h = 0)
    so the slow tunnelling between flipped ground states does not dominate.
    ``beta_scale`` builds the threshold tables for scaled temperatures: the chain
    then samples the wrong distribution and the statistic must blow up."""
    L, G, NT, C, seed = 2, 2, 4, 2, 2024
    bonds = doubled_bond_cube(G, 5)
    sim, inp = make_sim(L, G, NT, C, seed, 12, tmin=0.7, tmax=3.0, bonds=bonds, lib=lib,
                        table_betas_scale=beta_scale)
    betas = inp["betas"]
    sim.sweep(200, 1)
    idx = np.zeros((n_samples, G, NT, C, 32), np.int64)
    lanes = np.arange(32, dtype=np.uint32)
    for n in range(n_samples):
        sim.sweep(thin, 1)
        sp = sim.spins()                                   # [G][NT][C][8]
        bits = (sp[..., None] >> lanes) & 1                # [G][NT][C][8][32]
        idx[n] = (bits.astype(np.int64) << np.arange(8)[:, None]).sum(axis=3)
    worst = 0.0
    for g in range(G):
        J = refimpl.couplings(inp["bonds"][g], L)
        for t in range(NT):
            p, _ = _exact_distribution(J, betas[t])
            for c in range(C):
                for b in range(32):
                    obs = np.bincount(idx[:, g, t, c, b], minlength=256).astype(np.float64)
                    exp = p[:, b] * n_samples
                    # state s and its global flip 255 - s have equal weight
                    obs = (obs + obs[::-1])[:128]
                    exp = (exp + exp[::-1])[:128]
                    big = exp >= 5
                    e_bins = np.append(exp[big], exp[~big].sum())
                    o_bins = np.append(obs[big], obs[~big].sum())
                    keep = e_bins > 0
                    chi2 = ((o_bins[keep] - e_bins[keep]) ** 2 / e_bins[keep]).sum()
                    dof = max(int(keep.sum()) - 1, 1)
                    worst = max(worst, chi2 / dof)
    return worst


ENUM_LIMIT = 8.0


@pytest.mark.slow
def test_stationary_distribution_2x2x2_enumeration():
    stat = enumeration_statistic()
    # Independent samples give chi2/dof ~ 1; the maximum over 512 cells with mild
    # autocorrelation stays below ~5.  A chain sampling the wrong distribution
    # gives far more (see the next test).
    assert stat < ENUM_LIMIT, stat


@pytest.mark.slow
@pytest.mark.parametrize("scale", [1.15, 0.85])
def test_enumeration_detects_wrong_temperatures(scale):
    assert enumeration_statistic(n_samples=3000, beta_scale=scale) > ENUM_LIMIT


# ------------------------------------------------------------------ mutations

MUTANTS = {
    "dE_sign": ("int dE = 2 * sp[i] * local_field(m, sp, g, b, i);",
                "int dE = -2 * sp[i] * local_field(m, sp, g, b, i);"),
    "threshold_index": ("m->metro[t * 3 + (12 - dE) / 4]", "m->metro[t * 3 + 2 - (12 - dE) / 4]"),
    "swap_sign": ("int64_t delta = m->h_num == 0 ? e[l[p]] - e[l[p + 1]]",
                  "int64_t delta = m->h_num == 0 ? e[l[p + 1]] - e[l[p]]"),
    "minus_bond_J": ("h += jb(m, g, b, d)[im] * s[im];", "h += jb(m, g, b, d)[i] * s[im];"),
    "colour_order": ("for (int colour = 0; colour < 2; ++colour) {",
                     "for (int colour = 1; colour >= 0; --colour) {"),
    "energy_update": ("en(m, g, c, b)[rr] += dE;", "en(m, g, c, b)[rr] -= dE;"),
    "counter_layout": ("(uint32_t)s, (uint32_t)(m->group_base + g), (int)(k & 3u));",
                       "(uint32_t)(m->group_base + g), (uint32_t)s, (int)(k & 3u));"),
    "z_step": ("if (d == 2) z += step;", "if (d == 2) z += 1;"),
}


def _build_mutant(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "ea_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    path = tmp_path / f"mut_{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"mut_{name}.so"
    oracle.build(str(path), str(so))
    return oracle.load(str(so))


def _fast_pins(lib):
    """The cheap pins; returns the list of those that fail."""
    failed = []
    # closed form + quench
    L, N = 4, 64
    bonds = np.zeros((1, 3, N), np.uint32)
    spins = np.full((1, 2, 1, N), 0xFFFFFFFF, np.uint32)
    try:
        sim, _ = make_sim(L, 1, 2, 1, 9, 1, bonds=bonds, spins=spins,
                          metro=np.zeros((2, 3), np.uint32), lib=lib)
        sim.sweep(3, 1, check=True)
        if not (sim.energies() == -3 * N).all():
            failed.append("ferro")
    except AssertionError:
        failed.append("ferro")
    # incremental == recomputed
    try:
        sim, _ = make_sim(4, 1, 3, 1, 3, 2, lib=lib)
        sim.sweep(5, 1, check=True)
    except AssertionError:
        failed.append("recompute")
    # brute-force sweep
    Lb, seed = 4, 0x1234_5678_9ABC
    sim, inp = make_sim(Lb, 2, 2, 2, seed, 5, lib=lib)
    sim.sweep(2, 0)
    before = sim.spins()
    sim.sweep(1, 0)
    after = sim.spins()
    metro = oracle.metro_table(inp["betas"])
    J = refimpl.couplings(inp["bonds"][1], Lb)
    sig = refimpl.unpack_lanes(before[1, 1, 1], Lb)
    refimpl.brute_sweep(sig, J, metro[1], seed, Lb, 1, 1, 1, 2)
    if not np.array_equal(refimpl.pack_lanes(sig), after[1, 1, 1]):
        failed.append("brute_sweep")
    # brute-force swap
    sim, inp = make_sim(4, 1, 6, 1, 77, 6, tmin=1.5, tmax=2.0, lib=lib)
    E0 = sim.energies()
    masks = sim.pt_swap()
    sw = oracle.swap_table_trimmed(inp["betas"], 64)
    _, m = refimpl.brute_swap(E0[0, :, 0, :], sw, refimpl.swap_rn(77, 0, 0, 0, 6))
    if not np.array_equal(masks[0, 0], m):
        failed.append("brute_swap")
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_are_caught(name, tmp_path):
    lib = _build_mutant(name, tmp_path)
    failed = _fast_pins(lib)
    if not failed:
        # The stationary-distribution pin covers what the cheap pins cannot.
        failed = ["enumeration"] if enumeration_statistic(lib, n_samples=2000) > ENUM_LIMIT else []
    assert failed, f"mutant {name} passed every pin"


def test_unmutated_oracle_passes_fast_pins():
    assert _fast_pins(oracle.load()) == []


def test_group_subset_reproduces_full_ensemble():
    """Groups never interact, and counters use global group indices: a run on
    one group (with its global index) equals that group inside the full run."""
    sim, inp = make_sim(4, 4, 3, 2, 17, 13)
    full = sim.sweep(12, 2, energy_log=True, swap_log=True)
    fs = sim.spins()
    for g in (0, 2, 3):
        sub = oracle.OracleSim(4, 1, 3, 2, 17, inp["bonds"][g:g + 1], inp["spins"][g:g + 1],
                               sim.metro, sim.swapt, group_base=g)
        out = sub.sweep(12, 2, energy_log=True, swap_log=True)
        np.testing.assert_array_equal(out["energy_log"][:, 0], full["energy_log"][:, g])
        np.testing.assert_array_equal(out["swap_log"][:, 0], full["swap_log"][:, g])
        np.testing.assert_array_equal(sub.spins()[0], fs[g])


def test_overlap_counts_match_numpy_definition():
    """n_diff = number of sites where the two copies at a slot differ (q = 1 - 2 n_diff / N)."""
    L, G, NT = 6, 2, 4
    sim, _ = make_sim(L, G, NT, 2, 41, 14)
    sim.sweep(9, 1)
    sp = sim.spins()
    ov = sim.overlaps()
    for g in range(G):
        for t in range(NT):
            a = refimpl.unpack_lanes(sp[g, t, 0], L)
            b = refimpl.unpack_lanes(sp[g, t, 1], L)
            want = (a != b).reshape(32, -1).sum(axis=1)
            np.testing.assert_array_equal(ov[g, t], want)
