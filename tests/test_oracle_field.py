"""Pins of the oracle's external field (Eq. 1 with h != 0): tables against
high-precision decimals, the field-free limit, a numpy restatement of one
sweep and one swap pass, ferromagnet closed forms, and the Boltzmann
distribution of a 2x2x2 lattice in a field."""
from __future__ import annotations

import decimal

import numpy as np
import pytest

import oracle
import refimpl
import workloads as W

ALWAYS = 1 << 32


def dec_threshold(beta, dE):
    decimal.getcontext().prec = 60
    v = (decimal.Decimal(-beta) * decimal.Decimal(dE)).exp() * (1 << 32)
    return min(int(v), (1 << 32) - 1)


def inputs(L, G, NT, C, seed, input_seed, tmin=0.8, tmax=2.0):
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=seed, tmin=tmin, tmax=tmax, input_seed=input_seed)
    return inst, W.draw_inputs(inst)


def field_sim(inst, inp, h_num, h_den, bonds=None, spins=None, betas=None):
    b = inp["betas"] if betas is None else betas
    mf = oracle.metro_table_field(b, h_num, h_den)
    sw = oracle.swap_table_field_trimmed(b, inst.N, h_num, h_den)
    metro = oracle.metro_table(b)
    sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed,
                           inp["bonds"] if bonds is None else bonds,
                           inp["spins"] if spins is None else spins, metro, sw,
                           field=(h_num, h_den, mf))
    return sim, mf, sw


def test_field_tables_against_decimals():
    betas = np.array([1.3, 0.9, 0.55])
    for h_num, h_den in ((1, 2), (-3, 4), (7, 1)):
        mf = oracle.metro_table_field(betas, h_num, h_den)
        h = h_num / h_den
        for t, beta in enumerate(betas):
            for sp in (0, 1):
                S = 1 if sp else -1
                for u in range(7):
                    dEt = h_den * (12 - 4 * u) + 2 * h_num * S
                    want = ALWAYS if dEt <= 0 else dec_threshold(beta, 12 - 4 * u + 2 * h * S)
                    assert int(mf[t, sp, u]) == want, (h_num, h_den, t, sp, u)
        step = oracle.field_step(h_num, h_den)
        assert step == np.gcd(4 * h_den, 2 * abs(h_num))
        sw = oracle.swap_table_field_trimmed(betas, 8, h_num, h_den)
        for p in range(2):
            db = betas[p] - betas[p + 1]
            for k in (1, 2, 5):
                if k <= sw.shape[1]:
                    assert int(sw[p, k - 1]) == dec_threshold(db, k * step / h_den)


def test_zero_field_tables_reduce_to_the_field_free_ones():
    betas = W.geometric_ladder(6, 0.8, 2.0)
    mf = oracle.metro_table_field(betas, 0, 1)
    m = oracle.metro_table(betas)
    for sp in (0, 1):
        np.testing.assert_array_equal(mf[:, sp, :3], m.astype(np.uint64))
        assert np.all(mf[:, sp, 3:] == ALWAYS)
    np.testing.assert_array_equal(oracle.swap_table_field_trimmed(betas, 64, 0, 1),
                                  oracle.swap_table_trimmed(betas, 64))


@pytest.mark.parametrize("h_den", [1, 3])
def test_zero_field_trajectory_equals_the_field_free_oracle(h_den):
    """h = 0 / h_den is no field whatever h_den: Et = h_den E, whose differences
    are multiples of 4 h_den, so the swap index is still (E_{p+1} - E_p) / 4."""
    inst, inp = inputs(4, 2, 6, 2, 41, 42)
    sim_f, _, _ = field_sim(inst, inp, 0, h_den)
    sim_0 = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                             oracle.metro_table(inp["betas"]),
                             oracle.swap_table_trimmed(inp["betas"], inst.N))
    sim_f.sweep(30, 1)
    sim_0.sweep(30, 1)
    np.testing.assert_array_equal(sim_f.spins(), sim_0.spins())
    np.testing.assert_array_equal(sim_f.energies(), sim_0.energies())


@pytest.mark.parametrize("h_num,h_den", [(1, 2), (-5, 3), (3, 1)])
def test_one_sweep_matches_numpy_with_field(h_num, h_den):
    """NT = 1 and no swaps: one checkerboard sweep restated on +-1 arrays."""
    L, g = 4, 1
    inst, inp = inputs(L, 2, 1, 1, 57, 58, tmin=1.1, tmax=1.1)
    sim, mf, _ = field_sim(inst, inp, h_num, h_den)
    J = refimpl.couplings(inp["bonds"][g], L)
    sigma = refimpl.unpack_lanes(inp["spins"][g, 0, 0], L).astype(np.int8).copy()   # [32][z][y][x]
    col = refimpl.colour_mask(L)
    for colour in (0, 1):
        r = refimpl.metropolis_rn(inst.seed, L, g, 0, 0, 0, colour)
        h = refimpl.local_field_pm(sigma, J)
        dE = 2 * sigma.astype(np.int64) * h
        S = sigma.astype(np.int64)
        dEt = h_den * dE + 2 * h_num * S
        u = (12 - dE) // 4
        thr = mf[0][(S > 0).astype(np.int64), u]
        accept = (dEt <= 0) | (r[None].astype(np.uint64) < thr)
        flip = accept & (col[None] == colour)
        sigma[flip] = -sigma[flip]
    sim.sweep(1, 0)
    got = refimpl.unpack_lanes(sim.spins()[g, 0, 0], L)
    np.testing.assert_array_equal(got, sigma)
    np.testing.assert_array_equal(sim.magnetisations()[g, 0, 0], sigma.reshape(32, -1).sum(axis=1))


def test_ferromagnet_closed_forms():
    """J = +1 everywhere, T -> 0 (tables built for beta = 60): all up stays up in
    h > 0; all down is metastable for h < 6 (every flip costs 12 - 2h); for h = 7
    every flip lowers the energy and one sweep turns all spins up."""
    L = 4
    N = L ** 3
    inst, inp = inputs(L, 1, 2, 1, 3, 4)
    bonds = np.zeros((1, 3, N), np.uint32)
    betas = np.array([60.0, 50.0])
    up = np.full((1, 2, 1, N), 0xFFFFFFFF, np.uint32)
    down = np.zeros((1, 2, 1, N), np.uint32)
    for spins, h_num, h_den, want_up in ((up, 1, 2, True), (down, 1, 2, False), (down, 7, 1, True)):
        sim, _, _ = field_sim(inst, inp, h_num, h_den, bonds=bonds, spins=spins, betas=betas)
        sim.sweep(3, 0)
        sp = sim.spins()
        assert np.all(sp == (0xFFFFFFFF if want_up else 0)), (h_num, h_den)
        assert np.all(sim.energies() == -3 * N)
        assert np.all(sim.magnetisations() == (N if want_up else -N))


def test_swap_pass_matches_numpy_with_field():
    """One pass on the oracle's own state, restated with Et = h_den E - h_num M."""
    inst, inp = inputs(4, 1, 6, 1, 71, 72, tmin=0.9, tmax=1.6)
    h_num, h_den = 3, 2
    sim, _, sw = field_sim(inst, inp, h_num, h_den)
    sim.sweep(9, 0)                                   # decorrelate, no swaps yet
    E = sim.energies()[0, :, 0].astype(np.int64)      # [NT][32]
    M = sim.magnetisations()[0, :, 0].astype(np.int64)
    Et = h_den * E - h_num * M
    step = oracle.field_step(h_num, h_den)
    X = (Et - Et[0]) * 4 // step                      # differences of X are 4x those of Et / step
    rn = refimpl.swap_rn(inst.seed, 0, 0, sim.pass_index, inst.NT)
    perm, masks = refimpl.brute_swap(X, sw, rn)
    before = sim.spins()[0, :, 0]
    got_masks = sim.pt_swap()[0, 0]
    after = sim.spins()[0, :, 0]
    np.testing.assert_array_equal(got_masks, masks)
    lanes = np.arange(32, dtype=np.uint32)
    for t in range(inst.NT):
        want = np.zeros_like(after[t])
        for b in range(32):
            want |= before[perm[t, b]] & (np.uint32(1) << lanes[b])
        np.testing.assert_array_equal(after[t], want)


def _field_distribution(J, beta, h):
    L = 2
    states = np.arange(256)
    bits = (states[:, None] >> np.arange(8)) & 1
    sig = (bits * 2 - 1).astype(np.int8).reshape(256, 1, L, L, L)
    sig = np.broadcast_to(sig, (256, 32, L, L, L))
    E = refimpl.energy_pm(sig, J) - h * sig.reshape(256, 32, -1).sum(axis=-1)
    w = np.exp(-beta * (E - E.min(axis=0)))
    return w / w.sum(axis=0)


def field_enumeration_statistic(h_num, h_den, n_samples=4000, thin=3, table_h=None):
    """Max chi-square per degree of freedom between sampled 2x2x2 states and the
    Boltzmann distribution in the field h = h_num / h_den (the chain's tables
    may be built for another field, `table_h`, to check that this is noticed)."""
    from test_oracle_pins import doubled_bond_cube
    L, G, NT, C, seed = 2, 1, 4, 2, 4048
    inst, inp = inputs(L, G, NT, C, seed, 13, tmin=0.7, tmax=3.0)
    bonds = doubled_bond_cube(G, 9)
    tn, td = table_h if table_h is not None else (h_num, h_den)
    mf = oracle.metro_table_field(inp["betas"], tn, td)
    sw = oracle.swap_table_field_trimmed(inp["betas"], inst.N, tn, td)
    sim = oracle.OracleSim(L, G, NT, C, seed, bonds, inp["spins"], oracle.metro_table(inp["betas"]), sw,
                           field=(tn, td, mf))
    sim.sweep(200, 1)
    lanes = np.arange(32, dtype=np.uint32)
    idx = np.zeros((n_samples, G, NT, C, 32), np.int64)
    for n in range(n_samples):
        sim.sweep(thin, 1)
        bits = (sim.spins()[..., None] >> lanes) & 1
        idx[n] = (bits.astype(np.int64) << np.arange(8)[:, None]).sum(axis=3)
    worst = 0.0
    J = refimpl.couplings(bonds[0], L)
    for t in range(NT):
        p = _field_distribution(J, inp["betas"][t], h_num / h_den)
        for c in range(C):
            for b in range(32):
                obs = np.bincount(idx[:, 0, t, c, b], minlength=256).astype(np.float64)
                exp = p[:, b] * n_samples
                big = exp >= 5
                e_bins = np.append(exp[big], exp[~big].sum())
                o_bins = np.append(obs[big], obs[~big].sum())
                keep = e_bins > 0
                chi2 = ((o_bins[keep] - e_bins[keep]) ** 2 / e_bins[keep]).sum()
                worst = max(worst, chi2 / max(int(keep.sum()) - 1, 1))
    return worst


@pytest.mark.slow
def test_stationary_distribution_2x2x2_in_a_field():
    assert field_enumeration_statistic(1, 2) < 8.0


@pytest.mark.slow
def test_enumeration_notices_a_wrong_field():
    assert field_enumeration_statistic(1, 2, n_samples=3000, table_h=(3, 2)) > 8.0
