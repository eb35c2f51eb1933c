"""Pins of the oracle's per-plane counts (the input of the Fourier-mode
observables): closed forms on constructed configurations, consistency with
the total overlap, and a numpy restatement over the slot-ordered spins."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W

from refimpl import unpack_lanes


def sim_with(L, spins, NT=2, C=2, seed=5):
    """Oracle holding the given spins [1][NT][C][N] (ferromagnetic bonds, unused here)."""
    N = L ** 3
    bonds = np.zeros((1, 3, N), np.uint32)
    metro = np.zeros((NT, 3), np.uint32)
    swapt = np.zeros((max(NT - 1, 0), 0), np.uint32)
    return oracle.OracleSim(L, 1, NT, C, seed, bonds, spins, metro, swapt)


def coords(L):
    i = np.arange(L ** 3)
    return i % L, (i // L) % L, i // (L * L)


@pytest.mark.parametrize("L", [2, 4, 6])
def test_one_flipped_plane(L):
    """Copy 1 = copy 0 with the plane x = 0 flipped in every lane."""
    N = L ** 3
    rng = np.random.default_rng(L)
    s0 = rng.integers(0, 2**32, N, dtype=np.uint64).astype(np.uint32)
    x, y, z = coords(L)
    s1 = np.where(x == 0, ~s0, s0).astype(np.uint32)
    spins = np.zeros((1, 2, 2, N), np.uint32)
    spins[0, :, 0] = s0
    spins[0, :, 1] = s1
    pc = sim_with(L, spins).plane_counts(0)          # [1][NT][3][L][32]
    expect_x = np.zeros(L, np.uint32)
    expect_x[0] = L * L
    for t in range(2):
        for b in range(32):
            np.testing.assert_array_equal(pc[0, t, 0, :, b], expect_x)
            np.testing.assert_array_equal(pc[0, t, 1, :, b], np.full(L, L, np.uint32))
            np.testing.assert_array_equal(pc[0, t, 2, :, b], np.full(L, L, np.uint32))


@pytest.mark.parametrize("L", [2, 4])
def test_up_spin_planes(L):
    """mode 1: all up -> L^2 per plane; up exactly where z is even -> planes
    along z alternate L^2 / 0, planes along x and y hold L^2 / 2."""
    N = L ** 3
    x, y, z = coords(L)
    spins = np.zeros((1, 2, 2, N), np.uint32)
    spins[0, :, 0] = 0xFFFFFFFF
    spins[0, :, 1] = np.where(z % 2 == 0, 0xFFFFFFFF, 0).astype(np.uint32)
    pc = sim_with(L, spins).plane_counts(1)          # [1][NT][C][3][L][32]
    assert np.all(pc[0, :, 0] == L * L)
    zp = np.array([L * L if p % 2 == 0 else 0 for p in range(L)], np.uint32)
    for t in range(2):
        for b in range(32):
            np.testing.assert_array_equal(pc[0, t, 1, 2, :, b], zp)
            np.testing.assert_array_equal(pc[0, t, 1, 0, :, b], np.full(L, L * L // 2, np.uint32))
            np.testing.assert_array_equal(pc[0, t, 1, 1, :, b], np.full(L, L * L // 2, np.uint32))


def test_after_a_run_matches_numpy_and_total_overlap():
    """After sweeps and swap passes (slot labels permuted inside the oracle)."""
    inst = W.Instance(L=6, G=2, NT=5, C=2, seed=21, tmin=0.9, tmax=2.0, input_seed=22)
    inp = W.draw_inputs(inst)
    metro = oracle.metro_table(inp["betas"])
    swapt = oracle.swap_table_trimmed(inp["betas"], inst.N)
    sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                           metro, swapt)
    sim.sweep(17, 1)
    pc0, pc1 = sim.plane_counts(0), sim.plane_counts(1)
    pm = unpack_lanes(sim.spins(), inst.L)              # [G][NT][C][32][z][y][x] of +-1
    diff = (pm[:, :, 0] != pm[:, :, 1])                 # [G][NT][32][z][y][x]
    up = pm > 0
    sums_d = [diff.sum(axis=(-3, -2)), diff.sum(axis=(-3, -1)), diff.sum(axis=(-2, -1))]  # by x, y, z
    sums_u = [up.sum(axis=(-3, -2)), up.sum(axis=(-3, -1)), up.sum(axis=(-2, -1))]
    for a in range(3):
        np.testing.assert_array_equal(pc0[:, :, a], np.moveaxis(sums_d[a], -2, -1))
        np.testing.assert_array_equal(pc1[:, :, :, a], np.moveaxis(sums_u[a], -2, -1))
    tot = sim.overlaps()                                 # [G][NT][32]
    for a in range(3):
        np.testing.assert_array_equal(pc0[:, :, a].sum(axis=2), tot)


def test_invalid_modes():
    spins = np.zeros((1, 2, 1, 8), np.uint32)
    s = sim_with(2, spins, C=1)
    with pytest.raises(ValueError):
        s.plane_counts(0)                                # overlaps need two copies
    with pytest.raises(ValueError):
        s.plane_counts(2)
