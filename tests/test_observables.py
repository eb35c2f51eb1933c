"""Pins of the observable estimators (closed forms) and of their agreement
between the two measurement outputs of the oracle (q histogram and plane counts)."""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import workloads as W
from paper_1311_5582_gb300 import observables as ob


def test_binder_ratio_closed_forms():
    N = 8
    h = np.zeros(N + 1)
    h[0] = h[N] = 5                       # q = +-1 only: <q^4> = <q^2>^2 = 1
    assert ob.binder_ratio(h, N) == pytest.approx(1.0)
    h = np.zeros(N + 1)
    h[[0, N // 2, N]] = 1                 # q in {1, 0, -1}, equal weights: g = (3 - 1.5) / 2
    assert ob.binder_ratio(h, N) == pytest.approx(0.75)
    # a binomial n (independent sites, p = 1/2): q = 1 - 2n/N has <q^2> = 1/N,
    # <q^4> = (3N - 2) / N^3, so g = (3 - (3N - 2)/N) / 2 = 1/N
    N = 40
    h = np.array([math.comb(N, n) for n in range(N + 1)], dtype=np.float64)
    assert ob.binder_ratio(h, N) == pytest.approx(1.0 / N, rel=1e-12)
    # rows are independent
    rows = np.stack([h, h * 3])
    np.testing.assert_allclose(ob.binder_ratio(rows, N), [1.0 / N, 1.0 / N], rtol=1e-12)


def test_fourier_modes_closed_forms():
    L = 8
    N = L ** 3
    p = np.arange(L)
    # a plane wave along x, plane sums A L^2 cos(2 pi p / L): f(k) = (A L^2 / N)(L / 2) = A / 2
    # on that axis and 0 on the others
    A = 0.5
    sums = np.zeros((3, L))
    sums[0] = A * L * L * np.cos(2 * math.pi * p / L)
    s0, sk = ob.fourier_squares(sums, L)
    assert s0 == pytest.approx(0.0, abs=1e-20)
    assert sk == pytest.approx((A * L ** 3 / 2 / N) ** 2 / 3)
    # a uniform field: f(0) = mean, no k_min component
    sums = np.full((3, L), 0.25 * L * L)
    s0, sk = ob.fourier_squares(sums, L)
    assert s0 == pytest.approx(0.0625)
    assert sk == pytest.approx(0.0, abs=1e-20)


def test_correlation_length_inverts_ornstein_zernike():
    L = 12
    for xi in (0.3, 1.0, 4.5):
        chi0 = 7.0
        chik = chi0 / (1.0 + (2.0 * math.sin(math.pi / L) * xi) ** 2)
        assert ob.correlation_length(chi0, chik, L) == pytest.approx(xi, rel=1e-12)


def test_plane_sums_of_constructed_configurations():
    L = 4
    # copies identical: every q_i = 1
    assert np.all(ob.overlap_plane_sums(np.zeros((3, L)), L) == L * L)
    # all spins down: every m_i = -1
    assert np.all(ob.magnetisation_plane_sums(np.zeros((3, L)), L) == -L * L)


def test_histogram_and_plane_counts_give_the_same_q_moments():
    """The oracle's q histogram (total differing sites) and its plane counts
    (summed over the planes of any axis) are two views of the same overlaps."""
    inst = W.Instance(L=4, G=2, NT=6, C=2, seed=31, tmin=0.8, tmax=2.0, input_seed=32)
    inp = W.draw_inputs(inst)
    metro = oracle.metro_table(inp["betas"])
    swapt = oracle.swap_table_trimmed(inp["betas"], inst.N)
    sim = oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                           metro, swapt)
    qh = np.zeros((inst.NT, inst.N + 1), np.uint64)
    sq = np.zeros(inst.NT)
    sq4 = np.zeros(inst.NT)
    for _ in range(12):
        sim.sweep(5, 1, qhist=qh, measure_from=sim.sweep_index + 4, measure_every=5)
        sums = ob.overlap_plane_sums(sim.plane_counts(0), inst.L)     # [G][NT][3][L][32]
        q = sums[:, :, 0, :, :].sum(axis=2) / inst.N                   # [G][NT][32]
        sq += (q ** 2).sum(axis=(0, 2))
        sq4 += (q ** 4).sum(axis=(0, 2))
    n = 12 * inst.G * 32
    g_planes = 0.5 * (3 - (sq4 / n) / (sq / n) ** 2)
    np.testing.assert_allclose(ob.binder_ratio(qh, inst.N), g_planes, rtol=1e-12)
