"""Statistical checks of the GPU path on the paper's validation systems (Sec. 5):
the 3D Ising ferromagnet (all J = +1), whose correlation lengths for two sizes
cross near the known critical point 1/T = 0.2217, and the ferromagnet in an
external field, where runs with and without replica exchange must give the
same equilibrium energy and magnetisation.  The 32 realizations of a word
share its random numbers (one uniform per site and sweep), and for a
ferromagnet they share the bonds too, so lanes of one word are correlated
chains; words of different groups and copies draw independent numbers, so the
errors are taken over (group, copy) words."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU hosts too; every test here needs a device
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1311_5582_gb300 as ea  # noqa: E402
from paper_1311_5582_gb300 import observables as ob  # noqa: E402

BETA_C = 0.2217   # the crossing the paper reports for the 3D Ising model (Sec. 5)


def ferromagnet(L, G, NT, C, seed):
    """All bonds J = +1 (bond bit 0), random initial spins."""
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=seed, tmin=1.0, tmax=2.0, input_seed=seed + 1)
    inp = W.draw_inputs(inst)
    return np.zeros_like(inp["bonds"]), inp["spins"]


def xi_over_L(L, betas, equil, n_meas, every, seed):
    G, C, NT = 8, 2, len(betas)
    bonds, spins = ferromagnet(L, G, NT, C, seed)
    metro, swapt = ea.ea_build_tables(betas, L ** 3)
    gpu = ea.Ensemble(L, G, NT, C, seed, bonds, spins, metro, swapt)
    gpu.sweep(equil, 1)
    s0 = np.zeros(NT)
    sk = np.zeros(NT)
    for _ in range(n_meas):
        gpu.sweep(every, 1)
        F = ob.magnetisation_plane_sums(gpu.measure_planes(1).cpu().numpy(), L)   # [G][NT][C][3][L][32]
        f0, fk = ob.fourier_squares(np.moveaxis(F, -1, 3), L)                      # [G][NT][C][32]
        s0 += f0.sum(axis=(0, 2, 3))
        sk += fk.sum(axis=(0, 2, 3))
    n = n_meas * G * C * 32
    chi0, chik = L ** 3 * s0 / n, L ** 3 * sk / n
    return ob.correlation_length(chi0, chik, L) / L


def test_ising_correlation_length_crossing():
    """xi / L of L = 8 and L = 16 cross within 0.004 of 1/T = 0.2217 (the paper's
    correlation-length figure), at a value near the universal 0.64."""
    betas = np.linspace(0.238, 0.206, 12)
    r8 = xi_over_L(8, betas, 3000, 600, 10, 11)
    r16 = xi_over_L(16, betas, 4000, 600, 10, 12)
    d = r16 - r8                          # > 0 in the ordered phase (large beta, slot 0)
    assert d[0] > 0 and d[-1] < 0, (r8, r16)
    i = int(np.nonzero((d[:-1] > 0) & (d[1:] <= 0))[0][0])
    beta_x = betas[i] + (betas[i + 1] - betas[i]) * d[i] / (d[i] - d[i + 1])
    value_x = r8[i] + (r8[i + 1] - r8[i]) * d[i] / (d[i] - d[i + 1])
    assert abs(beta_x - BETA_C) < 0.004, (beta_x, r8, r16)
    assert 0.5 < value_x < 0.8, value_x


def field_means(L, betas, h_num, h_den, swap_every, equil, n_meas, every, seed):
    G, C, NT = 16, 2, len(betas)
    bonds, spins = ferromagnet(L, G, NT, C, seed)
    mf, sw = ea.ea_build_tables_field(betas, L ** 3, h_num, h_den)
    gpu = ea.Ensemble(L, G, NT, C, seed, bonds, spins, None, sw, field=(h_num, h_den, mf))
    gpu.sweep(equil, swap_every)
    accE = torch.zeros((G, NT, C, 32), dtype=torch.float64, device="cuda")
    accM = torch.zeros_like(accE)
    for _ in range(n_meas):
        gpu.sweep(every, swap_every)
        accE += gpu.measure()[0].double()
        accM += gpu.magnetisations().double()
    N = L ** 3
    # per-word time and lane averages: [NT][G * C] independent samples
    e = (accE / n_meas / N).mean(dim=3).permute(1, 0, 2).reshape(NT, -1).cpu().numpy()
    m = (accM / n_meas / N).mean(dim=3).permute(1, 0, 2).reshape(NT, -1).cpu().numpy()
    return e, m


@pytest.mark.parametrize("h_num,h_den", [(1, 4), (1, 1)])
def test_field_ferromagnet_with_and_without_replica_exchange(h_num, h_den):
    """The paper's check of the swap pass (Sec. 5): energies and magnetisations of
    the ferromagnet in a field agree with and without parallel tempering."""
    L = 8
    betas = np.linspace(0.22, 0.12, 8)     # at and above the critical point: no metastable states
    e_pt, m_pt = field_means(L, betas, h_num, h_den, 1, 1000, 300, 5, 21)
    e_0, m_0 = field_means(L, betas, h_num, h_den, 0, 1000, 300, 5, 22)
    for a, b, what in ((e_pt, e_0, "E/N"), (m_pt, m_0, "M/N")):
        diff = a.mean(axis=1) - b.mean(axis=1)
        se = np.sqrt(a.var(axis=1, ddof=1) / a.shape[1] + b.var(axis=1, ddof=1) / b.shape[1])
        assert np.all(np.abs(diff) < 5 * se + 1e-12), (what, diff, se)
    # the field orders the spins along it: M > 0, growing with beta
    assert np.all(m_pt.mean(axis=1) > 0) and np.all(np.diff(m_pt.mean(axis=1)) < 0)
