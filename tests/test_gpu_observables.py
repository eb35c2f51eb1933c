"""Per-plane counts on the GPU (ea_measure_planes) against the oracle, bit for bit."""
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
from paper_1311_5582_gb300 import observables as ob  # noqa: E402


@pytest.mark.parametrize("L,G,NT,C,n,k", [
    (4, 2, 5, 2, 23, 1), (8, 3, 24, 2, 17, 1), (10, 1, 6, 2, 9, 2), (16, 1, 32, 2, 12, 10),
    (32, 1, 3, 2, 4, 2), (6, 2, 4, 1, 11, 3),
])
def test_plane_counts_match_the_oracle(L, G, NT, C, n, k):
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=600 + L, tmin=0.9, tmax=2.0, input_seed=700 + L)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    gpu = ea.Ensemble(L, G, NT, C, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    gpu.sweep(n, k)
    sim = oracle.OracleSim(L, G, NT, C, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    sim.sweep(n, k, threads=8)
    up = gpu.measure_planes(1).cpu().numpy()
    np.testing.assert_array_equal(up, sim.plane_counts(1).astype(np.int32))
    if C == 2:
        d = gpu.measure_planes(0).cpu().numpy()
        np.testing.assert_array_equal(d, sim.plane_counts(0).astype(np.int32))
        _, nd = gpu.measure(energies=False, ndiff=True)
        nd = nd.cpu().numpy().view(np.uint32).astype(np.int64)
        for a in range(3):
            np.testing.assert_array_equal(d[:, :, a].sum(axis=2), nd)
    else:
        with pytest.raises(ea.EAError):
            gpu.measure_planes(0)


def test_correlation_length_inputs_from_the_gpu():
    """The estimators run on GPU plane counts exactly as on the oracle's."""
    inst = W.Instance(L=8, G=2, NT=8, C=2, seed=77, tmin=0.9, tmax=2.0, input_seed=78)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    gpu = ea.Ensemble(8, 2, 8, 2, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    sim = oracle.OracleSim(8, 2, 8, 2, inst.seed, inp["bonds"], inp["spins"], metro, swapt)
    acc_g, acc_o = [], []
    for _ in range(4):
        gpu.sweep(10, 1)
        sim.sweep(10, 1, threads=8)
        acc_g.append(ob.overlap_plane_sums(gpu.measure_planes(0).cpu().numpy(), 8))
        acc_o.append(ob.overlap_plane_sums(sim.plane_counts(0), 8))
    sg = np.moveaxis(np.stack(acc_g), -1, -3)          # [meas][G][NT][32][3][L]
    so = np.moveaxis(np.stack(acc_o), -1, -3)
    chi_g = ob.susceptibilities(sg, 8, axis=(0, 1, 3))  # per slot
    chi_o = ob.susceptibilities(so, 8, axis=(0, 1, 3))
    np.testing.assert_array_equal(chi_g[0], chi_o[0])
    np.testing.assert_array_equal(chi_g[1], chi_o[1])
    assert np.all(np.isfinite(ob.correlation_length(chi_g[0], chi_g[1], 8)))
