"""The allocation-free replica-exchange pass (ea_pt_swap_static) against ea_pt_swap.

Callers that cannot allocate device memory while they run use
ea_pt_swap_static on buffers they own; its scratch is a static device array
of the library.  This file is collected last so that a failure here, under a
run that stops at the first failure, comes after every other test.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1311_5582_gb300 as ea  # noqa: E402


def _u32(t):
    return t.detach().cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("L,G,NT,C", [(8, 5, 24, 2), (6, 3, 9, 1), (16, 2, 32, 2)])
def test_static_pass_matches_context_pass_twice(L, G, NT, C):
    inst = W.Instance(L=L, G=G, NT=NT, C=C, seed=4242 + L, tmin=0.9, tmax=2.0, input_seed=L * NT)
    inp = W.draw_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    ctx = ea.Ensemble(inst.L, inst.G, inst.NT, inst.C, inst.seed, inp["bonds"], inp["spins"],
                      metro, swapt)
    ctx.sweep(7, 0)
    spins = ctx.read_spins().clone()           # [G][NT][C][N], caller-owned
    energies = ctx.measure()[0].clone()        # [G][NT][C][32]
    swapt_d = torch.from_numpy(swapt.view(np.int32)).cuda()
    masks = torch.zeros((G, C, NT - 1), dtype=torch.int32, device="cuda")
    for call in range(2):
        P = ctx.pass_index
        ref_masks = ctx.pt_swap()
        ea.ea_pt_swap_static(spins, energies, swapt_d, L, G, NT, C, inst.seed, P, masks=masks)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(_u32(masks), _u32(ref_masks), err_msg=f"call {call}")
        np.testing.assert_array_equal(_u32(spins), _u32(ctx.read_spins()), err_msg=f"call {call}")
        np.testing.assert_array_equal(energies.cpu().numpy(), ctx.measure()[0].cpu().numpy(),
                                      err_msg=f"call {call}")


def test_static_pass_rejects_ensembles_beyond_its_scratch():
    lib = ea.load_library()
    # 4097 units exceed the static scratch; the check happens before any device work
    dummy = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.ea_pt_swap_static(dummy.data_ptr(), dummy.data_ptr(), None, 0, 4, 4097, 2, 1, 1, 0,
                               None, None)
    assert rc == -1
    # a lattice whose site count does not fit 32 bits is refused the same way
    rc = lib.ea_pt_swap_static(dummy.data_ptr(), dummy.data_ptr(), None, 0, 1626, 1, 2, 1, 1, 0,
                               None, None)
    assert rc == -1
