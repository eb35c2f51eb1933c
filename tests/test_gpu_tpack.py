"""GPU parity of the temperature-packed form (ea_tp_*) against the CPU oracle.

Realization r of a temperature-packed ensemble draws the random numbers of
word-group r of the realization-packed method (its bit 0), so it must follow
exactly the trajectory the oracle computes for bit 0 of group r when the
oracle is given the same bonds, spins and tables in its own layout.  Energies,
swap masks and spins are compared bit for bit (tolerance 0) after every sweep,
across lattice sizes with ragged quad counts (L = 6, 10, 12, 14), the
shared-memory and global-memory bond paths (L <= 24, L = 32), one and two
copies, 1 to 64 temperatures (two words per site above 32), and calls split
at arbitrary sweeps.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1311_5582_gb300 as ea  # noqa: E402


def _inputs(L, R, NT, C, seed):
    inst = W.Instance(L=L, G=R, NT=NT, C=C, seed=seed, tmin=0.8, tmax=2.0, input_seed=900 + L * 37 + NT)
    inp = W.draw_tp_inputs(inst)
    metro, swapt = ea.ea_build_tables(inp["betas"], inst.N)
    return inst, inp, metro, swapt


def _oracle(inst, inp, metro, swapt):
    b, s = W.tp_as_groups(inp["bonds"], inp["spins"], inst.NT)
    return oracle.OracleSim(inst.L, inst.G, inst.NT, inst.C, inst.seed, b, s, metro, swapt)


def _tp_from_oracle_spins(sp, NT):
    """Oracle spins [R][NT][C][N] (bit 0) -> temperature-packed words [R][C][N]
    ([R][C][W][N], slot 32 w + b in bit b of word w, when NT > 32)."""
    R, _, C, N = sp.shape
    nw = -(-NT // 32)
    out = np.zeros((R, C, nw, N), np.uint32)
    for t in range(NT):
        out[:, :, t // 32] |= (sp[:, t] & np.uint32(1)) << np.uint32(t % 32)
    return out[:, :, 0] if nw == 1 else out


def _pairs_as_words(rl, NT):
    """Accepted-pair bits [...][NT-1] -> swap-log words [...] ([...][W] when NT > 32)."""
    nw = -(-NT // 32)
    want = np.zeros(rl.shape[:-1] + (nw,), np.uint32)
    for p in range(NT - 1):
        want[..., p // 32] |= rl[..., p] << np.uint32(p % 32)
    return want[..., 0] if nw == 1 else want


def _compare_calls(L, R, NT, C, calls, swap_every, seed=77, split=None):
    inst, inp, metro, swapt = _inputs(L, R, NT, C, seed)
    gpu = ea.TPEnsemble(L, R, NT, C, seed, inp["bonds"], inp["spins"], metro, swapt)
    if split is not None:
        gpu.set_split(split)
    sim = _oracle(inst, inp, metro, swapt)
    sp0, en0 = gpu.read()
    np.testing.assert_array_equal(en0.cpu().numpy(), sim.energies()[..., 0], err_msg="initial energies")
    for k, n in enumerate(calls):
        out = gpu.sweep(n, swap_every, energy_log=True, swap_log=True)
        ref = sim.sweep(n, swap_every, energy_log=True, swap_log=True, threads=8)
        el = out["energy_log"].cpu().numpy()
        np.testing.assert_array_equal(el, ref["energy_log"][..., 0], err_msg=f"energy log, call {k}")
        sl = out["swap_log"].cpu().numpy().view(np.uint32)
        rl = ref["swap_log"] & np.uint32(1)                          # [passes][R][C][NT-1]
        np.testing.assert_array_equal(sl, _pairs_as_words(rl, NT), err_msg=f"swap log, call {k}")
        sp, en = gpu.read()
        np.testing.assert_array_equal(sp.cpu().numpy().view(np.uint32),
                                      _tp_from_oracle_spins(sim.spins(), NT), err_msg=f"spins, call {k}")
        np.testing.assert_array_equal(en.cpu().numpy(), sim.energies()[..., 0], err_msg=f"energies, call {k}")
    assert gpu.sweep_index == sum(calls)
    assert gpu.pass_index == sim.pass_index
    return gpu


@pytest.mark.parametrize("L,R,NT,C,n,swap_every", [
    (4, 3, 16, 2, 60, 1),      # the smallest configuration's shape, one realization per word
    (6, 2, 5, 1, 40, 3),       # ragged quad count (27 quads), one copy
    (8, 4, 24, 2, 30, 1),      # the scale configuration's ladder
    (10, 2, 32, 2, 20, 2),     # full words, 125 quads
    (12, 2, 7, 2, 16, 1),      # two quads a thread group, ragged
    (14, 1, 2, 2, 12, 1),      # one pair
    (16, 2, 32, 2, 12, 10),    # the largest configuration's ladder
    (20, 1, 9, 1, 6, 2),
    (24, 1, 32, 2, 4, 1),      # 221 KB of shared memory
    (32, 1, 32, 2, 3, 1),      # bonds read from global memory
])
@pytest.mark.parametrize("split", [None, 1])
def test_tpack_matches_oracle(L, R, NT, C, n, swap_every, split):
    """split None: the slot groups ea_tp_create picks (several per unit for these
    few realizations); 1: one CTA per unit with the swap passes in the kernel."""
    _compare_calls(L, R, NT, C, [n], swap_every, split=split)


@pytest.mark.parametrize("L,R,NT,C,calls,swap_every,split", [
    (8, 2, 24, 2, [9, 12], 1, 8),      # groups of 3 slots
    (6, 2, 5, 1, [13, 20], 3, 4),      # groups of 2 slots: three groups in use
    (16, 1, 32, 2, [7, 8], 5, 32),     # one slot a group
    (10, 3, 17, 2, [11], 4, 16),       # groups of 2, the last of 1
    (32, 1, 32, 1, [3], 2, 2),
])
def test_tpack_slot_groups_match_oracle(L, R, NT, C, calls, swap_every, split):
    gpu = _compare_calls(L, R, NT, C, calls, swap_every, split=split)
    assert gpu.split == -(-NT // -(-NT // split))


@pytest.mark.parametrize("L,R,NT,C,calls,swap_every,split", [
    (8, 2, 33, 2, [12, 7], 1, None),   # slot 32 alone in the second word: pair 31 crosses
    (6, 3, 40, 1, [20], 2, None),      # ragged second word, ragged quads
    (8, 1, 56, 2, [9, 6], 3, 4),       # the paper's largest ladder (Sec. 5.2), groups of 8 slots
    (10, 2, 64, 2, [10], 1, 1),        # two full words, one group per word
    (16, 1, 48, 1, [6], 1, 32),        # one slot a group, sixteen empty groups in the second word
    (32, 1, 64, 1, [2], 1, 8),         # bonds read from global memory
])
def test_tpack_two_words_match_oracle(L, R, NT, C, calls, swap_every, split):
    """More than 32 temperatures: two words per site (slot 32 w + b in bit b of
    word w), slot groups within each word, the pass over both words in the merge
    (runs of accepted pairs carried across the words)."""
    gpu = _compare_calls(L, R, NT, C, calls, swap_every, split=split)
    assert gpu.W == 2
    if split is not None:
        assert gpu.split == 2 * -(-32 // -(-32 // split))


def test_tpack_two_words_match_the_realization_packed_form():
    """Realization r of a 48-slot temperature-packed ensemble equals realization
    32r of the realization-packed GPU form (which holds up to 64 slots)."""
    L, R, NT, C, n = 8, 2, 48, 2, 14
    inst, inp, metro, swapt = _inputs(L, R, NT, C, 9)
    tp = ea.TPEnsemble(L, R, NT, C, 9, inp["bonds"], inp["spins"], metro, swapt)
    b, s = W.tp_as_groups(inp["bonds"], inp["spins"], NT)
    rp = ea.Ensemble(L, R, NT, C, 9, b, s, metro, swapt)
    o1 = tp.sweep(n, 1, energy_log=True, swap_log=True)
    o2 = rp.sweep(n, 1, energy_log=True, swap_log=True)
    np.testing.assert_array_equal(o1["energy_log"].cpu().numpy(), o2["energy_log"].cpu().numpy()[..., 0])
    rl = o2["swap_log"].cpu().numpy().view(np.uint32) & np.uint32(1)
    np.testing.assert_array_equal(o1["swap_log"].cpu().numpy().view(np.uint32), _pairs_as_words(rl, NT))
    sp, _ = tp.read()
    np.testing.assert_array_equal(sp.cpu().numpy().view(np.uint32),
                                  _tp_from_oracle_spins(rp.read_spins().cpu().numpy().view(np.uint32), NT))


def test_tpack_single_temperature_has_no_swaps():
    gpu = _compare_calls(8, 2, 1, 2, [15], 1)
    assert gpu.split == 1
    assert gpu.pass_index == 15          # passes are counted; with one slot they exchange nothing


@pytest.mark.parametrize("split", [None, 1])
def test_tpack_calls_split_anywhere(split):
    # pass indices and sweep counters continue across calls, swap every 3 sweeps
    _compare_calls(8, 3, 12, 2, [5, 1, 7, 4], 3, split=split)


def test_tpack_realization_matches_bit0_of_the_packed_form():
    """Realization r equals realization 32r of the realization-packed GPU form."""
    L, R, NT, C, n = 8, 3, 16, 2, 25
    inst, inp, metro, swapt = _inputs(L, R, NT, C, 5)
    tp = ea.TPEnsemble(L, R, NT, C, 5, inp["bonds"], inp["spins"], metro, swapt)
    b, s = W.tp_as_groups(inp["bonds"], inp["spins"], NT)
    rng = np.random.Generator(np.random.PCG64(1))
    # the other 31 realizations of each group are unrelated random ones
    b = b | (rng.integers(0, 2**32, size=b.shape, dtype=np.uint64).astype(np.uint32) & np.uint32(~1 & 0xFFFFFFFF))
    s = s | (rng.integers(0, 2**32, size=s.shape, dtype=np.uint64).astype(np.uint32) & np.uint32(~1 & 0xFFFFFFFF))
    rp = ea.Ensemble(L, R, NT, C, 5, b, s, metro, swapt)
    o1 = tp.sweep(n, 1, energy_log=True)
    o2 = rp.sweep(n, 1, energy_log=True)
    np.testing.assert_array_equal(o1["energy_log"].cpu().numpy(), o2["energy_log"].cpu().numpy()[..., 0])
    sp, _ = tp.read()
    np.testing.assert_array_equal(sp.cpu().numpy().view(np.uint32),
                                  _tp_from_oracle_spins(rp.read_spins().cpu().numpy().view(np.uint32), NT))


def test_tpack_split_changes_between_calls_and_rejects_bad_values():
    L, R, NT, C = 8, 2, 12, 2
    inst, inp, metro, swapt = _inputs(L, R, NT, C, 3)
    gpu = ea.TPEnsemble(L, R, NT, C, 3, inp["bonds"], inp["spins"], metro, swapt)
    sim = _oracle(inst, inp, metro, swapt)
    for k in (4, 1, 8, 2):
        gpu.set_split(k)
        gpu.sweep(6, 2)
        sim.sweep(6, 2, threads=8)
    sp, en = gpu.read()
    np.testing.assert_array_equal(sp.cpu().numpy().view(np.uint32), _tp_from_oracle_spins(sim.spins(), NT))
    np.testing.assert_array_equal(en.cpu().numpy(), sim.energies()[..., 0])
    for bad in (0, 3, 16, 64):          # not a power of two, or more groups than slots
        with pytest.raises(ea.EAError):
            gpu.set_split(bad)
