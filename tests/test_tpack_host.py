"""The swap pass of the temperature-packed form as one bit permutation (CPU).

The kernel applies a replica-exchange pass (pairs p = 0..NT-2 in order, pair p
exchanging slots p and p+1 of a realization when bit p of the accepted mask M
is set; Sec. 2.4) to a word whose bit t is slot t by the closed form

    new = ((w >> 1) & M) | ((M + (starts & w)) & ends),
    ends = ~M & valid,  starts = ((~M << 1) | 1) & valid,

because an accepted run of pairs a..b-1 rotates slots a..b by one, and adding
the bit at a to M carries it through the run's ones to b.  This test checks that
identity against the pass applied pair by pair, exhaustively for NT <= 10 and
on random words and masks for NT up to 32, and the two-word form the merge
kernel evaluates for 33 <= NT <= 64 (slot 32 w + b in bit b of word w; the
shift and the addition carried across the words in 32-bit arithmetic).
"""
import numpy as np


def closed_form(w, M, NT):
    valid = (1 << NT) - 1
    ends = ~M & valid
    starts = ((~M << 1) | 1) & valid
    return (((w >> 1) & M) | ((M + (starts & w)) & ends)) & 0xFFFFFFFF


def pair_by_pair(w, M, NT):
    bits = [(w >> t) & 1 for t in range(NT)]
    for p in range(NT - 1):
        if (M >> p) & 1:
            bits[p], bits[p + 1] = bits[p + 1], bits[p]
    return sum(b << t for t, b in enumerate(bits))


def test_exhaustive_small_ladders():
    for NT in range(1, 9):
        for M in range(1 << max(NT - 1, 0)):
            for w in range(1 << NT):
                assert closed_form(w, M, NT) == pair_by_pair(w, M, NT), (NT, M, w)


def test_random_words_up_to_32_slots():
    rng = np.random.Generator(np.random.PCG64(7))
    for NT in (9, 10, 16, 24, 31, 32):
        for _ in range(3000):
            M = int(rng.integers(0, 1 << (NT - 1)))
            w = int(rng.integers(0, 1 << NT))
            assert closed_form(w, M, NT) == pair_by_pair(w, M, NT), (NT, M, w)
        # all pairs accepted: the coldest configuration moves to the hottest slot
        M = (1 << (NT - 1)) - 1
        assert closed_form(1, M, NT) == 1 << (NT - 1)


def test_tp_inputs_and_their_realization_packed_layout():
    """The temperature-packed inputs and their rewrite as bit 0 of word-groups
    (used to hand the same ensemble to the oracle) are a pure change of layout."""
    import workloads as W
    inst = W.Instance(L=6, G=3, NT=13, C=2, seed=1, tmin=0.9, tmax=2.0, input_seed=5)
    inp = W.draw_tp_inputs(inst)
    assert inp["bonds"].shape == (3, 3, 216) and set(np.unique(inp["bonds"])) <= {0, 1}
    assert inp["spins"].shape == (3, 2, 216) and int(inp["spins"].max()) < (1 << 13)
    b, s = W.tp_as_groups(inp["bonds"], inp["spins"], inst.NT)
    assert b.shape == (3, 3, 216) and s.shape == (3, 13, 2, 216)
    assert int(b.max()) <= 1 and int(s.max()) <= 1          # only bit 0 of each group is used
    back = np.zeros_like(inp["spins"])
    for t in range(inst.NT):
        back |= s[:, t] << np.uint32(t)
    np.testing.assert_array_equal(back, inp["spins"])
    np.testing.assert_array_equal(b, inp["bonds"].astype(np.uint32))
    # fair coins: about half the slot bits and half the bonds are set
    frac = np.mean([(inp["spins"] >> np.uint32(t)) & 1 for t in range(inst.NT)])
    assert 0.45 < frac < 0.55 and 0.45 < inp["bonds"].mean() < 0.55


def two_word_form(x0, x1, M0, M1, NT):
    """The merge kernel's expression on two 32-bit words (unsigned wraparound)."""
    F = 0xFFFFFFFF
    valid0 = F if NT >= 32 else (1 << NT) - 1
    valid1 = F if NT >= 64 else (1 << (NT - 32)) - 1
    ends0, ends1 = ~M0 & valid0, ~M1 & valid1
    starts0 = (((~M0 << 1) & F) | 1) & valid0
    starts1 = (((~M1 << 1) & F) | ((~M0 & F) >> 31)) & valid1
    sh0 = ((x0 >> 1) | (x1 << 31)) & F
    sh1 = x1 >> 1
    s0 = (M0 + (starts0 & x0)) & F
    cy = 1 if s0 < M0 else 0
    s1 = (M1 + (starts1 & x1) + cy) & F
    return (sh0 & M0) | (s0 & ends0), (sh1 & M1) | (s1 & ends1)


def test_two_words_33_to_64_slots():
    rng = np.random.Generator(np.random.PCG64(11))
    for NT in (33, 34, 40, 47, 56, 63, 64):
        cases = []
        for _ in range(3000):
            M = int(rng.integers(0, 2**32, dtype=np.uint64)) | (int(rng.integers(0, 2**32, dtype=np.uint64)) << 32)
            w = int(rng.integers(0, 2**32, dtype=np.uint64)) | (int(rng.integers(0, 2**32, dtype=np.uint64)) << 32)
            cases.append((M, w & ((1 << NT) - 1)))
        # runs that cross the word boundary, all-accepted and all-rejected ladders
        full = (1 << (NT - 1)) - 1
        cases += [(full, 1), (full, 1 << 31), (0, (1 << NT) - 1), (((1 << 40) - 1) ^ ((1 << 20) - 1), 1 << 20),
                  (1 << 31, 1 << 32), (1 << 31, 1 << 31)]
        for M, w in cases:
            M &= (1 << (NT - 1)) - 1
            x0, x1 = w & 0xFFFFFFFF, w >> 32
            y0, y1 = two_word_form(x0, x1, M & 0xFFFFFFFF, M >> 32, NT)
            assert y0 | (y1 << 32) == pair_by_pair(w, M, NT), (NT, M, w)

