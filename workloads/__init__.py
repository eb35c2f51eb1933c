"""Seeded synthetic workloads for the parallel-tempering Edwards-Anderson simulation.

This module only draws inputs: coupling bits, initial spin words and the
temperature ladder.  It contains none of the method's arithmetic (no energies,
no acceptance probabilities, no random numbers of the Markov chain), so both
the CUDA path and the CPU oracle can consume its arrays without sharing code.

Inputs follow the paper's workload shapes (Sec. 5.2): +-J couplings with equal
numbers of ferro- and antiferromagnetic bonds on average (Sec. 2.2), random
initial spins, and a set of temperature replicas per realization (Sec. 3.2).
Here 32 disorder realizations are packed per 32-bit word; bit b of word-group g
is realization 32*g + b.

Layouts (all uint32, C order):
  bonds  [G][3][N]        bit b of bonds[g][d][i] = 1  <=>  J = -1 on the bond
                          (i, i + e_d), d = 0 (+x), 1 (+y), 2 (+z)
  spins  [G][NT][C][N]    bit b = 1  <=>  S = +1, indexed by temperature slot
  betas  [NT] float64     inverse temperatures, slot 0 = coldest (largest beta)
Site index i = x + L*(y + L*z).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Instance:
    L: int
    G: int          # word-groups (realizations / 32)
    NT: int         # temperature slots
    C: int          # independent copies per temperature
    seed: int       # key of the Markov chain's counter-based generator
    tmin: float
    tmax: float
    input_seed: int  # seed of the numpy generator that draws bonds/spins

    @property
    def N(self) -> int:
        return self.L ** 3


def geometric_ladder(nt: int, tmin: float, tmax: float) -> np.ndarray:
    """Inverse temperatures of a geometric ladder T_j = tmin*(tmax/tmin)^(j/(nt-1)).

    Slot 0 is the coldest (largest beta); betas are non-increasing.
    """
    if nt == 1:
        return np.array([1.0 / tmin], dtype=np.float64)
    j = np.arange(nt, dtype=np.float64)
    T = tmin * (tmax / tmin) ** (j / (nt - 1))
    return (1.0 / T).astype(np.float64)


def draw_inputs(inst: Instance) -> dict:
    """Draw bonds and initial spins with numpy's PCG64 from ``inst.input_seed``.

    Each bit of a raw 32-bit draw is an independent fair coin, so every bond is
    +J or -J with probability 1/2 and every initial spin is up or down with
    probability 1/2.
    """
    rng = np.random.Generator(np.random.PCG64(inst.input_seed))
    N = inst.N
    bonds = rng.integers(0, 2**32, size=(inst.G, 3, N), dtype=np.uint64).astype(np.uint32)
    spins = rng.integers(0, 2**32, size=(inst.G, inst.NT, inst.C, N),
                         dtype=np.uint64).astype(np.uint32)
    betas = geometric_ladder(inst.NT, inst.tmin, inst.tmax)
    return {"bonds": bonds, "spins": spins, "betas": betas}


def draw_tp_inputs(inst: Instance) -> dict:
    """Inputs of the temperature-packed form for ``inst.G`` realizations.

    bonds [R][3][N] uint8 (1 <=> J = -1), each a fair coin; spins [R][C][N]
    uint32 with bit t (t < NT) the initial spin of slot t, each a fair coin
    (bits at or above NT zero) -- for NT > 32, [R][C][W][N] with W = ceil(NT/32)
    words, bit b of word w the spin of slot 32 w + b; betas as ``draw_inputs``.
    R = inst.G here: one realization per entry, not 32.
    """
    rng = np.random.Generator(np.random.PCG64(inst.input_seed))
    N = inst.N
    bonds = rng.integers(0, 2, size=(inst.G, 3, N), dtype=np.uint8)
    if inst.NT > 32:
        nw = -(-inst.NT // 32)
        spins = rng.integers(0, 2**32, size=(inst.G, inst.C, nw, N), dtype=np.uint64).astype(np.uint32)
        last = inst.NT - 32 * (nw - 1)
        if last < 32:
            spins[:, :, nw - 1] &= np.uint32((1 << last) - 1)
        betas = geometric_ladder(inst.NT, inst.tmin, inst.tmax)
        return {"bonds": bonds, "spins": spins, "betas": betas}
    spins = rng.integers(0, 2**32, size=(inst.G, inst.C, N), dtype=np.uint64).astype(np.uint32)
    if inst.NT < 32:
        spins &= np.uint32((1 << inst.NT) - 1)
    betas = geometric_ladder(inst.NT, inst.tmin, inst.tmax)
    return {"bonds": bonds, "spins": spins, "betas": betas}


def tp_as_groups(bonds: np.ndarray, spins: np.ndarray, NT: int) -> tuple[np.ndarray, np.ndarray]:
    """Temperature-packed inputs rewritten in the realization-packed layout with
    realization r as bit 0 of word-group r (the other 31 bits zero): bonds
    [R][3][N] uint32, spins [R][NT][C][N] uint32.  A pure change of layout
    (spins [R][C][N], or [R][C][W][N] with slot 32 w + b in bit b of word w)."""
    if spins.ndim == 3:
        spins = spins[:, :, None, :]
    R, C, _, N = spins.shape
    b = bonds.astype(np.uint32) & np.uint32(1)
    s = np.zeros((R, NT, C, N), np.uint32)
    for t in range(NT):
        s[:, t] = (spins[:, :, t // 32] >> np.uint32(t % 32)) & np.uint32(1)
    return b, s


# Few realizations, many temperatures: the temperature-packed form's workload
# (R = G realizations, one per word).
TPACK = Instance(L=16, G=76, NT=32, C=2, seed=6, tmin=0.95, tmax=2.0, input_seed=106)
TPACK_SWEEPS = 2000
TPACK_SWAP_EVERY = 10


# The five workloads of the hot path.  Shapes follow the ensembles of Sec. 5.2
# (lattices of 8^3..16^3, 24-56 temperatures, swaps every 1-10 sweeps) scaled to
# a GB300: realizations packed 32 per word, two copies per temperature for the
# overlap q.
SMALL = Instance(L=4, G=1, NT=16, C=2, seed=1, tmin=0.8, tmax=2.0, input_seed=101)
SMALL_SWEEPS = 2000
SMALL_SWAP_EVERY = 1

SCALE = Instance(L=8, G=64, NT=24, C=2, seed=2, tmin=0.9, tmax=2.0, input_seed=102)
SCALE_SWEEPS = 100_000
SCALE_SWAP_EVERY = 1

LARGE16 = Instance(L=16, G=256, NT=32, C=2, seed=3, tmin=0.95, tmax=2.0, input_seed=103)
LARGE32 = Instance(L=32, G=32, NT=32, C=2, seed=4, tmin=0.95, tmax=2.0, input_seed=104)
LARGE_SWEEPS = 100_000
LARGE_SWAP_EVERY = 10

# Mixed ensemble of the batched form: (L, realizations, temperatures).
BATCH_MIX = [(4, 4096, 16), (6, 2048, 20), (8, 2048, 24), (10, 1024, 28), (12, 512, 32), (16, 512, 32)]
BATCH_SWEEPS = 10_000
BATCH_SWAP_EVERY = 10


def batch_instances() -> list[Instance]:
    out = []
    for j, (L, R, NT) in enumerate(BATCH_MIX):
        out.append(Instance(L=L, G=R // 32, NT=NT, C=2, seed=10 + j, tmin=0.8, tmax=2.0,
                            input_seed=110 + j))
    return out


def served_trace(n_requests: int = 512, rate_hz: float = 200.0, seed: int = 5,
                 sweeps_lo: int = 1000, sweeps_hi: int = 100_000) -> list[dict]:
    """Poisson arrivals of simulation requests (the served form).

    Each request: L in {6,...,16} even, 32..2048 realizations (multiple of 32),
    16..32 temperatures in [0.8, 2.0], sweeps log-uniform in [sweeps_lo, sweeps_hi].
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    for r in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        L = int(rng.choice([6, 8, 10, 12, 14, 16]))
        G = int(rng.integers(1, 65))
        NT = int(rng.integers(16, 33))
        sweeps = int(round(math.exp(rng.uniform(math.log(sweeps_lo), math.log(sweeps_hi)))))
        inst = Instance(L=L, G=G, NT=NT, C=2, seed=1000 + r, tmin=0.8, tmax=2.0,
                        input_seed=2000 + r)
        reqs.append({"arrival_s": t, "inst": inst, "sweeps": sweeps, "swap_every": 10})
    return reqs
