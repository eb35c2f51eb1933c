"""Independent test-side restatements used to pin the oracle.

Nothing here is imported by the oracle or by the product.  These are written
from the definitions (Eq. 1, Sec. 2.3, Sec. 2.4, Sec. 3.1) in a different
style from the oracle (vectorised numpy on +-1 arrays with periodic rolls),
with random numbers taken from PyTorch's Philox engine instead of the oracle's.
"""
from __future__ import annotations

import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
_REF_SRC = os.path.join(HERE, "philox_torch_ref.cpp")
_REF_BIN = os.path.join(ROOT, "oracle", "_build", "philox_torch_ref")


def torch_philox_binary() -> str:
    """Build (once) the PyTorch-header Philox4x32-10 reference program."""
    if not os.path.exists(_REF_BIN) or os.path.getmtime(_REF_BIN) < os.path.getmtime(_REF_SRC):
        import torch
        inc = os.path.join(os.path.dirname(torch.__file__), "include")
        os.makedirs(os.path.dirname(_REF_BIN), exist_ok=True)
        tmp = _REF_BIN + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O1", "-std=c++17", f"-I{inc}", "-o", tmp, _REF_SRC], check=True)
        os.replace(tmp, _REF_BIN)
    return _REF_BIN


def torch_philox(ctrs: np.ndarray, keys: np.ndarray) -> np.ndarray:
    """Philox4x32-10 outputs [n][4] for counters [n][4] and keys [n][2] via PyTorch's engine."""
    ctrs = np.asarray(ctrs, np.uint64).reshape(-1, 4)
    keys = np.asarray(keys, np.uint64).reshape(-1, 2)
    lines = "\n".join(" ".join(str(int(v)) for v in (*c, *k)) for c, k in zip(ctrs, keys))
    res = subprocess.run([torch_philox_binary()], input=lines + "\n", capture_output=True,
                         text=True, check=True)
    out = np.array([[int(v) for v in ln.split()] for ln in res.stdout.strip().splitlines()],
                   dtype=np.uint64)
    return out.astype(np.uint32).reshape(-1, 4)


def unpack_lanes(words: np.ndarray, L: int) -> np.ndarray:
    """uint32 [..., N] -> int8 [..., 32, L(z), L(y), L(x)] with bit b -> lane b (1 -> +1)."""
    w = np.asarray(words, np.uint32)
    bits = (w[..., None, :] >> np.arange(32, dtype=np.uint32)[:, None]) & 1
    pm = bits.astype(np.int8) * 2 - 1
    return pm.reshape(*w.shape[:-1], 32, L, L, L)


def pack_lanes(pm: np.ndarray) -> np.ndarray:
    """Inverse of unpack_lanes: int8 [..., 32, L, L, L] (+-1) -> uint32 [..., N]."""
    s = pm.shape
    flat = (pm.reshape(*s[:-4], 32, -1) > 0).astype(np.uint32)
    return (flat << np.arange(32, dtype=np.uint32)[:, None]).sum(axis=-2).astype(np.uint32)


def couplings(bonds_g: np.ndarray, L: int) -> np.ndarray:
    """bonds [3][N] words -> J [3][32][L,L,L] as +-1 (bit 1 -> J = -1)."""
    return -unpack_lanes(bonds_g, L)


# Axis of each direction in a [z][y][x] array.
AXIS = {0: -1, 1: -2, 2: -3}


def energy_pm(sigma: np.ndarray, J: np.ndarray) -> np.ndarray:
    """Eq. 1 (h = 0): E = -sum_{i,d} J_{i,d} s_i s_{i+d}.  sigma [..., 32, L,L,L], J [3][32][L,L,L]."""
    E = 0
    for d in range(3):
        E = E - (J[d] * sigma * np.roll(sigma, -1, axis=AXIS[d])).sum(axis=(-1, -2, -3))
    return E.astype(np.int64)


def local_field_pm(sigma: np.ndarray, J: np.ndarray) -> np.ndarray:
    """h_i = sum over the 6 bonds J_ij s_j; -d bond's J stored at the neighbour i - e_d."""
    h = np.zeros(sigma.shape, np.int32)
    for d in range(3):
        ax = AXIS[d]
        h += J[d] * np.roll(sigma, -1, axis=ax)
        h += np.roll(J[d], 1, axis=ax) * np.roll(sigma, 1, axis=ax)
    return h


def colour_mask(L: int) -> np.ndarray:
    z, y, x = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    return ((x + y + z) & 1).astype(np.int8)


def metropolis_rn(seed: int, L: int, g: int, t: int, c: int, s: int, colour: int) -> np.ndarray:
    """The shared uniform of every site of one colour: array [L,L,L] (other colour = 0)."""
    N = L ** 3
    i = np.arange(N)
    x, y, z = i % L, (i // L) % L, i // (L * L)
    sel = i[((x + y + z) & 1) == colour]
    k = sel >> 1
    ctr = np.stack([k >> 2, np.full_like(k, (colour << 16) | (c << 8) | t), np.full_like(k, s),
                    np.full_like(k, g)], axis=1)
    keys = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint64), (len(k), 1))
    out = torch_philox(ctr, keys)
    r = np.zeros(N, np.uint64)
    r[sel] = out[np.arange(len(k)), k & 3]
    return r.reshape(L, L, L)


def swap_rn(seed: int, g: int, c: int, P: int, NT: int) -> np.ndarray:
    """Uniforms of one swap pass: array [NT-1][32]."""
    p, b = np.meshgrid(np.arange(NT - 1), np.arange(32), indexing="ij")
    p, b = p.ravel(), b.ravel()
    ctr = np.stack([(p << 3) | (b >> 2), np.full_like(p, (1 << 24) | (c << 8)), np.full_like(p, P),
                    np.full_like(p, g)], axis=1)
    keys = np.tile(np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint64), (len(p), 1))
    out = torch_philox(ctr, keys)
    return out[np.arange(len(p)), b & 3].reshape(NT - 1, 32)


def brute_sweep(sigma, J, metro_row, seed, L, g, t, c, s):
    """One checkerboard Metropolis sweep (Sec. 2.3, 3.1) of sigma [32][L,L,L] in place."""
    col = colour_mask(L)
    for colour in (0, 1):
        r = metropolis_rn(seed, L, g, t, c, s, colour)
        h = local_field_pm(sigma, J)
        dE = 2 * sigma.astype(np.int32) * h
        idx = np.clip((12 - dE) // 4, 0, 2)
        thr = np.asarray(metro_row, np.uint64)[idx]
        accept = (dE <= 0) | (r[None] < thr)
        flip = accept & (col[None] == colour)
        sigma[flip] = -sigma[flip]
    return sigma


def brute_swap(E_by_slot, swap_row_tables, rn):
    """One replica-exchange pass (Sec. 2.4) per lane.  E_by_slot [NT][32]; returns
    (permutation perm[NT][32]: slot -> source slot, masks [NT-1] uint32)."""
    NT = E_by_slot.shape[0]
    E = E_by_slot.astype(np.int64).copy()
    perm = np.tile(np.arange(NT)[:, None], (1, 32))
    masks = np.zeros(NT - 1, np.uint32)
    K = swap_row_tables.shape[1] if swap_row_tables.ndim == 2 else 0
    for b in range(32):
        for p in range(NT - 1):
            delta = int(E[p, b] - E[p + 1, b])
            if delta >= 0:
                acc = True
            else:
                k = -delta // 4
                acc = k <= K and int(rn[p, b]) < int(swap_row_tables[p, k - 1])
            if acc:
                E[[p, p + 1], b] = E[[p + 1, p], b]
                perm[[p, p + 1], b] = perm[[p + 1, p], b]
                masks[p] |= np.uint32(1 << b)
    return perm, masks
