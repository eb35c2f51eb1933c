"""The oracle's Philox4x32-10 against CURAND's device Philox4_32_10 (GPU).

CURAND keys its generator with the 64-bit seed and, for curand_init(seed,
subsequence, offset) with offset a multiple of 4, returns from curand4() the
block at counter (offset/4 as two low words, subsequence as two high words) --
the documented layout of its 2^66-element subsequences.  The oracle's
generator must give the same four words for that counter and key.  This pins
the generator with an implementation written by others, beside the PyTorch
engine of the CPU pins; the CUDA path's generator equals the oracle's through
every bit-exact trajectory test.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "curand_philox_ref.cu")
BIN = os.path.join(os.path.dirname(HERE), "oracle", "_build", "curand_philox_ref")


def _binary():
    if not os.path.exists(BIN) or os.path.getmtime(BIN) < os.path.getmtime(SRC):
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        os.makedirs(os.path.dirname(BIN), exist_ok=True)
        tmp = BIN + f".tmp{os.getpid()}"
        subprocess.run([nvcc, "-O2", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, SRC],
                       check=True)
        os.replace(tmp, BIN)
    return BIN


def test_oracle_philox_equals_curand():
    rng = np.random.Generator(np.random.PCG64(20131122))
    edges = [0, 1, 0xFFFFFFFF, 0x100000000, 0xFFFFFFFFFFFFFFFF >> 2]
    reqs = []
    for seed in [0, 1, 0xFFFFFFFF, 0xDEADBEEFCAFEF00D, *rng.integers(0, 2**63, 4).tolist()]:
        for sub in edges + rng.integers(0, 2**63, 3).tolist():
            for m in edges + rng.integers(0, 2**61, 3).tolist():
                reqs.append((int(seed), int(sub), 4 * int(m) & 0xFFFFFFFFFFFFFFFF))
    text = f"{len(reqs)}\n" + "\n".join(f"{s} {u} {o}" for s, u, o in reqs) + "\n"
    out = subprocess.run([_binary()], input=text, capture_output=True, text=True, check=True).stdout
    got = np.array([[int(x) for x in line.split()] for line in out.strip().splitlines()], np.uint64)
    assert got.shape == (len(reqs), 4)
    for (seed, sub, off), row in zip(reqs, got):
        m = off // 4
        ctr = [m & 0xFFFFFFFF, m >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        np.testing.assert_array_equal(oracle.philox4x32_10(ctr, key), row.astype(np.uint32),
                                      err_msg=f"seed={seed} subsequence={sub} offset={off}")
