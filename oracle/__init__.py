"""CPU oracle of the parallel-tempering Edwards-Anderson simulation (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

The C source ``ea_oracle.c`` is compiled with gcc into ``_build/libea_oracle.so``
on first use (or by ``build()``); this module is a ctypes wrapper with numpy
arrays in and out.  See ``ea_oracle.c`` for the conventions and citations.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ea_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libea_oracle.so")
_lock = threading.Lock()
_lib = None

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(src: str = _SRC, out: str = _LIB_PATH, extra_flags: tuple = ()) -> str:
    """Compile the oracle (plain C, -O2, no fast-math) into a shared library."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", *extra_flags,
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    vp = ctypes.c_void_p
    lib.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    lib.or_philox4x32_10.restype = None
    lib.or_metro_table.argtypes = [_f64p, ctypes.c_int, _u32p]
    lib.or_metro_table.restype = ctypes.c_int
    lib.or_swap_table.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, _u32p]
    lib.or_swap_table.restype = ctypes.c_int
    lib.or_metro_table_field.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _u64p]
    lib.or_metro_table_field.restype = ctypes.c_int
    lib.or_swap_table_field.argtypes = [_f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        _u32p]
    lib.or_swap_table_field.restype = ctypes.c_int
    lib.or_field_step.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.or_field_step.restype = ctypes.c_int
    lib.or_set_field.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp]
    lib.or_set_field.restype = ctypes.c_int
    lib.or_magnetisations.argtypes = [vp, _i32p]
    lib.or_magnetisations.restype = None
    lib.or_create.argtypes = [ctypes.c_int] * 4 + [ctypes.c_uint64, _u32p, _u32p, _u32p, vp,
                                                  ctypes.c_int, ctypes.c_int]
    lib.or_create.restype = vp
    lib.or_destroy.argtypes = [vp]
    lib.or_destroy.restype = None
    lib.or_sweep.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, ctypes.c_uint64,
                             ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.or_sweep.restype = ctypes.c_int
    lib.or_pt_swap.argtypes = [vp, vp]
    lib.or_pt_swap.restype = None
    lib.or_energies.argtypes = [vp, _i32p]
    lib.or_energies.restype = None
    lib.or_energies_recompute.argtypes = [vp, _i32p]
    lib.or_energies_recompute.restype = None
    lib.or_overlaps.argtypes = [vp, _u32p]
    lib.or_overlaps.restype = ctypes.c_int
    lib.or_plane_counts.argtypes = [vp, ctypes.c_int, _u32p]
    lib.or_plane_counts.restype = ctypes.c_int
    lib.or_read_spins.argtypes = [vp, _u32p]
    lib.or_read_spins.restype = None
    lib.or_sweep_index.argtypes = [vp]
    lib.or_sweep_index.restype = ctypes.c_uint64
    lib.or_pass_index.argtypes = [vp]
    lib.or_pass_index.restype = ctypes.c_uint64
    return lib


def load(path: str | None = None):
    """Load the oracle library, compiling it when missing or older than its source."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if (not os.path.exists(_LIB_PATH)
                    or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
                build()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter (4 words) under a 64-bit key (2 words)."""
    lib = load()
    out = np.zeros(4, np.uint32)
    lib.or_philox4x32_10(np.ascontiguousarray(ctr, np.uint32), np.ascontiguousarray(key, np.uint32),
                         out)
    return out


def metro_table(betas) -> np.ndarray:
    betas = np.ascontiguousarray(betas, np.float64)
    out = np.zeros((len(betas), 3), np.uint32)
    if load().or_metro_table(betas, len(betas), out) != 0:
        raise ValueError("betas must be >= 0")
    return out


def swap_table(betas, length: int) -> np.ndarray:
    betas = np.ascontiguousarray(betas, np.float64)
    out = np.zeros((max(len(betas) - 1, 0), length), np.uint32)
    if load().or_swap_table(betas, len(betas), length, out) != 0:
        raise ValueError("betas must be non-increasing (slot 0 coldest)")
    return out


def swap_table_trimmed(betas, n_sites: int) -> np.ndarray:
    """Swap table over k = 1..3N/2 with trailing all-zero columns removed."""
    full = swap_table(betas, 3 * n_sites // 2)
    if full.size == 0:
        return full[:, :0]
    nz = np.nonzero(full.any(axis=0))[0]
    length = int(nz[-1]) + 1 if len(nz) else 0
    return np.ascontiguousarray(full[:, :length])


def metro_table_field(betas, h_num: int, h_den: int) -> np.ndarray:
    """Field Metropolis table [NT][2][7] of 64-bit thresholds (2^32 = always)."""
    betas = np.ascontiguousarray(betas, np.float64)
    out = np.zeros((len(betas), 2, 7), np.uint64)
    if load().or_metro_table_field(betas, len(betas), int(h_num), int(h_den), out) != 0:
        raise ValueError("invalid temperatures or field")
    return out


def field_step(h_num: int, h_den: int) -> int:
    """Step of differences of Et = h_den E - h_num M."""
    return int(load().or_field_step(int(h_num), int(h_den)))


def swap_table_field_trimmed(betas, n_sites: int, h_num: int, h_den: int) -> np.ndarray:
    """Field swap table over k = 1..kmax (Et_p - Et_{p+1} = -k step), trailing zeros removed."""
    betas = np.ascontiguousarray(betas, np.float64)
    step = field_step(h_num, h_den)
    kmax = (6 * n_sites * int(h_den) + 2 * n_sites * abs(int(h_num))) // step
    out = np.zeros((max(len(betas) - 1, 0), kmax), np.uint32)
    if load().or_swap_table_field(betas, len(betas), int(h_num), int(h_den), kmax, out) != 0:
        raise ValueError("invalid temperatures or field")
    if out.size == 0:
        return out[:, :0]
    nz = np.nonzero(out.any(axis=0))[0]
    length = int(nz[-1]) + 1 if len(nz) else 0
    return np.ascontiguousarray(out[:, :length])


class OracleSim:
    """Scalar simulation state; mirrors the product's create/sweep/swap/measure calls."""

    def __init__(self, L, G, NT, C, seed, bonds, spins, metro, swapt, group_base=0, field=None):
        """group_base: global index of the first group passed (the random-number
        counters use global group indices, so a subset of groups reproduces the
        same trajectories as the full ensemble).  field: (h_num, h_den, metro_f)
        with metro_f from metro_table_field and swapt from swap_table_field_trimmed
        (metro is then unused)."""
        self.lib = load()
        self.L, self.G, self.NT, self.C = int(L), int(G), int(NT), int(C)
        self.N = self.L ** 3
        self.bonds = np.ascontiguousarray(bonds, np.uint32)
        spins = np.ascontiguousarray(spins, np.uint32)
        self.metro = np.ascontiguousarray(metro, np.uint32)
        self.swapt = np.ascontiguousarray(swapt, np.uint32)
        assert self.bonds.shape == (self.G, 3, self.N)
        assert spins.shape == (self.G, self.NT, self.C, self.N)
        assert self.metro.shape == (self.NT, 3)
        swap_len = self.swapt.shape[1] if self.swapt.ndim == 2 else 0
        self.swap_len = swap_len
        self.h = self.lib.or_create(self.L, self.G, self.NT, self.C, int(seed), self.bonds, spins,
                                    self.metro, self.swapt.ctypes.data if self.swapt.size else None,
                                    swap_len, int(group_base))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        if field is not None:
            h_num, h_den, metro_f = field
            self._metro_f = np.ascontiguousarray(metro_f, np.uint64)
            if self.lib.or_set_field(self.h, int(h_num), int(h_den),
                                     self._metro_f.ctypes.data if int(h_num) else None) != 0:
                raise ValueError("oracle rejected the field")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_destroy(h)
            self.h = None

    @property
    def sweep_index(self) -> int:
        return int(self.lib.or_sweep_index(self.h))

    @property
    def pass_index(self) -> int:
        return int(self.lib.or_pass_index(self.h))

    def n_passes(self, n_sweeps: int, swap_every: int) -> int:
        if swap_every <= 0:
            return 0
        s0 = self.sweep_index
        return sum(1 for s in range(s0, s0 + n_sweeps) if (s + 1) % swap_every == 0)

    def sweep(self, n_sweeps, swap_every, energy_log=False, swap_log=False, qhist=None,
              esum=None, measure_from=0, measure_every=0, check=False, threads=1):
        """Run sweeps; returns dict with requested logs.  qhist/esum arrays are accumulated."""
        out = {}
        elog = slog = None
        if energy_log:
            elog = np.zeros((n_sweeps, self.G, self.NT, self.C, 32), np.int32)
            out["energy_log"] = elog
        if swap_log:
            slog = np.zeros((self.n_passes(n_sweeps, swap_every), self.G, self.C,
                             max(self.NT - 1, 0)), np.uint32)
            out["swap_log"] = slog
        if qhist is not None:
            assert qhist.dtype == np.uint64 and qhist.shape == (self.NT, self.N + 1)
        if esum is not None:
            assert esum.dtype == np.int64 and esum.shape == (self.NT,)
        ptr = lambda a: a.ctypes.data if a is not None and a.size else None
        rc = self.lib.or_sweep(self.h, int(n_sweeps), int(swap_every), ptr(elog), ptr(slog),
                               ptr(qhist), ptr(esum), int(measure_from), int(measure_every),
                               int(bool(check)), int(threads))
        if rc != 0:
            raise AssertionError("oracle: tracked energy differs from recomputation")
        return out

    def pt_swap(self):
        masks = np.zeros((self.G, self.C, max(self.NT - 1, 0)), np.uint32)
        self.lib.or_pt_swap(self.h, masks.ctypes.data if masks.size else None)
        return masks

    def energies(self) -> np.ndarray:
        out = np.zeros((self.G, self.NT, self.C, 32), np.int32)
        self.lib.or_energies(self.h, out)
        return out

    def magnetisations(self) -> np.ndarray:
        out = np.zeros((self.G, self.NT, self.C, 32), np.int32)
        self.lib.or_magnetisations(self.h, out)
        return out

    def energies_recomputed(self) -> np.ndarray:
        out = np.zeros((self.G, self.NT, self.C, 32), np.int32)
        self.lib.or_energies_recompute(self.h, out)
        return out

    def overlaps(self) -> np.ndarray:
        out = np.zeros((self.G, self.NT, 32), np.uint32)
        if self.lib.or_overlaps(self.h, out) != 0:
            raise ValueError("overlaps need two copies")
        return out

    def plane_counts(self, mode: int) -> np.ndarray:
        """Per-plane counts (or_plane_counts): mode 0 differing sites between the
        copies [G][NT][3][L][32]; mode 1 up spins [G][NT][C][3][L][32]."""
        shape = (self.G, self.NT, 3, self.L, 32) if mode == 0 else (self.G, self.NT, self.C, 3, self.L, 32)
        out = np.zeros(shape, np.uint32)
        if self.lib.or_plane_counts(self.h, int(mode), out) != 0:
            raise ValueError("invalid mode (mode 0 needs two copies)")
        return out

    def spins(self) -> np.ndarray:
        out = np.zeros((self.G, self.NT, self.C, self.N), np.uint32)
        self.lib.or_read_spins(self.h, out)
        return out
