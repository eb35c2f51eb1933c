"""Python binding of the GB300 parallel-tempering Edwards-Anderson simulator.

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of ``_build/libea.so`` behind the C ABI of ``include/ea.h``.  PyTorch
provides device memory (output tensors) and the CUDA stream.  There is no CPU
fallback: if the library is missing, importing the binding's functions raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = _build.LIB

EA_OK, EA_PENDING = 0, 1
_ERRORS = {-1: "EA_EINVAL", -2: "EA_ENOMEM", -3: "EA_ECUDA", -4: "EA_ETIMEOUT",
           -5: "EA_EUNSUPPORTED", -6: "EA_ESTATE"}

_lib = None


class EAError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {_ERRORS.get(code, code)}")
        self.code = code


class _Config(ctypes.Structure):
    _fields_ = [("L", ctypes.c_uint32), ("n_groups", ctypes.c_uint32),
                ("n_temps", ctypes.c_uint32), ("n_copies", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("bonds", ctypes.c_void_p),
                ("spins0", ctypes.c_void_p), ("metro", ctypes.c_void_p),
                ("swapt", ctypes.c_void_p), ("swap_len", ctypes.c_uint32),
                ("group_base", ctypes.c_uint32)]


class _SweepArgs(ctypes.Structure):
    _fields_ = [("n_sweeps", ctypes.c_uint32), ("swap_every", ctypes.c_uint32),
                ("energy_log", ctypes.c_void_p), ("swap_log", ctypes.c_void_p),
                ("qhist", ctypes.c_void_p), ("esum", ctypes.c_void_p),
                ("measure_from", ctypes.c_uint64), ("measure_every", ctypes.c_uint32)]


class _ServerOpts(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_uint64), ("max_live", ctypes.c_uint32),
                ("round_ms", ctypes.c_uint32)]


class _Request(ctypes.Structure):
    _fields_ = [("n_sweeps", ctypes.c_uint32), ("swap_every", ctypes.c_uint32),
                ("spins_out", ctypes.c_void_p), ("energies_out", ctypes.c_void_p),
                ("magnetisations_out", ctypes.c_void_p)]


class _TpConfig(ctypes.Structure):
    _fields_ = [("L", ctypes.c_uint32), ("n_real", ctypes.c_uint32),
                ("n_temps", ctypes.c_uint32), ("n_copies", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("bonds", ctypes.c_void_p),
                ("spins0", ctypes.c_void_p), ("metro", ctypes.c_void_p),
                ("swapt", ctypes.c_void_p), ("swap_len", ctypes.c_uint32),
                ("real_base", ctypes.c_uint32)]


class _TpRequest(ctypes.Structure):
    _fields_ = [("n_sweeps", ctypes.c_uint32), ("swap_every", ctypes.c_uint32),
                ("spins_out", ctypes.c_void_p), ("energies_out", ctypes.c_void_p)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("live", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("flip_attempts", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("span_s", ctypes.c_double), ("mem_budget", ctypes.c_uint64),
                ("peak_bytes", ctypes.c_uint64)]


class _PlanDesc(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("group_threads", ctypes.c_int32), ("lattices_per_cta", ctypes.c_int32),
                ("smem_bytes", ctypes.c_uint64), ("units_per_cta", ctypes.c_int32)]


class _Field(ctypes.Structure):
    _fields_ = [("h_num", ctypes.c_int32), ("h_den", ctypes.c_int32), ("metro", ctypes.c_void_p)]


PLAN_FORMS = {0: "unit", 1: "unit-fast", 2: "chunked", 3: "unit-wave"}

EXPORTS = ["ea_build_tables", "ea_build_tables_field", "ea_supported_L", "ea_create",
           "ea_create_field", "ea_magnetisations", "ea_destroy", "ea_sweep",
           "ea_pt_swap", "ea_measure", "ea_measure_planes", "ea_read_spins", "ea_read_spins_host", "ea_write_spins",
           "ea_get_counters", "ea_sync", "ea_launch_count", "ea_plan_count", "ea_plan_current",
           "ea_plan_info", "ea_plan_select", "ea_autotune", "ea_batch_create", "ea_batch_add",
           "ea_batch_clear", "ea_batch_plan_count", "ea_batch_plan_info", "ea_batch_plan_current",
           "ea_batch_set_plan", "ea_batch_set_width", "ea_batch_set_wait_limit", "ea_batch_inject_stall",
           "ea_batch_set_segment", "ea_batch_sweep",
           "ea_batch_sweep_each", "ea_batch_sync", "ea_batch_autotune", "ea_batch_launch_count", "ea_batch_destroy",
           "ea_server_create", "ea_submit", "ea_submit_field", "ea_submit_tp", "ea_poll", "ea_server_stats_get",
           "ea_server_destroy",
           "ea_run",
           "ea_pt_swap_static", "ea_tp_create", "ea_tp_sweep", "ea_tp_read", "ea_tp_info",
           "ea_tp_set_split", "ea_tp_destroy", "ea_strerror"]


def load_library(path: str | None = None):
    """Loads libea.so (building it with nvcc when the source is newer).

    Raises when the library cannot be built or loaded: the simulator has no
    other implementation to fall back to."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    if path is None:
        path = LIB_PATH
        if not os.path.exists(path) or _build._stale(path, [
                os.path.join(_build.CSRC, f) for f in os.listdir(_build.CSRC)]):
            _build.build()
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
    lib.ea_build_tables.argtypes = [vp, u32, u32, vp, vp, u32, ctypes.POINTER(u32)]
    lib.ea_supported_L.argtypes = [u32]
    lib.ea_create.argtypes = [ctypes.POINTER(_Config), vp, ctypes.POINTER(vp)]
    lib.ea_build_tables_field.argtypes = [vp, u32, u32, ctypes.c_int32, ctypes.c_int32, vp, vp, u32,
                                          ctypes.POINTER(u32)]
    lib.ea_create_field.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Field), vp,
                                    ctypes.POINTER(vp)]
    lib.ea_magnetisations.argtypes = [vp, vp]
    lib.ea_destroy.argtypes = [vp]
    lib.ea_destroy.restype = None
    lib.ea_sweep.argtypes = [vp, ctypes.POINTER(_SweepArgs)]
    lib.ea_pt_swap.argtypes = [vp, vp]
    lib.ea_measure.argtypes = [vp, vp, vp, vp]
    lib.ea_measure_planes.argtypes = [vp, i32, vp]
    lib.ea_read_spins.argtypes = [vp, vp]
    lib.ea_read_spins_host.argtypes = [vp, vp]
    lib.ea_write_spins.argtypes = [vp, vp, u64, u64]
    lib.ea_get_counters.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
    lib.ea_sync.argtypes = [vp]
    lib.ea_launch_count.argtypes = [vp]
    lib.ea_launch_count.restype = u64
    lib.ea_plan_count.argtypes = [vp]
    lib.ea_plan_current.argtypes = [vp]
    lib.ea_plan_info.argtypes = [vp, i32, ctypes.POINTER(_PlanDesc)]
    lib.ea_plan_select.argtypes = [vp, i32]
    lib.ea_autotune.argtypes = [vp, u32, u32, ctypes.POINTER(ctypes.c_float)]
    lib.ea_run.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_SweepArgs), vp, vp, vp, vp, vp]
    lib.ea_pt_swap_static.argtypes = [vp, vp, vp, u32, u32, u32, u32, u32, u64, u64, vp, vp]
    lib.ea_batch_create.argtypes = [vp, ctypes.POINTER(vp)]
    lib.ea_batch_add.argtypes = [vp, vp]
    lib.ea_batch_clear.argtypes = [vp]
    lib.ea_batch_plan_count.argtypes = [vp, u32]
    lib.ea_batch_plan_info.argtypes = [vp, u32, i32, ctypes.POINTER(_PlanDesc)]
    lib.ea_batch_plan_current.argtypes = [vp, u32]
    lib.ea_batch_set_plan.argtypes = [vp, u32, i32]
    lib.ea_batch_set_width.argtypes = [vp, i32]
    lib.ea_batch_set_wait_limit.argtypes = [vp, u32]
    lib.ea_batch_inject_stall.argtypes = [vp]
    lib.ea_batch_autotune.argtypes = [vp, u32, u32, ctypes.POINTER(ctypes.c_float)]
    lib.ea_batch_set_segment.argtypes = [vp, u32]
    lib.ea_batch_sweep.argtypes = [vp, u32, u32]
    lib.ea_batch_sweep_each.argtypes = [vp, vp, vp]
    lib.ea_batch_sync.argtypes = [vp]
    lib.ea_batch_launch_count.argtypes = [vp]
    lib.ea_batch_launch_count.restype = u64
    lib.ea_batch_destroy.argtypes = [vp]
    lib.ea_batch_destroy.restype = None
    lib.ea_server_create.argtypes = [ctypes.POINTER(_ServerOpts), ctypes.POINTER(vp)]
    lib.ea_submit.argtypes = [vp, ctypes.POINTER(_Config), ctypes.POINTER(_Request),
                              ctypes.POINTER(u64)]
    lib.ea_submit_tp.argtypes = [vp, ctypes.POINTER(_TpConfig), ctypes.POINTER(_TpRequest),
                                 ctypes.POINTER(u64)]
    lib.ea_poll.argtypes = [vp, u64, u32]
    lib.ea_server_stats_get.argtypes = [vp, ctypes.POINTER(_ServerStats)]
    lib.ea_server_destroy.argtypes = [vp]
    lib.ea_server_destroy.restype = None
    lib.ea_strerror.argtypes = [i32]
    lib.ea_strerror.restype = ctypes.c_char_p
    lib.ea_tp_create.argtypes = [ctypes.POINTER(_TpConfig), vp, ctypes.POINTER(vp)]
    lib.ea_tp_sweep.argtypes = [vp, u32, u32, vp, vp]
    lib.ea_tp_read.argtypes = [vp, vp, vp]
    lib.ea_tp_info.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64),
                               ctypes.POINTER(u32)]
    lib.ea_tp_set_split.argtypes = [vp, u32]
    lib.ea_tp_destroy.argtypes = [vp]
    lib.ea_tp_destroy.restype = None
    for name in ("ea_build_tables", "ea_build_tables_field", "ea_create_field", "ea_magnetisations",
                 "ea_supported_L", "ea_create", "ea_sweep", "ea_pt_swap",
                 "ea_measure_planes",
                 "ea_measure", "ea_read_spins", "ea_read_spins_host", "ea_write_spins",
                 "ea_get_counters", "ea_sync", "ea_run", "ea_plan_count", "ea_plan_current",
                 "ea_plan_info", "ea_plan_select", "ea_autotune", "ea_pt_swap_static",
                 "ea_batch_create", "ea_batch_add", "ea_batch_clear", "ea_batch_set_plan",
                 "ea_batch_set_segment", "ea_batch_sweep", "ea_batch_sync", "ea_batch_plan_count",
                 "ea_batch_plan_info", "ea_batch_plan_current", "ea_batch_set_width",
                 "ea_batch_autotune", "ea_batch_sweep_each", "ea_batch_set_wait_limit",
                 "ea_batch_inject_stall", "ea_server_create", "ea_submit",
                 "ea_poll", "ea_server_stats_get", "ea_tp_create", "ea_tp_sweep", "ea_tp_read",
                 "ea_tp_info", "ea_tp_set_split"):
        getattr(lib, name).restype = i32
    if path == LIB_PATH:
        _lib = lib
    return lib


def _plan_dict(d: _PlanDesc) -> dict:
    return {"form": PLAN_FORMS.get(d.form, d.form), "threads": d.threads,
            "group_threads": d.group_threads, "lattices_per_cta": d.lattices_per_cta,
            "smem_bytes": d.smem_bytes, "units_per_cta": d.units_per_cta}


def _check(rc: int, what: str):
    if rc != EA_OK:
        raise EAError(rc, what)


def _ptr(x):
    """Device or host address of a torch tensor / numpy array, or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def ea_build_tables(betas, n_sites: int):
    """FP64 threshold tables (metro [NT][3], swapt [NT-1][swap_len]) as uint32 numpy arrays."""
    lib = load_library()
    betas = np.ascontiguousarray(betas, np.float64)
    nt = len(betas)
    metro = np.zeros((nt, 3), np.uint32)
    ln = ctypes.c_uint32(0)
    _check(lib.ea_build_tables(betas.ctypes.data, nt, n_sites, metro.ctypes.data, None, 0,
                               ctypes.byref(ln)), "ea_build_tables")
    swapt = np.zeros((max(nt - 1, 0), ln.value), np.uint32)
    if swapt.size:
        _check(lib.ea_build_tables(betas.ctypes.data, nt, n_sites, None, swapt.ctypes.data,
                                   ln.value, ctypes.byref(ln)), "ea_build_tables")
    return metro, swapt


def ea_build_tables_field(betas, n_sites: int, h_num: int, h_den: int):
    """Field tables for h = h_num / h_den: metro [NT][2][7] uint64 (2^32 = always) and
    swapt [NT-1][swap_len] uint32 in steps of gcd(4 h_den, 2 |h_num|) of Et."""
    lib = load_library()
    betas = np.ascontiguousarray(betas, np.float64)
    nt = len(betas)
    metro = np.zeros((nt, 2, 7), np.uint64)
    ln = ctypes.c_uint32(0)
    _check(lib.ea_build_tables_field(betas.ctypes.data, nt, n_sites, int(h_num), int(h_den),
                                     metro.ctypes.data, None, 0, ctypes.byref(ln)), "ea_build_tables_field")
    swapt = np.zeros((max(nt - 1, 0), ln.value), np.uint32)
    if swapt.size:
        _check(lib.ea_build_tables_field(betas.ctypes.data, nt, n_sites, int(h_num), int(h_den), None,
                                         swapt.ctypes.data, ln.value, ctypes.byref(ln)),
               "ea_build_tables_field")
    return metro, swapt


def ea_supported_L(L: int) -> bool:
    return bool(load_library().ea_supported_L(L))


def _config(L, G, NT, C, seed, bonds, spins, metro, swapt, group_base=0):
    if metro is None:   # field ensembles: the field carries the Metropolis table
        metro = np.zeros((0, 3), np.uint32)
    keep = [np.ascontiguousarray(a, np.uint32) for a in (bonds, spins, metro, swapt)]
    b, s, m, w = keep
    N = L ** 3
    assert b.shape == (G, 3, N) and s.shape == (G, NT, C, N) and m.shape in ((NT, 3), (0, 3))
    cfg = _Config(L, G, NT, C, int(seed), b.ctypes.data, s.ctypes.data, m.ctypes.data if m.size else None,
                  w.ctypes.data if w.size else None, w.shape[1] if w.ndim == 2 else 0, int(group_base))
    return cfg, keep


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream, stream


class Ensemble:
    """One simulated ensemble (an ea_ctx): G word-groups x NT slots x C copies of an L^3 lattice.

    field=(h_num, h_den, metro_field) runs it in the external field h = h_num / h_den
    (ea_create_field); metro is then unused and swapt is the field swap table.
    group_base: global index of group 0 in the random-number counters, so that
    groups [group_base, group_base + G) of a larger ensemble run exactly as they
    would inside it."""

    def __init__(self, L, G, NT, C, seed, bonds, spins, metro, swapt, stream=None, field=None,
                 group_base=0):
        import torch
        self.lib = load_library()
        self.L, self.G, self.NT, self.C = int(L), int(G), int(NT), int(C)
        self.N = self.L ** 3
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.handle, self.stream = _stream_handle(stream)
        cfg, _keep = _config(self.L, self.G, self.NT, self.C, seed, bonds, spins, metro, swapt,
                             group_base)
        self.group_base = int(group_base)
        self.swap_len = cfg.swap_len
        h = ctypes.c_void_p(None)
        if field is None:
            _check(self.lib.ea_create(ctypes.byref(cfg), self.handle, ctypes.byref(h)), "ea_create")
        else:
            h_num, h_den, mf = field
            mf = np.ascontiguousarray(mf, np.uint64)
            assert mf.shape == (self.NT, 2, 7)
            fld = _Field(int(h_num), int(h_den), mf.ctypes.data)
            _check(self.lib.ea_create_field(ctypes.byref(cfg), ctypes.byref(fld), self.handle,
                                            ctypes.byref(h)), "ea_create_field")
        self.ctx = h

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ea_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- counters
    @property
    def counters(self):
        s, p = ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(self.lib.ea_get_counters(self.ctx, ctypes.byref(s), ctypes.byref(p)), "ea_get_counters")
        return s.value, p.value

    @property
    def sweep_index(self) -> int:
        return self.counters[0]

    @property
    def pass_index(self) -> int:
        return self.counters[1]

    @property
    def launches(self) -> int:
        return int(self.lib.ea_launch_count(self.ctx))

    def n_passes(self, n_sweeps: int, swap_every: int) -> int:
        if swap_every <= 0:
            return 0
        s0 = self.sweep_index
        return (s0 + n_sweeps) // swap_every - s0 // swap_every

    def _empty(self, shape, dtype):
        import torch
        return torch.empty(shape, dtype=dtype, device=self.device)

    # -- the C ABI calls
    def sweep(self, n_sweeps, swap_every, energy_log=False, swap_log=False, qhist=None, esum=None,
              measure_from=0, measure_every=0):
        """Runs sweeps; returns dict of requested device logs.  qhist/esum tensors accumulate."""
        import torch
        out = {}
        elog = slog = None
        if energy_log:
            elog = self._empty((n_sweeps, self.G, self.NT, self.C, 32), torch.int32)
            out["energy_log"] = elog
        if swap_log:
            slog = self._empty((self.n_passes(n_sweeps, swap_every), self.G, self.C,
                                max(self.NT - 1, 0)), torch.int32)
            out["swap_log"] = slog
        args = _SweepArgs(int(n_sweeps), int(swap_every), _ptr(elog), _ptr(slog), _ptr(qhist),
                          _ptr(esum), int(measure_from), int(measure_every))
        _check(self.lib.ea_sweep(self.ctx, ctypes.byref(args)), "ea_sweep")
        return out

    def pt_swap(self):
        import torch
        masks = self._empty((self.G, self.C, max(self.NT - 1, 0)), torch.int32)
        _check(self.lib.ea_pt_swap(self.ctx, _ptr(masks) if masks.numel() else None), "ea_pt_swap")
        return masks

    def measure(self, energies=True, ndiff=False, qhist=None):
        import torch
        e = self._empty((self.G, self.NT, self.C, 32), torch.int32) if energies else None
        nd = self._empty((self.G, self.NT, 32), torch.int32) if ndiff else None
        _check(self.lib.ea_measure(self.ctx, _ptr(e), _ptr(nd), _ptr(qhist)), "ea_measure")
        return e, nd

    def measure_planes(self, mode: int):
        """Per-plane counts (ea_measure_planes): mode 0 -> int32 [G][NT][3][L][32] of
        sites where the copies differ; mode 1 -> [G][NT][C][3][L][32] of up spins."""
        import torch
        shape = ((self.G, self.NT, 3, self.L, 32) if mode == 0
                 else (self.G, self.NT, self.C, 3, self.L, 32))
        out = self._empty(shape, torch.int32)
        _check(self.lib.ea_measure_planes(self.ctx, int(mode), _ptr(out)), "ea_measure_planes")
        return out

    def magnetisations(self):
        """M = sum_i S_i of every lattice by slot (ea_magnetisations): int32 [G][NT][C][32]."""
        import torch
        out = self._empty((self.G, self.NT, self.C, 32), torch.int32)
        _check(self.lib.ea_magnetisations(self.ctx, _ptr(out)), "ea_magnetisations")
        return out

    def read_spins(self, out=None):
        import torch
        if out is None:
            out = self._empty((self.G, self.NT, self.C, self.N), torch.int32)
        _check(self.lib.ea_read_spins(self.ctx, _ptr(out)), "ea_read_spins")
        return out

    def read_spins_host(self) -> np.ndarray:
        out = np.zeros((self.G, self.NT, self.C, self.N), np.uint32)
        _check(self.lib.ea_read_spins_host(self.ctx, out.ctypes.data), "ea_read_spins_host")
        return out

    def write_spins(self, spins_dev, sweep_index: int, pass_index: int):
        _check(self.lib.ea_write_spins(self.ctx, _ptr(spins_dev), int(sweep_index), int(pass_index)),
               "ea_write_spins")

    def sync(self):
        _check(self.lib.ea_sync(self.ctx), "ea_sync")

    # -- kernel plans and the autotuner
    def plans(self) -> list[dict]:
        out = []
        for i in range(self.lib.ea_plan_count(self.ctx)):
            d = _PlanDesc()
            _check(self.lib.ea_plan_info(self.ctx, i, ctypes.byref(d)), "ea_plan_info")
            out.append(_plan_dict(d))
        return out

    @property
    def plan(self) -> int:
        return int(self.lib.ea_plan_current(self.ctx))

    def select_plan(self, index: int):
        _check(self.lib.ea_plan_select(self.ctx, int(index)), "ea_plan_select")

    def autotune(self, probe_sweeps: int = 200, swap_every: int = 1) -> list[float]:
        """Times every plan from the current state (restored after each run), selects the fastest."""
        n = self.lib.ea_plan_count(self.ctx)
        ms = (ctypes.c_float * n)()
        _check(self.lib.ea_autotune(self.ctx, int(probe_sweeps), int(swap_every), ms), "ea_autotune")
        return list(ms)


class Batch:
    """Several ensembles advanced together by one persistent launch (ea_batch_*).

    Members keep their own state and counters; after ``sweep(n, k)`` each is
    exactly where ``member.sweep(n, k)`` alone would have left it."""

    def __init__(self, ensembles=(), stream=None):
        self.lib = load_library()
        self.handle, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p(None)
        _check(self.lib.ea_batch_create(self.handle, ctypes.byref(h)), "ea_batch_create")
        self.b = h
        self.members = []
        for e in ensembles:
            self.add(e)

    def add(self, ens: Ensemble):
        _check(self.lib.ea_batch_add(self.b, ens.ctx), "ea_batch_add")
        self.members.append(ens)

    def clear(self):
        _check(self.lib.ea_batch_clear(self.b), "ea_batch_clear")
        self.members = []

    def plans(self, member: int) -> list[dict]:
        """The member's batch plans (its own list for the batch kernel)."""
        n = self.lib.ea_batch_plan_count(self.b, int(member))
        if n < 0:
            raise EAError(n, "ea_batch_plan_count")
        out = []
        for i in range(n):
            d = _PlanDesc()
            _check(self.lib.ea_batch_plan_info(self.b, int(member), i, ctypes.byref(d)),
                   "ea_batch_plan_info")
            out.append(_plan_dict(d))
        return out

    def plan(self, member: int) -> int:
        r = self.lib.ea_batch_plan_current(self.b, int(member))
        if r < -1:
            raise EAError(r, "ea_batch_plan_current")
        return int(r)

    def set_plan(self, member: int, plan_index: int):
        _check(self.lib.ea_batch_set_plan(self.b, int(member), int(plan_index)), "ea_batch_set_plan")

    def set_wait_limit(self, naps: int):
        _check(self.lib.ea_batch_set_wait_limit(self.b, int(naps)), "ea_batch_set_wait_limit")

    def inject_stall(self):
        _check(self.lib.ea_batch_inject_stall(self.b), "ea_batch_inject_stall")

    def set_width(self, threads: int):
        _check(self.lib.ea_batch_set_width(self.b, int(threads)), "ea_batch_set_width")

    def autotune(self, probe_sweeps: int = 100, swap_every: int = 10) -> float:
        """Times plan choices on the whole batch (state restored); keeps the fastest."""
        ms = ctypes.c_float(0.0)
        _check(self.lib.ea_batch_autotune(self.b, int(probe_sweeps), int(swap_every),
                                          ctypes.byref(ms)), "ea_batch_autotune")
        return float(ms.value)

    def set_segment(self, site_words: int):
        _check(self.lib.ea_batch_set_segment(self.b, int(site_words)), "ea_batch_set_segment")

    def sweep(self, n_sweeps: int, swap_every: int):
        _check(self.lib.ea_batch_sweep(self.b, int(n_sweeps), int(swap_every)), "ea_batch_sweep")

    def sweep_each(self, n_sweeps, swap_every):
        """Member i advances n_sweeps[i] sweeps (0: not this call), swap every swap_every[i]."""
        n = np.ascontiguousarray(n_sweeps, dtype=np.uint32)
        k = np.ascontiguousarray(swap_every, dtype=np.uint32)
        assert n.shape == k.shape == (len(self.members),)
        _check(self.lib.ea_batch_sweep_each(self.b, n.ctypes.data, k.ctypes.data), "ea_batch_sweep_each")

    def sync(self):
        _check(self.lib.ea_batch_sync(self.b), "ea_batch_sync")

    @property
    def launches(self) -> int:
        return int(self.lib.ea_batch_launch_count(self.b))

    def close(self):
        if getattr(self, "b", None):
            self.lib.ea_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop (ea_server_*): requests are admitted by device memory, kept
    resident and advanced together in batched rounds; results land in host arrays."""

    def __init__(self, mem_budget: int = 0, max_live: int = 0, round_ms: int = 0):
        self.lib = load_library()
        opts = _ServerOpts(int(mem_budget), int(max_live), int(round_ms))
        h = ctypes.c_void_p(None)
        _check(self.lib.ea_server_create(ctypes.byref(opts), ctypes.byref(h)), "ea_server_create")
        self.s = h
        self._out = {}          # ticket -> (outputs dict, inputs kept alive)

    def submit(self, L, G, NT, C, seed, bonds, spins, metro, swapt, n_sweeps, swap_every,
               want_spins=True, want_energies=True, group_base=0, field=None) -> int:
        """field=(h_num, h_den, metro_field) submits the request in that external
        field (ea_submit_field); its outputs then include "magnetisations"."""
        cfg, keep = _config(L, G, NT, C, seed, bonds, spins, metro, swapt, group_base)
        N = int(L) ** 3
        in_field = field is not None and int(field[0]) != 0
        out = {"spins": np.zeros((G, NT, C, N), np.uint32) if want_spins else None,
               "energies": np.zeros((G, NT, C, 32), np.int32) if want_energies else None,
               "magnetisations": np.zeros((G, NT, C, 32), np.int32) if in_field else None}
        req = _Request(int(n_sweeps), int(swap_every), _ptr(out["spins"]), _ptr(out["energies"]),
                       _ptr(out["magnetisations"]))
        t = ctypes.c_uint64(0)
        if field is None:
            _check(self.lib.ea_submit(self.s, ctypes.byref(cfg), ctypes.byref(req), ctypes.byref(t)),
                   "ea_submit")
        else:
            h_num, h_den, mf = field
            mf = np.ascontiguousarray(mf, np.uint64)
            assert mf.shape == (NT, 2, 7)
            fld = _Field(int(h_num), int(h_den), mf.ctypes.data)
            _check(self.lib.ea_submit_field(self.s, ctypes.byref(cfg), ctypes.byref(fld), ctypes.byref(req),
                                            ctypes.byref(t)), "ea_submit_field")
        self._out[t.value] = out
        return t.value

    def submit_tp(self, L, R, NT, C, seed, bonds, spins, metro, swapt, n_sweeps, swap_every,
                  want_spins=True, want_energies=True, real_base=0) -> int:
        """A temperature-packed request (ea_submit_tp; inputs as TPEnsemble).  Its
        outputs: "spins" [R][C][N] ([R][C][W][N] for NT > 32) uint32 words, bit t =
        slot t, and "energies" [R][NT][C] int32."""
        N = int(L) ** 3
        W = max(1, -(-int(NT) // 32))
        b = np.ascontiguousarray(bonds, np.uint8)
        sp = np.ascontiguousarray(spins, np.uint32)
        m = np.ascontiguousarray(metro, np.uint32)
        w = np.ascontiguousarray(swapt, np.uint32)
        shape = (R, C, N) if W == 1 else (R, C, W, N)
        if b.shape != (R, 3, N) or sp.shape != shape or m.shape != (NT, 3):
            raise ValueError("submit_tp: bonds [R][3][N] uint8, spins [R][C](W)[N], metro [NT][3]")
        swap_len = w.shape[1] if w.ndim == 2 else 0
        cfg = _TpConfig(int(L), int(R), int(NT), int(C), int(seed), b.ctypes.data, sp.ctypes.data,
                        m.ctypes.data, w.ctypes.data if w.size else None, swap_len, int(real_base))
        out = {"spins": np.zeros(shape, np.uint32) if want_spins else None,
               "energies": np.zeros((R, NT, C), np.int32) if want_energies else None}
        req = _TpRequest(int(n_sweeps), int(swap_every), _ptr(out["spins"]), _ptr(out["energies"]))
        t = ctypes.c_uint64(0)
        _check(self.lib.ea_submit_tp(self.s, ctypes.byref(cfg), ctypes.byref(req), ctypes.byref(t)),
               "ea_submit_tp")
        self._out[t.value] = out
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0):
        """None while pending; the outputs dict when done; raises on a failed request."""
        rc = self.lib.ea_poll(self.s, int(ticket), int(timeout_us))
        if rc == EA_PENDING:
            return None
        out = self._out.pop(int(ticket), None)
        _check(rc, f"request {ticket}")
        return out

    def wait(self, ticket: int, timeout_s: float = 600.0):
        import time
        end = time.monotonic() + timeout_s
        while True:
            r = self.poll(ticket, 100_000)
            if r is not None:
                return r
            if time.monotonic() > end:
                raise TimeoutError(f"request {ticket} still pending")

    def stats(self) -> dict:
        st = _ServerStats()
        _check(self.lib.ea_server_stats_get(self.s, ctypes.byref(st)), "ea_server_stats_get")
        return {name: getattr(st, name) for name, _ in _ServerStats._fields_}

    def close(self):
        if getattr(self, "s", None):
            self.lib.ea_server_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ea_run(L, G, NT, C, seed, bonds, spins, metro, swapt, n_sweeps, swap_every, measure_from=0,
           measure_every=0, want_spins=True, want_qhist=False, want_esum=False, host_out=None,
           stream=None, group_base=0):
    """Host-buffer entry point: host arrays in, host arrays out (ea_run)."""
    lib = load_library()
    handle, _ = _stream_handle(stream)
    cfg, _keep = _config(L, G, NT, C, seed, bonds, spins, metro, swapt, group_base)
    N = L ** 3
    ho = host_out or {}
    energies = ho.get("energies", np.zeros((G, NT, C, 32), np.int32))
    sp = ho.get("spins", np.zeros((G, NT, C, N), np.uint32)) if want_spins else None
    qh = ho.get("qhist", np.zeros((NT, N + 1), np.uint64)) if want_qhist else None
    es = ho.get("esum", np.zeros(NT, np.int64)) if want_esum else None
    args = _SweepArgs(int(n_sweeps), int(swap_every), None, None, None, None, int(measure_from),
                      int(measure_every))
    _check(lib.ea_run(ctypes.byref(cfg), ctypes.byref(args), handle, _ptr(energies), _ptr(sp),
                      _ptr(qh), _ptr(es)), "ea_run")
    return {"energies": energies, "spins": sp, "qhist": qh, "esum": es}


def _check_static_args(spins, energies, swapt, L, G, NT, C, masks):
    """Shapes, dtypes and devices of ea_pt_swap_static's tensors, checked before
    anything reaches the GPU: the kernels index every buffer by (L, G, NT, C)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else None
    N = int(L) ** 3
    want = {"spins": (spins, G * NT * C * N), "energies": (energies, G * NT * C * 32)}
    if masks is not None:
        want["masks"] = (masks, G * C * max(NT - 1, 0))
    if swapt is not None:
        want["swapt"] = (swapt, None)
    for name, (t, numel) in want.items():
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name} must be a torch tensor on the current CUDA device")
        if not t.is_cuda or t.device != dev:
            raise ValueError(f"{name} must live on the current CUDA device, not {t.device}")
        if not t.is_contiguous() or t.element_size() != 4:
            raise ValueError(f"{name} must be contiguous with 4-byte elements")
        if numel is not None and t.numel() != numel:
            raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    if swapt is not None and (swapt.dim() != 2 or swapt.shape[0] != NT - 1):
        raise ValueError(f"swapt must be [NT-1][swap_len] = [{NT - 1}][...], got {tuple(swapt.shape)}")


def ea_pt_swap_static(spins, energies, swapt, L, n_groups, n_temps, n_copies, seed, pass_index,
                      masks=None, stream=None):
    """Allocation-free replica-exchange pass on caller-owned device tensors (in place).

    spins: int32/uint32 device tensor [G][NT][C][N]; energies: int32 [G][NT][C][32];
    swapt: device tensor [NT-1][swap_len]; masks: optional int32 [G][C][NT-1].
    Raises ValueError, before any launch, for a tensor of the wrong size, dtype
    width or device."""
    _check_static_args(spins, energies, swapt, int(L), int(n_groups), int(n_temps), int(n_copies),
                       masks)
    lib = load_library()
    handle, _ = _stream_handle(stream)
    swap_len = int(swapt.shape[1]) if swapt is not None and swapt.dim() == 2 else 0
    _check(lib.ea_pt_swap_static(_ptr(spins), _ptr(energies),
                                 _ptr(swapt) if swap_len else None, swap_len, int(L),
                                 int(n_groups), int(n_temps), int(n_copies), int(seed),
                                 int(pass_index), _ptr(masks), handle), "ea_pt_swap_static")


class TPEnsemble:
    """Temperature-packed ensemble (an ea_tp): R realizations x C copies of an L^3
    lattice, W = ceil(NT / 32) words per (realization, copy, site) with bit b of
    word w = temperature slot 32 w + b (NT <= 64).  Realization r draws the random
    numbers of word-group r of the realization-packed form (its bit 0), so it
    follows the trajectory of realization 32r of an Ensemble with the same inputs.

    bonds: [R][3][N] uint8 (1 <=> J = -1); spins: [R][C][N] uint32 (bit t = slot t)
    when W = 1, [R][C][W][N] otherwise.  real_base: global index of realization 0
    in the random-number counters."""

    def __init__(self, L, R, NT, C, seed, bonds, spins, metro, swapt, stream=None, real_base=0):
        import torch
        self.lib = load_library()
        self.L, self.R, self.NT, self.C = int(L), int(R), int(NT), int(C)
        self.N = self.L ** 3
        self.W = max(1, -(-self.NT // 32))
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.handle, self.stream = _stream_handle(stream)
        b = np.ascontiguousarray(bonds, np.uint8)
        sp = np.ascontiguousarray(spins, np.uint32)
        m = np.ascontiguousarray(metro, np.uint32)
        w = np.ascontiguousarray(swapt, np.uint32)
        assert b.shape == (self.R, 3, self.N) and sp.shape == self._spin_shape()
        assert m.shape == (self.NT, 3)
        self.swap_len = w.shape[1] if w.ndim == 2 else 0
        cfg = _TpConfig(self.L, self.R, self.NT, self.C, int(seed), b.ctypes.data, sp.ctypes.data,
                        m.ctypes.data, w.ctypes.data if w.size else None, self.swap_len,
                        int(real_base))
        h = ctypes.c_void_p(None)
        _check(self.lib.ea_tp_create(ctypes.byref(cfg), self.handle, ctypes.byref(h)), "ea_tp_create")
        self.ctx = h

    def _spin_shape(self):
        return (self.R, self.C, self.N) if self.W == 1 else (self.R, self.C, self.W, self.N)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.ea_tp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _info(self):
        s, p, n, k = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint32(0)
        _check(self.lib.ea_tp_info(self.ctx, ctypes.byref(s), ctypes.byref(p), ctypes.byref(n),
                                   ctypes.byref(k)), "ea_tp_info")
        return s.value, p.value, n.value, k.value

    @property
    def split(self) -> int:
        """Slot groups (CTAs) per (realization, copy) unit, over all its words."""
        return self._info()[3]

    def set_split(self, k: int):
        """ea_tp_set_split: k slot groups per word of a unit (a power of two <= min(32, NT))."""
        _check(self.lib.ea_tp_set_split(self.ctx, int(k)), "ea_tp_set_split")

    @property
    def sweep_index(self) -> int:
        return self._info()[0]

    @property
    def pass_index(self) -> int:
        return self._info()[1]

    @property
    def launches(self) -> int:
        return self._info()[2]

    def n_passes(self, n_sweeps: int, swap_every: int) -> int:
        if swap_every <= 0:
            return 0
        s0 = self.sweep_index
        return (s0 + n_sweeps) // swap_every - s0 // swap_every

    def sweep(self, n_sweeps: int, swap_every: int, energy_log=False, swap_log=False) -> dict:
        """ea_tp_sweep; returns the requested logs as device tensors:
        energy_log [n][R][NT][C] int32, swap_log [passes][R][C] int32 (bit p = pair p)
        when W = 1, [passes][R][C][W] (bit b of word w = pair 32 w + b) otherwise."""
        import torch
        out = {}
        el = sl = None
        if energy_log:
            el = torch.empty((n_sweeps, self.R, self.NT, self.C), dtype=torch.int32, device=self.device)
            out["energy_log"] = el
        if swap_log:
            shape = (self.n_passes(n_sweeps, swap_every), self.R, self.C) + ((self.W,) if self.W > 1 else ())
            sl = torch.zeros(shape, dtype=torch.int32, device=self.device)
            out["swap_log"] = sl
        _check(self.lib.ea_tp_sweep(self.ctx, int(n_sweeps), int(swap_every), _ptr(el),
                                    _ptr(sl) if sl is not None and sl.numel() else None), "ea_tp_sweep")
        return out

    def read(self):
        """(spins [R][C][N] ([R][C][W][N] when W > 1) int32 view of the words,
        energies [R][NT][C] int32), device tensors."""
        import torch
        sp = torch.empty(self._spin_shape(), dtype=torch.int32, device=self.device)
        en = torch.empty((self.R, self.NT, self.C), dtype=torch.int32, device=self.device)
        _check(self.lib.ea_tp_read(self.ctx, _ptr(sp), _ptr(en)), "ea_tp_read")
        return sp, en
