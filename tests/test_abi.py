"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point include/ea.h declares, and its host-only pieces (threshold
tables, argument validation) behave as documented."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1311_5582_gb300 as ea
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ea.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ea_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ea.load_library()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(ea.EXPORTS)


def test_library_is_built_for_sm_103a():
    import subprocess
    out = subprocess.run(["cuobjdump", "--list-elf", ea.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


@pytest.mark.parametrize("nt,tmin,tmax,L", [(16, 0.8, 2.0, 4), (24, 0.9, 2.0, 8), (32, 0.95, 2.0, 16),
                                            (32, 0.95, 2.0, 32), (1, 1.0, 1.0, 6), (20, 0.8, 2.0, 10)])
def test_tables_match_oracle_bit_for_bit(nt, tmin, tmax, L):
    betas = W.geometric_ladder(nt, tmin, tmax)
    m, s = ea.ea_build_tables(betas, L ** 3)
    np.testing.assert_array_equal(m, oracle.metro_table(betas))
    np.testing.assert_array_equal(s, oracle.swap_table_trimmed(betas, L ** 3))


def test_table_builder_rejects_bad_ladders():
    with pytest.raises(ea.EAError):
        ea.ea_build_tables(np.array([0.5, 1.0]), 64)      # increasing beta
    with pytest.raises(ea.EAError):
        ea.ea_build_tables(np.array([-1.0]), 64)


def test_supported_sizes_and_strerror():
    for L in (4, 6, 8, 10, 12, 14, 16, 20, 24, 32):
        assert ea.ea_supported_L(L)
    for L in (2, 3, 5, 18, 64):
        assert not ea.ea_supported_L(L)
    lib = ea.load_library()
    assert lib.ea_strerror(-1) == b"invalid argument"


def _cfg(**over):
    inst = W.Instance(L=4, G=1, NT=4, C=2, seed=1, tmin=1.0, tmax=2.0, input_seed=1)
    inp = W.draw_inputs(inst)
    m, s = ea.ea_build_tables(inp["betas"], 64)
    arrays = dict(bonds=inp["bonds"], spins=inp["spins"], metro=m, swapt=s)
    arrays.update({k: v for k, v in over.items() if k in arrays})
    dims = dict(L=4, G=1, NT=4, C=2)
    dims.update({k: v for k, v in over.items() if k in dims})
    cfg, keep = ea._config(dims["L"], dims["G"], dims["NT"], dims["C"], 1, arrays["bonds"],
                           arrays["spins"], arrays["metro"], arrays["swapt"])
    return cfg, keep


def _create_rc(cfg):
    lib = ea.load_library()
    h = ctypes.c_void_p(None)
    return lib.ea_create(ctypes.byref(cfg), None, ctypes.byref(h))


def test_create_validates_arguments_before_touching_the_device():
    cfg, keep = _cfg()
    bad = []
    c = ea._Config.from_buffer_copy(cfg); c.L = 5; bad.append((c, -1))
    c = ea._Config.from_buffer_copy(cfg); c.L = 18; bad.append((c, -5))
    c = ea._Config.from_buffer_copy(cfg); c.n_copies = 3; bad.append((c, -1))
    c = ea._Config.from_buffer_copy(cfg); c.n_temps = 65; bad.append((c, -1))
    c = ea._Config.from_buffer_copy(cfg); c.bonds = None; bad.append((c, -1))
    c = ea._Config.from_buffer_copy(cfg); c.group_base = 2**32 - 1; c.n_groups = 2; bad.append((c, -1))
    for c, want in bad:
        assert _create_rc(c) == want
    # non-monotone Metropolis row
    m = keep[2].copy(); m[0] = [5, 4, 3]
    cfg2, keep2 = _cfg(metro=m)
    assert _create_rc(cfg2) == -1
    # increasing swap row
    s = keep[3].copy(); s[0, 1] = s[0, 0] + 1 if s[0, 0] < 2**32 - 1 else s[0, 0]; s[0, 0] = 0
    cfg3, keep3 = _cfg(swapt=s)
    assert _create_rc(cfg3) == -1


def test_null_context_calls_fail_cleanly():
    lib = ea.load_library()
    assert lib.ea_sweep(None, None) == -1
    assert lib.ea_pt_swap(None, None) == -1
    assert lib.ea_measure(None, None, None, None) == -1
    assert lib.ea_sync(None) == -1
    lib.ea_destroy(None)


@pytest.mark.parametrize("h_num,h_den,nt,L", [(1, 2, 8, 4), (-3, 4, 16, 8), (7, 1, 12, 6), (5, 3, 32, 16),
                                              (1, 10, 24, 32), (0, 1, 6, 4)])
def test_field_tables_match_oracle_bit_for_bit(h_num, h_den, nt, L):
    betas = W.geometric_ladder(nt, 0.8, 2.0)
    m, s = ea.ea_build_tables_field(betas, L ** 3, h_num, h_den)
    np.testing.assert_array_equal(m, oracle.metro_table_field(betas, h_num, h_den))
    np.testing.assert_array_equal(s, oracle.swap_table_field_trimmed(betas, L ** 3, h_num, h_den))


def test_field_builder_and_create_reject_bad_fields():
    betas = W.geometric_ladder(4, 1.0, 2.0)
    with pytest.raises(ea.EAError):
        ea.ea_build_tables_field(betas, 64, 1, 0)              # h_den < 1
    with pytest.raises(ea.EAError):
        ea.ea_build_tables_field(betas, 64, 1 << 15, 1)        # Et would overflow int32
    lib = ea.load_library()
    cfg, keep = _cfg()
    mf, sw = ea.ea_build_tables_field(betas, 64, 1, 2)

    def rc(h_num, h_den, table):
        t = np.ascontiguousarray(table, np.uint64)
        f = ea._Field(h_num, h_den, t.ctypes.data)
        h = ctypes.c_void_p(None)
        return lib.ea_create_field(ctypes.byref(cfg), ctypes.byref(f), None, ctypes.byref(h))

    bad = mf.copy(); bad[1, 0, 2], bad[1, 0, 3] = bad[1, 0, 3], bad[1, 0, 2]   # decreasing in u
    assert rc(1, 2, bad) == -1
    big = mf.copy(); big[0, 1, 6] = (1 << 32) + 1                              # above "always"
    assert rc(1, 2, big) == -1
    assert rc(1, 0, mf) == -1
    # h_num = 0 must carry the field-free table: both spin rows equal, 2^32 for u >= 3
    assert rc(0, 1, mf) == -1


def _tp_create(L=4, R=2, NT=4, C=2, metro=None, swapt=None, bonds=True, spins=True, real_base=0):
    lib = ea.load_library()
    N = L ** 3
    b = np.zeros((R, 3, N), np.uint8)
    s = np.zeros((R, C, N), np.uint32)
    betas = W.geometric_ladder(max(min(NT, 64), 1), 1.0, 2.0)
    m, w = ea.ea_build_tables(betas, N)
    m = m if metro is None else metro
    w = w if swapt is None else swapt
    cfg = ea._TpConfig(L, R, NT, C, 1, b.ctypes.data if bonds else None, s.ctypes.data if spins else None,
                       m.ctypes.data, w.ctypes.data if w.size else None, w.shape[1] if w.ndim == 2 else 0,
                       real_base)
    h = ctypes.c_void_p(None)
    return lib.ea_tp_create(ctypes.byref(cfg), None, ctypes.byref(h)), h


def test_tp_create_validates_arguments_before_touching_the_device():
    """The temperature-packed form rejects bad shapes and tables on the host."""
    assert _tp_create(NT=65)[0] == -1                    # more slots than two words hold
    assert _tp_create(NT=0)[0] == -1
    assert _tp_create(R=0)[0] == -1
    assert _tp_create(C=3)[0] == -1
    assert _tp_create(L=5)[0] == -1                      # odd L
    assert _tp_create(L=18)[0] == -5                     # even but not compiled
    assert _tp_create(bonds=False)[0] == -1
    assert _tp_create(spins=False)[0] == -1
    assert _tp_create(real_base=2**32 - 1)[0] == -1      # realizations past the 32-bit counter word
    bad = np.array([[5, 3, 9]] * 4, np.uint32)           # thresholds must not decrease in u
    assert _tp_create(metro=bad)[0] == -1
    w = ea.ea_build_tables(W.geometric_ladder(4, 1.0, 2.0), 64)[1].copy()
    w[0, :2] = [1, 2]                                    # swap rows must not increase in k
    assert _tp_create(swapt=w)[0] == -1
    lib = ea.load_library()
    assert lib.ea_tp_sweep(None, 1, 1, None, None) == -1
    assert lib.ea_tp_read(None, None, None) == -1
    assert lib.ea_tp_info(None, None, None, None, None) == -1
    assert lib.ea_tp_set_split(None, 1) == -1
    lib.ea_tp_destroy(None)


def test_static_pass_wrapper_rejects_bad_tensors_before_any_launch():
    """ea_pt_swap_static indexes its buffers by (L, G, NT, C): the binding refuses
    host tensors, wrong sizes, wrong element widths and a malformed table."""
    torch = pytest.importorskip("torch")
    L, G, NT, C = 4, 2, 3, 2
    N = L ** 3
    host = dict(spins=torch.zeros(G * NT * C * N, dtype=torch.int32),
                energies=torch.zeros(G * NT * C * 32, dtype=torch.int32),
                swapt=torch.zeros((NT - 1, 5), dtype=torch.int32))
    with pytest.raises(ValueError):
        ea.ea_pt_swap_static(host["spins"], host["energies"], host["swapt"], L, G, NT, C, 1, 0)
    if not torch.cuda.is_available():
        return
    dev = {k: v.cuda() for k, v in host.items()}
    bad = [
        dict(dev, spins=dev["spins"][:-1]),                              # one word short
        dict(dev, energies=dev["energies"].to(torch.int64)),             # 8-byte elements
        dict(dev, swapt=torch.zeros((NT, 5), dtype=torch.int32, device="cuda")),   # NT rows
        dict(dev, energies=host["energies"]),                            # host tensor
    ]
    for b in bad:
        with pytest.raises(ValueError):
            ea.ea_pt_swap_static(b["spins"], b["energies"], b["swapt"], L, G, NT, C, 1, 0)
    with pytest.raises(ValueError):
        ea.ea_pt_swap_static(dev["spins"], dev["energies"], dev["swapt"], L, G, NT, C, 1, 0,
                             masks=torch.zeros(3, dtype=torch.int32, device="cuda"))
