"""The C ABI library builds, loads and exports every function declared in include/snac.h; host-side
validation of block layouts (no GPU needed: these calls return before touching the device)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2106_03583_gb300 import build, inputs, snac

from layouts import homogeneous_along, make

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return snac.lib()


def declared_functions():
    names = set()
    for h in ("snac.h", "snac_engine.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(snac_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(snac.EXPORTS)


def test_status_strings(lib):
    assert lib.snac_status_string(0) == b"ok"
    for code in range(-8, 0):
        assert lib.snac_status_string(code) not in (b"", b"unknown status")
    assert lib.snac_status_string(-99) == b"unknown status"


def _create(lib, blocks, homog=2, opt=None):
    arr, keep = snac._marshal_blocks(blocks)
    h = ctypes.c_void_p()
    st = lib.snac_plan_create(ctypes.byref(h), len(blocks), arr, homog, opt)
    return st, lib.snac_last_error_message().decode()


def test_layout_validation(lib):
    good = make("2x2", n=4, nz=8, zpair="NN")
    bad = [dict(b) for b in good]
    bad[0] = dict(bad[0], nbr=((-1, 2), (-1, 2), (-1, -1)))           # asymmetric connectivity
    st, msg = _create(lib, bad)
    assert st == -2 and "symmetric" in msg
    odd = make("1", n=4, nz=7, zpair="PP")
    st, msg = _create(lib, odd)
    assert st == -2 and "even" in msg
    nonuni = make("1", n=4, nz=8, zpair="NN")
    nonuni[0] = dict(nonuni[0], dx=(nonuni[0]["dx"][0], nonuni[0]["dx"][1], np.linspace(0.1, 0.2, 8)))
    st, msg = _create(lib, nonuni)
    assert st == -2 and "uniform" in msg
    cong = [dict(b) for b in make("1x2", n=4, nz=8, zpair="NN")]
    wy = cong[1]["dx"][1].copy()
    wy[0] *= 1.5
    cong[1] = dict(cong[1], dx=(cong[1]["dx"][0], wy, cong[1]["dx"][2]))
    st, msg = _create(lib, cong)
    assert st == -2 and "congruent" in msg
    st, _ = _create(lib, good, homog=0)     # split into blocks along x: x cannot be the homogeneous axis
    assert st == -2
    neg = [dict(good[0], dx=(-good[0]["dx"][0], good[0]["dx"][1], good[0]["dx"][2]))] + good[1:]
    st, _ = _create(lib, neg)
    assert st == -1


def test_null_arguments(lib):
    assert lib.snac_plan_create(None, 1, None, 2, None) == -1
    assert lib.snac_poisson_solve(None, None, None, 1e-10, None) == -1
    assert lib.snac_plan_info(None, None) == -1
    assert lib.snac_plan_destroy(None) == 0


def test_engine_argument_checks(lib):
    """Engine calls reject bad arguments before touching a device."""
    h = ctypes.c_void_p()
    for bad in ((0, 64, 10**9, 0, 16), (4, -1, 10**9, 0, 16), (4, 8, 0, 0, 16), (4, 8, 10**9, 2, 16),
                (4, 8, 10**9, 0, 0), (4, 8, 10**9, 0, 257)):
        opt = snac._EngineOptions(*bad)
        assert lib.snac_engine_create(ctypes.byref(h), ctypes.byref(opt)) == -1, bad
    assert lib.snac_engine_create(None, None) == -1
    t = ctypes.c_int64()
    assert lib.snac_engine_submit(None, 1, None, 2, None, None, None, 1e-10, ctypes.byref(t)) == -1
    assert lib.snac_engine_wait(None, 1, None, None) == -1
    assert lib.snac_engine_get_stats(None, None) == -1
    assert lib.snac_engine_destroy(None) == 0
    assert lib.snac_engine_clock() >= 0.0


def test_option_validation(lib):
    """Bad options are refused before any device work (including a positive Helmholtz shift)."""
    blocks = make("1", n=4, nz=8, zpair="NN")
    for kw in ({"shift": 1.0}, {"shift": float("nan")}, {"inner_reduction": 1.5}, {"nu1": 0, "nu2": 0},
               {"max_coarse": 1000}):
        o = dict(precision=0, nu1=2, nu2=2, max_outer=20, max_cycles=40, max_coarse=64, fused=-1,
                 inner_reduction=1e-3, shift=0.0)
        o.update(kw)
        opt = snac._Options(o["precision"], o["nu1"], o["nu2"], o["max_outer"], o["max_cycles"], o["max_coarse"],
                            o["fused"], o["inner_reduction"], o["shift"])
        st, msg = _create(lib, blocks, opt=ctypes.byref(opt))
        assert st == -1 and "options" in msg, (kw, st, msg)


def test_bottom_and_onchip_option_validation(lib):
    """onchip is 0 or -1; bottom_cells is 0, -1 or 16 .. 8192; refused before any device work."""
    blocks = make("1", n=4, nz=8, zpair="NN")
    for oc, bc, word in ((1, 0, "onchip"), (0, 5, "bottom_cells"), (0, 8193, "bottom_cells"),
                         (0, -2, "bottom_cells")):
        opt = snac._Options(0, 2, 2, 20, 40, 64, -1, 1e-3, 0.0, 0, 0, oc, bc)
        st, msg = _create(lib, blocks, opt=ctypes.byref(opt))
        assert st == -1 and word in msg, (oc, bc, st, msg)


def test_homogeneous_axis_validation(lib):
    """homog_axis is 0, 1 or 2; the chosen axis must be the one the blocks are not split along."""
    blocks = make("L", n=4, nz=6, zpair="DN", walls=("D", "N", "N", "N"))
    f = np.zeros(inputs.total_cells(blocks))
    st, msg = _create(lib, blocks, homog=3)
    assert st == -1 and "homog_axis" in msg
    relabelled, _, _ = homogeneous_along(blocks, f, 0)     # homogeneous direction now along caller x
    st, msg = _create(lib, relabelled, homog=2)             # caller z is split into blocks
    assert st == -2
    st, msg = _create(lib, relabelled, homog=1)
    assert st == -2


def test_autotune_argument_checks(lib):
    blocks = make("1", n=4, nz=8, zpair="NN")
    arr, keep = snac._marshal_blocks(blocks)
    best = snac._Options()
    assert lib.snac_autotune(0, arr, 2, None, ctypes.c_void_p(8), 1e-10, ctypes.byref(best), None, None) == -1
    assert lib.snac_autotune(1, arr, 2, None, None, 1e-10, ctypes.byref(best), None, None) == -1
    assert lib.snac_autotune(1, arr, 2, None, ctypes.c_void_p(8), 0.0, ctypes.byref(best), None, None) == -1
    assert lib.snac_autotune(1, arr, 5, None, ctypes.c_void_p(8), 1e-10, ctypes.byref(best), None, None) == -1


def test_wavenumber_range_validation(lib):
    """mode_begin/mode_end outside 0 <= begin < end <= n_z are refused before any device work."""
    blocks = make("1", n=4, nz=8, zpair="NN")
    for rng in ((3, 3), (-1, 2), (2, 9), (5, 4)):
        opt = snac._Options(0, 2, 2, 20, 40, 64, -1, 1e-3, 0.0, rng[0], rng[1])
        st, msg = _create(lib, blocks, opt=ctypes.byref(opt))
        assert st == -1 and "mode_begin" in msg, (rng, st, msg)


def test_pencil_calls_check_their_arguments(lib):
    assert lib.snac_pencil_forward(None, 4, None, None, None) == -1
    assert lib.snac_pencil_backward_update(None, 4, None, None, None) == -1
    n = ctypes.c_int64()
    assert lib.snac_pencil_setup(None, 0, 4, None, 0, ctypes.byref(n)) == -1
    assert lib.snac_pencil_residual(None, None, None, None, 0.0, None, None) == -1
    assert lib.snac_mode_solve(None, None, None, 1.0, None) == -1
    assert lib.snac_mode_fix_mean(None, None, 0.0, None) == -1
