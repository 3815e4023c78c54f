"""The C-ABI library on a machine without a GPU: it builds, loads, exports
every symbol include/hh.h declares, and rejects bad arguments before any
device work (no compute call is made here)."""

import ctypes as ct
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="session")
def hh():
    from paper_1211_4752_gb300 import _binding as B, build
    if not B.lib_path().exists():
        build.build()
    return B


def declared_functions():
    text = (ROOT / "include" / "hh.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hh_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("hh_setup", "hh_solve", "hh_adjoint", "hh_grad_k2", "hh_destroy",
                 "hh_last_error", "hh_solve_host", "hh_apply"):
        assert need in names


def test_library_exports_every_declared_symbol(hh):
    lib = ct.CDLL(str(hh.lib_path()))
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in hh.SIGNATURES, name
    assert set(hh.SIGNATURES) == set(declared_functions())


def test_default_options(hh):
    L = hh.lib()
    o = hh.HHOptions()
    L.hh_default_options(ct.byref(o))
    assert (o.omega_re, o.omega_im, o.nu1, o.nu2, o.coarsest) == (0.8, 0.0, 1, 1, 4)
    assert o.precision == hh.HH_FP64 and o.max_cycles > 0
    s = hh.HHShift()
    L.hh_default_shift(ct.byref(s))
    assert s.form == hh.HH_FORM_CSL and abs(s.theta_max - 3.141592653589793 / 6) < 1e-15


@pytest.mark.parametrize("dim,n,lo,hi,angle", [
    (4, 64, 0, 0, 0.5),      # dim
    (2, 63, 0, 0, 0.5),      # not a power of two
    (2, 4, 0, 0, 0.5),       # too small
    (2, 64, 40, 30, 0.5),    # layers overlap
    (2, 64, -1, 0, 0.5),     # negative layer
    (2, 64, 4, 4, 2.0),      # ECS angle >= pi/2
    (3, 1024, 0, 0, 0.5),    # 3-D too large
])
def test_setup_rejects_bad_grids(hh, dim, n, lo, hi, angle):
    L = hh.lib()
    g = hh.HHGrid(dim, n, lo, hi, angle)
    h = ct.c_void_p()
    st = L.hh_setup(ct.byref(g), None, 100.0, None, None, 1, None, ct.byref(h))
    assert st == hh.HH_ERR_ARG
    assert h.value is None
    assert L.hh_last_error()


def test_setup_rejects_bad_options(hh):
    L = hh.lib()
    g = hh.HHGrid(2, 64, 0, 0, 0.5)
    for field, val in (("nu1", 0), ("coarsest", 8), ("precision", 7), ("max_cycles", 0),
                       ("inner_tol", 2.0)):
        o = hh.HHOptions()
        L.hh_default_options(ct.byref(o))
        setattr(o, field, val)
        h = ct.c_void_p()
        assert L.hh_setup(ct.byref(g), None, 1.0, None, ct.byref(o), 1, None, ct.byref(h)) == hh.HH_ERR_ARG
    h = ct.c_void_p()
    assert L.hh_setup(ct.byref(g), None, 1.0, None, None, 0, None, ct.byref(h)) == hh.HH_ERR_ARG


def test_calls_with_null_handle_fail_cleanly(hh):
    L = hh.lib()
    info = (hh.HHSolveInfo * 1)()
    assert L.hh_solve(None, None, None, 1, 1e-6, 0, info, None) == hh.HH_ERR_ARG
    assert L.hh_adjoint(None, None, None, 1, 1e-6, 0, info, None) == hh.HH_ERR_ARG
    assert L.hh_fgmres(None, None, None, 1, 1e-6, 10, 0, 0, info, None) == hh.HH_ERR_ARG
    assert L.hh_solve_group(None, 1, 1e-6, None) == hh.HH_ERR_ARG
    assert L.hh_solve_group(None, 0, 1e-6, None) == hh.HH_OK
    assert L.hh_destroy(None) == hh.HH_OK
    assert L.hh_num_levels(None) == 0
    assert L.hh_cycle_kernels(None) == 0
    assert L.hh_solve_kernels(None) == -1
    bx, by = ct.c_int(7), ct.c_int(7)
    assert L.hh_tile_shape(None, 0, ct.byref(bx), ct.byref(by)) == 0
    assert (bx.value, by.value) == (0, 0)


def test_python_layer_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1211_4752_gb300 import _binding as B
    monkeypatch.setattr(B, "_LIB_PATH", tmp_path / "missing.so")
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        B.lib()


def test_setup_rejects_bad_radiating_condition(hh):
    L = hh.lib()
    h = ct.c_void_p()
    for grid, field, k2 in ((hh.HHGrid(2, 64, 8, 8, 0.5, 1), None, 100.0),   # no end without a layer
                            (hh.HHGrid(2, 64, 0, 0, 0.5, 2), None, 100.0),   # bad flag
                            (hh.HHGrid(2, 64, 0, 0, 0.5, 1), None, 0.0),     # k = 0
                            (hh.HHGrid(2, 64, 0, 0, 0.5, 1), ct.c_void_p(8), 100.0)):  # k^2 field
        assert L.hh_setup(ct.byref(grid), field, k2, None, None, 1, None, ct.byref(h)) == hh.HH_ERR_ARG
        assert h.value is None
