"""The C-ABI library loads on a machine without a GPU and exports every
function that include/*.h declares; host-side argument checks reject bad
calls before any device work."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:int|void|size_t|double|unsigned long long|long long|const char\s*\*)\s+\**(\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def native():
    from paper_2010_05975_gb300 import build
    build.build()
    import paper_2010_05975_gb300 as g
    return g


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ["lu_factor", "lu_factor_ex", "lu_solve"]:
        assert n in names


def test_every_declared_symbol_is_exported(native):
    lib = native.library()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_errors_before_device_work(native):
    lib = native.library()
    s = ctypes.c_void_p(0)
    dummy = ctypes.c_void_p(16)
    assert lib.lu_factor(-1, dummy, 1, dummy, dummy, s) == -1
    assert lib.lu_factor(4, dummy, 3, dummy, dummy, s) == -3
    assert lib.lu_factor(4, None, 4, dummy, dummy, s) == -2
    assert lib.lu_factor(4, dummy, 4, None, dummy, s) == -4
    assert lib.lu_factor(4, dummy, 4, dummy, None, s) == -5
    opts = native._native.lu_opts(512, 128, 0)
    assert lib.lu_factor_ex(8, 8, dummy, 8, dummy, dummy, ctypes.byref(opts), s) == -7
    opts = native._native.lu_opts(32, 100000, 0)
    assert lib.lu_factor_ex(200000, 64, dummy, 64, dummy, dummy, ctypes.byref(opts), s) == -7
    assert lib.lu_solve(4, -1, dummy, 4, dummy, dummy, 1, s) == -2
    assert lib.lu_solve(4, 2, dummy, 4, dummy, dummy, 1, s) == -7


def test_python_layer_refuses_cpu_tensors(native):
    import torch
    with pytest.raises(TypeError):
        native.lu_factor(torch.zeros(4, 4, dtype=torch.float64))


def test_chol_argument_errors_before_device_work(native):
    lib = native.library()
    s = ctypes.c_void_p(0)
    dummy = ctypes.c_void_p(16)
    nat = native._native
    for fn in (lib.chol_factor, lib.chol_factor_f32):
        assert fn(-1, dummy, 1, dummy, None, s) == -1
        assert fn(4, None, 4, dummy, None, s) == -2
        assert fn(4, dummy, 3, dummy, None, s) == -3
        assert fn(4, dummy, 4, None, None, s) == -4
        assert fn(4, dummy, 4, dummy, ctypes.byref(nat.lu_opts(129, 0, 0)), s) == -5   # b > 128
        assert fn(4, dummy, 4, dummy, ctypes.byref(nat.lu_opts(64, 128, 0)), s) == -5  # h must be 0
        assert fn(4, dummy, 4, dummy, ctypes.byref(nat.lu_opts(-1, 0, 0)), s) == -5
    bad = nat.lu_opts(64, 0, nat.LU_PREC_BF16)
    assert lib.chol_factor(4, dummy, 4, dummy, ctypes.byref(bad), s) == -5
    assert lib.chol_factor_f32(4, dummy, 4, dummy, ctypes.byref(bad), s) == -5


def test_chol_solve_argument_errors(native):
    lib = native.library()
    s = ctypes.c_void_p(0)
    dummy = ctypes.c_void_p(16)
    for fn in (lib.chol_solve, lib.chol_solve_f32):
        assert fn(-1, 1, dummy, 1, dummy, 1, s) == -1
        assert fn(4, -1, dummy, 4, dummy, 1, s) == -2
        assert fn(4, 385, dummy, 4, dummy, 385, s) == -2
        assert fn(4, 1, None, 4, dummy, 1, s) == -3
        assert fn(4, 1, dummy, 3, dummy, 1, s) == -4
        assert fn(4, 1, dummy, 4, None, 1, s) == -5
        assert fn(4, 2, dummy, 4, dummy, 1, s) == -6
        assert fn(0, 0, None, 1, None, 1, s) == 0


def test_python_cholesky_refuses_bad_tensors(native):
    import torch
    with pytest.raises(TypeError):
        native.chol_factor(torch.zeros(4, 4, dtype=torch.float64))          # host tensor
    with pytest.raises(TypeError):
        native.chol_factor(torch.zeros(4, 4, dtype=torch.int32))
    with pytest.raises(TypeError):
        native.chol_solve(torch.zeros(4, 4, dtype=torch.float16), torch.zeros(4))
    with pytest.raises(TypeError):
        native.chol_solve(torch.zeros(4, 4, dtype=torch.float64), torch.zeros(4, dtype=torch.float64))


def test_host_factor_argument_errors(native):
    """lu_factor_host checks its host arguments before it allocates or copies."""
    lib = native.library()
    s = ctypes.c_void_p(0)
    dummy = ctypes.c_void_p(16)
    assert lib.lu_factor_host(-1, 4, dummy, 4, dummy, dummy, None, s) == -1
    assert lib.lu_factor_host(4, -1, dummy, 4, dummy, dummy, None, s) == -2
    assert lib.lu_factor_host(4, 4, None, 4, dummy, dummy, None, s) == -3
    assert lib.lu_factor_host(4, 4, dummy, 3, dummy, dummy, None, s) == -4
    assert lib.lu_factor_host(4, 4, dummy, 4, None, dummy, None, s) == -5
    assert lib.lu_factor_host(4, 4, dummy, 4, dummy, None, None, s) == -6
    bf16 = native._native.lu_opts(32, 128, native.LU_PREC_BF16)
    info = ctypes.c_int(7)
    assert lib.lu_factor_host(4, 4, dummy, 4, dummy, ctypes.byref(info), ctypes.byref(bf16), s) == \
        native.LU_EUNSUPPORTED
    # an empty matrix needs no device: info is set, nothing else happens
    assert lib.lu_factor_host(0, 0, None, 1, None, ctypes.byref(info), None, s) == 0
    assert info.value == 0


def test_wait_deadline_config_host_side(native):
    """The wait-deadline hook: argument checks, the 4 s default, a set value
    and its reset (host-side state only; no device work)."""
    lib = native.library()
    TC, SOLVE = native.LU_WAIT_SITE_TC, native.LU_WAIT_SITE_SOLVE
    assert lib.lu_test_wait_config(2, 0, 0) == -1
    assert lib.lu_test_wait_config(-1, 0, 0) == -1
    assert lib.lu_test_wait_config(TC, -5, 0) == -2
    assert lib.lu_test_wait_config(TC, 601 * 10 ** 9, 0) == -2
    assert lib.lu_test_wait_config(TC, 0, 2) == -3
    assert lib.lu_wait_deadline_ns(3) == -1
    assert lib.lu_wait_deadline_ns(TC) == 4 * 10 ** 9
    assert lib.lu_wait_deadline_ns(SOLVE) == 4 * 10 ** 9
    try:
        assert lib.lu_test_wait_config(SOLVE, 12345, 1) == 0
        assert lib.lu_wait_deadline_ns(SOLVE) == 12345
        assert lib.lu_wait_deadline_ns(TC) == 4 * 10 ** 9      # sites are independent
    finally:
        assert lib.lu_test_wait_config(SOLVE, 0, 0) == 0
    assert lib.lu_wait_deadline_ns(SOLVE) == 4 * 10 ** 9


def test_batched_width_table_host_side(native):
    """The batched size-class table: lookups, a replacement, its checks and
    the restore (host-side state only)."""
    import torch
    lib = native.library()
    F64, F32 = native.LU_PREC_F64, native.LU_PREC_F32
    assert lib.lu_batched_panel_width_dt(100, 7) == -2
    default = [native.batched_panel_width(n, torch.float32) for n in (20, 50, 100, 200, 400, 1000)]
    arr = (ctypes.c_int * 6)(8, 8, 16, 16, 32, 32)
    assert lib.lu_batched_set_panel_widths(9, arr, 6) == -1
    assert lib.lu_batched_set_panel_widths(F32, arr, 5) == -3
    bad = (ctypes.c_int * 6)(8, 8, 16, 16, 33, 32)
    assert lib.lu_batched_set_panel_widths(F32, bad, 6) == -2
    try:
        assert lib.lu_batched_set_panel_widths(F32, arr, 6) == 0
        got = [lib.lu_batched_panel_width_dt(n, F32) for n in (1, 32, 33, 64, 65, 128, 129, 256, 257, 512, 513, 1024)]
        assert got == [8, 8, 8, 8, 16, 16, 16, 16, 32, 32, 32, 32]
        # the binary64 table is separate
        assert lib.lu_batched_panel_width_dt(20, F64) == lib.lu_batched_panel_width(20)
    finally:
        assert lib.lu_batched_set_panel_widths(F32, None, 6) == 0
    assert [native.batched_panel_width(n, torch.float32) for n in (20, 50, 100, 200, 400, 1000)] == default
