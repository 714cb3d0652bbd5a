"""CPU checks of the C-ABI library: it loads, exports every function that
include/fcn.h declares, and rejects invalid arguments before touching the
GPU.  No compute call is made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def fcn():
    from paper_1507_05988_gb300 import build
    build.build()
    from paper_1507_05988_gb300 import fcn as m
    return m


def _declared():
    names = []
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(fcn_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("fcn_create", "fcn_step", "fcn_get_field", "fcn_get_rho", "fcn_get_diag",
              "fcn_op_rows", "fcn_op_cn", "fcn_op_cn_table", "fcn_propagate"):
        assert n in names


def test_library_exports_every_declared_symbol(fcn):
    missing = [n for n in _declared() if not hasattr(fcn.lib, n)]
    assert not missing, missing
    assert fcn.fcn_version().decode().startswith("fcn-gb300")


def test_binding_uses_the_c_names(fcn):
    for n in _declared():
        assert callable(getattr(fcn, n)), n


@pytest.mark.parametrize("nr,nt,code", [(2, 64, -1), (16, 12, -1), (16, 16384, -5),
                                         (4096, 64, -5), (16, 1, -1)])
def test_create_rejects_bad_grids_without_gpu(fcn, nr, nt, code):
    g = fcn.make_grid(nr, nt, 1e-3, 1e-12)
    p = fcn.make_params()
    ctx = C.c_void_p()
    assert fcn.fcn_create(C.byref(g), C.byref(p), fcn.FCN_FP64, None, C.byref(ctx)) == code
    assert ctx.value is None
    assert len(fcn.fcn_last_error(None)) > 0


def test_ops_reject_bad_arguments_without_gpu(fcn):
    g = fcn.make_grid(8, 16, 1e-3, 1e-12)
    p = fcn.make_params()
    assert fcn.fcn_op_rows(C.byref(g), C.byref(p), 1, fcn.FCN_OP_FFT, 0.0, None, None, None) == -1
    assert fcn.fcn_op_rows(C.byref(g), C.byref(p), 7, fcn.FCN_OP_FFT, 0.0, None, None, None) == -1
    assert fcn.fcn_op_cn(C.byref(g), C.byref(p), 1, -1.0, None, None, None) == -1
    assert fcn.fcn_cn_table_entries(C.byref(g)) == 8 * 9
    bad = fcn.make_params(K=0)
    assert fcn.fcn_op_cn_table(C.byref(g), C.byref(bad), 1, 1e-3, None, None) == -1


def test_context_calls_reject_null_context(fcn):
    assert fcn.fcn_step(None, 1e-3, 1) == -1
    assert fcn.fcn_set_stream(None, None) == -1
    fcn.fcn_destroy(None)


@pytest.mark.parametrize("nx,ny,nt,xw,code", [(2, 8, 16, 1e-3, -1), (8, 2, 16, 1e-3, -1),
                                              (8, 8, 12, 1e-3, -1), (4096, 8, 16, 1e-3, -5),
                                              (8, 8, 16384, 1e-3, -5), (8, 8, 16, -1.0, -1)])
def test_xy_create_rejects_bad_grids_without_gpu(fcn, nx, ny, nt, xw, code):
    g = fcn.fcn_grid_xy(nx, ny, nt, 0, xw, 1e-3, 1e-12)
    p = fcn.make_params()
    ctx = C.c_void_p()
    assert fcn.fcn_xy_create(C.byref(g), C.byref(p), fcn.FCN_FP64, None, C.byref(ctx)) == code
    assert ctx.value is None
    assert len(fcn.fcn_xy_last_error(None)) > 0


def test_xy_calls_reject_null_context(fcn):
    assert fcn.fcn_xy_step(None, 1e-3, 1) == -1
    assert fcn.fcn_xy_get_diag(None, None) == -1
    assert fcn.fcn_xy_profile_read(None, None, None, 0) == -1
    fcn.fcn_xy_destroy(None)


def test_noalloc_column_stage_checks_arguments_like_the_others_without_gpu(fcn):
    """The allocation-free column stage validates through the same routine
    as fcn_op_cn, before any GPU work: an unknown flag, a non-finite k'', a
    photon number outside 1..16, a bad dz or pointer are FCN_ERR_ARG, and a
    grid beyond the library's range is FCN_ERR_UNSUPPORTED."""
    g = fcn.make_grid(8, 16, 1e-3, 1e-12)
    dummy = C.c_void_p(16)          # never dereferenced: the checks come first
    for bad in (fcn.make_params(k2=float("nan")), fcn.make_params(flags=1 << 10),
                fcn.make_params(K=0), fcn.make_params(K=17)):
        assert fcn.fcn_op_cn_noalloc(C.byref(g), C.byref(bad), 1, 1e-3, dummy, None) == -1
        assert fcn.fcn_op_cn(C.byref(g), C.byref(bad), 1, 1e-3, dummy, dummy, None) == -1
    p = fcn.make_params()
    assert fcn.fcn_op_cn_noalloc(C.byref(g), C.byref(p), 1, float("inf"), dummy, None) == -1
    assert fcn.fcn_op_cn_noalloc(C.byref(g), C.byref(p), 1, 1e-3, None, None) == -1
    assert fcn.fcn_op_cn_noalloc(C.byref(g), C.byref(p), 3, 1e-3, dummy, None) == -1
    big = fcn.make_grid(16, 16384, 1e-3, 1e-12)
    assert fcn.fcn_op_cn_noalloc(C.byref(big), C.byref(p), 1, 1e-3, dummy, None) == -5
