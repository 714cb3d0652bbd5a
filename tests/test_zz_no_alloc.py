"""fcn_op_cn_noalloc: the Crank-Nicolson column stage for callers that cannot
allocate device memory (a framework's caching allocator owns the GPU, or a
loop must never block on cudaMalloc/cudaFree).  Its scratch lives in a
static device array inside the library.

Checked through the C-ABI against the regular entry points (fcn_op_cn_table
into a caller buffer + fcn_op_cn) on two calls in a row, with different dz,
so the second call runs on the array the first one left behind.  This file
is collected last and must pass both alone in a fresh process and after the
other GPU tests."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1507_05988_gb300 import workloads as W
from tests.conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}   # FP64, FP32-mixed (as in the column-stage parity tests)


@pytest.fixture(scope="module")
def fcn():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1507_05988_gb300 import build
    build.build()
    from paper_1507_05988_gb300 import fcn as m
    return m


def _reference(fcn, g, p, prec, dz, f):
    ent = fcn.fcn_cn_table_entries(C.byref(g))
    table = torch.zeros(ent, dtype=f.dtype, device="cuda")
    st = fcn.stream_ptr()
    assert fcn.fcn_op_cn_table(C.byref(g), C.byref(p), prec, dz, fcn.tensor_ptr(table), st) == 0
    assert fcn.fcn_op_cn(C.byref(g), C.byref(p), prec, dz, fcn.tensor_ptr(table),
                         fcn.tensor_ptr(f), st) == 0


@pytest.mark.parametrize("prec,nr,nt", [(0, 128, 256), (1, 128, 256), (1, 1024, 1024), (0, 37, 64)])
def test_noalloc_column_stage_matches_regular_entry_points(fcn, prec, nr, nt):
    wl = W.small(nr, nt, noise_seed=1).with_(k2=2e-27)
    g, p = fcn.grid_params(wl.physics())
    ctype = torch.complex128 if prec == 0 else torch.complex64
    rng = np.random.default_rng(nr + nt)
    F = rng.standard_normal((nr, nt)) + 1j * rng.standard_normal((nr, nt))
    a = torch.from_numpy(F).to("cuda", ctype)     # regular path
    b = a.clone()                                  # no-alloc path
    st = fcn.stream_ptr()
    for dz in (2e-2, 7e-3):                        # two calls in a row
        _reference(fcn, g, p, prec, dz, a)
        rc = fcn.fcn_op_cn_noalloc(C.byref(g), C.byref(p), prec, dz, fcn.tensor_ptr(b), st)
        assert rc == 0
        torch.cuda.synchronize()
        ref = a.cpu().numpy().astype(np.complex128)
        out = b.cpu().numpy().astype(np.complex128)
        assert rel_l2(out, ref) < TOL[prec]


def test_noalloc_rejects_grids_beyond_the_static_array(fcn):
    g = fcn.make_grid(1024, 1024, 1e-2, 1e-12)     # FP64 table: 8.4 MB > 8 MiB
    p = fcn.make_params()
    f = torch.zeros(1024 * 1024, dtype=torch.complex128, device="cuda")
    assert fcn.fcn_op_cn_noalloc(C.byref(g), C.byref(p), 0, 1e-3, fcn.tensor_ptr(f),
                                 fcn.stream_ptr()) == fcn.FCN_ERR_UNSUPPORTED
    assert fcn.fcn_op_cn_noalloc(C.byref(g), C.byref(p), 0, -1.0, fcn.tensor_ptr(f),
                                 fcn.stream_ptr()) == fcn.FCN_ERR_ARG
