"""Host logic of the GPU path, checked on the CPU: the two FFT decompositions
of the row stage (every Nt from 2 to 8192), the twiddle-table layout that
follows from them, the pivot-table row pitch, and the closed-form fixed point
of the pivot recurrence that FP32 context tables are stored against.  A
small host program including the kernels' header prints them (nvcc, host
code only)."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dump():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "host_plans")
    subprocess.run([nvcc, "-std=c++17", "-x", "cu", os.path.join(ROOT, "tests", "host_plans.cu"), "-o", exe],
                   check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    shutil.rmtree(d, ignore_errors=True)
    plans, lims = [], []
    for line in out.splitlines():
        f = line.split()
        if f[0] == "plan":
            nt, plan, npass, tws, pitch = map(int, f[1:6])
            passes = [tuple(map(int, x.split(":"))) for x in f[6:]]
            plans.append((nt, plan, npass, tws, pitch, passes))
        else:
            lims.append((float(f[1]), float(f[2]), int(f[3]), complex(float(f[4]), float(f[5]))))
    return plans, lims


def test_fft_plans_factor_nt_and_end_in_the_thread_radix(dump):
    plans, _ = dump
    assert len(plans) == 2 * 13
    for nt, plan, npass, tws, pitch, passes in plans:
        radices = [r for r, _, _ in passes]
        assert len(radices) == npass
        assert int(np.prod(radices)) == nt
        assert radices[-1] == min(nt, 16)                 # a thread's samples: the last pass
        ns = 1
        off = 0
        for p, (r, nsp, o) in enumerate(passes):
            assert nsp == ns                              # product of the earlier radices
            assert o == off                               # blocks of (R-1) Ns entries from pass 1 on
            if p >= 1:
                off += (r - 1) * nsp
            ns *= r
        assert tws == off
        assert pitch % 2 == 0 and pitch >= nt // 2 + 1 and pitch <= nt // 2 + 2
        if plan == 0 or nt < 256:
            # radix-16 passes after one radix 2/4/8 pass (plan 1 falls back below Nt = 256)
            assert all(r == 16 for r in radices[1:]) or nt < 16
        else:
            assert all(r == 8 for r in radices[1:-1])
            assert radices[0] in (2, 4, 8)
            plan0 = [r for r, _, _ in [q for q in plans if q[0] == nt and q[1] == 0][0][5]]
            assert radices != plan0                       # a different decomposition


def test_pivot_limit_is_the_attracting_fixed_point(dump):
    """1/p with p = b + s^2/p, b = 1 + i(2s - dk q^2), and |p| the larger
    root (the one the recurrence piv_j = b + s^2 / piv_{j-1} tends to)."""
    _, lims = dump
    for s, dk, q, inv in lims:
        b = 1 + 1j * (2 * s - dk * q * q)
        p = 1 / inv
        assert abs(p - (b + s * s / p)) <= 1e-12 * abs(p)
        other = b - p                                     # the two roots sum to b
        assert abs(p) >= abs(other) - 1e-12 * abs(p)
        # the recurrence from piv_0 = b converges to it
        piv = b
        for _ in range(4000):
            piv = b + s * s / piv
        assert abs(1 / piv - inv) <= 1e-9 * abs(inv) or s > 10


def test_chunked_row_io_is_a_permutation_and_cuts_bank_conflicts():
    """The head and tail row launches move time-domain rows between HBM and
    the digit-reversed shared-memory layout in 16-byte chunks (RowIo,
    row_chunks): every value of the row once, at its digit-reversed
    position, whole 32-byte sectors per warp instruction, and no more
    shared-memory wavefronts than the per-value loop: for the 4096-point
    float rows 2 instead of 16.  The same for the rho output's rows of
    reals (FFT plan 0)."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tempfile.mkdtemp()
    exe = os.path.join(d, "row_io")
    subprocess.run([nvcc, "-std=c++17", "-x", "cu", "-diag-suppress", "20013,1886",
                    os.path.join(ROOT, "tests", "row_io.cu"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    shutil.rmtree(d, ignore_errors=True)
    rows, reals = {}, {}
    for line in out.splitlines():
        f = line.split()
        if f[0] not in ("io", "rio") or f[-1] == "skip":
            continue
        (rows if f[0] == "io" else reals)[(f[1], int(f[2]), int(f[3]))] = dict(zip(f[4::2], map(int, f[5::2])))
    # float rows from 512 points, double rows from 512 points (whole warps, whole line groups)
    assert len(rows) == 2 * 2 * 5
    for (prec, nt, plan), r in rows.items():
        assert r["bad"] == 0, (prec, nt, plan)
        assert r["sectors"] == 16                       # 16 full 32-byte sectors per instruction
        assert r["wf_new"] <= r["wf_old"], (prec, nt, plan)
    assert rows[("f32", 4096, 0)]["wf_new"] == 2 and rows[("f32", 4096, 0)]["wf_old"] == 16
    assert rows[("f32", 1024, 0)]["wf_new"] == 2
    assert rows[("f64", 4096, 0)]["wf_new"] == 4        # 512 bytes: the minimum
    # the rho output's chunks of reals (FFT plan 0, from 512 points)
    assert len(reals) == 2 * 5
    for key, r in reals.items():
        assert key[2] == 0 and r["bad"] == 0, key
        assert r["wf_new"] <= r["wf_old"], key
    assert reals[("f32", 4096, 0)]["wf_new"] == 2 and reals[("f32", 4096, 0)]["wf_old"] == 8
