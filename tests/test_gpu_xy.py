"""GPU parity of the Cartesian transverse grid (3D+1): the CUDA path through
the C-ABI (fcn_xy_*) against the FP64 oracle (orc_xy_*), element by element
on the same seeded inputs.

Tolerances (relative L2 over the compared array):
  FP64 path: 1e-10 on the field and rho;
  FP32-mixed path: 1e-4 on the field and 1e-5 on the energy.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05988_gb300 import workloads as W
from tests.conftest import rel_l2

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1


@pytest.fixture(scope="module")
def fcn():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1507_05988_gb300 import build
    build.build()
    from paper_1507_05988_gb300 import fcn as m
    return m


def _oracle_run(wl, n, A0=None, **kw):
    d = wl.physics()
    d.update(kw)
    pb = oracle.Problem(**d)
    g = oracle.GridXY(**wl.grid())
    A, rho = oracle.xy_run(pb, g, wl.dz, n, wl.field() if A0 is None else A0)
    return pb, g, A, rho


def _gpu_run(fcn, wl, n, prec, graph=True, variants=None, A0=None, **kw):
    d = wl.physics()
    d.update(kw)
    s = fcn.SolverXY(wl.grid(), d, precision=prec)
    if variants is not None:
        s.set_variants(*variants)
    s.set_field(wl.field() if A0 is None else A0)
    s.step(wl.dz, n, graph=graph)
    A = s.get_field()
    rho = s.get_rho()
    diag = s.diag()
    s.close()
    return A, rho, diag


# ragged grids: chunk counts that leave a partial last chunk, lines longer
# than one warp of chunks, Nx != Ny, the smallest grid, tiny and wide Nt
GRIDS = [(37, 29, 64), (21, 45, 16), (3, 4, 4), (130, 7, 8), (11, 19, 512)]


@pytest.mark.parametrize("nx,ny,nt", GRIDS)
def test_fp64_steps_match_the_oracle(fcn, nx, ny, nt):
    wl = W.small_xy(nx, ny, nt, p_over_pcr=3.0, noise_seed=5, dz=1e-2)
    n = 10                               # head, one graph block of 8, one step, tail
    _, _, Ao, ro = _oracle_run(wl, n)
    A, rho, _ = _gpu_run(fcn, wl, n, FP64)
    assert rel_l2(A, Ao) < 1e-10
    assert rel_l2(rho, ro) < 1e-10
    assert rel_l2(Ao, wl.field()) > 1e-4       # the field changed


def test_fp64_physics_variants_match_the_oracle(fcn):
    """An intense elliptical beam (ionisation and loss active), the exact
    dispersion factor, saturated loss, n4 Kerr and a chirp."""
    wl = W.small_xy(33, 27, 64, w0=0.3e-3, w0y=0.2e-3, p_over_pcr=3.0, chirp=1.5,
                    n2j=(W.N2, W.N4, 0, 0), dz=1e-3, k2=2e-27)
    for flags in (W.ALL_PHYSICS, W.ALL_PHYSICS | W.EXACT_DISPERSION | W.MPI_SAT):
        _, _, Ao, ro = _oracle_run(wl, 9, flags=flags)
        A, rho, _ = _gpu_run(fcn, wl, 9, FP64, flags=flags)
        assert rel_l2(A, Ao) < 1e-10, flags
        assert rel_l2(rho, ro) < 1e-10, flags
        assert ro.max() > 1e12


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_graph_replay_equals_direct_launches_and_variants_agree(fcn, prec):
    wl = W.small_xy(25, 19, 256, noise_seed=1, dz=1e-2)
    A0, _, _ = _gpu_run(fcn, wl, 17, prec, graph=True)
    A1, _, _ = _gpu_run(fcn, wl, 17, prec, graph=False)
    assert np.array_equal(A0, A1)
    ref = _oracle_run(wl, 17)[2]
    tol = 1e-10 if prec == FP64 else 1e-4
    for v in ((0, 0), (1, 1), (2, 2), (0, 3), (1, 4), (2, 5), (1, 6), (2, 7)):
        A, _, _ = _gpu_run(fcn, wl, 17, prec, variants=v)
        assert rel_l2(A, ref) < tol, v


def test_fp32_field_and_energy_within_tolerance(fcn):
    wl = W.small_xy(65, 57, 256, p_over_pcr=3.0, noise_seed=2, dz=1e-2)
    n = 40
    pb, g, Ao, _ = _oracle_run(wl, n)
    A, _, d = _gpu_run(fcn, wl, n, FP32)
    assert rel_l2(A, Ao) < 1e-4
    eo = oracle.xy_diag(pb, g, Ao)["energy"]
    assert abs(d["energy"] / eo - 1) < 1e-5


def test_diagnostics_match_the_oracle(fcn):
    wl = W.small_xy(31, 23, 64, w0=0.3e-3, p_over_pcr=3.0, noise_seed=3, dz=1e-3)
    pb, g, Ao, ro = _oracle_run(wl, 5)
    A, rho, d = _gpu_run(fcn, wl, 5, FP64)
    do = oracle.xy_diag(pb, g, Ao, ro)
    for k in ("energy", "peak_intensity", "onaxis_peak", "spectral_rms", "peak_rho"):
        assert d[k] == pytest.approx(do[k], rel=1e-10), k
    assert d["steps"] == 5 and d["z"] == pytest.approx(5e-3)


def test_gaussian_beam_on_the_gpu(fcn):
    """Diffraction only, FP64 and FP32: the elliptical Gaussian beam's closed
    form (the oracle's pin) to the discretisation error."""
    wl = W.small_xy(81, 61, 4, w0y=0.7e-3, flags=W.DIFFRACTION, dz=2e-2)
    pb = oracle.Problem(**wl.physics())
    k0, z = pb.k0(), 50 * 2e-2
    g = oracle.GridXY(**wl.grid())
    qx, qy = 1 + 1j * z / (k0 * wl.w0 ** 2 / 2), 1 + 1j * z / (k0 * wl.w0y ** 2 / 2)
    tau = -0.5 * wl.t_window + np.arange(4) * (wl.t_window / 4)
    ref = (np.sqrt(wl.i0) * (qx ** -0.5 * np.exp(-g.x() ** 2 / (wl.w0 ** 2 * qx)))[:, None, None]
           * (qy ** -0.5 * np.exp(-g.y() ** 2 / (wl.w0y ** 2 * qy)))[None, :, None]
           * np.exp(-(tau / wl.tp) ** 2)[None, None, :])
    for prec in (FP64, FP32):
        A, _, _ = _gpu_run(fcn, wl, 50, prec)
        assert rel_l2(A, ref) < 4e-3


def test_full_size_grid_matches_the_oracle(fcn):
    """255 x 255 x 256 (config 1's pulse on a Cartesian grid, the measured
    workload): two FP32 steps and one FP64 step against the oracle, every
    element."""
    wl = W.cartesian_config1()
    _, _, A2, _ = _oracle_run(wl, 2)
    A, _, _ = _gpu_run(fcn, wl, 2, FP32)
    assert rel_l2(A, A2) < 1e-5
    _, _, A1, _ = _oracle_run(wl, 1)
    A, _, _ = _gpu_run(fcn, wl, 1, FP64)
    assert rel_l2(A, A1) < 1e-10


def test_c64_host_calls_and_state_errors(fcn):
    wl = W.small_xy(9, 7, 16, noise_seed=4)
    s = fcn.SolverXY(wl.grid(), wl.physics(), precision=FP32)
    with pytest.raises(fcn.FcnError) as e:
        s.step(1e-3, 1)
    assert e.value.code == fcn.FCN_ERR_STATE
    a = wl.field().astype(np.complex64)
    s.set_field_c64(a)
    assert np.array_equal(s.get_field_c64(), a)
    with pytest.raises(fcn.FcnError):
        s.step(-1.0, 1)
    s.close()
