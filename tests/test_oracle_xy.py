"""Pins of the oracle's Cartesian transverse grid (Sec. 2: Delta_perp =
d^2/dx^2 + d^2/dy^2; reading R9: per-axis Crank-Nicolson factors, x then y,
dispersion in the y factor, A = 0 on the walls) against closed forms, dense
linear algebra, invariants and the radial solver."""
import numpy as np
import pytest

import oracle
from paper_1507_05988_gb300 import workloads as W
from tests.conftest import rel_l2


def _pb(wl, flags=None, **kw):
    d = wl.physics()
    if flags is not None:
        d["flags"] = flags
    d.update(kw)
    return oracle.Problem(**d)


def _gaussian_beam(wl, z, wx, wy):
    """Paraxial solution of dA/dz = (i/2k0)(A_xx + A_yy) from the elliptical
    Gaussian sqrt(I0) exp(-x^2/wx^2 - y^2/wy^2) g(tau): each axis contributes
    (1 + i z/z_R)^(-1/2) exp(-x^2/(w^2 (1 + i z/z_R))), z_R = k0 w^2/2."""
    pb = _pb(wl)
    k0 = pb.k0()
    g = oracle.GridXY(**wl.grid())
    x, y = g.x(), g.y()
    qx, qy = 1 + 1j * z / (k0 * wx ** 2 / 2), 1 + 1j * z / (k0 * wy ** 2 / 2)
    tau = -0.5 * wl.t_window + np.arange(wl.nt) * (wl.t_window / wl.nt)
    return (np.sqrt(wl.i0) * (qx ** -0.5 * np.exp(-x ** 2 / (wx ** 2 * qx)))[:, None, None]
            * (qy ** -0.5 * np.exp(-y ** 2 / (wy ** 2 * qy)))[None, :, None]
            * np.exp(-(tau / wl.tp) ** 2)[None, None, :])


def test_elliptical_gaussian_beam_matches_the_closed_form():
    """Diffraction only: the field (amplitude and Gouy/curvature phase) follows
    the paraxial Gaussian beam with a different Rayleigh length per axis, with
    second-order convergence when dx, dy and dz are halved together.  The
    same run compared with the axes' waists swapped is far off, so an x/y
    mix-up cannot pass."""
    errs = []
    for nx, ny, dz, n in [(81, 61, 2e-2, 50), (161, 121, 1e-2, 100)]:
        wl = W.small_xy(nx, ny, 4, w0y=0.7e-3, flags=W.DIFFRACTION)
        A, _ = oracle.xy_run(_pb(wl), oracle.GridXY(**wl.grid()), dz, n, wl.field())
        errs.append(rel_l2(A, _gaussian_beam(wl, dz * n, wl.w0, wl.w0y)))
        swapped = rel_l2(A, _gaussian_beam(wl, dz * n, wl.w0y, wl.w0))
        assert swapped > 20 * errs[-1]
    assert errs[0] < 4e-3
    assert 3.5 < errs[0] / errs[1] < 4.5


def _dense_cayley(n, h, k0, dz, gvd=0.0):
    """(I - dz/2 L)^-1 (I + dz/2 L) on the interior nodes of a line of n
    nodes (walls held at 0), L = (i/2k0) D2/h^2 + i gvd with D2 the [1 -2 1]
    second difference: the Crank-Nicolson step of Eq. (diff1) written as
    matrices and inverted by LAPACK."""
    m = n - 2
    d2 = np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)
    L = 1j / (2 * k0) * d2 / h ** 2 + 1j * gvd * np.eye(m)
    full = np.zeros((n, n), np.complex128)
    full[1:-1, 1:-1] = np.linalg.solve(np.eye(m) - dz / 2 * L, np.eye(m) + dz / 2 * L)
    return full


def test_linear_step_equals_dense_solves_of_both_axes():
    """One linear step on a tiny ragged grid equals F^-1 (C_y(q) kron C_x) F
    with the 1-D Crank-Nicolson factors formed densely and inverted by
    LAPACK, and numpy's FFT: this pins the Thomas sweeps, the line strides,
    the wall rows and that the dispersion term sits in the y factor only."""
    wl = W.small_xy(7, 5, 8, flags=W.DIFFRACTION | W.DISPERSION, k2=3e-26)
    pb = _pb(wl)
    g = oracle.GridXY(**wl.grid())
    rng = np.random.default_rng(3)
    A0 = rng.normal(size=(7, 5, 8)) + 1j * rng.normal(size=(7, 5, 8))
    A0[[0, -1]] = 0          # the walls hold A = 0 (Eq. (bound))
    A0[:, [0, -1]] = 0
    dz = 0.05
    got = oracle.xy_linear_step(pb, g, dz, A0)
    k0 = pb.k0()
    F = np.fft.fft(A0, axis=2)
    Cx = _dense_cayley(7, g.dx, k0, dz)
    omega = 2 * np.pi * np.fft.fftfreq(8, wl.t_window / 8)
    out = np.empty_like(F)
    for q in range(8):
        Cy = _dense_cayley(5, g.dy, k0, dz, gvd=wl.k2 * omega[q] ** 2 / 2)
        out[:, :, q] = Cx @ F[:, :, q] @ Cy.T
    ref = np.fft.ifft(out, axis=2)
    assert rel_l2(got, ref) < 1e-13
    # the same with the dispersion in both factors differs clearly
    both = np.empty_like(F)
    for q in range(8):
        gv = wl.k2 * omega[q] ** 2 / 2
        both[:, :, q] = _dense_cayley(7, g.dx, k0, dz, gv) @ F[:, :, q] @ _dense_cayley(5, g.dy, k0, dz, gv).T
    assert rel_l2(got, np.fft.ifft(both, axis=2)) > 1e-3


def test_energy_is_conserved_without_loss():
    """Each 1-D Cayley factor is unitary (a real symmetric interior operator),
    Kerr and plasma are pure phases: with MPI off dx dy dtau sum |A|^2 is an
    invariant to round-off."""
    wl = W.small_xy(25, 19, 32, p_over_pcr=3.0, noise_seed=1)
    pb = _pb(wl, flags=W.ALL_PHYSICS & ~W.MPI)
    g = oracle.GridXY(**wl.grid())
    A0 = wl.field()
    A0[[0, -1]] = 0
    A0[:, [0, -1]] = 0
    A, _ = oracle.xy_run(pb, g, 1e-2, 100, A0)
    e0 = oracle.xy_diag(pb, g, A0)["energy"]
    assert abs(oracle.xy_diag(pb, g, A)["energy"] / e0 - 1) < 1e-12
    assert rel_l2(A, A0) > 1e-2
    # and MPI loss removes energy (a 25x more intense beam: w0 = 0.2 mm)
    wn = wl.with_(w0=0.2e-3, x_width=0.0, y_width=0.0, w0y=0.0)
    gn = oracle.GridXY(**wn.grid())
    An = wn.field()
    An[[0, -1]] = 0
    An[:, [0, -1]] = 0
    Al, _ = oracle.xy_run(_pb(wn, flags=W.ALL_PHYSICS), gn, 1e-3, 20, An)
    assert oracle.xy_diag(pb, gn, Al)["energy"] < oracle.xy_diag(pb, gn, An)["energy"] * (1 - 3e-7)


@pytest.mark.parametrize("exact", [False, True])
def test_dispersion_only_is_the_radial_scheme_factor(exact):
    """Diffraction and nonlinearity off: every interior node's spectrum is
    multiplied per step by (1 + i delta_q)/(1 - i delta_q), delta_q = k''
    omega_q^2 dz/4, exactly the radial scheme's factor (or by exp(i k''
    omega_q^2 dz/2) in the exact-dispersion variant); the walls become 0."""
    flags = W.DISPERSION | (W.EXACT_DISPERSION if exact else 0)
    wl = W.small_xy(5, 6, 64, tp=30e-15, t_window=480e-15, flags=flags, k2=2e-27)
    pb = _pb(wl)
    g = oracle.GridXY(**wl.grid())
    A0 = wl.field()
    n, dz = 20, 0.05
    A, _ = oracle.xy_run(pb, g, dz, n, A0)
    omega = 2 * np.pi * np.fft.fftfreq(64, wl.t_window / 64)
    if exact:
        fac = np.exp(1j * wl.k2 * omega ** 2 * dz / 2) ** n
    else:
        d = wl.k2 * omega ** 2 * dz / 4
        fac = ((1 + 1j * d) / (1 - 1j * d)) ** n
    ref = np.fft.ifft(np.fft.fft(A0, axis=2) * fac, axis=2)
    assert rel_l2(A[1:-1, 1:-1], ref[1:-1, 1:-1]) < 1e-13
    assert np.all(A[[0, -1]] == 0) and np.all(A[:, [0, -1]] == 0)


def test_pure_self_phase_modulation_is_exact():
    """Kerr (n2 + n4) only: A(z) = A0 exp(i k0/n0 (n2 I0 + n4 I0^2) z) at
    every interior node."""
    wl = W.small_xy(6, 5, 16, n2j=(W.N2, W.N4, 0, 0), flags=W.KERR)
    pb = _pb(wl)
    A0 = wl.field()
    n, dz = 25, 4e-3
    A, _ = oracle.xy_run(pb, oracle.GridXY(**wl.grid()), dz, n, A0)
    I0 = np.abs(A0) ** 2
    ref = A0 * np.exp(1j * pb.k0() / pb.n0 * (W.N2 * I0 + W.N4 * I0 ** 2) * n * dz)
    assert rel_l2(A[1:-1, 1:-1], ref[1:-1, 1:-1]) < 1e-13     # the walls hold 0


def test_round_beam_agrees_with_the_radial_solver():
    """All physics on, 3 P_cr, 20 steps: a round beam on a square grid whose
    nodes along +x are the radial grid's nodes gives, on the axis and along
    +x, the radial solver's field to the discretisation difference of the
    two Laplacians (measured 1.6e-4); both grids see the same nonlinear
    steps."""
    nr, nt = 48, 64
    wl = W.small(nr, nt, p_over_pcr=3.0)
    Ar, _ = oracle.run(oracle.Problem(**wl.physics()), 1e-2, 20, wl.field())
    wx = W.small_xy(2 * nr - 1, 2 * nr - 1, nt, p_over_pcr=3.0)
    assert np.isclose(wx.x_width / (wx.nx - 1), wl.r_max / (nr - 1))
    Ax, _ = oracle.xy_run(_pb(wx), oracle.GridXY(**wx.grid()), 1e-2, 20, wx.field())
    c = nr - 1
    assert rel_l2(Ax[c, c], Ar[0]) < 5e-4
    assert rel_l2(Ax[c:, c], Ar) < 5e-4
    assert rel_l2(Ar, wl.field()) > 1e-2


def test_square_grid_keeps_the_beam_symmetric_without_dispersion():
    """Without the dispersion term the two factors are the same operator on
    transposed axes and commute, so a beam symmetric under x <-> y stays
    symmetric to round-off through the nonlinear steps."""
    wl = W.small_xy(23, 23, 32, flags=W.ALL_PHYSICS & ~W.DISPERSION)
    A, _ = oracle.xy_run(_pb(wl), oracle.GridXY(**wl.grid()), 1e-2, 30, wl.field())
    assert rel_l2(A.transpose(1, 0, 2), A) < 1e-12
    assert rel_l2(A, wl.field()) > 1e-3


def test_diag_sums():
    wl = W.small_xy(9, 7, 16, noise_seed=2)
    pb = _pb(wl)
    g = oracle.GridXY(**wl.grid())
    A = wl.field()
    d = oracle.xy_diag(pb, g, A)
    I = np.abs(A) ** 2
    assert d["energy"] == pytest.approx(g.dx * g.dy * wl.t_window / wl.nt * I.sum(), rel=1e-14)
    assert d["peak_intensity"] == pytest.approx(I.max(), rel=1e-15)
    assert d["onaxis_peak"] == pytest.approx(I[4, 3].max(), rel=1e-15)
    assert not d["nonfinite"]


def test_cartesian_workload_grid_and_power():
    """The Cartesian input: nodes symmetric about 0 with the walls at +-5 w0,
    config 1's dr as spacing, and I0 = 2P/(pi wx wy) so that the transverse
    integral of |A|^2 at the pulse peak is the beam power P."""
    wl = W.cartesian_config1()
    g = oracle.GridXY(**wl.grid())
    assert g.x()[0] == pytest.approx(-5e-3) and g.x()[-1] == pytest.approx(5e-3)
    assert g.x()[(wl.nx - 1) // 2] == pytest.approx(0.0, abs=1e-15)
    assert g.dx == pytest.approx(W.config1().r_max / (W.config1().nr - 1))
    we = W.small_xy(161, 121, 8, w0y=0.6e-3)
    A = we.field()
    ge = oracle.GridXY(**we.grid())
    peak = np.abs(A[:, :, we.nt // 2]) ** 2
    p = peak.sum() * ge.dx * ge.dy
    assert p == pytest.approx(we.p_over_pcr * W.critical_power(), rel=1e-9)


def test_cpu_oracle_sample_of_the_cartesian_bench_leg():
    import bench
    r = bench.cpu_oracle_sample_xy(W.small_xy(9, 7, 16), budget_s=0.2)
    assert r["kind"] == "oracle" and r["cores"] >= 1 and r["value"] > 0 and r["single_thread_value"] > 0


def test_factored_step_differs_from_the_unsplit_2d_step_at_third_order():
    """Reading R9: the product of the x and y Cayley factors differs from the
    unsplit two-dimensional Crank-Nicolson step (Kronecker-sum operator,
    solved densely by LAPACK) by O(dz^3) per step: halving dz divides the
    one-step difference by about 8, while both stay unitary."""
    wl = W.small_xy(9, 7, 4, flags=W.DIFFRACTION | W.DISPERSION, k2=2e-27)
    pb = _pb(wl)
    g = oracle.GridXY(**wl.grid())
    rng = np.random.default_rng(11)
    A0 = rng.normal(size=(9, 7, 4)) + 1j * rng.normal(size=(9, 7, 4))
    A0[[0, -1]] = 0
    A0[:, [0, -1]] = 0
    k0 = pb.k0()
    mx, my = 7, 5

    def d2(m, h):
        return (np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1)
                + np.diag(np.ones(m - 1), -1)) / h ** 2

    omega = 2 * np.pi * np.fft.fftfreq(4, wl.t_window / 4)
    diffs = []
    for dz in (1.0, 0.5):
        F = np.fft.fft(A0, axis=2)
        out = np.zeros_like(F)
        for q in range(4):
            L = (1j / (2 * k0) * (np.kron(d2(mx, g.dx), np.eye(my)) + np.kron(np.eye(mx), d2(my, g.dy)))
                 + 1j * wl.k2 * omega[q] ** 2 / 2 * np.eye(mx * my))
            I = np.eye(mx * my)
            v = F[1:-1, 1:-1, q].reshape(-1)
            out[1:-1, 1:-1, q] = np.linalg.solve(I - dz / 2 * L, (I + dz / 2 * L) @ v).reshape(mx, my)
        unsplit = np.fft.ifft(out, axis=2)
        adi = oracle.xy_linear_step(pb, g, dz, A0)
        assert np.linalg.norm(adi) == pytest.approx(np.linalg.norm(A0), rel=1e-12)
        diffs.append(rel_l2(adi, unsplit))
    assert diffs[0] > 1e-6
    assert 6.5 < diffs[0] / diffs[1] < 9.5


@pytest.mark.parametrize("threads", [2, 5])
def test_threaded_oracle_is_bit_identical(threads):
    """Rows and frequency bins split over threads (Sec. 4's decomposition on
    the Cartesian grid) give exactly the serial result, field and rho."""
    wl = W.small_xy(13, 11, 32, w0=0.4e-3, p_over_pcr=3.0, noise_seed=9, dz=2e-3)
    pb = _pb(wl)
    g = oracle.GridXY(**wl.grid())
    A1, r1 = oracle.xy_run(pb, g, wl.dz, 7, wl.field())
    A2, r2 = oracle.xy_run(pb, g, wl.dz, 7, wl.field(), threads=threads)
    assert np.array_equal(A1, A2) and np.array_equal(r1, r2)
    assert r1.max() > 0
