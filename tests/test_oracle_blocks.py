"""Pins of the oracle's building blocks against facts that do not come from
the oracle itself: brute-force DFTs, dense linear algebra, exact discrete
operator identities and the Crank-Nicolson structure of Sec. 3.1."""
import mpmath
import numpy as np
import pytest

import oracle
from tests.conftest import rel_l2


# ---------------------------------------------------------------- FFT ---

def _brute_dft(x, sign):
    """O(N^2) DFT in 40-digit arithmetic."""
    mpmath.mp.dps = 40
    n = len(x)
    out = []
    for q in range(n):
        s = mpmath.mpc(0)
        for p in range(n):
            s += mpmath.mpc(x[p].real, x[p].imag) * mpmath.expjpi(sign * 2 * mpmath.mpf(p * q) / n)
        out.append(complex(s))
    return np.array(out)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64])
def test_fft_matches_brute_force_dft(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel_l2(oracle.fft(x), _brute_dft(x, -1)) < 1e-14
    inv = _brute_dft(x, +1) / n
    assert rel_l2(oracle.fft(x, inverse=True), inv) < 1e-14


@pytest.mark.parametrize("n", [128, 1024, 8192])
def test_fft_matches_numpy_and_roundtrips(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert rel_l2(oracle.fft(x), np.fft.fft(x)) < 1e-13
    assert rel_l2(oracle.fft(oracle.fft(x), inverse=True), x) < 1e-14


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.fft(np.zeros(12))


# ------------------------------------------------------------- Thomas ---

@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 40])
def test_thomas_matches_dense_solve(n):
    rng = np.random.default_rng(100 + n)
    cz = lambda: rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a, c, d = cz(), cz(), cz()
    b = cz() + 4.0 * (1 + 1j)            # keep the system well conditioned
    M = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    x = oracle.thomas(a, b, c, d)
    assert rel_l2(x, np.linalg.solve(M, d)) < 1e-13


# --------------------------------------------- Crank-Nicolson matrices ---

def _problem(nr=24, nt=16, flags=oracle.DIFFRACTION, **kw):
    base = dict(nr=nr, nt=nt, r_max=5e-3, t_window=1.6e-12, lambda0=800e-9, n0=1.0,
                n2j=(3.2e-23, 0, 0, 0), k2=2e-29, sigma_k=2.88e-131, rho_nt=5.4e24,
                K=8, flags=flags)
    base.update(kw)
    return oracle.Problem(**base)


def _dense(pb, dz, q):
    a, b, c, d, e, f = oracle.cn_coeffs(pb, dz, q)
    Mabc = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    Mdef = np.diag(e) + np.diag(d[1:], -1) + np.diag(f[:-1], 1)
    return Mabc, Mdef


def _radial_operator(pb, dz, q=0):
    """Returns L with (M_def - I) = i s dr^2 L on rows 0..nr-2 (dispersion off)."""
    _, Mdef = _dense(pb, dz, q)
    s = dz / (4.0 * pb.k0() * pb.dr ** 2)
    n = pb.nr - 1
    return ((Mdef - np.eye(pb.nr))[:n] / (1j * s * pb.dr ** 2)).real * pb.dr ** 2


def test_cn_operator_annihilates_constants_and_is_exact_on_r2():
    """Delta_perp 1 = 0 and Delta_perp r^2 = 4 hold exactly for the
    discretisation of Eqs. (diff2)-(diff3) with the r -> 0 row of Eq. (bound)."""
    pb = _problem()
    L = _radial_operator(pb, 1e-2)          # dimensionless: dr^2 * Delta_perp
    j = np.arange(pb.nr, dtype=float)
    assert np.max(np.abs(L @ np.ones(pb.nr))) < 1e-12
    assert np.max(np.abs(L @ j ** 2 - 4.0)) < 1e-11
    # r^4: Delta_perp r^4 = 16 r^2, second-order truncation 6 dr^2 for j >= 1
    lr4 = L @ j ** 4
    assert abs(lr4[0] - 4.0) < 1e-10
    assert np.max(np.abs(lr4[1:] - (16 * j[1:-1] ** 2 + 6))) < 1e-8


def test_printed_cj_reading_is_rejected_by_the_constant_pin():
    pb = _problem(flags=oracle.DIFFRACTION | oracle.PRINTED_CJ)
    L = _radial_operator(pb, 1e-2)
    assert np.max(np.abs(L @ np.ones(pb.nr))) > 0.1


def test_cn_matrices_have_crank_nicolson_structure():
    """M_abc = I - (dz/2) D and M_def = I + (dz/2) D: their sum is 2I on
    rows 0..nr-2, and the Dirichlet row forces x_{nr-1} = 0."""
    pb = _problem(flags=oracle.DIFFRACTION | oracle.DISPERSION)
    for q in (0, 3, pb.nt // 2, pb.nt - 1):
        Mabc, Mdef = _dense(pb, 2e-3, q)
        S = Mabc + Mdef
        assert np.max(np.abs(S[:-1] - 2 * np.eye(pb.nr)[:-1])) < 1e-14
        assert np.allclose(Mabc[-1], np.eye(pb.nr)[-1]) and np.allclose(Mdef[-1], 0)


def test_omega_grid_matches_numpy_fftfreq():
    pb = _problem(nt=64)
    ref = 2 * np.pi * np.fft.fftfreq(pb.nt, d=pb.dtau)
    got = np.array([pb.omega(q) for q in range(pb.nt)])
    assert np.allclose(np.abs(got), np.abs(ref), rtol=1e-14, atol=0)
    assert np.allclose(got[: pb.nt // 2], ref[: pb.nt // 2], rtol=1e-14, atol=0)


def test_cn_operator_is_self_adjoint_in_the_radial_weight():
    """W (M_def - I) is i times a real symmetric matrix with W_0 = 1/8,
    W_m = m: the step is then unitary in the energy norm."""
    pb = _problem(nr=33)
    _, Mdef = _dense(pb, 1e-2, 0)
    n = pb.nr - 1
    W = np.diag(np.r_[0.125, np.arange(1, n, dtype=float)])
    H = (W @ (Mdef - np.eye(pb.nr))[:n, :n]) / 1j
    assert np.max(np.abs(H.imag)) < 1e-15
    assert np.max(np.abs(H - H.T)) < 1e-12 * np.max(np.abs(H))
    pbx = _problem(nr=33, flags=oracle.DIFFRACTION | oracle.PRINTED_CJ)
    _, Mx = _dense(pbx, 1e-2, 0)
    Hx = (W @ (Mx - np.eye(pb.nr))[:n, :n]) / 1j
    assert np.max(np.abs(Hx - Hx.T)) > 1e-3 * np.max(np.abs(Hx))


def test_cn_update_preserves_weighted_norm():
    pb = _problem(nr=40, flags=oracle.DIFFRACTION | oracle.DISPERSION)
    rng = np.random.default_rng(7)
    W = np.r_[0.125, np.arange(1, pb.nr, dtype=float)]
    for q in (0, 5, pb.nt // 2):
        Mabc, Mdef = _dense(pb, 5e-2, q)
        v = rng.standard_normal(pb.nr) + 1j * rng.standard_normal(pb.nr)
        v[-1] = 0
        x = np.linalg.solve(Mabc, Mdef @ v)
        assert abs(np.sum(W * abs(x) ** 2) / np.sum(W * abs(v) ** 2) - 1) < 1e-13


def test_linear_step_equals_dense_column_solves():
    """orc_linear_step = row FFT, per-column dense solve, row inverse FFT."""
    pb = _problem(nr=12, nt=8, flags=oracle.DIFFRACTION | oracle.DISPERSION)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((pb.nr, pb.nt)) + 1j * rng.standard_normal((pb.nr, pb.nt))
    dz = 3e-2
    At = np.fft.fft(A, axis=1)
    for q in range(pb.nt):
        Mabc, Mdef = _dense(pb, dz, q)
        At[:, q] = np.linalg.solve(Mabc, Mdef @ At[:, q])
    ref = np.fft.ifft(At, axis=1)
    assert rel_l2(oracle.linear_step(pb, dz, A), ref) < 1e-13


def test_threaded_run_is_bit_identical():
    """The paper's row/column thread decomposition (timing mode) computes
    every row and column with the same code as the serial run."""
    from paper_1507_05988_gb300 import workloads as W
    wl = W.small(40, 128, p_over_pcr=4.0, noise_seed=5).with_(n2j=(W.N2, W.N4, 0, 0))
    pb = oracle.Problem(**wl.physics())
    a1, r1 = oracle.run(pb, 5e-3, 4, wl.field())
    for th in (2, 3, 7):
        a, r = oracle.run(pb, 5e-3, 4, wl.field(), threads=th)
        assert np.array_equal(a, a1) and np.array_equal(r, r1)
