"""Pins of the oracle's whole Strang step (Eq. (nlseq)) against closed-form
solutions of the NLSE's pieces, conservation laws and convergence orders."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_05988_gb300 import workloads as W
from tests.conftest import rel_l2


def _pb(wl: W.Workload, flags=None, **kw):
    d = wl.physics()
    if flags is not None:
        d["flags"] = flags
    d.update(kw)
    return oracle.Problem(**d)


def _weights(nr):
    return np.r_[0.125, np.arange(1, nr, dtype=float)]


def test_energy_is_conserved_without_loss():
    """Kerr and plasma are pure phases and the CN step is unitary in the
    radial weight, so with MPI off the discrete energy is an invariant."""
    wl = W.small(48, 64, p_over_pcr=3.0)
    pb = _pb(wl, flags=W.ALL_PHYSICS & ~W.MPI)
    A0 = wl.field()
    A0[-1] = 0                       # the Dirichlet node is zero from the start
    A, _ = oracle.run(pb, 1e-2, 200, A0)
    e0 = oracle.diag(pb, A0)["energy"]
    e1 = oracle.diag(pb, A)["energy"]
    assert abs(e1 / e0 - 1) < 1e-12
    assert rel_l2(A, A0) > 1e-2       # the field did change
    bad = _pb(wl, flags=(W.ALL_PHYSICS & ~W.MPI) | oracle.PRINTED_CJ)
    Ab, _ = oracle.run(bad, 1e-2, 200, A0)
    assert abs(oracle.diag(bad, Ab)["energy"] / e0 - 1) > 1e-6


def test_pure_self_phase_modulation_is_exact():
    """Diffraction, dispersion, plasma and MPI off: A(z) = A0 exp(i k0/n0
    (n2 I0 + n4 I0^2) z) pointwise (rows m < Nr-1; the Dirichlet row is 0)."""
    wl = W.small(8, 32).with_(n2j=(W.N2, W.N4, 0, 0))
    pb = _pb(wl, flags=W.KERR)
    A0 = wl.field()
    n, dz = 25, 4e-3
    A, _ = oracle.run(pb, dz, n, A0)
    I0 = np.abs(A0) ** 2
    ref = A0 * np.exp(1j * pb.k0() / pb.n0 * (W.N2 * I0 + W.N4 * I0 ** 2) * n * dz)
    assert rel_l2(A[:-1], ref[:-1]) < 1e-13
    assert np.all(A[-1] == 0)


def test_dispersion_only_matches_discrete_cayley_factor():
    """Diffraction and nonlinearity off: every frequency bin is multiplied by
    (1 + i delta_q)/(1 - i delta_q) per step, delta_q = k'' omega_q^2 dz/4,
    with omega_q = 2 pi fftfreq."""
    wl = W.small(4, 256).with_(tp=30e-15, t_window=480e-15)
    pb = _pb(wl, flags=W.DISPERSION, k2=2e-27)
    A0 = wl.field()
    n, dz = 30, 5e-2
    A, _ = oracle.run(pb, dz, n, A0)
    w = 2 * np.pi * np.fft.fftfreq(pb.nt, d=pb.dtau)
    delta = pb.k2 * w ** 2 * dz / 4
    g = ((1 + 1j * delta) / (1 - 1j * delta)) ** n
    ref = np.fft.ifft(np.fft.fft(A0, axis=1) * g[None, :], axis=1)
    assert rel_l2(A[:-1], ref[:-1]) < 1e-13
    assert rel_l2(A[:-1], A0[:-1]) > 0.1


def test_gvd_broadening_matches_closed_form():
    """Dispersion only: a Gaussian exp(-tau^2/tp^2) broadens as
    tp sqrt(1 + (2 k'' z / tp^2)^2); second moment <tau^2> = width^2/4."""
    tp = 100e-15
    L_D = 1.0
    k2 = tp ** 2 / (2 * L_D)
    wl = W.Workload("gvd", nr=3, nt=1024, w0=1e-3, tp=tp, p_over_pcr=1.0, t_window=64 * tp)
    pb = _pb(wl, flags=W.DISPERSION, k2=k2)
    A, _ = oracle.run(pb, 2e-3, 1000, wl.field())
    tau = -pb.t_window / 2 + np.arange(pb.nt) * pb.dtau
    I = np.abs(A[0]) ** 2
    width = np.sqrt(4 * np.sum(tau ** 2 * I) / np.sum(I))
    assert width == pytest.approx(tp * np.sqrt(1 + (2 * k2 * 2.0 / tp ** 2) ** 2), rel=1e-5)


def test_exact_dispersion_matches_continuous_gvd():
    """Dispersion as its exact factor (variant of reading R7): a Gaussian
    exp(-tau^2/tp^2) under dA/dz = -(i k''/2) d^2A/dtau^2 (Eq. (linearpart))
    is tp / sqrt(tp^2 - 2 i k'' z) exp(-tau^2 / (tp^2 - 2 i k'' z)) at z,
    which a wide periodic window reproduces to rounding; the CN form (the
    Cayley factor per step) does not."""
    tp = 100e-15
    k2 = tp ** 2 / 2.0                       # dispersion length 1 m
    wl = W.Workload("gvd", nr=3, nt=1024, w0=1e-3, tp=tp, p_over_pcr=1.0, t_window=64 * tp)
    z, n = 1.5, 150
    tau = -wl.t_window / 2 + np.arange(wl.nt) * (wl.t_window / wl.nt)
    T2 = tp ** 2 - 2j * k2 * z
    exact = np.sqrt(wl.i0) * tp / np.sqrt(T2) * np.exp(-tau ** 2 / T2)
    pb = _pb(wl, flags=W.DISPERSION | oracle.EXACT_DISPERSION, k2=k2)
    A, _ = oracle.run(pb, z / n, n, wl.field())
    assert rel_l2(A[0], exact) < 1e-11
    cn, _ = oracle.run(_pb(wl, flags=W.DISPERSION, k2=k2), z / n, n, wl.field())
    assert rel_l2(cn[0], exact) > 1e-6       # the CN form carries its O(dz^2) phase error


def test_exact_dispersion_keeps_the_energy_with_diffraction():
    """Diffraction (CN, unitary in the radial weight) and the exact
    dispersion factor (unit modulus) together conserve the discrete energy;
    the result differs from the CN form by the CN's dispersion phase error."""
    wl = W.small(48, 64, p_over_pcr=3.0).with_(tp=30e-15, t_window=480e-15)
    A0 = wl.field()
    A0[-1] = 0
    flags = W.DIFFRACTION | W.DISPERSION | W.KERR | W.PLASMA
    pb = _pb(wl, flags=flags | oracle.EXACT_DISPERSION, k2=2e-27)
    A, _ = oracle.run(pb, 1e-2, 100, A0)
    assert abs(oracle.diag(pb, A)["energy"] / oracle.diag(pb, A0)["energy"] - 1) < 1e-12
    B, _ = oracle.run(_pb(wl, flags=flags, k2=2e-27), 1e-2, 100, A0)
    assert rel_l2(A, B) > 1e-6


def _waist(pb, A):
    r = np.arange(pb.nr) * pb.dr
    w = _weights(pb.nr)
    I = np.sum(np.abs(A) ** 2, axis=1)
    return np.sqrt(2 * np.sum(w * r ** 2 * I) / np.sum(w * I))


def test_gaussian_beam_waist_converges_at_second_order():
    """Diffraction only: w(z) = w0 sqrt(1 + (z/z_R)^2), z_R = k0 w0^2 / 2.
    The error against the closed form falls as dr^2 (dz refined with it)."""
    w0 = 1e-3
    errs = []
    for nr, nz in ((65, 25), (129, 50), (257, 100)):
        wl = W.Workload("beam", nr=nr, nt=2, w0=w0, tp=100e-15, p_over_pcr=1.0, r_max=8 * w0)
        pb = _pb(wl, flags=W.DIFFRACTION)
        zr = pb.k0() * w0 ** 2 / 2
        A, _ = oracle.run(pb, zr / nz, nz, wl.field())
        exact = w0 * np.sqrt(2.0)
        errs.append(abs(_waist(pb, A) - exact) / exact)
    assert errs[-1] < 5e-4
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_strang_step_is_second_order_in_dz():
    """Kerr + diffraction + dispersion (no loss): global error vs a fine
    reference falls as dz^2."""
    wl = W.small(32, 64, p_over_pcr=2.0)
    pb = _pb(wl, flags=W.DIFFRACTION | W.DISPERSION | W.KERR)
    A0 = wl.field()
    z = 0.4
    ref, _ = oracle.run(pb, z / 256, 256, A0)
    errs = []
    for n in (8, 16, 32):
        A, _ = oracle.run(pb, z / n, n, A0)
        errs.append(rel_l2(A, ref))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_diagnostics_of_the_gaussian_input():
    """E = I0 (pi w0^2 / 2)(tp sqrt(pi/2)); peak = I0; spectral rms = 1/tp;
    power and fluence integrate to the energy."""
    wl = W.Workload("diag", nr=512, nt=512, w0=1e-3, tp=100e-15, p_over_pcr=1.0,
                    r_max=6e-3, t_window=2.4e-12)
    pb = _pb(wl)
    A = wl.field()
    d = oracle.diag(pb, A)
    i0 = wl.i0
    # the radial sum is a second-order quadrature: error ~ (dr/w0)^2 / 6
    assert d["energy"] == pytest.approx(i0 * np.pi * wl.w0 ** 2 / 2 * wl.tp * np.sqrt(np.pi / 2),
                                        rel=(pb.dr / wl.w0) ** 2 / 3)
    # the Gaussian's peak sits on the grid (m = 0, p = nt/2)
    assert d["peak_intensity"] == pytest.approx(i0, rel=1e-14)
    assert d["onaxis_peak"] == pytest.approx(i0, rel=1e-14)
    assert d["spectral_rms"] == pytest.approx(1 / wl.tp, rel=1e-9)
    assert np.sum(d["power"]) * pb.dtau == pytest.approx(d["energy"], rel=1e-12)
    area = 2 * np.pi * pb.dr ** 2 * _weights(pb.nr)
    assert np.sum(area * d["fluence"]) == pytest.approx(d["energy"], rel=1e-12)
    assert not d["nonfinite"]
    A[3, 7] = np.nan
    assert oracle.diag(pb, A)["nonfinite"]


# ------------------------------------------------- step-doubling controller

def test_adaptive_controller_accepts_exact_steps_and_lands_on_z_end():
    """Pure SPM is integrated exactly by any dz (err ~ round-off), so every
    step is accepted, dz doubles each step and the run ends exactly at z_end."""
    wl = W.small(6, 16)
    pb = _pb(wl, flags=W.KERR)
    A0 = wl.field()
    A, _, st = oracle.propagate_adaptive(pb, A0, 0.0, 1.0, 0.01, rtol=1e-8)
    assert st["status"] == 0 and st["rejected"] == 0
    assert st["z"] == 1.0
    # 0.01 + 0.02 + ... + 0.32 = 0.63, then the clipped 0.37
    assert st["accepted"] == 7
    I0 = np.abs(A0) ** 2
    ref = A0 * np.exp(1j * pb.k0() * W.N2 * I0 * 1.0)
    assert rel_l2(A[:-1], ref[:-1]) < 1e-12


def test_adaptive_controller_error_estimate_is_the_step_doubling_difference():
    """Dispersion only: one step and two half steps have closed forms, so the
    rejected first attempt's error and the shrink factor are known."""
    wl = W.small(3, 128).with_(tp=30e-15, t_window=480e-15)
    k2 = 2e-26
    pb = _pb(wl, flags=W.DISPERSION, k2=k2)
    A0 = wl.field()
    dz = 0.5
    w = 2 * np.pi * np.fft.fftfreq(pb.nt, d=pb.dtau)
    d1 = k2 * w ** 2 * dz / 4
    g1 = (1 + 1j * d1) / (1 - 1j * d1)
    g2 = ((1 + 1j * d1 / 2) / (1 - 1j * d1 / 2)) ** 2
    F = np.fft.fft(A0[:-1], axis=1)
    a1 = np.fft.ifft(F * g1, axis=1)
    a2 = np.fft.ifft(F * g2, axis=1)
    err = rel_l2(a1, a2)
    rtol = err / 3
    _, _, st = oracle.propagate_adaptive(pb, A0, 0.0, dz, dz, rtol=rtol, max_reject=0)
    # first attempt rejected, then max_reject = 0 aborts with that error
    assert st["status"] == -1 and st["rejected"] == 1 and st["accepted"] == 0
    assert st["last_err"] == pytest.approx(err, rel=1e-10)
    fac = min(2.0, max(0.2, 0.9 * (rtol / err) ** (1 / 3)))
    assert st["dz_next"] == pytest.approx(dz * fac, rel=1e-12)


# ------------------------------------------------------------------- MLP

def _torch_mlp(params, nin, nh):
    p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    o = np.cumsum([0, nh * nin, nh, nh * nh, nh, nh, 1])
    W1 = p[o[0]:o[1]].view(nh, nin)
    b1 = p[o[1]:o[2]]
    W2 = p[o[2]:o[3]].view(nh, nh)
    b2 = p[o[3]:o[4]]
    W3 = p[o[4]:o[5]].view(1, nh)
    b3 = p[o[5]:o[6]]

    def f(x):
        h = torch.tanh(torch.nn.functional.linear(x, W1, b1))
        h = torch.tanh(torch.nn.functional.linear(h, W2, b2))
        return torch.nn.functional.linear(h, W3, b3)[:, 0]
    return p, f


def test_mlp_forward_and_gradient_match_torch_autograd():
    nin, nh, batch = 6, 64, 37
    rng = np.random.default_rng(5)
    npar = oracle.mlp_param_count(nin, nh)
    params = 0.3 * rng.standard_normal(npar)
    x = rng.standard_normal((batch, nin))
    t = rng.standard_normal(batch)
    y = oracle.mlp_forward(params, x, nin, nh)
    p, f = _torch_mlp(params, nin, nh)
    yt = f(torch.tensor(x))
    assert np.max(np.abs(y - yt.detach().numpy())) < 1e-13
    loss, g = oracle.mlp_loss_grad(params, x, t, nin, nh)
    lt = torch.mean((yt - torch.tensor(t)) ** 2)
    lt.backward()
    assert loss == pytest.approx(lt.item(), rel=1e-13)
    assert rel_l2(g, p.grad.numpy()) < 1e-12


def test_mlp_gradient_matches_finite_differences():
    nin, nh, batch = 6, 8, 5
    rng = np.random.default_rng(9)
    params = 0.5 * rng.standard_normal(oracle.mlp_param_count(nin, nh))
    x = rng.standard_normal((batch, nin))
    t = rng.standard_normal(batch)
    _, g = oracle.mlp_loss_grad(params, x, t, nin, nh)
    eps = 1e-6
    fd = np.zeros_like(params)
    for i in range(params.size):
        pp, pm = params.copy(), params.copy()
        pp[i] += eps
        pm[i] -= eps
        fd[i] = (oracle.mlp_loss_grad(pp, x, t, nin, nh)[0]
                 - oracle.mlp_loss_grad(pm, x, t, nin, nh)[0]) / (2 * eps)
    assert rel_l2(g, fd) < 1e-7
