"""Seeded synthetic workloads: grids, physics parameters and initial pulses.

This module only *generates inputs*.  It holds none of the FCN step's
arithmetic, imports neither the CUDA binding nor the oracle, and serves both
of them: the same host arrays it returns are handed to the oracle and to the
CUDA path.

Physics parameters are SI.  The MPI cross section sigma_8 = 2.88e-99
s^-1 cm^16 W^-8 and rho_nt = 5.4e18 cm^-3 are converted here (1 cm^16 =
1e-32 m^16, 1 cm^-3 = 1e6 m^-3).  k'' = 0.2 fs^2/cm (Sec. 2) is 2e-29 s^2/m.

Initial pulse (Sec. 5, Eq. (gauss)):
    A(r, 0, tau) = sqrt(I0) exp(-r^2/w0^2 - tau^2/tp^2 - i C tau^2/tp^2)
with I0 = 2 P / (pi w0^2) (peak intensity of a Gaussian beam of power P) and
P a multiple of the critical power P_cr = 3.77 lambda0^2 / (8 pi n0 n2)
(Sec. 2, below Eq. (kerrsource)).  The grid samples r_m = m R/(Nr-1) and
tau_p = -T/2 + p T/Nt.  An optional multiplicative amplitude perturbation
(1 + u), u uniform in [-0.01, 0.01], is drawn row-major from numpy's PCG64
with the given seed.
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

LAMBDA0 = 800e-9
N0 = 1.0
N2 = 3.2e-23                 # m^2/W
N4 = -2.5e-37                # m^4/W^2
K2 = 0.2e-30 / 1e-2          # 0.2 fs^2/cm in s^2/m
K_MPI = 8
SIGMA_K = 2.88e-99 * 1e-32   # s^-1 m^16 W^-8
RHO_NT = 5.4e18 * 1e6        # m^-3

# physics switches (same bit meaning on both sides of the parity tests)
DIFFRACTION, DISPERSION, KERR, PLASMA, MPI, MPI_SAT = 1, 2, 4, 8, 16, 32
ALL_PHYSICS = DIFFRACTION | DISPERSION | KERR | PLASMA | MPI
EXACT_DISPERSION = 128        # dispersion as its exact factor per frequency (variant of R7)


def critical_power(lambda0: float = LAMBDA0, n0: float = N0, n2: float = N2) -> float:
    """P_cr = 3.77 lambda0^2 / (8 pi n0 n2) (Sec. 2)."""
    return 3.77 * lambda0 ** 2 / (8.0 * np.pi * n0 * n2)


def peak_intensity(power: float, w0: float) -> float:
    """I0 of sqrt(I0) exp(-r^2/w0^2): 2 P / (pi w0^2)."""
    return 2.0 * power / (np.pi * w0 ** 2)


@dataclass
class Workload:
    """One pulse: grid + physics + the input pulse recipe + the run length."""
    name: str
    nr: int
    nt: int
    w0: float
    tp: float
    p_over_pcr: float
    r_max: float = 0.0          # default 5 w0
    t_window: float = 0.0       # default 16 tp
    chirp: float = 0.0
    n2j: tuple = (N2, 0.0, 0.0, 0.0)
    k2: float = K2
    sigma_k: float = SIGMA_K
    rho_nt: float = RHO_NT
    K: int = K_MPI
    lambda0: float = LAMBDA0
    n0: float = N0
    flags: int = ALL_PHYSICS
    dz: float = 1e-2
    nsteps: int = 200
    noise_seed: int | None = None
    noise_amp: float = 0.01

    def __post_init__(self):
        if self.r_max <= 0:
            self.r_max = 5.0 * self.w0
        if self.t_window <= 0:
            self.t_window = 16.0 * self.tp

    @property
    def i0(self) -> float:
        return peak_intensity(self.p_over_pcr * critical_power(self.lambda0, self.n0, self.n2j[0]),
                              self.w0)

    @property
    def points(self) -> int:
        return self.nr * self.nt

    def physics(self) -> dict:
        """Keyword arguments shared by oracle.Problem and the CUDA binding."""
        return dict(nr=self.nr, nt=self.nt, r_max=self.r_max, t_window=self.t_window,
                    lambda0=self.lambda0, n0=self.n0, n2j=tuple(self.n2j), k2=self.k2,
                    sigma_k=self.sigma_k, rho_nt=self.rho_nt, K=self.K, flags=self.flags)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)

    def field(self) -> np.ndarray:
        """Initial field (nr, nt) complex128 per Eq. (gauss) (+ optional noise)."""
        r = np.arange(self.nr, dtype=np.float64) * (self.r_max / (self.nr - 1))
        tau = -0.5 * self.t_window + np.arange(self.nt, dtype=np.float64) * (self.t_window / self.nt)
        rr = (r / self.w0) ** 2
        tt = (tau / self.tp) ** 2
        a = np.sqrt(self.i0) * np.exp(-rr[:, None] - tt[None, :] - 1j * self.chirp * tt[None, :])
        if self.noise_seed is not None:
            rng = np.random.Generator(np.random.PCG64(self.noise_seed))
            u = rng.uniform(-self.noise_amp, self.noise_amp, size=(self.nr, self.nt))
            a = a * (1.0 + u)
        return np.ascontiguousarray(a.astype(np.complex128))


def config1() -> Workload:
    """Plain FCN, FP64: 128 x 256, w0 = 1 mm, tp = 100 fs, 3 P_cr, n2 only,
    200 steps of 1 cm (deterministic)."""
    return Workload("cfg1_128x256", nr=128, nt=256, w0=1e-3, tp=100e-15, p_over_pcr=3.0,
                    dz=1e-2, nsteps=200)


def config2(seed: int | None = 0) -> Workload:
    """Filamentation regime: 1024 x 4096, w0 = 2 mm, tp = 50 fs, 5 P_cr,
    n2 + n4, 1 % uniform amplitude noise (seed 0), 1000 steps of 2 mm."""
    return Workload("cfg2_1024x4096", nr=1024, nt=4096, w0=2e-3, tp=50e-15, p_over_pcr=5.0,
                    n2j=(N2, N4, 0.0, 0.0), dz=2e-3, nsteps=1000, noise_seed=seed)


def config3() -> Workload:
    """Long-distance run: 2048 x 8192, w0 = 5 mm, tp = 100 fs, 10 P_cr,
    n2 + n4, 1 km adaptive (rtol 1e-4)."""
    return Workload("cfg3_2048x8192", nr=2048, nt=8192, w0=5e-3, tp=100e-15, p_over_pcr=10.0,
                    n2j=(N2, N4, 0.0, 0.0), dz=1.0, nsteps=0)


def config4(n: int = 64, seed: int = 0) -> list[Workload]:
    """Batched form: n pulses drawn in order (Nr, Nt, P, w0, tp) per pulse from
    PCG64(seed); R = 5 w0, T = 16 tp, dz = 2 mm, 500 steps, n2 only."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        nr = int(rng.choice([256, 512, 1024, 2048]))
        nt = int(rng.choice([512, 1024, 4096, 8192]))
        p = float(rng.uniform(1.0, 10.0))
        w0 = float(rng.uniform(0.5e-3, 5e-3))
        tp = float(rng.uniform(30e-15, 200e-15))
        out.append(Workload(f"cfg4_{i:02d}_{nr}x{nt}", nr=nr, nt=nt, w0=w0, tp=tp,
                            p_over_pcr=p, dz=2e-3, nsteps=500))
    return out


def config5(seed: int | None = 0) -> Workload:
    """Learned-dz form on the config-2 grid over 1 km."""
    return config2(seed).with_(name="cfg5_1024x4096_1km", nsteps=0)


def application_1km() -> Workload:
    """The paper's application run (Sec. 5, Fig. 4): Nr = 1350, Nt = 1024,
    1.1e6 steps over 1.1 km; peak intensity 3.14e14 W/m^2, r0 = 18 mm,
    tau0 = 300 fs (P = 53.3 P_cr), n2 only.  The paper gives no windows:
    R = 5 r0 and T = 16 tau0 as for the other workloads."""
    w0, i0 = 18e-3, 3.14e14
    p_cr = 3.77 * LAMBDA0 ** 2 / (8.0 * np.pi * N0 * N2)
    p = i0 * np.pi * w0 ** 2 / 2.0
    return Workload("app_1350x1024_1km", nr=1350, nt=1024, w0=w0, tp=300e-15,
                    p_over_pcr=p / p_cr, dz=1e-3, nsteps=1_100_000)


@dataclass
class WorkloadXY:
    """One pulse on a Cartesian transverse grid (Sec. 2: Delta_perp = d^2/dx^2
    + d^2/dy^2): nx x ny nodes over x_width x y_width (default 10 w0 each,
    walls at +-5 w0 holding A = 0), Nt points over t_window (default 16 tp).
    Input: sqrt(I0) exp(-x^2/wx^2 - y^2/wy^2 - tau^2/tp^2 - i C tau^2/tp^2)
    with I0 = 2 P/(pi wx wy) (the peak intensity of an elliptical Gaussian
    beam of power P), times (1 + u) with optional noise as for Workload."""
    name: str
    nx: int
    ny: int
    nt: int
    w0: float
    tp: float
    p_over_pcr: float
    w0y: float = 0.0            # default w0 (round beam)
    x_width: float = 0.0        # default 10 w0
    y_width: float = 0.0        # default 10 w0y
    t_window: float = 0.0       # default 16 tp
    chirp: float = 0.0
    n2j: tuple = (N2, 0.0, 0.0, 0.0)
    k2: float = K2
    sigma_k: float = SIGMA_K
    rho_nt: float = RHO_NT
    K: int = K_MPI
    lambda0: float = LAMBDA0
    n0: float = N0
    flags: int = ALL_PHYSICS
    dz: float = 1e-2
    nsteps: int = 200
    noise_seed: int | None = None
    noise_amp: float = 0.01

    def __post_init__(self):
        if self.w0y <= 0:
            self.w0y = self.w0
        if self.x_width <= 0:
            self.x_width = 10.0 * self.w0
        if self.y_width <= 0:
            self.y_width = 10.0 * self.w0y
        if self.t_window <= 0:
            self.t_window = 16.0 * self.tp

    @property
    def i0(self) -> float:
        p = self.p_over_pcr * critical_power(self.lambda0, self.n0, self.n2j[0])
        return 2.0 * p / (np.pi * self.w0 * self.w0y)

    @property
    def points(self) -> int:
        return self.nx * self.ny * self.nt

    def grid(self) -> dict:
        """Keyword arguments of the Cartesian grid (oracle.GridXY and the binding)."""
        return dict(nx=self.nx, ny=self.ny, x_width=self.x_width, y_width=self.y_width)

    def physics(self) -> dict:
        """Physics and time grid, as Workload.physics (nr, r_max unused: 3, 0)."""
        return dict(nr=3, nt=self.nt, r_max=0.0, t_window=self.t_window, lambda0=self.lambda0,
                    n0=self.n0, n2j=tuple(self.n2j), k2=self.k2, sigma_k=self.sigma_k,
                    rho_nt=self.rho_nt, K=self.K, flags=self.flags)

    def with_(self, **kw) -> "WorkloadXY":
        return replace(self, **kw)

    def field(self) -> np.ndarray:
        """Initial field (nx, ny, nt) complex128."""
        x = -0.5 * self.x_width + np.arange(self.nx) * (self.x_width / (self.nx - 1))
        y = -0.5 * self.y_width + np.arange(self.ny) * (self.y_width / (self.ny - 1))
        tau = -0.5 * self.t_window + np.arange(self.nt) * (self.t_window / self.nt)
        tt = (tau / self.tp) ** 2
        a = (np.sqrt(self.i0) * np.exp(-(x / self.w0) ** 2)[:, None, None]
             * np.exp(-(y / self.w0y) ** 2)[None, :, None]
             * np.exp(-tt - 1j * self.chirp * tt)[None, None, :])
        if self.noise_seed is not None:
            rng = np.random.Generator(np.random.PCG64(self.noise_seed))
            u = rng.uniform(-self.noise_amp, self.noise_amp, size=a.shape)
            a = a * (1.0 + u)
        return np.ascontiguousarray(a.astype(np.complex128))


def cartesian_config1() -> WorkloadXY:
    """Config 1's pulse (w0 = 1 mm, tp = 100 fs, 3 P_cr, n2 only, 200 steps
    of 1 cm) on a Cartesian grid of 255 x 255 x 256: the walls at +-5 w0 and
    dx = dy = 10 mm/254, the radial grid's dr, so the centre node and the
    nodes along the axes coincide with the radial grid's."""
    return WorkloadXY("cart_cfg1_255x255x256", nx=255, ny=255, nt=256, w0=1e-3, tp=100e-15,
                      p_over_pcr=3.0, dz=1e-2, nsteps=200)


def small_xy(nx: int = 21, ny: int = 17, nt: int = 32, **kw) -> WorkloadXY:
    """A small Cartesian grid with config-1 physics for fast tests."""
    base = dict(name=f"small_xy_{nx}x{ny}x{nt}", nx=nx, ny=ny, nt=nt, w0=1e-3, tp=100e-15,
                p_over_pcr=3.0, dz=1e-2, nsteps=10)
    base.update(kw)
    return WorkloadXY(**base)


def small(nr: int = 48, nt: int = 64, **kw) -> Workload:
    """A small grid with config-1 physics for fast tests."""
    base = dict(name=f"small_{nr}x{nt}", nr=nr, nt=nt, w0=1e-3, tp=100e-15, p_over_pcr=3.0,
                dz=1e-2, nsteps=10)
    base.update(kw)
    return Workload(**base)
