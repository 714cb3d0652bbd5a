"""FP64 CPU oracle of the FCN z-step (Ma & Lin, arXiv:1507.05988, Sec. 3).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it and shares no code with it.

This module is a ctypes wrapper around ``fcn_oracle.c`` (plain C, FP64).  It
compiles the C file with gcc on first use if the shared object is missing.
Complex arrays are numpy ``complex128`` of shape ``(nr, nt)``; the wrapper
copies in and out, so the caller's arrays are never aliased.

Parity status (per function; the pins live in ``tests/test_oracle_*.py``):
pinned: fft, thomas, cn_coeffs, rho_row, nl_half, linear_step, step, diag,
propagate_adaptive, mlp_forward, mlp_loss_grad, and the Cartesian-grid
functions xy_cn_coeffs, xy_linear_step, xy_run (serial and threaded), xy_diag.  The full coupled run with
all physics on is parity unpinned beyond the invariants those tests check,
because the paper prints no values for it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fcn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

DIFFRACTION = 1
DISPERSION = 2
KERR = 4
PLASMA = 8
MPI = 16
MPI_SAT = 32
PRINTED_CJ = 64
EXACT_DISPERSION = 128
ALL_PHYSICS = DIFFRACTION | DISPERSION | KERR | PLASMA | MPI


def build(force: bool = False) -> str:
    """Compile fcn_oracle.c into liboracle.so (portable flags: x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fno-fast-math",
             "-ffp-contract=off", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("nr", C.c_int), ("nt", C.c_int),
        ("r_max", C.c_double), ("t_window", C.c_double),
        ("lambda0", C.c_double), ("n0", C.c_double),
        ("n2j", C.c_double * 4), ("k2", C.c_double),
        ("sigma_k", C.c_double), ("rho_nt", C.c_double),
        ("K", C.c_int), ("flags", C.c_uint),
    ]


class _Diag(C.Structure):
    _fields_ = [
        ("energy", C.c_double), ("peak_intensity", C.c_double),
        ("peak_rho", C.c_double), ("onaxis_peak", C.c_double),
        ("spectral_rms", C.c_double), ("nonfinite", C.c_int),
    ]


class _Adaptive(C.Structure):
    _fields_ = [
        ("z", C.c_double), ("dz_next", C.c_double),
        ("accepted", C.c_long), ("rejected", C.c_long),
        ("last_err", C.c_double), ("status", C.c_int),
    ]


class _GridXY(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x_width", C.c_double), ("y_width", C.c_double)]


_lib = None
_D = C.POINTER(C.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.POINTER(_Problem)
        sig = {
            "orc_k0": (C.c_double, [P]), "orc_omega0": (C.c_double, [P]),
            "orc_rho_c": (C.c_double, [P]), "orc_beta_k": (C.c_double, [P]),
            "orc_omega": (C.c_double, [P, C.c_int]),
            "orc_fft": (C.c_int, [_D, C.c_int, C.c_int]),
            "orc_thomas": (C.c_int, [C.c_int, _D, _D, _D, _D, _D]),
            "orc_cn_coeffs": (None, [P, C.c_double, C.c_int, _D, _D, _D, _D, _D, _D]),
            "orc_rho_row": (None, [P, _D, _D]),
            "orc_nl_half": (None, [P, C.c_double, _D, _D]),
            "orc_linear_step": (C.c_int, [P, C.c_double, _D]),
            "orc_step": (C.c_int, [P, C.c_double, _D, _D]),
            "orc_run": (C.c_int, [P, C.c_double, C.c_long, _D, _D]),
            "orc_run_threads": (C.c_int, [P, C.c_double, C.c_long, _D, _D, C.c_int]),
            "orc_diag_compute": (None, [P, _D, _D, C.POINTER(_Diag), _D, _D]),
            "orc_propagate_adaptive": (C.c_int, [P, _D, _D, C.c_double, C.c_double,
                                                  C.c_double, C.c_double, C.c_double,
                                                  C.c_int, C.POINTER(_Adaptive)]),
            "orc_xy_cn_coeffs": (None, [P, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int,
                                        _D, _D, _D, _D, _D, _D]),
            "orc_xy_linear_step": (C.c_int, [P, C.POINTER(_GridXY), C.c_double, _D]),
            "orc_xy_run": (C.c_int, [P, C.POINTER(_GridXY), C.c_double, C.c_long, _D, _D]),
            "orc_xy_run_threads": (C.c_int, [P, C.POINTER(_GridXY), C.c_double, C.c_long, _D, _D,
                                             C.c_int]),
            "orc_xy_diag": (None, [P, C.POINTER(_GridXY), _D, _D, C.POINTER(_Diag)]),
            "orc_mlp_forward": (C.c_int, [C.c_int, C.c_int, C.c_int, _D, _D, _D]),
            "orc_mlp_loss_grad": (C.c_int, [C.c_int, C.c_int, C.c_int, _D, _D, _D, _D, _D]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


@dataclass
class Problem:
    """Grid and physics of one FCN problem, SI units (mirrors orc_problem)."""
    nr: int
    nt: int
    r_max: float
    t_window: float
    lambda0: float = 800e-9
    n0: float = 1.0
    n2j: tuple = (0.0, 0.0, 0.0, 0.0)
    k2: float = 0.0
    sigma_k: float = 0.0
    rho_nt: float = 0.0
    K: int = 8
    flags: int = ALL_PHYSICS

    def _c(self) -> _Problem:
        p = _Problem()
        p.nr, p.nt = int(self.nr), int(self.nt)
        p.r_max, p.t_window = float(self.r_max), float(self.t_window)
        p.lambda0, p.n0 = float(self.lambda0), float(self.n0)
        for i in range(4):
            p.n2j[i] = float(self.n2j[i]) if i < len(self.n2j) else 0.0
        p.k2, p.sigma_k, p.rho_nt = float(self.k2), float(self.sigma_k), float(self.rho_nt)
        p.K, p.flags = int(self.K), int(self.flags)
        return p

    # derived constants
    def k0(self) -> float:
        return _load().orc_k0(C.byref(self._c()))

    def omega0(self) -> float:
        return _load().orc_omega0(C.byref(self._c()))

    def rho_c(self) -> float:
        return _load().orc_rho_c(C.byref(self._c()))

    def beta_k(self) -> float:
        return _load().orc_beta_k(C.byref(self._c()))

    def omega(self, q: int) -> float:
        return _load().orc_omega(C.byref(self._c()), int(q))

    @property
    def dr(self) -> float:
        return self.r_max / (self.nr - 1)

    @property
    def dtau(self) -> float:
        return self.t_window / self.nt


def fft(x, inverse: bool = False) -> np.ndarray:
    """Radix-2 transform of a 1-D complex vector (see orc_fft)."""
    a = _c128(x).copy()
    if _load().orc_fft(_ptr(a), a.size, 1 if inverse else 0) != 0:
        raise ValueError("length must be a power of two")
    return a


def thomas(a, b, c, d) -> np.ndarray:
    """Solve a tridiagonal system by the Thomas algorithm (see orc_thomas)."""
    a, b, c, d = (_c128(v) for v in (a, b, c, d))
    n = b.size
    x = np.zeros(n, np.complex128)
    rc = _load().orc_thomas(n, _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(x))
    if rc != 0:
        raise ZeroDivisionError("zero pivot")
    return x


def cn_coeffs(pb: Problem, dz: float, q: int):
    """(a, b, c, d, e, f) diagonals of M_abc^q and M_def^q (see orc_cn_coeffs)."""
    arrs = [np.zeros(pb.nr, np.complex128) for _ in range(6)]
    _load().orc_cn_coeffs(C.byref(pb._c()), float(dz), int(q), *[_ptr(v) for v in arrs])
    return tuple(arrs)


def rho_row(pb: Problem, intensity) -> np.ndarray:
    i = _f64(intensity)
    rho = np.zeros(pb.nt, np.float64)
    _load().orc_rho_row(C.byref(pb._c()), _ptr(i), _ptr(rho))
    return rho


def nl_half(pb: Problem, h: float, row):
    """One nonlinear half step of length h on one row; returns (row, rho)."""
    r = _c128(row).copy()
    rho = np.zeros(pb.nt, np.float64)
    _load().orc_nl_half(C.byref(pb._c()), float(h), _ptr(r), _ptr(rho))
    return r, rho


def linear_step(pb: Problem, dz: float, A) -> np.ndarray:
    a = _c128(A).copy()
    rc = _load().orc_linear_step(C.byref(pb._c()), float(dz), _ptr(a))
    if rc != 0:
        raise RuntimeError(f"orc_linear_step failed ({rc})")
    return a


def run(pb: Problem, dz: float, nsteps: int, A, threads: int = 1):
    """nsteps Strang steps of length dz; returns (field, rho of the last half step).
    threads > 1 runs the paper's row/column thread decomposition (same bits)."""
    a = _c128(A).copy()
    assert a.shape == (pb.nr, pb.nt)
    rho = np.zeros((pb.nr, pb.nt), np.float64)
    if threads > 1:
        rc = _load().orc_run_threads(C.byref(pb._c()), float(dz), int(nsteps), _ptr(a), _ptr(rho),
                                     int(threads))
    else:
        rc = _load().orc_run(C.byref(pb._c()), float(dz), int(nsteps), _ptr(a), _ptr(rho))
    if rc != 0:
        raise RuntimeError(f"orc_run failed ({rc})")
    return a, rho


def step(pb: Problem, dz: float, A):
    return run(pb, dz, 1, A)


def diag(pb: Problem, A, rho=None) -> dict:
    a = _c128(A)
    r = _f64(rho) if rho is not None else None
    out = _Diag()
    power = np.zeros(pb.nt, np.float64)
    fluence = np.zeros(pb.nr, np.float64)
    _load().orc_diag_compute(C.byref(pb._c()), _ptr(a), _ptr(r) if r is not None else None,
                             C.byref(out), _ptr(power), _ptr(fluence))
    return dict(energy=out.energy, peak_intensity=out.peak_intensity,
                peak_rho=out.peak_rho, onaxis_peak=out.onaxis_peak,
                spectral_rms=out.spectral_rms, nonfinite=bool(out.nonfinite),
                power=power, fluence=fluence)


def propagate_adaptive(pb: Problem, A, z0: float, z_end: float, dz0: float,
                       rtol: float = 1e-4, dz_min: float = 1e-9, max_reject: int = 20):
    a = _c128(A).copy()
    rho = np.zeros((pb.nr, pb.nt), np.float64)
    res = _Adaptive()
    _load().orc_propagate_adaptive(C.byref(pb._c()), _ptr(a), _ptr(rho), float(z0),
                                   float(z_end), float(dz0), float(rtol), float(dz_min),
                                   int(max_reject), C.byref(res))
    return a, rho, dict(z=res.z, dz_next=res.dz_next, accepted=res.accepted,
                        rejected=res.rejected, last_err=res.last_err, status=res.status)


@dataclass
class GridXY:
    """Cartesian transverse grid (mirrors orc_xy_grid): nx x ny nodes over
    widths x_width, y_width [m]; the walls (first and last node of each axis)
    hold A = 0.  The field is complex128 of shape (nx, ny, nt)."""
    nx: int
    ny: int
    x_width: float
    y_width: float

    def _c(self) -> _GridXY:
        g = _GridXY()
        g.nx, g.ny = int(self.nx), int(self.ny)
        g.x_width, g.y_width = float(self.x_width), float(self.y_width)
        return g

    @property
    def dx(self) -> float:
        return self.x_width / (self.nx - 1)

    @property
    def dy(self) -> float:
        return self.y_width / (self.ny - 1)

    def x(self) -> np.ndarray:
        return -0.5 * self.x_width + self.dx * np.arange(self.nx)

    def y(self) -> np.ndarray:
        return -0.5 * self.y_width + self.dy * np.arange(self.ny)


def xy_cn_coeffs(pb: Problem, dz: float, q: int, n: int, h: float, with_disp: bool):
    """(a, b, c, d, e, f) of one transverse line's Crank-Nicolson system."""
    arrs = [np.zeros(n, np.complex128) for _ in range(6)]
    _load().orc_xy_cn_coeffs(C.byref(pb._c()), float(dz), int(q), int(n), float(h),
                             1 if with_disp else 0, *[_ptr(v) for v in arrs])
    return tuple(arrs)


def xy_linear_step(pb: Problem, g: GridXY, dz: float, A) -> np.ndarray:
    a = _c128(A).copy()
    assert a.shape == (g.nx, g.ny, pb.nt)
    rc = _load().orc_xy_linear_step(C.byref(pb._c()), C.byref(g._c()), float(dz), _ptr(a))
    if rc != 0:
        raise RuntimeError(f"orc_xy_linear_step failed ({rc})")
    return a


def xy_run(pb: Problem, g: GridXY, dz: float, nsteps: int, A, threads: int = 1):
    """nsteps Strang steps on the Cartesian grid; returns (field, rho).
    threads > 1 splits rows and frequency bins over threads (same bits)."""
    a = _c128(A).copy()
    assert a.shape == (g.nx, g.ny, pb.nt)
    rho = np.zeros(a.shape, np.float64)
    if threads > 1:
        rc = _load().orc_xy_run_threads(C.byref(pb._c()), C.byref(g._c()), float(dz), int(nsteps),
                                        _ptr(a), _ptr(rho), int(threads))
    else:
        rc = _load().orc_xy_run(C.byref(pb._c()), C.byref(g._c()), float(dz), int(nsteps), _ptr(a),
                                _ptr(rho))
    if rc != 0:
        raise RuntimeError(f"orc_xy_run failed ({rc})")
    return a, rho


def xy_diag(pb: Problem, g: GridXY, A, rho=None) -> dict:
    a = _c128(A)
    r = _f64(rho) if rho is not None else None
    out = _Diag()
    _load().orc_xy_diag(C.byref(pb._c()), C.byref(g._c()), _ptr(a),
                        _ptr(r) if r is not None else None, C.byref(out))
    return dict(energy=out.energy, peak_intensity=out.peak_intensity, peak_rho=out.peak_rho,
                onaxis_peak=out.onaxis_peak, spectral_rms=out.spectral_rms,
                nonfinite=bool(out.nonfinite))


def mlp_param_count(nin: int, nh: int) -> int:
    return nh * nin + nh + nh * nh + nh + nh + 1


def mlp_forward(params, x, nin: int, nh: int) -> np.ndarray:
    p = _f64(params)
    xx = _f64(x)
    batch = xx.size // nin
    y = np.zeros(batch, np.float64)
    _load().orc_mlp_forward(batch, nin, nh, _ptr(p), _ptr(xx), _ptr(y))
    return y


def mlp_loss_grad(params, x, target, nin: int, nh: int):
    p = _f64(params)
    xx = _f64(x)
    t = _f64(target)
    batch = xx.size // nin
    loss = C.c_double()
    g = np.zeros(p.size, np.float64)
    _load().orc_mlp_loss_grad(batch, nin, nh, _ptr(p), _ptr(xx), _ptr(t), C.byref(loss), _ptr(g))
    return loss.value, g
