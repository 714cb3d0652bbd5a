"""Thin ctypes binding of the C-ABI in ``include/fcn.h``.

Every function keeps its C name and only marshals arguments: numpy host
arrays become ``double*``, torch CUDA tensors become device pointers, and a
torch stream becomes a ``cudaStream_t``.  All computation happens in the
CUDA library ``libfcn_gb300.so``; importing this module fails loudly if that
library is missing (build it with ``paper_1507_05988_gb300.build.build()``).

``Solver`` is a small convenience wrapper over one context.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfcn_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python -c 'import __graft_entry__ as g; g.build()')")

lib = C.CDLL(LIB_PATH)

# ---- constants (mirror include/fcn.h) ----
FCN_OK = 0
FCN_ERR_ARG = -1
FCN_ERR_CUDA = -2
FCN_ERR_NONFINITE = -3
FCN_ERR_STEP_UNDERFLOW = -4
FCN_ERR_UNSUPPORTED = -5
FCN_ERR_NOMEM = -6
FCN_ERR_STATE = -7
FCN_DIFFRACTION, FCN_DISPERSION, FCN_KERR, FCN_PLASMA, FCN_MPI, FCN_MPI_SAT = 1, 2, 4, 8, 16, 32
FCN_ALL_PHYSICS = 31
FCN_EXACT_DISPERSION = 128
FCN_FP64 = 0
FCN_FP32_MIXED = 1
FCN_OP_IFFT, FCN_OP_NL, FCN_OP_NL2, FCN_OP_FFT, FCN_OP_RHO = 1, 2, 4, 8, 16
FCN_MLP_NIN, FCN_MLP_NH, FCN_MLP_NPARAM = 6, 64, 4673
FCN_MLP_LOG_FLOATS = 9
FCN_NOALLOC_SCRATCH_BYTES = 8 * 1024 * 1024
FCN_PROF_ROW_HEAD, FCN_PROF_ROW_MID, FCN_PROF_ROW_TAIL, FCN_PROF_COLUMN, FCN_PROF_KINDS = 0, 1, 2, 3, 4
FCN_XY_PROF_KINDS = 5


class fcn_grid(C.Structure):
    _fields_ = [("nr", C.c_int32), ("nt", C.c_int32), ("r_max", C.c_double),
                ("t_window", C.c_double)]


class fcn_params(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("n0", C.c_double), ("n2j", C.c_double * 4),
                ("k2", C.c_double), ("sigma_k", C.c_double), ("rho_nt", C.c_double),
                ("K", C.c_int32), ("flags", C.c_uint32)]


class fcn_grid_xy(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nt", C.c_int32), ("pad_", C.c_int32),
                ("x_width", C.c_double), ("y_width", C.c_double), ("t_window", C.c_double)]


class fcn_diag(C.Structure):
    _fields_ = [("z", C.c_double), ("energy", C.c_double), ("peak_intensity", C.c_double),
                ("peak_rho", C.c_double), ("onaxis_peak", C.c_double),
                ("spectral_rms", C.c_double), ("steps", C.c_int64), ("rejected", C.c_int64),
                ("nonfinite", C.c_int32), ("pad_", C.c_int32)]


class fcn_stats(C.Structure):
    _fields_ = [("z", C.c_double), ("dz_next", C.c_double), ("last_err", C.c_double),
                ("accepted", C.c_int64), ("rejected", C.c_int64), ("substeps", C.c_int64),
                ("mlp_proposals", C.c_int64)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_G = C.POINTER(fcn_grid)
_PR = C.POINTER(fcn_params)
_CTX = C.c_void_p

_SIGS = {
    "fcn_version": (C.c_char_p, []),
    "fcn_create": (C.c_int, [_G, _PR, C.c_int32, _P, C.POINTER(_CTX)]),
    "fcn_create_batch": (C.c_int, [C.c_int32, _G, _PR, C.c_int32, _P, C.POINTER(_CTX)]),
    "fcn_destroy": (None, [_CTX]),
    "fcn_last_error": (C.c_char_p, [_CTX]),
    "fcn_set_stream": (C.c_int, [_CTX, _P]),
    "fcn_set_field": (C.c_int, [_CTX, C.c_int32, _D]),
    "fcn_set_field_device": (C.c_int, [_CTX, C.c_int32, _P]),
    "fcn_get_field": (C.c_int, [_CTX, C.c_int32, _D]),
    "fcn_get_field_device": (C.c_int, [_CTX, C.c_int32, _P]),
    "fcn_get_rho": (C.c_int, [_CTX, C.c_int32, _D]),
    "fcn_step": (C.c_int, [_CTX, C.c_double, C.c_int64]),
    "fcn_step_nograph": (C.c_int, [_CTX, C.c_double, C.c_int64]),
    "fcn_propagate": (C.c_int, [_CTX, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.c_int32, C.c_int32, C.POINTER(fcn_stats)]),
    "fcn_get_diag": (C.c_int, [_CTX, C.c_int32, C.POINTER(fcn_diag)]),
    "fcn_get_profiles": (C.c_int, [_CTX, C.c_int32, _D, _D]),
    "fcn_get_state": (C.c_int, [_CTX, C.c_int32, _D]),
    "fcn_set_state": (C.c_int, [_CTX, C.c_int32, _D]),
    "fcn_set_variants": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "fcn_get_variants": (C.c_int, [_CTX, C.c_int32, C.POINTER(C.c_int32)]),
    "fcn_set_batching": (C.c_int, [_CTX, C.c_int32]),
    "fcn_set_pairing": (C.c_int, [_CTX, C.c_int32]),
    "fcn_get_pairing": (C.c_int, [_CTX]),
    "fcn_alu_peak": (C.c_int, [C.c_int32, _D, C.c_void_p]),
    "fcn_set_sequential_columns": (C.c_int, [_CTX, C.c_int32]),
    "fcn_get_sequential_columns": (C.c_int, [_CTX]),
    "fcn_set_field_c64": (C.c_int, [_CTX, C.c_int32, C.POINTER(C.c_float)]),
    "fcn_get_field_c64": (C.c_int, [_CTX, C.c_int32, C.POINTER(C.c_float)]),
    "fcn_set_graph_branches": (C.c_int, [_CTX, C.c_int32]),
    "fcn_get_graph_branches": (C.c_int, [_CTX]),
    "fcn_set_multi_launch": (C.c_int, [_CTX, C.c_int32]),
    "fcn_get_multi_launch": (C.c_int, [_CTX]),
    "fcn_profile_enable": (C.c_int, [_CTX, C.c_int32]),
    "fcn_profile_read": (C.c_int, [_CTX, _D, C.POINTER(C.c_int64), C.c_int32]),
    "fcn_mlp_set": (C.c_int, [_CTX, _F]),
    "fcn_mlp_get": (C.c_int, [_CTX, _F]),
    "fcn_mlp_set_log": (C.c_int, [_CTX, _F, C.c_int64]),
    "fcn_mlp_log_count": (C.c_int64, [_CTX]),
    "fcn_mlp_train": (C.c_int, [_CTX, _F, _F, C.c_int32, C.c_int32, C.c_int32, C.c_float,
                                C.c_uint64, _F]),
    "fcn_mlp_loss_grad": (C.c_int, [_F, _F, _F, C.c_int32, _F, _F]),
    "fcn_op_rows": (C.c_int, [_G, _PR, C.c_int32, C.c_int32, C.c_double, _P, _P, _P]),
    "fcn_cn_table_entries": (C.c_int64, [_G]),
    "fcn_op_cn_table": (C.c_int, [_G, _PR, C.c_int32, C.c_double, _P, _P]),
    "fcn_op_cn": (C.c_int, [_G, _PR, C.c_int32, C.c_double, _P, _P, _P]),
    "fcn_op_cn_noalloc": (C.c_int, [_G, _PR, C.c_int32, C.c_double, _P, _P]),
    "fcn_xy_create": (C.c_int, [C.POINTER(fcn_grid_xy), _PR, C.c_int32, _P, C.POINTER(_CTX)]),
    "fcn_xy_destroy": (None, [_CTX]),
    "fcn_xy_last_error": (C.c_char_p, [_CTX]),
    "fcn_xy_set_field": (C.c_int, [_CTX, _D]),
    "fcn_xy_get_field": (C.c_int, [_CTX, _D]),
    "fcn_xy_set_field_c64": (C.c_int, [_CTX, _F]),
    "fcn_xy_get_field_c64": (C.c_int, [_CTX, _F]),
    "fcn_xy_set_field_device": (C.c_int, [_CTX, _P]),
    "fcn_xy_get_field_device": (C.c_int, [_CTX, _P]),
    "fcn_xy_get_rho": (C.c_int, [_CTX, _D]),
    "fcn_xy_step": (C.c_int, [_CTX, C.c_double, C.c_int64]),
    "fcn_xy_step_nograph": (C.c_int, [_CTX, C.c_double, C.c_int64]),
    "fcn_xy_get_diag": (C.c_int, [_CTX, C.POINTER(fcn_diag)]),
    "fcn_xy_set_variants": (C.c_int, [_CTX, C.c_int32, C.c_int32]),
    "fcn_xy_get_variants": (C.c_int, [_CTX, C.POINTER(C.c_int32)]),
    "fcn_xy_profile_enable": (C.c_int, [_CTX, C.c_int32]),
    "fcn_xy_profile_read": (C.c_int, [_CTX, _D, C.POINTER(C.c_int64), C.c_int32]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args
    globals()[_name] = _fn


class FcnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fcn error {code}: {msg}")
        self.code = code


def check(rc: int, ctx=None) -> int:
    if rc != FCN_OK:
        raise FcnError(rc, (fcn_last_error(ctx) or b"").decode())
    return rc


def make_grid(nr, nt, r_max, t_window) -> fcn_grid:
    return fcn_grid(int(nr), int(nt), float(r_max), float(t_window))


def make_params(lambda0=800e-9, n0=1.0, n2j=(0.0, 0.0, 0.0, 0.0), k2=0.0, sigma_k=0.0,
                rho_nt=0.0, K=8, flags=FCN_ALL_PHYSICS) -> fcn_params:
    p = fcn_params()
    p.lambda0, p.n0, p.k2 = float(lambda0), float(n0), float(k2)
    for i in range(4):
        p.n2j[i] = float(n2j[i]) if i < len(n2j) else 0.0
    p.sigma_k, p.rho_nt, p.K, p.flags = float(sigma_k), float(rho_nt), int(K), int(flags)
    return p


def grid_params(phys: dict):
    """(fcn_grid, fcn_params) from a dict with the keys of Workload.physics()."""
    g = make_grid(phys["nr"], phys["nt"], phys["r_max"], phys["t_window"])
    p = make_params(phys["lambda0"], phys["n0"], phys["n2j"], phys["k2"], phys["sigma_k"],
                    phys["rho_nt"], phys["K"], phys["flags"])
    return g, p


def mlp_loss_grad(params, x, y):
    """GPU mean squared error and gradient of the dz network (stateless)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    yy = np.ascontiguousarray(y, dtype=np.float32)
    loss = C.c_float()
    g = np.zeros(FCN_MLP_NPARAM, np.float32)
    check(fcn_mlp_loss_grad(p.ctypes.data_as(_F), xx.ctypes.data_as(_F), yy.ctypes.data_as(_F),
                            yy.size, C.byref(loss), g.ctypes.data_as(_F)), None)
    return loss.value, g


def stream_ptr(stream=None):
    """cudaStream_t of a torch stream (None: torch's current stream)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def tensor_ptr(t):
    return C.c_void_p(t.data_ptr())


class Solver:
    """One FCN context (single pulse, or a batch of pulses)."""

    def __init__(self, phys, precision=FCN_FP64, stream=None):
        plist = phys if isinstance(phys, (list, tuple)) else [phys]
        gs, ps = zip(*(grid_params(p) for p in plist))
        self.grids = list(gs)
        self.n = len(plist)
        self.precision = precision
        ctx = _CTX()
        st = stream if stream is not None else C.c_void_p(0)
        if self.n == 1:
            rc = fcn_create(C.byref(self.grids[0]), C.byref(ps[0]), precision, st, C.byref(ctx))
        else:
            ga = (fcn_grid * self.n)(*self.grids)
            pa = (fcn_params * self.n)(*ps)
            rc = fcn_create_batch(self.n, ga, pa, precision, st, C.byref(ctx))
        check(rc, None)
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", None):
            fcn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _shape(self, pulse):
        g = self.grids[pulse]
        return g.nr, g.nt

    def set_field(self, a: np.ndarray, pulse: int = 0):
        a = np.ascontiguousarray(a, dtype=np.complex128)
        assert a.shape == self._shape(pulse)
        check(fcn_set_field(self.ctx, pulse, a.ctypes.data_as(_D)), self.ctx)

    def get_field(self, pulse: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        out = np.empty(self._shape(pulse), np.complex128) if out is None else out
        check(fcn_get_field(self.ctx, pulse, out.ctypes.data_as(_D)), self.ctx)
        return out

    def set_field_c64(self, a: np.ndarray, pulse: int = 0):
        a = np.ascontiguousarray(a, dtype=np.complex64)
        assert a.shape == self._shape(pulse)
        check(fcn_set_field_c64(self.ctx, pulse, a.ctypes.data_as(_F)), self.ctx)

    def set_field_device(self, t, pulse: int = 0):
        """From a contiguous CUDA tensor in the working precision
        (complex128 for FCN_FP64, complex64 for FCN_FP32_MIXED)."""
        check(fcn_set_field_device(self.ctx, pulse, tensor_ptr(t)), self.ctx)

    def get_field_device(self, t, pulse: int = 0):
        """Into a contiguous CUDA tensor in the working precision."""
        check(fcn_get_field_device(self.ctx, pulse, tensor_ptr(t)), self.ctx)
        return t

    def get_field_c64(self, pulse: int = 0, out: np.ndarray | None = None) -> np.ndarray:
        out = np.empty(self._shape(pulse), np.complex64) if out is None else out
        check(fcn_get_field_c64(self.ctx, pulse, out.ctypes.data_as(_F)), self.ctx)
        return out

    def get_rho(self, pulse: int = 0) -> np.ndarray:
        out = np.empty(self._shape(pulse), np.float64)
        check(fcn_get_rho(self.ctx, pulse, out.ctypes.data_as(_D)), self.ctx)
        return out

    def step(self, dz: float, n: int = 1, graph: bool = True):
        fn = fcn_step if graph else fcn_step_nograph
        check(fn(self.ctx, float(dz), int(n)), self.ctx)

    def propagate(self, z_end, dz0, rtol=1e-4, dz_min=1e-9, max_reject=20, controller=0) -> dict:
        st = fcn_stats()
        rc = fcn_propagate(self.ctx, float(z_end), float(dz0), float(rtol), float(dz_min),
                           int(max_reject), int(controller), C.byref(st))
        check(rc, self.ctx)
        return {k: getattr(st, k) for k, _ in fcn_stats._fields_}

    def diag(self, pulse: int = 0) -> dict:
        d = fcn_diag()
        check(fcn_get_diag(self.ctx, pulse, C.byref(d)), self.ctx)
        return {k: getattr(d, k) for k, _ in fcn_diag._fields_ if k != "pad_"}

    def profiles(self, pulse: int = 0):
        nr, nt = self._shape(pulse)
        p = np.empty(nt, np.float64)
        f = np.empty(nr, np.float64)
        check(fcn_get_profiles(self.ctx, pulse, p.ctypes.data_as(_D), f.ctypes.data_as(_D)), self.ctx)
        return p, f

    def get_state(self, pulse: int = 0) -> np.ndarray:
        s = np.zeros(4, np.float64)
        check(fcn_get_state(self.ctx, pulse, s.ctypes.data_as(_D)), self.ctx)
        return s

    def set_variants(self, row: int = -1, col: int = -1):
        check(fcn_set_variants(self.ctx, int(row), int(col)), self.ctx)

    def set_batching(self, mode: int):
        check(fcn_set_batching(self.ctx, int(mode)), self.ctx)

    def set_pairing(self, mode: int):
        check(fcn_set_pairing(self.ctx, int(mode)), self.ctx)

    def pairing(self) -> int:
        return int(fcn_get_pairing(self.ctx))

    def set_sequential_columns(self, mode: int):
        check(fcn_set_sequential_columns(self.ctx, int(mode)), self.ctx)

    def sequential_columns(self) -> int:
        return int(fcn_get_sequential_columns(self.ctx))

    def set_graph_branches(self, n: int):
        check(fcn_set_graph_branches(self.ctx, int(n)), self.ctx)

    def graph_branches(self) -> int:
        return int(fcn_get_graph_branches(self.ctx))

    def set_multi_launch(self, mode: int):
        check(fcn_set_multi_launch(self.ctx, int(mode)), self.ctx)

    def multi_launch(self) -> int:
        return int(fcn_get_multi_launch(self.ctx))

    def variants(self, pulse: int = 0):
        out = (C.c_int32 * 2)()
        check(fcn_get_variants(self.ctx, pulse, out), self.ctx)
        return out[0], out[1]

    def profile(self, on):
        """False/0: off; True/1: direct launches, an event pair around each;
        2: graphs captured with event nodes around each kernel (the launch
        structure and timing of an unprofiled graph replay)."""
        mode = (1 if on else 0) if isinstance(on, bool) else int(on)
        check(fcn_profile_enable(self.ctx, mode), self.ctx)

    def profile_read(self, reset: bool = True) -> dict:
        ms = (C.c_double * FCN_PROF_KINDS)()
        n = (C.c_int64 * FCN_PROF_KINDS)()
        check(fcn_profile_read(self.ctx, ms, n, 1 if reset else 0), self.ctx)
        names = ("row_head", "row_mid", "row_tail", "column")
        return {names[k]: (ms[k], n[k]) for k in range(FCN_PROF_KINDS)}

    # ---- learned dz ----
    def mlp_set(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == FCN_MLP_NPARAM
        check(fcn_mlp_set(self.ctx, p.ctypes.data_as(_F)), self.ctx)

    def mlp_get(self) -> np.ndarray:
        p = np.empty(FCN_MLP_NPARAM, np.float32)
        check(fcn_mlp_get(self.ctx, p.ctypes.data_as(_F)), self.ctx)
        return p

    def mlp_log(self, capacity: int):
        """Starts logging adaptive attempts; returns the buffer (kept alive here)."""
        self._log = np.zeros((max(capacity, 0), FCN_MLP_LOG_FLOATS), np.float32)
        check(fcn_mlp_set_log(self.ctx, self._log.ctypes.data_as(_F), int(capacity)), self.ctx)
        return self._log

    def mlp_log_records(self) -> np.ndarray:
        n = fcn_mlp_log_count(self.ctx)
        return self._log[:n].copy()

    def mlp_train(self, x, y, epochs=50, batch=256, lr=1e-3, seed=0) -> float:
        xx = np.ascontiguousarray(x, dtype=np.float32)
        yy = np.ascontiguousarray(y, dtype=np.float32)
        loss = C.c_float()
        check(fcn_mlp_train(self.ctx, xx.ctypes.data_as(_F), yy.ctypes.data_as(_F), yy.size,
                            int(epochs), int(batch), float(lr), int(seed), C.byref(loss)), self.ctx)
        return loss.value

    def set_state(self, s, pulse: int = 0):
        s = np.ascontiguousarray(s, dtype=np.float64)
        check(fcn_set_state(self.ctx, pulse, s.ctypes.data_as(_D)), self.ctx)


def check_xy(rc: int, ctx=None) -> int:
    if rc != FCN_OK:
        raise FcnError(rc, (fcn_xy_last_error(ctx) or b"").decode())
    return rc


class SolverXY:
    """One Cartesian-grid (3D+1) context: field (nx, ny, nt)."""

    def __init__(self, grid: dict, phys: dict, precision=FCN_FP64, stream=None):
        """grid: nx, ny, x_width, y_width (WorkloadXY.grid()); phys: the
        physics and time-grid keys of Workload.physics() (nr, r_max unused)."""
        self.g = fcn_grid_xy(int(grid["nx"]), int(grid["ny"]), int(phys["nt"]), 0,
                             float(grid["x_width"]), float(grid["y_width"]), float(phys["t_window"]))
        _, p = grid_params(phys)
        self.precision = precision
        ctx = _CTX()
        st = stream if stream is not None else C.c_void_p(0)
        check_xy(fcn_xy_create(C.byref(self.g), C.byref(p), precision, st, C.byref(ctx)), None)
        self.ctx = ctx

    @property
    def shape(self):
        return self.g.nx, self.g.ny, self.g.nt

    def close(self):
        if getattr(self, "ctx", None):
            fcn_xy_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_field(self, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.complex128)
        assert a.shape == self.shape
        check_xy(fcn_xy_set_field(self.ctx, a.ctypes.data_as(_D)), self.ctx)

    def get_field(self, out: np.ndarray | None = None) -> np.ndarray:
        out = np.empty(self.shape, np.complex128) if out is None else out
        check_xy(fcn_xy_get_field(self.ctx, out.ctypes.data_as(_D)), self.ctx)
        return out

    def set_field_c64(self, a: np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.complex64)
        assert a.shape == self.shape
        check_xy(fcn_xy_set_field_c64(self.ctx, a.ctypes.data_as(_F)), self.ctx)

    def get_field_c64(self, out: np.ndarray | None = None) -> np.ndarray:
        out = np.empty(self.shape, np.complex64) if out is None else out
        check_xy(fcn_xy_get_field_c64(self.ctx, out.ctypes.data_as(_F)), self.ctx)
        return out

    def set_field_device(self, t):
        """From a contiguous CUDA tensor in the working precision."""
        check_xy(fcn_xy_set_field_device(self.ctx, tensor_ptr(t)), self.ctx)

    def get_field_device(self, t):
        """Into a contiguous CUDA tensor in the working precision."""
        check_xy(fcn_xy_get_field_device(self.ctx, tensor_ptr(t)), self.ctx)
        return t

    def get_rho(self) -> np.ndarray:
        out = np.empty(self.shape, np.float64)
        check_xy(fcn_xy_get_rho(self.ctx, out.ctypes.data_as(_D)), self.ctx)
        return out

    def step(self, dz: float, n: int = 1, graph: bool = True):
        fn = fcn_xy_step if graph else fcn_xy_step_nograph
        check_xy(fn(self.ctx, float(dz), int(n)), self.ctx)

    def diag(self) -> dict:
        d = fcn_diag()
        check_xy(fcn_xy_get_diag(self.ctx, C.byref(d)), self.ctx)
        return {k: getattr(d, k) for k, _ in fcn_diag._fields_ if k != "pad_"}

    def set_variants(self, row: int = -1, line: int = -1):
        check_xy(fcn_xy_set_variants(self.ctx, int(row), int(line)), self.ctx)

    def variants(self):
        out = (C.c_int32 * 2)()
        check_xy(fcn_xy_get_variants(self.ctx, out), self.ctx)
        return out[0], out[1]

    def profile(self, on: bool):
        check_xy(fcn_xy_profile_enable(self.ctx, 1 if on else 0), self.ctx)

    def profile_read(self, reset: bool = True) -> dict:
        ms = (C.c_double * FCN_XY_PROF_KINDS)()
        n = (C.c_int64 * FCN_XY_PROF_KINDS)()
        check_xy(fcn_xy_profile_read(self.ctx, ms, n, 1 if reset else 0), self.ctx)
        names = ("row_head", "row_mid", "row_tail", "line_x", "line_y")
        return {names[k]: (ms[k], n[k]) for k in range(FCN_XY_PROF_KINDS)}


def alu_peak(kind: int) -> float:
    """FLOP/s of the library's FMA microkernel on the current device (kind 0:
    FP64 fma, 1: FP32 fmaf, 2: FP32 packed f32x2), on the current stream."""
    out = C.c_double()
    check(fcn_alu_peak(int(kind), C.byref(out), stream_ptr()), None)
    return out.value
