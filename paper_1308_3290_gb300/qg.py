"""Thin ctypes binding of libqgcgp (the C ABI declared in include/qg.h).

The functions ``qg_create`` ... ``qg_last_error`` marshal arguments to the
C calls of the same names and raise :class:`QGError` on a non-zero status.
Fields may be torch tensors (device or host) or numpy arrays (host); they
are passed by pointer, so they must be C-contiguous and of the handle's
dtype.  :class:`Basin` wraps a handle for convenience.

Every step of the computation runs in the library's CUDA kernels; this
module does no arithmetic of the method.  Loading fails loudly when the
library has not been built (``paper_1308_3290_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqgcgp.so")

QG_F32, QG_F64 = 0, 1
QG_FAULT_NONE, QG_FAULT_BARRIER_STALL = 0, 1
QG_SOLVER_FFT, QG_SOLVER_MULTIGRID = 0, 1
QG_OK, QG_ERR_ARG, QG_ERR_SHAPE, QG_ERR_CUDA, QG_ERR_OOM = 0, 1, 2, 3, 4
QG_ERR_NONFINITE, QG_ERR_CFL, QG_ERR_TIMEOUT, QG_ERR_UNSUPPORTED = 5, 6, 7, 8

STATUS = {
    0: "QG_OK", 1: "QG_ERR_ARG", 2: "QG_ERR_SHAPE", 3: "QG_ERR_CUDA",
    4: "QG_ERR_OOM", 5: "QG_ERR_NONFINITE", 6: "QG_ERR_CFL",
    7: "QG_ERR_TIMEOUT", 8: "QG_ERR_UNSUPPORTED", 9: "QG_ERR_NO_DEVICE",
}

# Every symbol include/qg.h declares.
EXPORTS = [
    "qg_create", "qg_destroy", "qg_set_state", "qg_get_state", "qg_get_psi",
    "qg_set_forcing", "qg_poisson_solve", "qg_restrict", "qg_prolong",
    "qg_step", "qg_diagnostics", "qg_set_timing", "qg_read_timing",
    "qg_step_kernel_count", "qg_synchronize", "qg_status_string",
    "qg_last_error", "qg_poisson_solve_noalloc", "qg_inject_fault",
    "qg_ensemble_create", "qg_ensemble_member", "qg_ensemble_step",
    "qg_ensemble_kernel_count", "qg_ensemble_synchronize", "qg_ensemble_destroy",
    "qg_tape_begin", "qg_tape_end", "qg_adjoint_step", "qg_energy_gradient",
    "qg_set_cfl", "qg_set_solver", "qg_get_time", "qg_stats_begin", "qg_stats_mean_psi", "qg_stats_end",
    "qg_set_timing_mask", "qg_solve_engine", "qg_energy_accumulate", "qg_stencil_tile",
    "qg_bounds_check_result", "qg_stats_mean_q", "qg_get_state_async",
]

KERNEL_CLASSES = ["restrict", "solve", "prolong", "fine", "cfl"]


class QGError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class qg_basin(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("forcing_amp", ctypes.c_double), ("delta", ctypes.c_double),
                ("sigma", ctypes.c_double), ("dt", ctypes.c_double),
                ("flags", ctypes.c_uint32)]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libqgcgp.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_1308_3290_gb300.build.build()")
    lib = ctypes.CDLL(p)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "qg_create": [ctypes.POINTER(qg_basin), i32, dbl, dbl, dbl, i32, i32, vp,
                      ctypes.POINTER(vp)],
        "qg_destroy": [vp],
        "qg_set_state": [vp, vp, i32],
        "qg_get_state": [vp, vp, i32],
        "qg_get_psi": [vp, vp, i32],
        "qg_set_forcing": [vp, vp],
        "qg_poisson_solve": [vp, vp, vp, i32],
        "qg_restrict": [vp, vp, vp, i32],
        "qg_prolong": [vp, vp, vp, i32],
        "qg_step": [vp, i64],
        "qg_diagnostics": [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl)],
        "qg_set_timing": [vp, i32],
        "qg_read_timing": [vp, ctypes.POINTER(dbl), ctypes.POINTER(ctypes.c_int32)],
        "qg_step_kernel_count": [vp, ctypes.POINTER(i64)],
        "qg_synchronize": [vp],
        "qg_poisson_solve_noalloc": [i32, i32, dbl, dbl, i32, vp, vp, vp],
        "qg_last_error": [vp],
        "qg_inject_fault": [vp, i32],
        "qg_ensemble_create": [ctypes.POINTER(qg_basin), ctypes.POINTER(dbl),
                               ctypes.POINTER(dbl), ctypes.POINTER(i32), i32, i32, vp,
                               ctypes.POINTER(vp)],
        "qg_ensemble_member": [vp, i32, ctypes.POINTER(vp)],
        "qg_ensemble_step": [vp, i64],
        "qg_ensemble_kernel_count": [vp, ctypes.POINTER(i64)],
        "qg_ensemble_synchronize": [vp],
        "qg_ensemble_destroy": [vp],
        "qg_tape_begin": [vp, i64, i64],
        "qg_tape_end": [vp],
        "qg_adjoint_step": [vp, i64, vp, vp],
        "qg_energy_gradient": [vp, dbl, vp],
        "qg_set_cfl": [vp, dbl],
        "qg_set_solver": [vp, i32, i32],
        "qg_solve_engine": [vp, ctypes.POINTER(i32)],
        "qg_get_time": [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)],
        "qg_stats_begin": [vp],
        "qg_stats_mean_psi": [vp, vp, i32, ctypes.POINTER(i64)],
        "qg_stats_end": [vp],
        "qg_set_timing_mask": [vp, ctypes.c_uint32],
        "qg_energy_accumulate": [vp, dbl, vp],
        "qg_stencil_tile": [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "qg_bounds_check_result": [ctypes.POINTER(i32)],
        "qg_stats_mean_q": [vp, vp, i32, ctypes.POINTER(i64)],
        "qg_get_state_async": [vp, vp, i32],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.qg_status_string.argtypes = [ctypes.c_int]
    lib.qg_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, where: str) -> None:
    if status != 0:
        raise QGError(status, where)


def _ptr(x) -> int:
    """Address of a C-contiguous torch tensor or numpy array."""
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


# --- the C calls, by name --------------------------------------------------

def qg_create(basin: qg_basin, layers: int, Re: float, Ro: float, Fr: float,
              levels: int, dtype: int, stream: int | None = None) -> int:
    h = ctypes.c_void_p()
    _check(load().qg_create(ctypes.byref(basin), layers, Re, Ro, Fr, levels, dtype,
                            stream or None, ctypes.byref(h)), "qg_create")
    return h.value


def qg_destroy(h: int) -> None:
    _check(load().qg_destroy(h), "qg_destroy")


def qg_set_state(h: int, field, layer: int = 0) -> None:
    _check(load().qg_set_state(h, _ptr(field), layer), "qg_set_state")


def qg_get_state(h: int, field, layer: int = 0) -> None:
    _check(load().qg_get_state(h, _ptr(field), layer), "qg_get_state")


def qg_get_psi(h: int, psi, layer: int = 0) -> None:
    _check(load().qg_get_psi(h, _ptr(psi), layer), "qg_get_psi")


def qg_set_forcing(h: int, forcing) -> None:
    _check(load().qg_set_forcing(h, None if forcing is None else _ptr(forcing)), "qg_set_forcing")


def qg_poisson_solve(h: int, rhs, psi, level: int) -> None:
    _check(load().qg_poisson_solve(h, _ptr(rhs), _ptr(psi), level), "qg_poisson_solve")


def qg_restrict(h: int, fine, coarse, levels: int) -> None:
    _check(load().qg_restrict(h, _ptr(fine), _ptr(coarse), levels), "qg_restrict")


def qg_prolong(h: int, coarse, fine, levels: int) -> None:
    _check(load().qg_prolong(h, _ptr(coarse), _ptr(fine), levels), "qg_prolong")


def qg_step(h: int, n: int) -> None:
    _check(load().qg_step(h, n), "qg_step")


def qg_diagnostics(h: int) -> tuple[float, float, float]:
    ke, z, u = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().qg_diagnostics(h, ctypes.byref(ke), ctypes.byref(z), ctypes.byref(u)),
           "qg_diagnostics")
    return ke.value, z.value, u.value


def qg_energy_accumulate(h: int, scale: float, acc) -> None:
    """acc (a device float64 tensor of one element) += scale * kinetic
    energy of the current state; asynchronous on the handle's stream."""
    _check(load().qg_energy_accumulate(h, scale, _ptr(acc)), "qg_energy_accumulate")


def qg_set_timing(h: int, enable: bool) -> None:
    _check(load().qg_set_timing(h, 1 if enable else 0), "qg_set_timing")


def qg_set_timing_mask(h: int, classes) -> None:
    """Bracket only the kernels of the named classes (see KERNEL_CLASSES)."""
    mask = 0
    for c in classes:
        mask |= 1 << KERNEL_CLASSES.index(c)
    _check(load().qg_set_timing_mask(h, mask), "qg_set_timing_mask")


def qg_read_timing(h: int) -> dict:
    """{kernel class: (milliseconds, launches)} of the last timed step."""
    n = len(KERNEL_CLASSES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int32 * n)()
    _check(load().qg_read_timing(h, ms, cnt), "qg_read_timing")
    return {KERNEL_CLASSES[k]: (ms[k], cnt[k]) for k in range(n)}


def qg_step_kernel_count(h: int) -> int:
    c = ctypes.c_int64()
    _check(load().qg_step_kernel_count(h, ctypes.byref(c)), "qg_step_kernel_count")
    return c.value


def qg_poisson_solve_noalloc(nx: int, ny: int, dx: float, dy: float, dtype: int,
                             rhs, psi, stream: int | None = None) -> None:
    """Handle-free Poisson solve that allocates no device memory (its
    workspace is a fixed library-owned device array); rhs and psi are device
    buffers of shape (ny-1, nx-1)."""
    _check(load().qg_poisson_solve_noalloc(nx, ny, dx, dy, dtype, _ptr(rhs), _ptr(psi),
                                           stream or None), "qg_poisson_solve_noalloc")


def qg_inject_fault(h: int, kind: int) -> None:
    """Failure-detection test switch: QG_FAULT_BARRIER_STALL makes the
    handle's solves run out of their bounded grid-barrier wait (the next
    synchronisation raises QGError with QG_ERR_TIMEOUT); QG_FAULT_NONE
    restores normal operation."""
    _check(load().qg_inject_fault(h, kind), "qg_inject_fault")


def qg_tape_begin(h: int, every: int, max_steps: int) -> None:
    _check(load().qg_tape_begin(h, every, max_steps), "qg_tape_begin")


def qg_tape_end(h: int) -> None:
    _check(load().qg_tape_end(h), "qg_tape_end")


def qg_adjoint_step(h: int, n: int, lam, dJdF) -> None:
    _check(load().qg_adjoint_step(h, n, _ptr(lam), _ptr(dJdF)), "qg_adjoint_step")


def qg_energy_gradient(h: int, scale: float, g) -> None:
    _check(load().qg_energy_gradient(h, scale, _ptr(g)), "qg_energy_gradient")


def qg_set_cfl(h: int, c: float) -> None:
    _check(load().qg_set_cfl(h, c), "qg_set_cfl")


def qg_set_solver(h: int, kind: int, cycles: int = 4) -> None:
    _check(load().qg_set_solver(h, kind, cycles), "qg_set_solver")


def qg_solve_engine(h: int) -> int:
    """The elliptic-solve kernel of the handle's step: 4, 16 (shared-memory
    FFT), 32, 33, 34 (warp-group FFT), 40 (matrix form on the tensor cores),
    0 (multigrid)."""
    e = ctypes.c_int32()
    _check(load().qg_solve_engine(h, ctypes.byref(e)), "qg_solve_engine")
    return e.value


def qg_bounds_check_result() -> int:
    """Checked builds only: the first failed index check's site (0: none);
    raises QGError (QG_ERR_UNSUPPORTED) in normal builds."""
    r = ctypes.c_int32()
    _check(load().qg_bounds_check_result(ctypes.byref(r)), "qg_bounds_check_result")
    return r.value


def qg_stencil_tile(h: int) -> tuple[int, int]:
    """(fine rows per CTA, fine rows per thread) of the fused fine-grid
    kernel (autotuned)."""
    r, y = ctypes.c_int32(), ctypes.c_int32()
    _check(load().qg_stencil_tile(h, ctypes.byref(r), ctypes.byref(y)), "qg_stencil_tile")
    return r.value, y.value


def qg_get_time(h: int) -> tuple[float, float]:
    """(model time, last step size)."""
    t, dt = ctypes.c_double(), ctypes.c_double()
    _check(load().qg_get_time(h, ctypes.byref(t), ctypes.byref(dt)), "qg_get_time")
    return t.value, dt.value


def qg_stats_begin(h: int) -> None:
    _check(load().qg_stats_begin(h), "qg_stats_begin")


def qg_stats_mean_psi(h: int, out=None, layer: int = 0) -> int:
    """Write the time-mean first-stage psi into `out` (if given); returns the
    number of steps averaged."""
    c = ctypes.c_int64()
    _check(load().qg_stats_mean_psi(h, _ptr(out) if out is not None else None, layer,
                                    ctypes.byref(c)), "qg_stats_mean_psi")
    return c.value


def qg_get_state_async(h: int, field, layer: int = 0) -> None:
    """Copy the state into a page-locked host buffer without holding up the
    handle's later steps; complete after qg_synchronize."""
    _check(load().qg_get_state_async(h, _ptr(field), layer), "qg_get_state_async")


def qg_stats_mean_q(h: int, out=None, layer: int = 0) -> int:
    """Write the time-mean potential vorticity into `out` (if given); returns
    the number of steps averaged."""
    c = ctypes.c_int64()
    _check(load().qg_stats_mean_q(h, _ptr(out) if out is not None else None, layer,
                                  ctypes.byref(c)), "qg_stats_mean_q")
    return c.value


def qg_stats_end(h: int) -> None:
    _check(load().qg_stats_end(h), "qg_stats_end")


def qg_synchronize(h: int) -> None:
    _check(load().qg_synchronize(h), "qg_synchronize")


def qg_last_error(h: int) -> int:
    return load().qg_last_error(h)


def qg_status_string(status: int) -> str:
    return load().qg_status_string(status).decode()


# --- convenience wrapper ---------------------------------------------------

class Basin:
    """One basin handle.  Fields in and out are torch tensors on the current
    CUDA device in the exchange layout (interior nodes, shape (ny-1, nx-1)).

    One layer (Section 2.1): Re, Ro; the state is w = (q - y)/Ro.
    Two layers (Section 2.2): Ro, Fr, delta, sigma and A = Ro/Re; the state
    planes are Q_i = q_i - y.
    """

    def __init__(self, nx: int, ny: int, *, Re: float, Ro: float, levels: int,
                 dt: float, dtype: str = "f32", layers: int = 1, Fr: float = 0.0,
                 delta: float = 0.5, sigma: float = 0.0, amp: float = 1.0,
                 x0: float = 0.0, x1: float = 1.0, y0: float = -1.0, y1: float = 1.0,
                 stream=None):
        import torch
        self.torch = torch
        self.nx, self.ny, self.levels, self.layers = nx, ny, levels, layers
        self.tdtype = torch.float32 if dtype == "f32" else torch.float64
        b = qg_basin(nx, ny, x0, x1, y0, y1, amp, delta, sigma, dt, 0)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        self._keep = {}
        self.h = qg_create(b, layers, Re, Ro, Fr, levels,
                           QG_F32 if dtype == "f32" else QG_F64, s.cuda_stream)

    def _empty(self, nx, ny, planes=1):
        shape = (ny - 1, nx - 1) if planes == 1 else (planes, ny - 1, nx - 1)
        return self.torch.empty(shape, dtype=self.tdtype, device="cuda")

    def _dev(self, a):
        t = self.torch.as_tensor(a, dtype=self.tdtype, device="cuda")
        return t.contiguous()

    def set_state(self, field, layer: int = 0):
        t = self._dev(field)
        qg_set_state(self.h, t, layer)
        self._keep[layer] = t     # keep alive until the copy has run
        return self

    def state(self, layer: int = 0):
        out = self._empty(self.nx, self.ny)
        qg_get_state(self.h, out, layer)
        return out

    def psi(self, layer: int = 0):
        out = self._empty(self.nx, self.ny)
        qg_get_psi(self.h, out, layer)
        return out

    def set_forcing(self, field):
        t = None if field is None else self._dev(field)
        qg_set_forcing(self.h, t)
        self._keep_f = t

    def step(self, n: int = 1):
        qg_step(self.h, n)
        return self

    def diagnostics(self):
        return qg_diagnostics(self.h)

    def poisson_solve(self, rhs, level: int = 0):
        mx, my = self.nx >> level, self.ny >> level
        r = self._dev(rhs)
        out = self._empty(mx, my, self.layers)
        qg_poisson_solve(self.h, r, out, level)
        self.synchronize()
        return out

    def restrict(self, fine, levels: int):
        f = self._dev(fine)
        out = self._empty(self.nx >> levels, self.ny >> levels)
        qg_restrict(self.h, f, out, levels)
        self.synchronize()
        return out

    def prolong(self, coarse, levels: int):
        c = self._dev(coarse)
        out = self._empty(self.nx, self.ny)
        qg_prolong(self.h, c, out, levels)
        self.synchronize()
        return out

    def synchronize(self):
        qg_synchronize(self.h)

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):   # ensemble members are not
                qg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Independent one-layer basins stepped together (one graph launch per
    step).  ``members`` is a list of dicts with the keys of ``Basin``'s
    constructor (nx, ny, Re, Ro, levels, dt and optionally amp, x0, x1, y0,
    y1).  ``member(i)`` returns a ``Basin`` view of member i for state I/O
    and diagnostics (owned by the ensemble)."""

    def __init__(self, members, *, dtype: str = "f32", stream=None):
        import torch
        self.torch = torch
        n = len(members)
        bs = (qg_basin * n)()
        Re = (ctypes.c_double * n)()
        Ro = (ctypes.c_double * n)()
        lv = (ctypes.c_int * n)()
        for i, m in enumerate(members):
            bs[i] = qg_basin(m["nx"], m["ny"], m.get("x0", 0.0), m.get("x1", 1.0),
                             m.get("y0", -1.0), m.get("y1", 1.0), m.get("amp", 1.0),
                             0.5, 0.0, m["dt"], 0)
            Re[i], Ro[i], lv[i] = m["Re"], m["Ro"], m["levels"]
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        e = ctypes.c_void_p()
        _check(load().qg_ensemble_create(bs, Re, Ro, lv, n,
                                         QG_F32 if dtype == "f32" else QG_F64,
                                         s.cuda_stream, ctypes.byref(e)), "qg_ensemble_create")
        self.e = e.value
        self.views = []
        for i, m in enumerate(members):
            h = ctypes.c_void_p()
            _check(load().qg_ensemble_member(self.e, i, ctypes.byref(h)), "qg_ensemble_member")
            v = Basin.__new__(Basin)
            v.torch = torch
            v.nx, v.ny, v.levels, v.layers = m["nx"], m["ny"], m["levels"], 1
            v.tdtype = torch.float32 if dtype == "f32" else torch.float64
            v.stream = s
            v._keep = {}
            v.h = h.value
            v._owned = False
            self.views.append(v)

    def __len__(self):
        return len(self.views)

    def member(self, i: int) -> "Basin":
        return self.views[i]

    def step(self, n: int = 1):
        _check(load().qg_ensemble_step(self.e, n), "qg_ensemble_step")
        return self

    def kernel_count(self) -> int:
        c = ctypes.c_int64()
        _check(load().qg_ensemble_kernel_count(self.e, ctypes.byref(c)),
               "qg_ensemble_kernel_count")
        return c.value

    def synchronize(self):
        _check(load().qg_ensemble_synchronize(self.e), "qg_ensemble_synchronize")

    def close(self):
        if getattr(self, "e", None):
            for v in self.views:
                v.h = None
            load().qg_ensemble_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
