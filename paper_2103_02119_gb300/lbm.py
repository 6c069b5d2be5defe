"""Thin ctypes binding of the C ABI in ``include/lbm.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``liblbm_gb300.so``.  Importing this module raises ImportError when the
library has not been built (``__graft_entry__.build()`` or
``python -m paper_2103_02119_gb300.build``); there is no CPU fallback.

Functions carry the C names.  Host arrays are numpy float64 arrays; device
arrays are CUDA tensors (anything with ``data_ptr()`` and ``is_cuda``) of
float64, contiguous.  Fields are ``(ny, nx)``, distributions ``(9, ny, nx)``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_gb300.so")

LBM_OK = 0
LBM_ERR_INVALID = -1
LBM_ERR_OOM = -2
LBM_ERR_CUDA = -3
LBM_ERR_UNSTABLE = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_STATE = -6
LBM_DIAG_COUNT = 7
DIAG_NAMES = ("mass", "mom_x", "mom_y", "energy", "residual", "nonfinite", "step")
_STATUS = {0: "LBM_OK", -1: "LBM_ERR_INVALID", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA",
           -4: "LBM_ERR_UNSTABLE", -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_STATE"}


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class lbm_params(ctypes.Structure):
    """Mirror of ``lbm_params``."""

    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("a", ctypes.c_double), ("cs2", ctypes.c_double),
        ("omega", ctypes.c_double * 9),
        ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("precision", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("wall_u", (ctypes.c_double * 2) * 4),
        ("use_iso_corr", ctypes.c_int32), ("use_gi_corr", ctypes.c_int32),
        ("block_x", ctypes.c_int32), ("bands", ctypes.c_int32),
        ("scheme", ctypes.c_int32),
    ]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is not built; build it with __graft_entry__.build() "
            "(nvcc, sm_103a).  There is no CPU fallback.")
    L = ctypes.CDLL(LIB_PATH)
    L.lbm_params_init.argtypes = [ctypes.POINTER(lbm_params)]
    L.lbm_create.argtypes = [ctypes.POINTER(lbm_params), ctypes.POINTER(ctypes.c_uint8), _P,
                             ctypes.POINTER(_P)]
    L.lbm_destroy.argtypes = [_P]
    L.lbm_destroy.restype = None
    L.lbm_init_fields.argtypes = [_P, _P, _P, _P, ctypes.c_int]
    L.lbm_step.argtypes = [_P, ctypes.c_int64]
    L.lbm_set_force.argtypes = [_P, ctypes.c_double, ctypes.c_double]
    L.lbm_moments.argtypes = [_P, _P, _P, _P, ctypes.c_int]
    L.lbm_get_f.argtypes = [_P, _P, ctypes.c_int]
    L.lbm_set_f.argtypes = [_P, _P, ctypes.c_int]
    L.lbm_diagnostics.argtypes = [_P, _D]
    L.lbm_diagnostics_noalloc.argtypes = [_P, _D]
    L.lbm_state_bytes.argtypes = [_P]
    L.lbm_state_bytes.restype = ctypes.c_size_t
    L.lbm_get_state.argtypes = [_P, _P, ctypes.c_size_t]
    L.lbm_set_state.argtypes = [_P, _P, ctypes.c_size_t]
    L.lbm_step_count.argtypes = [_P]
    L.lbm_step_count.restype = ctypes.c_int64
    L.lbm_launch_count.argtypes = [_P]
    L.lbm_launch_count.restype = ctypes.c_int64
    L.lbm_last_error.argtypes = [_P]
    L.lbm_last_error.restype = ctypes.c_char_p
    return L


lib = _load()


def _check(status: int, h=None):
    if status != LBM_OK:
        raise LbmError(status, lib.lbm_last_error(h).decode())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None  # torch.cuda.Stream


def _arr(x, n, on_device):
    """Pointer to n contiguous float64 values (numpy host array or CUDA tensor)."""
    if x is None:
        return None, None
    if on_device:
        if not getattr(x, "is_cuda", False):
            raise TypeError("on_device arrays must be CUDA tensors")
        if x.numel() != n or str(x.dtype) != "torch.float64" or not x.is_contiguous():
            raise ValueError("device array must be a contiguous float64 tensor of "
                             f"{n} elements")
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"host array must have {n} elements, got {a.size}")
    return a.ctypes.data, a


def _is_device(*xs):
    return any(getattr(x, "is_cuda", False) for x in xs if x is not None)


# ----------------------------------------------------------------- C names --

def lbm_params_init() -> lbm_params:
    p = lbm_params()
    _check(lib.lbm_params_init(ctypes.byref(p)))
    return p


def lbm_create(params: lbm_params, solid_mask=None, stream=None):
    """Returns an opaque handle (c_void_p)."""
    h = _P()
    m = None
    if solid_mask is not None:
        m = np.ascontiguousarray(solid_mask, dtype=np.uint8).reshape(-1)
        if m.size != params.nx * params.ny:
            raise ValueError("solid_mask must hold nx*ny bytes")
    st = lib.lbm_create(ctypes.byref(params),
                        None if m is None else m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                        _stream_ptr(stream), ctypes.byref(h))
    _check(st, None)
    return h


def lbm_destroy(h):
    lib.lbm_destroy(h)


def lbm_init_fields(h, N, rho=None, ux=None, uy=None):
    dev = _is_device(rho, ux, uy)
    keep = [_arr(v, N, dev) for v in (rho, ux, uy)]
    _check(lib.lbm_init_fields(h, keep[0][0], keep[1][0], keep[2][0], int(dev)), h)


def lbm_step(h, nsteps: int):
    _check(lib.lbm_step(h, int(nsteps)), h)


def lbm_set_force(h, Fx: float, Fy: float):
    _check(lib.lbm_set_force(h, float(Fx), float(Fy)), h)


def lbm_moments(h, N, rho=None, ux=None, uy=None):
    """Writes into the given outputs (numpy host arrays or CUDA tensors)."""
    dev = _is_device(rho, ux, uy)
    ptrs = []
    for v in (rho, ux, uy):
        if v is None:
            ptrs.append(None)
        elif dev:
            ptrs.append(_arr(v, N, True)[0])
        else:
            if not (isinstance(v, np.ndarray) and v.dtype == np.float64
                    and v.flags.c_contiguous and v.size == N):
                raise ValueError("host outputs must be contiguous float64 arrays of N elements")
            ptrs.append(v.ctypes.data)
    _check(lib.lbm_moments(h, ptrs[0], ptrs[1], ptrs[2], int(dev)), h)


def lbm_get_f(h, N, out):
    dev = _is_device(out)
    if dev:
        ptr = _arr(out, 9 * N, True)[0]
    else:
        if not (out.dtype == np.float64 and out.flags.c_contiguous and out.size == 9 * N):
            raise ValueError("output must be a contiguous float64 array of 9*N elements")
        ptr = out.ctypes.data
    _check(lib.lbm_get_f(h, ptr, int(dev)), h)


def lbm_set_f(h, N, f):
    dev = _is_device(f)
    ptr, keep = _arr(f, 9 * N, dev)
    _check(lib.lbm_set_f(h, ptr, int(dev)), h)


def lbm_diagnostics(h):
    """Returns (status, out[7]); LBM_ERR_UNSTABLE is reported, not raised."""
    out = (ctypes.c_double * LBM_DIAG_COUNT)()
    st = lib.lbm_diagnostics(h, out)
    if st not in (LBM_OK, LBM_ERR_UNSTABLE):
        _check(st, h)
    return st, np.array(out[:], dtype=np.float64)


def lbm_diagnostics_noalloc(h):
    """As lbm_diagnostics, without allocating (fixed in-library scratch)."""
    out = (ctypes.c_double * LBM_DIAG_COUNT)()
    st = lib.lbm_diagnostics_noalloc(h, out)
    if st not in (LBM_OK, LBM_ERR_UNSTABLE):
        _check(st, h)
    return st, np.array(out[:], dtype=np.float64)


def lbm_state_bytes(h) -> int:
    return int(lib.lbm_state_bytes(h))


def lbm_get_state(h) -> bytes:
    n = lbm_state_bytes(h)
    buf = ctypes.create_string_buffer(n)
    _check(lib.lbm_get_state(h, buf, n), h)
    return buf.raw


def lbm_set_state(h, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(lib.lbm_set_state(h, buf, len(state)), h)


def lbm_step_count(h) -> int:
    return int(lib.lbm_step_count(h))


def lbm_launch_count(h) -> int:
    return int(lib.lbm_launch_count(h))


def lbm_last_error(h=None) -> str:
    return lib.lbm_last_error(h).decode()


# ------------------------------------------------------------ convenience --

class Lattice:
    """A lattice owned by one handle of the CUDA library."""

    def __init__(self, nx, ny, a, cs2, omega, Fx=0.0, Fy=0.0, rho0=1.0, precision=32,
                 periodic_x=1, periodic_y=1, wall_u=None, use_iso_corr=1, use_gi_corr=1,
                 mask=None, stream=None, block_x=0, bands=0, scheme=0):
        p = lbm_params_init()
        p.nx, p.ny, p.a, p.cs2 = int(nx), int(ny), float(a), float(cs2)
        for j in range(9):
            p.omega[j] = float(omega[j])
        p.Fx, p.Fy, p.rho0 = float(Fx), float(Fy), float(rho0)
        p.precision = int(precision)
        p.periodic_x, p.periodic_y = int(periodic_x), int(periodic_y)
        for k in range(4):
            for d in range(2):
                p.wall_u[k][d] = 0.0 if wall_u is None else float(wall_u[k][d])
        p.use_iso_corr, p.use_gi_corr = int(use_iso_corr), int(use_gi_corr)
        p.block_x, p.bands, p.scheme = int(block_x), int(bands), int(scheme)
        self.params = p
        self.nx, self.ny, self.N = p.nx, p.ny, p.nx * p.ny
        self.h = lbm_create(p, mask, stream)

    @classmethod
    def from_workload(cls, wl, precision=32, stream=None, **kw):
        lat = cls(wl.nx, wl.ny, wl.a, wl.cs2, wl.omega, Fx=wl.Fx, Fy=wl.Fy,
                  precision=precision, periodic_x=wl.periodic_x, periodic_y=wl.periodic_y,
                  wall_u=wl.wall_u, use_iso_corr=wl.use_iso_corr, use_gi_corr=wl.use_gi_corr,
                  mask=wl.mask, stream=stream, **kw)
        if wl.rho is not None or wl.ux is not None or wl.uy is not None:
            lat.init_fields(wl.rho, wl.ux, wl.uy)
        return lat

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init_fields(self, rho=None, ux=None, uy=None):
        lbm_init_fields(self.h, self.N, rho, ux, uy)

    def step(self, n=1):
        lbm_step(self.h, n)

    def set_force(self, Fx, Fy):
        lbm_set_force(self.h, Fx, Fy)

    def moments(self):
        r, u, v = (np.empty((self.ny, self.nx)) for _ in range(3))
        lbm_moments(self.h, self.N, r, u, v)
        return r, u, v

    def get_f(self):
        f = np.empty((9, self.ny, self.nx))
        lbm_get_f(self.h, self.N, f)
        return f

    def set_f(self, f):
        lbm_set_f(self.h, self.N, f)

    def diagnostics(self):
        return lbm_diagnostics(self.h)

    def get_state(self) -> bytes:
        return lbm_get_state(self.h)

    def set_state(self, s: bytes):
        lbm_set_state(self.h, s)

    @property
    def step_count(self) -> int:
        return lbm_step_count(self.h)

    @property
    def launch_count(self) -> int:
        return lbm_launch_count(self.h)
