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
# LBM_CHECKED=1 in the environment loads the checked build (device bounds
# checks in the step kernels; ``build(checked=True)``) instead.
CHECKED = os.environ.get("LBM_CHECKED", "") == "1"
LIB_PATH = os.path.join(_HERE, "liblbm_gb300_checked.so" if CHECKED else "liblbm_gb300.so")

LBM_OK = 0
LBM_ERR_INVALID = -1
LBM_ERR_OOM = -2
LBM_ERR_CUDA = -3
LBM_ERR_UNSTABLE = -4
LBM_ERR_TIMEOUT = -5
LBM_ERR_STATE = -6
LBM_ERR_BOUNDS = -7
LBM_BUILD_CHECKED = 1
LBM_DIAG_COUNT = 8
DIAG_NAMES = ("mass", "mom_x", "mom_y", "energy", "residual", "nonfinite", "step",
              "step_change")
_STATUS = {0: "LBM_OK", -1: "LBM_ERR_INVALID", -2: "LBM_ERR_OOM", -3: "LBM_ERR_CUDA",
           -4: "LBM_ERR_UNSTABLE", -5: "LBM_ERR_TIMEOUT", -6: "LBM_ERR_STATE",
           -7: "LBM_ERR_BOUNDS"}


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
            "(nvcc, sm_103a; the checked build with build(checked=True)).  "
            "There is no CPU fallback.")
    L = ctypes.CDLL(LIB_PATH)
    L.lbm_build_flags.argtypes = []
    L.lbm_params_init.argtypes = [ctypes.POINTER(lbm_params)]
    L.lbm_create.argtypes = [ctypes.POINTER(lbm_params), ctypes.POINTER(ctypes.c_uint8), _P,
                             ctypes.POINTER(_P)]
    L.lbm_destroy.argtypes = [_P]
    L.lbm_destroy.restype = None
    L.lbm_init_fields.argtypes = [_P, _P, _P, _P, ctypes.c_int]
    L.lbm_step.argtypes = [_P, ctypes.c_int64]
    L.lbm_set_force.argtypes = [_P, ctypes.c_double, ctypes.c_double]
    L.lbm_set_wait_limit.argtypes = [_P, ctypes.c_int64]
    L.lbm_set_small_path.argtypes = [_P, ctypes.c_int]
    L.lbm_debug_fail_alloc.argtypes = [ctypes.c_int64]
    L.lbm_moments.argtypes = [_P, _P, _P, _P, ctypes.c_int]
    L.lbm_get_f.argtypes = [_P, _P, ctypes.c_int]
    L.lbm_stress.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int]
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
    I64 = ctypes.c_int64
    L.lbm_batch_create.argtypes = [ctypes.POINTER(lbm_params), ctypes.c_int, _P, _P,
                                   ctypes.POINTER(_P)]
    L.lbm_batch_destroy.argtypes = [_P]
    L.lbm_batch_destroy.restype = None
    L.lbm_batch_count.argtypes = [_P]
    L.lbm_batch_init_fields.argtypes = [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int]
    L.lbm_batch_step.argtypes = [_P, I64]
    L.lbm_batch_residuals.argtypes = [_P, _D]
    L.lbm_batch_run.argtypes = [_P, ctypes.c_double, I64, I64, _D]
    L.lbm_batch_set_active.argtypes = [_P, ctypes.c_int, ctypes.c_int]
    L.lbm_batch_is_active.argtypes = [_P, ctypes.c_int]
    L.lbm_batch_set_shape.argtypes = [_P, ctypes.c_int, ctypes.c_int]
    L.lbm_batch_set_wait_limit.argtypes = [_P, ctypes.c_int64]
    L.lbm_batch_set_table_path.argtypes = [_P, ctypes.c_int]
    L.lbm_batch_table_groups.argtypes = [_P]
    _IP = ctypes.POINTER(ctypes.c_int)
    L.lbm_batch_get_shape.argtypes = [_P, _IP, _IP]
    L.lbm_batch_tune.argtypes = [_P, ctypes.c_int, _IP, _IP]
    L.lbm_batch_moments.argtypes = [_P, ctypes.c_int, _P, _P, _P, ctypes.c_int]
    L.lbm_batch_get_f.argtypes = [_P, ctypes.c_int, _P, ctypes.c_int]
    L.lbm_batch_diagnostics.argtypes = [_P, ctypes.c_int, _D]
    L.lbm_batch_step_count.argtypes = [_P, ctypes.c_int]
    L.lbm_batch_step_count.restype = I64
    L.lbm_batch_launch_count.argtypes = [_P]
    L.lbm_batch_launch_count.restype = I64
    L.lbm_batch_last_error.argtypes = [_P]
    L.lbm_batch_last_error.restype = ctypes.c_char_p
    _F = ctypes.POINTER(ctypes.c_float)
    L.lbm_nn_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _P,
                                ctypes.POINTER(_P)]
    L.lbm_nn_destroy.argtypes = [_P]
    L.lbm_nn_destroy.restype = None
    L.lbm_nn_param_count.argtypes = [_P]
    L.lbm_nn_param_count.restype = ctypes.c_size_t
    L.lbm_nn_get_params.argtypes = [_P, _F]
    L.lbm_nn_set_params.argtypes = [_P, _F]
    L.lbm_nn_forward.argtypes = [_P, _F, ctypes.c_int, _F]
    L.lbm_nn_prolong.argtypes = [_P, _F, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_uint8), _F]
    L.lbm_nn_gradients.argtypes = [_P, _F, _F, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int,
                                   _F, _F]
    L.lbm_nn_train_step.argtypes = [_P, _F, _F, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int,
                                    ctypes.c_float, _F]
    L.lbm_nn_launch_count.argtypes = [_P]
    L.lbm_nn_launch_count.restype = ctypes.c_int64
    L.lbm_nn_last_error.argtypes = [_P]
    L.lbm_nn_last_error.restype = ctypes.c_char_p
    L.lbm_peak_copy_gbs.argtypes = [ctypes.c_size_t, ctypes.c_int, _P, _D]
    L.lbm_peak_fp64_gflops.argtypes = [ctypes.c_int, _P, _D]
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


def lbm_set_small_path(h, enable: bool):
    _check(lib.lbm_set_small_path(h, int(bool(enable))), h)


def lbm_set_wait_limit(h, polls: int):
    _check(lib.lbm_set_wait_limit(h, int(polls)), h)


def lbm_debug_fail_alloc(nth: int):
    _check(lib.lbm_debug_fail_alloc(int(nth)), None)


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


def lbm_stress(h, N, dxux=None, dyuy=None, sxy=None, txx=None, tyy=None, txy=None):
    """Writes the local strain rates and viscous stress into the given
    outputs (numpy host arrays or CUDA tensors, float64, N elements)."""
    outs = (dxux, dyuy, sxy, txx, tyy, txy)
    dev = _is_device(*outs)
    ptrs = []
    for v in outs:
        if v is None:
            ptrs.append(None)
        elif dev:
            ptrs.append(_arr(v, N, True)[0])
        else:
            if not (isinstance(v, np.ndarray) and v.dtype == np.float64
                    and v.flags.c_contiguous and v.size == N):
                raise ValueError("host outputs must be contiguous float64 arrays of N elements")
            ptrs.append(v.ctypes.data)
    _check(lib.lbm_stress(h, *ptrs, int(dev)), h)


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
    """Returns (status, out[LBM_DIAG_COUNT]); LBM_ERR_UNSTABLE is reported, not raised."""
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

def make_params(nx, ny, a, cs2, omega, Fx=0.0, Fy=0.0, rho0=1.0, precision=32,
                periodic_x=1, periodic_y=1, wall_u=None, use_iso_corr=1, use_gi_corr=1,
                block_x=0, bands=0, scheme=0) -> lbm_params:
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
    return p


def params_of_workload(wl, precision=32, **kw) -> lbm_params:
    return make_params(wl.nx, wl.ny, wl.a, wl.cs2, wl.omega, Fx=wl.Fx, Fy=wl.Fy,
                       precision=precision, periodic_x=wl.periodic_x,
                       periodic_y=wl.periodic_y, wall_u=wl.wall_u,
                       use_iso_corr=wl.use_iso_corr, use_gi_corr=wl.use_gi_corr, **kw)


# ------------------------------------------------------------- batch ABI --

def _bcheck(status: int, b=None):
    if status != LBM_OK:
        raise LbmError(status, lib.lbm_batch_last_error(b).decode())


def lbm_batch_create(params, masks=None, stream=None):
    """params: sequence of lbm_params; masks: None or a sequence of
    (ny, nx) uint8 arrays / None.  Returns an opaque batch (c_void_p)."""
    n = len(params)
    arr = (lbm_params * n)(*params)
    keep, mptrs = [], None
    if masks is not None:
        if len(masks) != n:
            raise ValueError("one mask (or None) per lattice")
        mptrs = (ctypes.c_void_p * n)()
        for k, m in enumerate(masks):
            if m is None:
                continue
            m = np.ascontiguousarray(m, dtype=np.uint8).reshape(-1)
            if m.size != params[k].nx * params[k].ny:
                raise ValueError(f"mask {k} must hold nx*ny bytes")
            keep.append(m)
            mptrs[k] = m.ctypes.data
    b = _P()
    st = lib.lbm_batch_create(arr, n, None if mptrs is None else ctypes.cast(mptrs, _P),
                              _stream_ptr(stream), ctypes.byref(b))
    _bcheck(st, None)
    return b


def lbm_batch_destroy(b):
    lib.lbm_batch_destroy(b)


def lbm_batch_count(b) -> int:
    return int(lib.lbm_batch_count(b))


def lbm_batch_init_fields(b, k, N, rho=None, ux=None, uy=None):
    dev = _is_device(rho, ux, uy)
    keep = [_arr(v, N, dev) for v in (rho, ux, uy)]
    _bcheck(lib.lbm_batch_init_fields(b, int(k), keep[0][0], keep[1][0], keep[2][0],
                                      int(dev)), b)


def lbm_batch_step(b, nsteps: int):
    _bcheck(lib.lbm_batch_step(b, int(nsteps)), b)


def lbm_batch_residuals(b, count):
    """Returns (status, res[count]); LBM_ERR_UNSTABLE is reported, not raised."""
    out = (ctypes.c_double * count)()
    st = lib.lbm_batch_residuals(b, out)
    if st not in (LBM_OK, LBM_ERR_UNSTABLE):
        _bcheck(st, b)
    return st, np.array(out[:], dtype=np.float64)


def lbm_batch_run(b, count, tol, check_every, max_steps):
    """Returns (status, res[count]); LBM_ERR_UNSTABLE is reported, not raised."""
    out = (ctypes.c_double * count)()
    st = lib.lbm_batch_run(b, float(tol), int(check_every), int(max_steps), out)
    if st not in (LBM_OK, LBM_ERR_UNSTABLE):
        _bcheck(st, b)
    return st, np.array(out[:], dtype=np.float64)


def lbm_batch_set_active(b, k, on):
    _bcheck(lib.lbm_batch_set_active(b, int(k), int(bool(on))), b)


def lbm_batch_is_active(b, k) -> int:
    return int(lib.lbm_batch_is_active(b, int(k)))


def lbm_batch_set_shape(b, block_x, rows_per_band):
    _bcheck(lib.lbm_batch_set_shape(b, int(block_x), int(rows_per_band)), b)


def lbm_batch_set_wait_limit(b, polls: int):
    _bcheck(lib.lbm_batch_set_wait_limit(b, int(polls)), b)


def lbm_batch_set_table_path(b, enable: bool):
    _bcheck(lib.lbm_batch_set_table_path(b, int(enable)), b)


def lbm_batch_table_groups(b) -> int:
    return lib.lbm_batch_table_groups(b)


def lbm_batch_get_shape(b):
    bx, rows = ctypes.c_int(), ctypes.c_int()
    _bcheck(lib.lbm_batch_get_shape(b, ctypes.byref(bx), ctypes.byref(rows)), b)
    return bx.value, rows.value


def lbm_batch_tune(b, trial_steps):
    bx, rows = ctypes.c_int(), ctypes.c_int()
    _bcheck(lib.lbm_batch_tune(b, int(trial_steps), ctypes.byref(bx), ctypes.byref(rows)), b)
    return bx.value, rows.value


def lbm_batch_moments(b, k, N, rho=None, ux=None, uy=None):
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
    _bcheck(lib.lbm_batch_moments(b, int(k), ptrs[0], ptrs[1], ptrs[2], int(dev)), b)


def lbm_batch_get_f(b, k, N, out):
    dev = _is_device(out)
    if dev:
        ptr = _arr(out, 9 * N, True)[0]
    else:
        if not (out.dtype == np.float64 and out.flags.c_contiguous and out.size == 9 * N):
            raise ValueError("output must be a contiguous float64 array of 9*N elements")
        ptr = out.ctypes.data
    _bcheck(lib.lbm_batch_get_f(b, int(k), ptr, int(dev)), b)


def lbm_batch_diagnostics(b, k):
    out = (ctypes.c_double * LBM_DIAG_COUNT)()
    st = lib.lbm_batch_diagnostics(b, int(k), out)
    if st not in (LBM_OK, LBM_ERR_UNSTABLE):
        _bcheck(st, b)
    return st, np.array(out[:], dtype=np.float64)


def lbm_batch_step_count(b, k) -> int:
    return int(lib.lbm_batch_step_count(b, int(k)))


def lbm_batch_launch_count(b) -> int:
    return int(lib.lbm_batch_launch_count(b))


def lbm_batch_last_error(b=None) -> str:
    return lib.lbm_batch_last_error(b).decode()


# ---------------------------------------------------------- surrogate ABI --

def _ncheck(status: int, nn=None):
    if status != LBM_OK:
        raise LbmError(status, lib.lbm_nn_last_error(nn).decode())


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def lbm_nn_create(channels, max_batch, height, width, seed=0, stream=None):
    ch = (ctypes.c_int * len(channels))(*[int(c) for c in channels])
    nn = _P()
    _ncheck(lib.lbm_nn_create(len(channels), ch, int(max_batch), int(height), int(width),
                              int(seed), _stream_ptr(stream), ctypes.byref(nn)), None)
    return nn


def lbm_nn_destroy(nn):
    lib.lbm_nn_destroy(nn)


def lbm_nn_param_count(nn) -> int:
    return int(lib.lbm_nn_param_count(nn))


def lbm_nn_get_params(nn):
    out = np.empty(lbm_nn_param_count(nn), np.float32)
    _ncheck(lib.lbm_nn_get_params(nn, _fptr(out)), nn)
    return out


def lbm_nn_set_params(nn, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != lbm_nn_param_count(nn):
        raise ValueError("parameter vector of the wrong length")
    _ncheck(lib.lbm_nn_set_params(nn, _fptr(p)), nn)


def lbm_nn_forward(nn, x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty(x.shape[:3] + (3,), np.float32)
    _ncheck(lib.lbm_nn_forward(nn, _fptr(x), x.shape[0], _fptr(y)), nn)
    return y


def lbm_nn_prolong(nn, y, factor, fluid):
    """y (n, h, w, 3) network outputs, fluid (n, h f, w f) fine fluid flags ->
    (n, h f, w f, 3) prolonged fields after the output stage."""
    y = np.ascontiguousarray(y, dtype=np.float32)
    f = np.ascontiguousarray(fluid, dtype=np.uint8)
    n, h, w = y.shape[:3]
    if factor >= 1 and f.shape != (n, h * factor, w * factor):
        raise ValueError(f"fluid must have shape {(n, h * factor, w * factor)}")
    out = np.empty((n, h * max(factor, 0), w * max(factor, 0), 3), np.float32)
    _ncheck(lib.lbm_nn_prolong(nn, _fptr(y), n, int(factor),
                               f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _fptr(out)), nn)
    return out


def lbm_nn_gradients(nn, x, target, fluid):
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(target, dtype=np.float32)
    f = np.ascontiguousarray(fluid, dtype=np.uint8)
    loss = ctypes.c_float()
    g = np.empty(lbm_nn_param_count(nn), np.float32)
    _ncheck(lib.lbm_nn_gradients(nn, _fptr(x), _fptr(t),
                                 f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), x.shape[0],
                                 ctypes.byref(loss), _fptr(g)), nn)
    return float(loss.value), g


def lbm_nn_train_step(nn, x, target, fluid, lr):
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.ascontiguousarray(target, dtype=np.float32)
    f = np.ascontiguousarray(fluid, dtype=np.uint8)
    loss = ctypes.c_float()
    _ncheck(lib.lbm_nn_train_step(nn, _fptr(x), _fptr(t),
                                  f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), x.shape[0],
                                  float(lr), ctypes.byref(loss)), nn)
    return float(loss.value)


def lbm_nn_launch_count(nn) -> int:
    return int(lib.lbm_nn_launch_count(nn))


def lbm_nn_last_error(nn=None) -> str:
    return lib.lbm_nn_last_error(nn).decode()


def params_to_list(vec, shapes):
    """Flat parameter vector -> [(w (3, 3, cin, cout), b (cout,))]."""
    out, k = [], 0
    for ci, co in shapes:
        w = np.asarray(vec[k:k + 9 * ci * co], dtype=np.float64).reshape(3, 3, ci, co)
        k += 9 * ci * co
        b = np.asarray(vec[k:k + co], dtype=np.float64)
        k += co
        out.append((w, b))
    return out


def params_to_vec(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


# ------------------------------------------------------------ convenience --

class Batch:
    """Many FP32 lattices owned by one batch of the CUDA library."""

    def __init__(self, workloads, stream=None, schemes=None):
        """schemes: None (all RC-LBM) or one scheme per workload (0 RC-LBM,
        1 RNR-LBM, -1 no collision)."""
        if schemes is None:
            schemes = [0] * len(workloads)
        self.params = [params_of_workload(w, precision=32, scheme=int(sc))
                       for w, sc in zip(workloads, schemes)]
        self.shapes = [(w.ny, w.nx) for w in workloads]
        self.count = len(workloads)
        self.b = lbm_batch_create(self.params, [w.mask for w in workloads], stream)
        for k, w in enumerate(workloads):
            if w.rho is not None or w.ux is not None or w.uy is not None:
                self.init_fields(k, w.rho, w.ux, w.uy)

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _N(self, k):
        ny, nx = self.shapes[k]
        return nx * ny

    def init_fields(self, k, rho=None, ux=None, uy=None):
        lbm_batch_init_fields(self.b, k, self._N(k), rho, ux, uy)

    def step(self, n=1):
        lbm_batch_step(self.b, n)

    def residuals(self):
        return lbm_batch_residuals(self.b, self.count)

    def run(self, tol, check_every=100, max_steps=10**6):
        return lbm_batch_run(self.b, self.count, tol, check_every, max_steps)

    def set_active(self, k, on):
        lbm_batch_set_active(self.b, k, on)

    def is_active(self, k) -> bool:
        return lbm_batch_is_active(self.b, k) == 1

    def set_table_path(self, enable):
        lbm_batch_set_table_path(self.b, enable)

    @property
    def table_groups(self) -> int:
        return lbm_batch_table_groups(self.b)

    def set_shape(self, block_x, rows_per_band):
        lbm_batch_set_shape(self.b, block_x, rows_per_band)

    @property
    def shape(self):
        return lbm_batch_get_shape(self.b)

    def tune(self, trial_steps=20):
        return lbm_batch_tune(self.b, trial_steps)

    def moments(self, k):
        ny, nx = self.shapes[k]
        r, u, v = (np.empty((ny, nx)) for _ in range(3))
        lbm_batch_moments(self.b, k, nx * ny, r, u, v)
        return r, u, v

    def get_f(self, k):
        ny, nx = self.shapes[k]
        f = np.empty((9, ny, nx))
        lbm_batch_get_f(self.b, k, nx * ny, f)
        return f

    def diagnostics(self, k):
        return lbm_batch_diagnostics(self.b, k)

    def step_count(self, k) -> int:
        return lbm_batch_step_count(self.b, k)

    @property
    def launch_count(self) -> int:
        return lbm_batch_launch_count(self.b)


class Lattice:
    """A lattice owned by one handle of the CUDA library."""

    def __init__(self, nx, ny, a, cs2, omega, Fx=0.0, Fy=0.0, rho0=1.0, precision=32,
                 periodic_x=1, periodic_y=1, wall_u=None, use_iso_corr=1, use_gi_corr=1,
                 mask=None, stream=None, block_x=0, bands=0, scheme=0):
        p = make_params(nx, ny, a, cs2, omega, Fx=Fx, Fy=Fy, rho0=rho0, precision=precision,
                        periodic_x=periodic_x, periodic_y=periodic_y, wall_u=wall_u,
                        use_iso_corr=use_iso_corr, use_gi_corr=use_gi_corr,
                        block_x=block_x, bands=bands, scheme=scheme)
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

    def stress(self):
        """(d_x u_x, d_y u_y, d_y u_x + d_x u_y, tau_xx, tau_yy, tau_xy)."""
        out = [np.empty((self.ny, self.nx)) for _ in range(6)]
        lbm_stress(self.h, self.N, *out)
        return tuple(out)

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


# ------------------------------------------------------------ measurement --

def lbm_peak_copy_gbs(nbytes, iters, stream=None) -> float:
    """Device-to-device copy bandwidth in GB/s (read plus write)."""
    out = ctypes.c_double()
    st = lib.lbm_peak_copy_gbs(int(nbytes), int(iters), _stream_ptr(stream), ctypes.byref(out))
    if st != LBM_OK:
        raise LbmError(st, "lbm_peak_copy_gbs failed")
    return out.value


def lbm_peak_fp64_gflops(iters, stream=None) -> float:
    """FP64 fused multiply-add rate in GFLOP/s (an FMA counts two)."""
    out = ctypes.c_double()
    st = lib.lbm_peak_fp64_gflops(int(iters), _stream_ptr(stream), ctypes.byref(out))
    if st != LBM_OK:
        raise LbmError(st, "lbm_peak_fp64_gflops failed")
    return out.value
