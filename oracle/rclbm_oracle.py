"""ctypes wrapper of the FP64 CPU oracle (``rclbm_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Array layout follows
the C header: distributions are plane-major ``(9, ny, nx)`` float64 arrays,
fields are ``(ny, nx)`` float64 arrays, cell (x, y) at ``[y, x]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rclbm_oracle.c")
_LIB = os.path.join(_HERE, "librclbm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/librclbm_oracle.so`` with gcc.

    Plain IEEE double arithmetic: no fast-math and no FMA contraction, so the
    oracle rounds the same way on every host.
    """
    stale = (not os.path.exists(_LIB)
             or os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC),
                                             os.path.getmtime(_SRC[:-2] + ".h")))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class OracleParams(ctypes.Structure):
    """Mirror of ``orc_params`` in rclbm_oracle.h."""

    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("a", ctypes.c_double), ("cs2", ctypes.c_double),
        ("omega", ctypes.c_double * 9),
        ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
        ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
        ("wall_u", (ctypes.c_double * 2) * 4),
        ("use_iso_corr", ctypes.c_int), ("use_gi_corr", ctypes.c_int),
        ("scheme", ctypes.c_int), ("nthreads", ctypes.c_int),
    ]

    @classmethod
    def make(cls, nx, ny, a, cs2, omega, Fx=0.0, Fy=0.0, periodic_x=1,
             periodic_y=1, wall_u=None, use_iso_corr=1, use_gi_corr=1,
             scheme="rc", nthreads=0):
        p = cls()
        p.nx, p.ny, p.a, p.cs2 = int(nx), int(ny), float(a), float(cs2)
        for j in range(9):
            p.omega[j] = float(omega[j])
        p.Fx, p.Fy = float(Fx), float(Fy)
        p.periodic_x, p.periodic_y = int(periodic_x), int(periodic_y)
        for k in range(4):
            for d in range(2):
                p.wall_u[k][d] = 0.0 if wall_u is None else float(wall_u[k][d])
        p.use_iso_corr, p.use_gi_corr = int(use_iso_corr), int(use_gi_corr)
        p.scheme = {"rc": 0, "rnr": 1}[scheme] if isinstance(scheme, str) else int(scheme)
        p.nthreads = int(nthreads)
        return p


_D = ctypes.POINTER(ctypes.c_double)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_matrices.argtypes = [ctypes.c_double] * 3 + [_D] * 4
            L.orc_central_moments.argtypes = [ctypes.c_double, _D, ctypes.c_double,
                                              ctypes.c_double, _D]
            L.orc_feq.argtypes = [ctypes.c_double] * 5 + [_D]
            L.orc_collide_cell.argtypes = [ctypes.POINTER(OracleParams), _D,
                                           ctypes.c_double, ctypes.c_double, _D, _D]
            L.orc_create.argtypes = [ctypes.POINTER(OracleParams), _U8]
            L.orc_create.restype = ctypes.c_void_p
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_init_fields.argtypes = [ctypes.c_void_p, _D, _D, _D]
            L.orc_set_f.argtypes = [ctypes.c_void_p, _D]
            L.orc_get_f.argtypes = [ctypes.c_void_p, _D]
            L.orc_set_force.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
            L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
            L.orc_moments.argtypes = [ctypes.c_void_p, _D, _D, _D]
            L.orc_strain.argtypes = [ctypes.c_void_p, _D, _D]
            L.orc_stress.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
            L.orc_solid.argtypes = [ctypes.c_void_p, _U8]
            L.orc_threads.argtypes = [ctypes.c_void_p]
            _lib = L
    return _lib


def _dp(x):
    return None if x is None else x.ctypes.data_as(_D)


def _f64(x, shape=None):
    if x is None:
        return None
    x = np.ascontiguousarray(x, dtype=np.float64)
    if shape is not None and x.shape != shape:
        x = x.reshape(shape)
    return x


def matrices(a, ux=0.0, uy=0.0):
    """Return (T, T^-1, F(u), F(-u)) as 9x9 arrays."""
    out = [np.zeros((9, 9)) for _ in range(4)]
    if lib().orc_matrices(a, ux, uy, *[_dp(m) for m in out]):
        raise ValueError("invalid aspect ratio")
    return tuple(out)


def central_moments(a, f, ux, uy):
    f = _f64(f)
    k = np.zeros(9)
    lib().orc_central_moments(a, _dp(f), ux, uy, _dp(k))
    return k


def feq(a, cs2, rho, ux, uy):
    out = np.zeros(9)
    if lib().orc_feq(a, cs2, rho, ux, uy, _dp(out)):
        raise ValueError("invalid aspect ratio")
    return out


def collide_cell(params: OracleParams, f, dxrho=0.0, dyrho=0.0):
    """One-cell collision; returns (post-collision f, (d_x u_x, d_y u_y))."""
    f = _f64(f)
    ft = np.zeros(9)
    st = np.zeros(2)
    if lib().orc_collide_cell(ctypes.byref(params), _dp(f), dxrho, dyrho,
                              _dp(ft), _dp(st)):
        raise ValueError("invalid parameters")
    return ft, (st[0], st[1])


class Oracle:
    """A lattice advanced by the FP64 oracle."""

    def __init__(self, params: OracleParams, solid=None):
        self.p = params
        self.nx, self.ny = params.nx, params.ny
        self.N = self.nx * self.ny
        m = None
        if solid is not None:
            m = np.ascontiguousarray(solid, dtype=np.uint8).reshape(self.N)
        self._m = m
        self.h = lib().orc_create(ctypes.byref(params),
                                  None if m is None else m.ctypes.data_as(_U8))
        if not self.h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def threads(self) -> int:
        return lib().orc_threads(self.h)

    def init_fields(self, rho=None, ux=None, uy=None):
        sh = (self.ny, self.nx)
        r, u, v = _f64(rho, sh), _f64(ux, sh), _f64(uy, sh)
        lib().orc_init_fields(self.h, _dp(r), _dp(u), _dp(v))

    def set_f(self, f):
        f = _f64(f, (9, self.ny, self.nx))
        lib().orc_set_f(self.h, _dp(f))

    def get_f(self):
        f = np.zeros((9, self.ny, self.nx))
        lib().orc_get_f(self.h, _dp(f))
        return f

    def set_force(self, Fx, Fy):
        self.p.Fx, self.p.Fy = float(Fx), float(Fy)
        lib().orc_set_force(self.h, float(Fx), float(Fy))

    def step(self, n=1):
        if lib().orc_step(self.h, int(n)):
            raise ValueError("bad step count")

    def moments(self):
        r, u, v = (np.zeros((self.ny, self.nx)) for _ in range(3))
        lib().orc_moments(self.h, _dp(r), _dp(u), _dp(v))
        return r, u, v

    def strain(self):
        dx, dy = np.zeros((self.ny, self.nx)), np.zeros((self.ny, self.nx))
        lib().orc_strain(self.h, _dp(dx), _dp(dy))
        return dx, dy

    def stress(self):
        """(d_y u_x + d_x u_y, tau_xx, tau_yy, tau_xy), each (ny, nx)."""
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        lib().orc_stress(self.h, *(_dp(x) for x in out))
        return tuple(out)

    def solid(self):
        s = np.zeros((self.ny, self.nx), dtype=np.uint8)
        lib().orc_solid(self.h, s.ctypes.data_as(_U8))
        return s
