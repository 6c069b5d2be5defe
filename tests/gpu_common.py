"""Shared helpers of the GPU tests: build a CUDA-library lattice and an
oracle lattice from the same seeded workload, and compare them.

The two sides share only the inputs (paper_2103_02119_gb300.workloads): each
computes its own initial equilibrium from the same (rho, u) fields, and the
same seeded perturbation is then added on each side.
"""
import numpy as np

from paper_2103_02119_gb300 import workloads as W

# FP64: differences come only from the order of rounding (matrix form in the
# oracle, factorized form on the GPU): a few ulp per step, far below 1e-12.
F64_ATOL_F = 1e-12
F64_RTOL_U = 1e-10
# FP32: stored deviations |f - w rho0| <~ 3e-2 round at ~2e-9 per step, the
# collision adds errors of the same order; after tens of steps the
# population error stays far below 1e-6, and the velocity error below the
# 1e-5 relative target.
F32_ATOL_F = 1e-6
F32_RTOL_U = 1e-5


def oracle_of(orc, wl, scheme="rc"):
    p = orc.OracleParams.make(wl.nx, wl.ny, wl.a, wl.cs2, wl.omega, Fx=wl.Fx, Fy=wl.Fy,
                              periodic_x=wl.periodic_x, periodic_y=wl.periodic_y,
                              wall_u=wl.wall_u, use_iso_corr=wl.use_iso_corr,
                              use_gi_corr=wl.use_gi_corr, scheme=scheme)
    o = orc.Oracle(p, wl.mask)
    o.init_fields(wl.rho, wl.ux, wl.uy)
    return o


def gpu_of(wl, precision, stream=None, **kw):
    from paper_2103_02119_gb300.lbm import Lattice
    return Lattice.from_workload(wl, precision=precision, stream=stream, **kw)


def pair(orc, wl, precision, noise_seed=None, noise_amp=1e-3, scheme=0, **kw):
    """(oracle, gpu) lattices in the same initial state; scheme 0 = RC-LBM,
    1 = RNR-LBM."""
    o = oracle_of(orc, wl, scheme={0: "rc", 1: "rnr"}[scheme])
    g = gpu_of(wl, precision, scheme=scheme, **kw)
    if noise_seed is not None:
        fluid = 1.0 - o.solid()[None].astype(float)
        n = W.perturbation(wl.nx, wl.ny, noise_seed, noise_amp) * fluid
        o.set_f(o.get_f() + n)
        g.set_f(g.get_f() + n)
    return o, g


def rel_l2(a, b):
    return float(np.sqrt(((a - b) ** 2).sum()) / max(np.sqrt((b ** 2).sum()), 1e-300))


def compare(o, g, precision):
    """Element-wise comparison of the populations and the velocity fields."""
    fo, fg = o.get_f(), g.get_f()
    ro, uo, vo = o.moments()
    rg, ug, vg = g.moments()
    df = float(np.abs(fg - fo).max())
    dr = float(np.abs(rg - ro).max())
    uscale = max(float(np.abs(uo).max()), float(np.abs(vo).max()), 1e-300)
    du = float(max(np.abs(ug - uo).max(), np.abs(vg - vo).max())) / uscale
    if precision == 64:
        assert df <= F64_ATOL_F, df
        assert dr <= F64_ATOL_F, dr
        assert du <= F64_RTOL_U, du
    else:
        assert df <= F32_ATOL_F, df
        assert dr <= F32_ATOL_F, dr
        u_err = rel_l2(np.stack([ug, vg]), np.stack([uo, vo]))
        assert u_err <= F32_RTOL_U, u_err
    return df, du
