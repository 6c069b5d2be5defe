"""Configurations that the checked build (device bounds checks) is run on,
and the runner that steps them with whichever library the process loaded.

Run as a script (``python tests/checked_cases.py OUT.npz``) under
LBM_CHECKED=1 it builds and loads the checked library, steps every case,
checks that no bounds test failed, and saves the final populations; the GPU
test compares them with the normal build's, bit for bit.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2103_02119_gb300 import workloads as W  # noqa: E402

STEPS = (1, 2, 37)   # both parities, direct launches only (under 50)


def _fields(wl, seed, u_amp=0.02):
    r, u, v = W.smooth_random_fields(wl.nx, wl.ny, seed, u_amp=u_amp, rho_amp=2e-3)
    return wl.with_(rho=r, ux=u, uy=v)


def single_cases():
    """(name, workload, precision, scheme, small path): tiny and ragged
    grids, walls on every side, a moving lid, masks, a > 1 and a < 1, a
    force, both schemes, both step kernels."""
    c = []
    tiny = _fields(W.cavity(5, 3, 1.0, 1 / 3, 0.03, 20.0), 1)
    c.append(("cavity_5x3", tiny))
    c.append(("cavity_7x9_mask", _fields(W.cavity(7, 9, 0.5, 0.075, 0.03, 20.0), 2).with_(
        mask=W.random_obstacles(7, 9, seed=3, coverage=0.1))))
    c.append(("tgv_5x3_force", W.taylor_green(5, 3, 2.0, 1 / 3, 0.05, seed=4).with_(
        Fx=1e-5, Fy=-2e-5)))
    c.append(("poiseuille_130x33_mask", _fields(
        W.poiseuille(ny=33, nx=130, a=0.25, cs2=0.01875, nu=0.02, U=0.03), 5).with_(
        mask=W.random_obstacles(130, 33, seed=6, coverage=0.08))))
    c.append(("cavity_300x21", _fields(W.cavity(300, 21, 0.8, W.stable_cs2(0.8), 0.04, 300.0), 7)))
    c.append(("cavity_600x70_mask", _fields(W.cavity(600, 70, 0.5, 0.075, 0.05, 400.0), 8).with_(
        mask=W.random_obstacles(600, 70, seed=9, coverage=0.05))))
    c.append(("tgv_257x129", W.taylor_green(257, 129, 1.0, 1 / 3, 0.02, seed=10)))
    out = []
    for name, wl in c:
        for prec in (32, 64):
            for scheme in (0, 1):
                small = [True, False] if wl.nx * wl.ny <= 4096 else [False]
                for sp in small:
                    out.append((f"{name}_p{prec}_s{scheme}_{'cluster' if sp else 'bands'}",
                                wl, prec, scheme, sp))
    return out


def batch_cases():
    s = [_fields(W.cavity(70, 45, 0.5, 0.075, 0.05, 100.0), 11),
         _fields(W.poiseuille(ny=33, nx=130, a=0.25, cs2=0.01875, nu=0.02, U=0.03), 12).with_(
             mask=W.random_obstacles(130, 33, seed=13, coverage=0.08)),
         _fields(W.taylor_green(5, 4, 1.5, 1 / 3, 0.05, seed=14), 14),
         _fields(W.cavity(300, 21, 0.8, W.stable_cs2(0.8), 0.04, 300.0), 15)]
    return s


def run_all():
    """{name: final populations} of every case with the loaded library;
    raises when a diagnostics call reports an error."""
    from paper_2103_02119_gb300 import lbm
    from paper_2103_02119_gb300.lbm import Batch, Lattice
    out = {}
    for name, wl, prec, scheme, small in single_cases():
        g = Lattice.from_workload(wl, precision=prec, scheme=scheme)
        if not small and wl.nx * wl.ny <= 4096:
            lbm.lbm_set_small_path(g.h, False)
        for n in STEPS:
            g.step(n)
            st, _ = g.diagnostics()
            if st not in (lbm.LBM_OK, lbm.LBM_ERR_UNSTABLE):
                raise RuntimeError(f"{name}: status {st}")
        out[name] = g.get_f()
        g.close()
    for shape in ((32, 1), (64, 8), (128, 64)):
        b = Batch(batch_cases())
        b.set_shape(*shape)
        for n in STEPS:
            b.step(n)
            b.residuals()         # raises LbmError on a failed bounds check
        for k in range(len(batch_cases())):
            out[f"batch_{shape[0]}x{shape[1]}_{k}"] = b.get_f(k)
        b.close()
    return out


if __name__ == "__main__":
    assert os.environ.get("LBM_CHECKED") == "1"
    from paper_2103_02119_gb300 import build
    build.build(checked=True)
    from paper_2103_02119_gb300 import lbm
    assert lbm.lib.lbm_build_flags() & lbm.LBM_BUILD_CHECKED
    res = run_all()
    np.savez(sys.argv[1], **res)
    print(f"checked build: {len(res)} final states, no bounds check failed")
