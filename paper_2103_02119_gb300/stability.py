"""Numerical stability sweeps of the two rectangular schemes (Sec. 6).

Both studies run many small lid-driven cavities at once through the batch
API of the CUDA library (FP32, one persistent launch per step) and call a
run unstable when any of its fluid cells turns non-finite within the step
budget.

* ``lid_velocity_thresholds``: the largest lid speed U that stays stable for
  a fixed number of steps, against the relaxation time tau, for RC-LBM and
  RNR-LBM on 21 x ny cavities of physical aspect 1 (ny = 20/a + 1), the
  study of Fig. 17.
* ``max_reynolds``: the largest Re = U nx / nu that stays stable at a = 0.5,
  U = 0.2, c_s^2 = 0.1 on nx x 2nx cavities, the study of Table 6.

The speed of sound of the first study is not given in the paper; it is
c_s^2 = min(1/3, f a^2) with f = 0.3 by default, inside the range the
paper's own cavity runs use at a = 0.5 (Table 3: c_s^2 = 0.02 to 0.18, i.e.
f = 0.08 to 0.72).  The RC-LBM advantage of Fig. 17 shows at f = 0.3 and
0.15; at f = 0.6 the two schemes stay within a step or two of each other.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W


def fig17_cs2(a: float, factor: float = 0.3) -> float:
    """c_s^2 of the lid-speed sweep: min(1/3, factor a^2)."""
    return min(1.0 / 3.0, factor * a * a)


def largest_stable(runs) -> float:
    """The largest value v of [(v, stable), ...] such that v and every
    smaller value stayed stable (0 when the smallest one did not)."""
    best = 0.0
    for v, ok in sorted(runs):
        if not ok:
            break
        best = v
    return best


def _run(wls, schemes, steps, check, stream):
    from .lbm import Batch
    b = Batch(wls, stream=stream, schemes=schemes)
    try:
        # tol = 0: only a lattice that stops changing exactly is retired early
        st, res = b.run(0.0, check_every=check, max_steps=steps)
        done = np.array([b.step_count(k) for k in range(len(wls))])
    finally:
        b.close()
    return ~np.isnan(res), done


def lid_velocity_thresholds(a_values=(1.0, 0.5, 0.3), taus=(0.51, 0.55, 0.6, 0.7, 0.8, 1.0),
                            u_values=None, steps=100_000, check=1000, nx=21, stream=None,
                            cs2_factor=0.3):
    """Returns {(a, tau, scheme): largest U of u_values such that it and
    every smaller U stayed stable}; scheme 0 = RC-LBM, 1 = RNR-LBM."""
    if u_values is None:
        u_values = np.round(np.arange(0.02, 0.62, 0.02), 4)
    wls, schemes, keys = [], [], []
    for a in a_values:
        ny = int(round((nx - 1) / a)) + 1
        cs2 = fig17_cs2(a, cs2_factor)
        for tau in taus:
            nu = cs2 * (tau - 0.5)
            for U in u_values:
                for scheme in (0, 1):
                    wls.append(W.cavity(nx, ny, a, cs2, float(U), float(U) * nx / nu))
                    schemes.append(scheme)
                    keys.append((a, tau, scheme, float(U)))
    stable, _ = _run(wls, schemes, steps, check, stream)
    out = {}
    for (a, tau, scheme, U), ok in zip(keys, stable):
        out.setdefault((a, tau, scheme), []).append((U, bool(ok)))
    return {key: largest_stable(runs) for key, runs in out.items()}


def max_reynolds(grids=((100, 200), (200, 400), (300, 600)), a=0.5, U=0.2, cs2=0.1,
                 re_values=None, steps=100_000, check=1000, stream=None):
    """Returns {(nx, ny, scheme): largest Re of re_values such that it and
    every smaller Re stayed stable}."""
    if re_values is None:
        re_values = np.round(np.geomspace(2000, 32000, 17))
    wls, schemes, keys = [], [], []
    for nx, ny in grids:
        for Re in re_values:
            for scheme in (0, 1):
                wls.append(W.cavity(nx, ny, a, cs2, U, float(Re)))
                schemes.append(scheme)
                keys.append((nx, ny, scheme, float(Re)))
    stable, _ = _run(wls, schemes, steps, check, stream)
    out = {}
    for (nx, ny, scheme, Re), ok in zip(keys, stable):
        out.setdefault((nx, ny, scheme), []).append((Re, bool(ok)))
    return {key: largest_stable(runs) for key, runs in out.items()}


def main(argv=None):
    """python -m paper_2103_02119_gb300.stability [--steps N] [--table6-grids G]
    [--cs2-factor F] prints the two sweeps as JSON lines (an empty G skips
    the second)."""
    import argparse
    import json

    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=100_000)
    ap.add_argument("--table6-grids", default="100x200,200x400,300x600")
    ap.add_argument("--cs2-factor", type=float, default=0.3,
                    help="c_s^2 = min(1/3, factor a^2) in the lid-speed sweep")
    args = ap.parse_args(argv)
    thr = lid_velocity_thresholds(steps=args.steps, cs2_factor=args.cs2_factor)
    print(json.dumps({"fig17_max_lid_speed": [
        {"a": a, "tau": tau, "scheme": "RC" if sc == 0 else "RNR", "U_max": u}
        for (a, tau, sc), u in sorted(thr.items())], "steps": args.steps,
        "cs2_factor": args.cs2_factor}), flush=True)
    grids = [tuple(int(v) for v in g.split("x")) for g in args.table6_grids.split(",") if g]
    if not grids:  # --table6-grids "": the lid-speed sweep only
        return
    best = max_reynolds(grids=grids, steps=args.steps)
    print(json.dumps({"table6_max_re": [
        {"grid": f"{nx}x{ny}", "scheme": "RC" if sc == 0 else "RNR", "Re_max": r}
        for (nx, ny, sc), r in sorted(best.items())], "steps": args.steps}), flush=True)


if __name__ == "__main__":
    main()
