"""Writes tests/golden/cavity_256x1024_20k.json: the FP64 oracle's velocity
after 20,000 steps of the lid-driven cavity of Sec. 5.4 on the benchmark's
lattice shape scaled down to 256 x 1024 cells (a = 0.25, c_s^2 = 0.04, lid
speed 0.05, Re = 1000 on the cavity width, every other relaxation rate 1),
started from rest.

The stored values come from the oracle only: the density and velocity at a
seeded sample of 2,048 cells, plus sums over the whole field (mass, the
velocity's L2 norm) for the global checks.  Run from the repository root:

    python tests/golden/make_cavity_downscale.py

(about 10 minutes on 8 cores).
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2103_02119_gb300 import workloads as W  # noqa: E402

NX, NY, STEPS, SAMPLES, SEED = 256, 1024, 20_000, 2048, 20


def workload():
    return W.cavity(NX, NY, 0.25, 0.04, 0.05, 1000.0)


def sample_cells():
    rng = np.random.default_rng(SEED)
    return rng.integers(0, NY, SAMPLES), rng.integers(0, NX, SAMPLES)


def main():
    wl = workload()
    p = oracle.OracleParams.make(wl.nx, wl.ny, wl.a, wl.cs2, wl.omega, periodic_x=0,
                                 periodic_y=0, wall_u=wl.wall_u)
    o = oracle.Oracle(p)
    t = time.time()
    o.step(STEPS)
    r, u, v = o.moments()
    ys, xs = sample_cells()
    out = {
        "what": "FP64 oracle, lid-driven cavity (Sec. 5.4) 256 x 1024 cells, a = 0.25, "
                "c_s^2 = 0.04, lid u = 0.05, Re = 1000 (nu = 0.0128), rest start, "
                f"{STEPS} steps",
        "script": "tests/golden/make_cavity_downscale.py",
        "seconds": round(time.time() - t, 1), "threads": o.threads,
        "nx": NX, "ny": NY, "steps": STEPS, "sample_seed": SEED,
        "y": ys.tolist(), "x": xs.tolist(),
        "rho": [float(r[j, i]) for j, i in zip(ys, xs)],
        "ux": [float(u[j, i]) for j, i in zip(ys, xs)],
        "uy": [float(v[j, i]) for j, i in zip(ys, xs)],
        "mass": math.fsum(r.ravel()),
        "u_l2": math.sqrt(math.fsum((u * u + v * v).ravel())),
        "ux_max": float(np.abs(u).max()), "uy_max": float(np.abs(v).max()),
    }
    path = os.path.join(ROOT, "tests", "golden", "cavity_256x1024_20k.json")
    with open(path, "w") as fh:
        json.dump(out, fh)
    print(path, out["seconds"], "s")


if __name__ == "__main__":
    main()
