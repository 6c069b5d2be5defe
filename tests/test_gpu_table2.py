"""Table 2 of Sec. 5.1 on the GPU FP64 path: the body-force channel at
a = 0.5, tau = 0.6, Re = 50, N = 100, 200, 400 cells across, both schemes
(set-up, error and run length as in tests/test_oracle_table2.py).  At N = 100
the GPU's final velocity equals the oracle's element by element; over the
three resolutions both schemes converge at second order and agree with each
other to well under 1 %."""
import numpy as np
import pytest

from gpu_common import F64_RTOL_U
from test_oracle_table2 import channel, global_error, oracle_fields, steps_for

pytestmark = pytest.mark.gpu


def gpu_fields(N, scheme):
    from paper_2103_02119_gb300.lbm import Lattice
    wl, ua = channel(N)
    g = Lattice.from_workload(wl, precision=64, scheme={"rc": 0, "rnr": 1}[scheme])
    g.init_fields(np.ones_like(ua), ua, np.zeros_like(ua))
    g.step(steps_for(N))
    _, u, v = g.moments()
    g.close()
    return u, v, ua


@pytest.fixture(scope="module")
def runs():
    out = {}
    for N in (100, 200, 400):
        for s in ("rc", "rnr"):
            out[(N, s)] = gpu_fields(N, s)
    print("Table 2 (GPU FP64):",
          {f"{N} {s}": f"{global_error(*f):.3e}" for (N, s), f in out.items()})
    return out


@pytest.mark.parametrize("scheme", ["rc", "rnr"])
def test_n100_matches_the_oracle(orc, runs, scheme):
    """Element by element after 110,000 steps (FP64 on both sides: only the
    order of rounding differs)."""
    u, v, ua = runs[(100, scheme)]
    uo, vo, _ = oracle_fields(orc, 100, scheme)
    du = max(np.abs(u - uo).max(), np.abs(v - vo).max()) / np.abs(uo).max()
    assert du <= F64_RTOL_U, du


def test_second_order_and_schemes_agree(runs):
    errors = {k: global_error(*f) for k, f in runs.items()}
    for s in ("rc", "rnr"):
        for N in (100, 200):
            ratio = errors[(N, s)] / errors[(2 * N, s)]
            assert 3.7 < ratio < 4.3, (s, N, ratio)
    for N in (100, 200, 400):
        rc, rnr = errors[(N, "rc")], errors[(N, "rnr")]
        assert abs(rc - rnr) < 0.01 * rc, (N, rc, rnr)
