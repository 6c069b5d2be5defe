"""The checked build: step kernels compiled with device bounds checks on
every computed global, link-mask and shared-memory index (a failed check
skips the access and is reported as LBM_ERR_BOUNDS, without a trap).

A child process loads the checked library (LBM_CHECKED=1), steps tiny and
ragged grids with walls, masks, a moving lid, a force and both schemes on
both single-lattice kernels and on the batch kernel at three launch shapes,
and checks that no bounds test failed; its final states must equal the
normal build's bit for bit (the checks add no arithmetic).  The tiny grids
are also compared with the FP64 oracle element by element.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import checked_cases as C
from gpu_common import F64_ATOL_F, pair

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_reports_no_violation_and_matches_normal_build(tmp_path):
    out = tmp_path / "checked.npz"
    env = dict(os.environ, LBM_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-4000:]
    assert "no bounds check failed" in r.stdout
    got = np.load(out)
    ref = C.run_all()                 # the normal build, loaded by this process
    assert sorted(got.files) == sorted(ref)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("name", ["cavity_5x3", "cavity_7x9_mask", "tgv_5x3_force"])
def test_tiny_grids_match_oracle(orc, name, scheme):
    from paper_2103_02119_gb300 import lbm
    wl = dict((n, w) for n, w, p, s, sp in C.single_cases())[f"{name}_p64_s{scheme}_cluster"]
    for small in (True, False):
        o, g = pair(orc, wl, 64, scheme=scheme)
        lbm.lbm_set_small_path(g.h, small)
        o.step(40)
        g.step(40)
        assert float(np.abs(g.get_f() - o.get_f()).max()) <= F64_ATOL_F
        g.close()
