"""lbm_diagnostics_noalloc against lbm_diagnostics.

lbm_diagnostics_noalloc serves callers that cannot allocate device memory
(device memory fully reserved by another allocator, or loops that must not
pay cudaMalloc's device synchronisation): its scratch is a fixed device array
inside the library.  It must give the values lbm_diagnostics gives, on two
calls in a row (the second one with a residual), whether it runs first in a
fresh process or after the other tests.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2103_02119_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _lattice(precision):
    from paper_2103_02119_gb300.lbm import Lattice
    wl = W.cavity(64, 128, 0.25, 0.01875, 0.03, 200.0)
    r, u, v = W.smooth_random_fields(64, 128, seed=4, u_amp=0.02, rho_amp=2e-3)
    wl = wl.with_(rho=r, ux=u, uy=v, mask=W.random_obstacles(64, 128, seed=5))
    g = Lattice.from_workload(wl, precision=precision)
    g.set_f(g.get_f() + W.perturbation(64, 128, 11, 5e-4))
    return g


@pytest.mark.parametrize("precision", [64, 32])
def test_noalloc_matches_diagnostics_on_two_calls(precision):
    from paper_2103_02119_gb300 import lbm
    g = _lattice(precision)
    for call in range(2):
        g.step(7)
        st_ref, ref = lbm.lbm_diagnostics(g.h)
        st_na, na = lbm.lbm_diagnostics_noalloc(g.h)
        assert st_ref == st_na == lbm.LBM_OK
        assert na[0] == ref[0]                      # exact fixed-point mass
        np.testing.assert_allclose(na[1:4], ref[1:4], rtol=1e-12, atol=1e-300)
        assert na[5] == ref[5] == 0 and na[6] == ref[6] == 7 * (call + 1)
        if call == 0:
            assert na[4] == ref[4] == -1.0
        else:
            assert ref[4] > 0
            np.testing.assert_allclose(na[4], ref[4], rtol=1e-12)
    g.close()


def test_noalloc_rejects_lattices_above_its_limit():
    from paper_2103_02119_gb300 import lbm
    from paper_2103_02119_gb300.lbm import Lattice
    g = Lattice(1100, 1000, 0.5, 0.075, [1.0] * 9, precision=32)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_diagnostics_noalloc(g.h)
    assert e.value.status == lbm.LBM_ERR_INVALID
    assert "1048576" in str(e.value)
    g.close()
