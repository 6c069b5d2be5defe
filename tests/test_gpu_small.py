"""Small lattices (at most 4096 cells) on the cluster kernel.

The cluster kernel runs up to 1024 steps per launch; a lattice must go
through exactly the states of the row-band kernel (bit for bit, FP32 and
FP64), whatever the number of steps per call and its parity, with masks,
both wall types, a force, a > 1, fewer rows than CTAs in a cluster and the
largest lattice the path takes.  Agreement with the FP64 oracle follows from
the parity tests, whose lattices of at most 4096 cells run on this path.
"""
import numpy as np
import pytest

from paper_2103_02119_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fields(wl, seed, u_amp=0.02):
    r, u, v = W.smooth_random_fields(wl.nx, wl.ny, seed, u_amp=u_amp, rho_amp=2e-3)
    return wl.with_(rho=r, ux=u, uy=v)


def cases():
    c = {}
    c["poiseuille_32x32"] = W.poiseuille(ny=32, nx=32, a=1.0, cs2=1 / 3, nu=0.1, U=0.05)
    c["cavity_45x70_mask"] = _fields(W.cavity(45, 70, 0.5, 0.075, 0.05, 100.0), 1).with_(
        mask=W.random_obstacles(45, 70, seed=2, coverage=0.08))
    c["tgv_64x64_a2_force"] = W.taylor_green(64, 64, 2.0, 1 / 3, 0.05, u0=0.02, seed=3).with_(
        Fx=2e-5, Fy=-1e-5)
    c["cavity_300x5"] = _fields(W.cavity(300, 5, 0.8, W.stable_cs2(0.8), 0.04, 300.0), 4)
    c["poiseuille_7x3_mask"] = W.poiseuille(ny=3, nx=7, a=0.5, cs2=0.075, nu=0.02, U=0.01).with_(
        mask=np.array([[0, 0, 0, 1, 0, 0, 0], [0, 0, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0, 0]],
                      np.uint8))
    return c


CASES = cases()


def _pair(wl, precision):
    from paper_2103_02119_gb300 import lbm
    from paper_2103_02119_gb300.lbm import Lattice
    a = Lattice.from_workload(wl, precision=precision)
    b = Lattice.from_workload(wl, precision=precision)
    lbm.lbm_set_small_path(b.h, False)
    return a, b


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("name", sorted(CASES))
def test_cluster_kernel_matches_row_band_kernel(name, precision):
    wl = CASES[name]
    assert wl.nx * wl.ny <= 4096
    a, b = _pair(wl, precision)
    total = 0
    for n in (1, 2, 57, 1100):            # both parities; 1100 takes two launches
        a.step(n)
        b.step(n)
        total += n
        assert np.array_equal(a.get_f(), b.get_f()), n
    assert a.step_count == b.step_count == total
    assert a.launch_count == 5 and b.launch_count == total
    da, db = a.diagnostics()[1], b.diagnostics()[1]
    assert np.array_equal(da, db)         # including the step-to-step change
    a.close()
    b.close()


def test_switching_paths_mid_run():
    from paper_2103_02119_gb300 import lbm
    wl = CASES["cavity_45x70_mask"]
    a, b = _pair(wl, 32)
    a.step(33)
    lbm.lbm_set_small_path(a.h, False)
    a.step(20)
    lbm.lbm_set_small_path(a.h, True)
    a.step(11)
    b.step(64)
    assert np.array_equal(a.get_f(), b.get_f())
    assert a.launch_count == 22
    a.close()
    b.close()


def test_path_is_refused_for_larger_lattices():
    from paper_2103_02119_gb300 import lbm
    from paper_2103_02119_gb300.lbm import Lattice
    g = Lattice.from_workload(W.cavity(65, 64, 1.0, 1 / 3, 0.05, 100.0), precision=32)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_set_small_path(g.h, True)
    assert e.value.status == lbm.LBM_ERR_INVALID
    lbm.lbm_set_small_path(g.h, False)    # already the row-band kernel: accepted
    g.step(2)
    assert g.launch_count == 2
    g.close()


def test_small_lattice_allocation_failures():
    """The density field of the cluster path is one allocation more than a
    larger lattice makes; failing any of them gives LBM_ERR_OOM."""
    from paper_2103_02119_gb300 import lbm
    wl = CASES["cavity_45x70_mask"]
    p = lbm.params_of_workload(wl, precision=64)
    for nth in range(1, 7):
        lbm.lbm_debug_fail_alloc(nth)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(p, wl.mask)
        assert e.value.status == lbm.LBM_ERR_OOM
    lbm.lbm_debug_fail_alloc(7)
    h = lbm.lbm_create(p, wl.mask)
    lbm.lbm_debug_fail_alloc(0)
    lbm.lbm_destroy(h)
