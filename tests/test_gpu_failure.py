"""Failure paths on the GPU, made without faulting it.

A bounded wait that runs out: the test sets the step kernel's poll limit to
0, so each block's wait for its first staged row gives up at once; the block
records it in the status word, waits with the full bound for its copies in
flight and returns.  The host reads the word (LBM_ERR_TIMEOUT) and the
context stays usable.  A device allocation that fails: the host-side hook
fails the n-th allocation before any CUDA call, for every allocation an
entry point makes in turn; each gives LBM_ERR_OOM and leaves nothing behind.
"""
import numpy as np
import pytest

from paper_2103_02119_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FULL = 1 << 22


def _wl():
    wl = W.cavity(96, 64, 0.5, 0.075, 0.05, 100.0)
    return wl.with_(mask=W.random_obstacles(96, 64, seed=2))


@pytest.mark.parametrize("precision", [32, 64])
def test_wait_that_runs_out_is_reported(precision):
    from paper_2103_02119_gb300 import lbm
    from paper_2103_02119_gb300.lbm import Lattice
    g = Lattice.from_workload(_wl(), precision=precision)
    g.step(3)
    assert g.diagnostics()[0] == lbm.LBM_OK
    lbm.lbm_set_wait_limit(g.h, 0)
    for n in (2, 50):                        # launched directly, then from a graph
        g.step(n)
        for call in (lbm.lbm_diagnostics, lbm.lbm_diagnostics_noalloc):
            with pytest.raises(lbm.LbmError) as e:
                call(g.h)
            assert e.value.status == lbm.LBM_ERR_TIMEOUT
            assert "gave up waiting" in str(e.value)
    # the report stays until the state is replaced; the context stays usable
    lbm.lbm_set_wait_limit(g.h, FULL)
    g.init_fields()
    g.step(60)
    st, d = g.diagnostics()
    assert st == lbm.LBM_OK and d[5] == 0 and d[6] == 60
    st, d2 = lbm.lbm_diagnostics_noalloc(g.h)
    assert st == lbm.LBM_OK and d2[0] == d[0]
    # the same state as a lattice that never timed out
    h = Lattice.from_workload(_wl(), precision=precision)
    h.step(60)
    assert np.array_equal(g.get_f(), h.get_f())
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_wait_limit(g.h, FULL + 1)
    g.close()
    h.close()


def test_batch_wait_that_runs_out_is_reported():
    from paper_2103_02119_gb300 import lbm
    from paper_2103_02119_gb300.lbm import Batch
    ws = [_wl(), W.cavity(40, 70, 0.8, W.stable_cs2(0.8), 0.04, 50.0)]
    b = Batch(ws)
    b.step(3)
    assert b.residuals()[0] == lbm.LBM_OK
    lbm.lbm_batch_set_wait_limit(b.b, 0)
    b.step(2)
    with pytest.raises(lbm.LbmError) as e:
        b.residuals()
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    with pytest.raises(lbm.LbmError) as e:
        b.run(1e-8, check_every=10, max_steps=20)
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    # reported once; re-initialised lattices step normally again
    lbm.lbm_batch_set_wait_limit(b.b, FULL)
    for k in range(len(ws)):
        b.init_fields(k)
    b.step(60)
    st, res = b.residuals()
    assert st == lbm.LBM_OK
    ref = Batch(ws)
    ref.step(60)
    for k in range(len(ws)):
        assert np.array_equal(b.get_f(k), ref.get_f(k))
    b.close()
    ref.close()


def _count_failures(make, destroy, lbm, limit=40):
    """Fails allocation 1, 2, ... of make() until it succeeds; returns how
    many allocations failed (each must give LBM_ERR_OOM)."""
    for nth in range(1, limit):
        lbm.lbm_debug_fail_alloc(nth)
        try:
            obj = make()
        except lbm.LbmError as e:
            assert e.status == lbm.LBM_ERR_OOM, (nth, str(e))
            continue
        lbm.lbm_debug_fail_alloc(0)      # the countdown outlived make()
        destroy(obj)
        return nth - 1
    lbm.lbm_debug_fail_alloc(0)
    raise AssertionError("make() kept failing")


def test_every_allocation_failure_gives_oom():
    import torch
    from paper_2103_02119_gb300 import lbm
    wl = _wl()
    free0 = torch.cuda.mem_get_info()[0]
    p = lbm.params_of_workload(wl, precision=32)
    n = _count_failures(lambda: lbm.lbm_create(p, wl.mask), lbm.lbm_destroy, lbm)
    assert n == 5                        # link mask, two buffers, partial sums, status
    q = [lbm.params_of_workload(w, precision=32) for w in (wl, wl)]
    n = _count_failures(lambda: lbm.lbm_batch_create(q, [wl.mask, None]),
                        lbm.lbm_batch_destroy, lbm)
    assert n >= 8
    n = _count_failures(lambda: lbm.lbm_nn_create([8, 16], 2, 16, 16), lbm.lbm_nn_destroy, lbm)
    assert n >= 8
    # the residual field of the first lbm_diagnostics call
    h = lbm.lbm_create(p, wl.mask)
    lbm.lbm_debug_fail_alloc(1)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_diagnostics(h)
    assert e.value.status == lbm.LBM_ERR_OOM
    st, d = lbm.lbm_diagnostics(h)          # the handle stays valid
    assert st == lbm.LBM_OK
    lbm.lbm_destroy(h)
    torch.cuda.synchronize()
    # nothing leaked (the library's own allocations bypass torch's cache)
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
