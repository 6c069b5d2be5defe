"""Batches of uneven lattices advanced by the persistent batch kernel.

A lattice of a batch must go through exactly the states of a single-lattice
handle with the same parameters and mask (bit for bit: the batch kernel runs
the same per-block step), whatever the launch shape, graph replay, retiring
and re-activation; one batch lattice is also checked against the FP64
oracle element by element.  The residual sums and the run-to-steady loop are
checked against the single-lattice diagnostics.
"""
import numpy as np
import pytest

from paper_2103_02119_gb300 import workloads as W
from gpu_common import F32_ATOL_F, F32_RTOL_U, oracle_of, rel_l2

pytestmark = pytest.mark.gpu


def _fields(wl, seed, u_amp=0.02):
    r, u, v = W.smooth_random_fields(wl.nx, wl.ny, seed, u_amp=u_amp, rho_amp=2e-3)
    return wl.with_(rho=r, ux=u, uy=v)


def uneven_set():
    """Ragged sizes (not multiples of any block width), both wall types, masks,
    a > 1, a tiny lattice and one lattice wider than a 256-column segment."""
    s = []
    s.append(_fields(W.cavity(70, 45, 0.5, 0.075, 0.05, 100.0), 1))
    s.append(_fields(W.poiseuille(ny=33, nx=130, a=0.25, cs2=0.01875, nu=0.02, U=0.03), 2)
             .with_(mask=W.random_obstacles(130, 33, seed=3, coverage=0.08)))
    s.append(W.taylor_green(33, 97, 0.25, 0.01875, 0.01, u0=0.02, seed=4))
    s.append(_fields(W.cavity(300, 21, 0.8, 0.19, 0.04, 300.0), 5)
             .with_(mask=W.random_obstacles(300, 21, seed=6, coverage=0.05)))
    s.append(_fields(W.taylor_green(5, 4, 1.5, 1 / 3, 0.05, seed=7), 7))
    s.append(W.taylor_green(64, 64, 1.0, 1 / 3, 0.02, u0=0.03, seed=8).with_(
        mask=W.random_obstacles(64, 64, seed=9, coverage=0.1)))
    return s


def singles(ws):
    """Single-lattice handles of the same workloads.  The batch always
    stores a link mask, so the handles get one too (all fluid where the
    workload has none): the same kernel code path, hence the same bits."""
    from paper_2103_02119_gb300.lbm import Lattice
    out = []
    for w in ws:
        if w.mask is None:
            w = w.with_(mask=np.zeros((w.ny, w.nx), np.uint8))
        out.append(Lattice.from_workload(w, precision=32))
    return out


def same_state(batch, k, lat):
    assert np.array_equal(batch.get_f(k), lat.get_f()), k


@pytest.fixture(scope="module")
def ws():
    return uneven_set()


@pytest.mark.parametrize("table", [True, False])
def test_batch_matches_single_handles_bit_for_bit(ws, table):
    """Either parameter path: the constant-memory tables (one group here) or
    the global table."""
    from paper_2103_02119_gb300.lbm import Batch
    b = Batch(ws)
    b.set_table_path(table)
    assert b.table_groups == (1 if table else 0)
    ref = singles(ws)
    for n in (1, 2, 57, 120):        # direct launches and graph replays, both parities
        b.step(n)
        for lat in ref:
            lat.step(n)
        for k, lat in enumerate(ref):
            same_state(b, k, lat)
            assert b.step_count(k) == lat.step_count
    assert b.launch_count == 180
    b.close()


@pytest.mark.parametrize("bx,rows", [(32, 1), (64, 8), (128, 64), (32, 7)])
def test_launch_shape_does_not_change_results(ws, bx, rows):
    from paper_2103_02119_gb300.lbm import Batch
    b = Batch(ws)
    b.set_shape(bx, rows)
    assert b.shape == (bx, rows)
    ref = singles(ws)
    b.step(53)
    for lat in ref:
        lat.step(53)
    for k, lat in enumerate(ref):
        same_state(b, k, lat)


def test_batch_lattice_matches_oracle(orc, ws):
    from paper_2103_02119_gb300.lbm import Batch
    b = Batch(ws)
    b.step(30)
    for k in (0, 1, 3):
        o = oracle_of(orc, ws[k])
        o.step(30)
        fo, fg = o.get_f(), b.get_f(k)
        assert float(np.abs(fg - fo).max()) <= F32_ATOL_F
        _, uo, vo = o.moments()
        _, ug, vg = b.moments(k)
        assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) <= F32_RTOL_U


@pytest.mark.parametrize("table", [True, False])
def test_retire_and_reactivate(ws, table):
    from paper_2103_02119_gb300.lbm import Batch
    b = Batch(ws)
    b.set_table_path(table)
    ref = singles(ws)
    b.step(3)
    for lat in ref:
        lat.step(3)
    frozen = b.get_f(2)
    b.set_active(2, False)
    b.set_active(4, False)
    assert not b.is_active(2) and b.is_active(0)
    b.step(51)                        # odd: the active lattices change parity
    for k, lat in enumerate(ref):
        if k not in (2, 4):
            lat.step(51)
    assert np.array_equal(b.get_f(2), frozen)
    assert b.step_count(2) == 3 and b.step_count(0) == 54
    b.set_active(2, True)             # re-joins at the other parity
    b.step(8)
    for k, lat in enumerate(ref):
        if k != 4:
            lat.step(8)
    for k, lat in enumerate(ref):
        same_state(b, k, lat)
    # retiring every lattice leaves an empty work list: stepping is a no-op
    for k in range(len(ws)):
        b.set_active(k, False)
    before = b.launch_count
    b.step(10)
    assert b.launch_count == before


def _many(count, seed):
    """`count` small lattices of both schemes, ragged sizes, masks."""
    rng = np.random.default_rng(seed)
    ws, schemes = [], []
    for k in range(count):
        nx, ny = int(rng.integers(5, 40)), int(rng.integers(4, 30))
        if k % 2:
            w = _fields(W.cavity(nx, ny, 0.5, 0.075, 0.04, 100.0), 100 + k)
        else:
            w = W.taylor_green(nx, ny, 0.8, 0.19, 0.02, u0=0.02, seed=k).with_(
                mask=W.random_obstacles(nx, ny, seed=k, coverage=0.05))
        ws.append(w)
        schemes.append(1 if k % 3 == 0 else 0)
    return ws, schemes


@pytest.mark.parametrize("count,groups", [(400, 3), (900, 0)])
def test_table_groups_and_fallback(count, groups):
    """400 lattices (266 RC-LBM, 134 RNR-LBM) fill three constant-memory
    tables (at most 180 lattices each, one scheme each); 900 would need six
    of the four and step from the global table.  Either way a sample of lattices equals single-lattice
    handles bit for bit, across graph replays and a retirement that changes
    the groups."""
    from paper_2103_02119_gb300.lbm import Batch, Lattice
    ws, schemes = _many(count, count)
    b = Batch(ws, schemes=schemes)
    assert b.table_groups == groups
    sample = list(range(0, count, 37)) + [count - 1]
    ref = []
    for k in sample:
        w = ws[k] if ws[k].mask is not None else ws[k].with_(
            mask=np.zeros((ws[k].ny, ws[k].nx), np.uint8))
        ref.append(Lattice.from_workload(w, precision=32, scheme=schemes[k]))
    b.step(57)
    for lat in ref:
        lat.step(57)
    for j, k in enumerate(sample):
        same_state(b, k, ref[j])
    # retire every third lattice: new groups, new graphs, same results
    for k in range(0, count, 3):
        if k not in sample:
            b.set_active(k, False)
    b.step(50)
    for lat in ref:
        lat.step(50)
    for j, k in enumerate(sample):
        same_state(b, k, ref[j])


def test_two_batches_share_the_tables(ws):
    """Two batches on one device take turns with the constant-memory tables:
    each re-uploads its own before it steps."""
    from paper_2103_02119_gb300.lbm import Batch
    a, c = Batch(ws), Batch(ws[::-1])
    ra, rc = singles(ws), singles(ws[::-1])
    for n in (3, 50, 7):
        a.step(n)
        c.step(n)
        for lat in ra + rc:
            lat.step(n)
    for k in range(len(ws)):
        same_state(a, k, ra[k])
        same_state(c, k, rc[k])
    assert a.table_groups == 1 and c.table_groups == 1


def test_residuals_match_single_diagnostics(ws):
    from paper_2103_02119_gb300.lbm import Batch
    b = Batch(ws)
    ref = singles(ws)
    st, r0 = b.residuals()
    assert st == 0 and np.all(r0 == -1.0)      # no reference yet
    for lat in ref:
        lat.diagnostics()
    b.step(40)
    for lat in ref:
        lat.step(40)
    st, r1 = b.residuals()
    assert st == 0
    for k, lat in enumerate(ref):
        _, d = lat.diagnostics()
        assert d[4] > 0 and abs(r1[k] - d[4]) <= 1e-12 * d[4], (k, r1[k], d[4])
        _, db = b.diagnostics(k)
        assert db[0] == d[0]                    # exact mass: same state, same bits
        assert db[4] == r1[k]


def test_run_to_steady_state():
    """Small body-force channels converge; each retires at the first check
    with R <= tol and keeps its state afterwards."""
    from paper_2103_02119_gb300.lbm import Batch, Lattice
    ws = [W.poiseuille(ny=ny, nx=nx, a=a, cs2=W.stable_cs2(a), nu=0.05, U=0.01)
          for nx, ny, a in ((8, 12, 0.5), (16, 20, 0.8), (4, 9, 1.0), (40, 7, 0.3))]
    b = Batch(ws)
    tol = 1e-7
    st, res = b.run(tol, check_every=100, max_steps=40000)
    assert st == 0
    assert all(not b.is_active(k) for k in range(len(ws)))
    assert np.all((res >= 0) & (res <= tol)), res
    for k, w in enumerate(ws):
        n = b.step_count(k)
        assert n % 100 == 0 and n < 40000
        lat = singles([w])[0]
        lat.diagnostics()
        lat.step(n - 100)
        lat.diagnostics()
        lat.step(100)
        _, d = lat.diagnostics()
        assert abs(d[4] - res[k]) <= 1e-9 * res[k] + 1e-15
        same_state(b, k, lat)


def test_tune_keeps_results(ws):
    from paper_2103_02119_gb300.lbm import Batch
    b = Batch(ws)
    bx, rows = b.tune(trial_steps=3)
    assert bx in (32, 64, 128) and rows in (1, 2, 4, 8, 16, 32, 64)
    assert b.shape == (bx, rows)
    n = b.step_count(0)
    assert n == 21 * 4
    ref = singles(ws)
    for lat in ref:
        lat.step(n)
    for k, lat in enumerate(ref):
        same_state(b, k, lat)


def test_mask_and_maskless_paths_agree():
    """A lattice without solid cells runs the same arithmetic with or without
    a stored link mask (the two kernels may round differently only where the
    compiler contracts operations differently)."""
    from paper_2103_02119_gb300.lbm import Lattice
    w = _fields(W.cavity(70, 45, 0.5, 0.075, 0.05, 100.0), 1)
    a = Lattice.from_workload(w, precision=32)
    b = Lattice.from_workload(w.with_(mask=np.zeros((w.ny, w.nx), np.uint8)), precision=32)
    a.step(50)
    b.step(50)
    assert float(np.abs(a.get_f() - b.get_f()).max()) <= F32_ATOL_F


def test_batch_errors():
    from paper_2103_02119_gb300 import lbm as L
    from paper_2103_02119_gb300.lbm import Batch, LbmError, LBM_ERR_INVALID
    b = Batch([W.taylor_green(16, 16, 1.0, 1 / 3, 0.05, seed=1)])
    out = np.empty(9 * 256)
    with pytest.raises(LbmError) as e:
        L.lbm_batch_get_f(b.b, 1, 256, out)
    assert e.value.status == LBM_ERR_INVALID and "outside" in str(e.value)
    with pytest.raises(LbmError):
        L.lbm_batch_set_active(b.b, -1, 1)
    with pytest.raises(LbmError):
        b.set_shape(48, 8)
    with pytest.raises(LbmError):
        b.set_shape(32, 0)
    with pytest.raises(LbmError):
        b.step(-1)
    with pytest.raises(LbmError):
        L.lbm_batch_set_table_path(b.b, 2)
    assert b.shape == (32, 16)
