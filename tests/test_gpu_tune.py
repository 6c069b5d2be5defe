"""Launch-shape tuner on the GPU: the chosen shape is a candidate and is
cached, and a lattice stepped with it goes through the same states, bit for
bit, as one with the automatic shape."""
import json

import numpy as np
import pytest

from paper_2103_02119_gb300 import tune
from paper_2103_02119_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _wl():
    r, u, v = W.smooth_random_fields(300, 200, 3, u_amp=0.02, rho_amp=2e-3)
    return W.cavity(300, 200, 0.5, 0.075, 0.05, 300.0).with_(
        rho=r, ux=u, uy=v, mask=W.random_obstacles(300, 200, seed=4, coverage=0.05))


@pytest.mark.parametrize("precision", [32, 64])
def test_tuned_shape_is_cached_and_changes_no_result(tmp_path, precision):
    from paper_2103_02119_gb300.lbm import Lattice
    path = str(tmp_path / "tune.json")
    wl = _wl()
    shape = tune.tune_lattice(wl, precision, path=path, steps=5)
    assert shape in tune.lattice_candidates(wl.nx, wl.ny)
    entry = json.load(open(path))[tune.lattice_key(wl.nx, wl.ny, precision, True)]
    assert tuple(entry["shape"]) == shape and entry["ms_per_step"] > 0
    a = tune.tuned_lattice(wl, precision, path=path)
    b = Lattice.from_workload(wl, precision=precision)
    a.step(61)
    b.step(61)
    assert np.array_equal(a.get_f(), b.get_f())
    a.close()
    b.close()


def test_batch_shape_is_cached(tmp_path):
    from paper_2103_02119_gb300.lbm import Batch
    path = str(tmp_path / "tune.json")
    ws = [W.cavity(70, 45, 0.5, 0.075, 0.05, 100.0), W.cavity(200, 90, 0.8, W.stable_cs2(0.8),
                                                              0.04, 300.0)]
    b = Batch(ws)
    shape = tune.tune_batch(b, ws, path=path, trial_steps=3)
    assert b.shape == shape
    b.close()
    c = Batch(ws)
    c.set_shape(32, 1)
    assert tune.tune_batch(c, ws, path=path) == shape     # from the cache
    assert c.shape == shape
    c.close()
