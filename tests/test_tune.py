"""Launch-shape tuner: cache keys, the choice of the fastest candidate, and
the JSON cache's reuse, on the CPU with an injected measurement."""
import json

from paper_2103_02119_gb300 import tune


def test_keys_name_size_precision_layout_and_mask():
    k = tune.lattice_key(2048, 8192, 32, False)
    assert k == f"lattice:2048x8192:fp32:{tune.LAYOUT}:nomask"
    assert tune.lattice_key(2048, 8192, 64, True) != k
    # a batch key ignores the order of its lattices, not their sizes
    a = tune.batch_key([(64, 32), (128, 70), (64, 32)])
    assert a == tune.batch_key([(128, 70), (64, 32), (64, 32)])
    assert a != tune.batch_key([(64, 32), (128, 70)])
    assert a.startswith("batch:3:fp32:")


def test_candidates_fit_the_lattice():
    c = tune.lattice_candidates(50, 40)
    assert all(bx * 2 <= 100 for bx, _ in c) and (32, 0) in c
    assert {bx for bx, _ in tune.lattice_candidates(2048, 8192)} == {32, 64, 128, 256}
    assert all(nb >= 0 for _, nb in tune.lattice_candidates(3, 2))


def test_choose_measures_once_then_reads_the_cache(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    cost = {(32, 0): 3.0, (64, 0): 1.5, (64, 10): 2.0}
    calls = []

    def measure(s):
        calls.append(s)
        return cost[s]

    assert tune.choose("k", list(cost), measure, path) == (64, 0)
    assert sorted(calls) == sorted(cost)
    d = json.load(open(path))
    assert d["k"]["shape"] == [64, 0] and d["k"]["ms_per_step"] == 1.5
    calls.clear()
    assert tune.choose("k", list(cost), measure, path) == (64, 0)
    assert calls == []                       # from the cache
    cost[(32, 0)] = 0.5
    assert tune.choose("k", list(cost), measure, path, force=True) == (32, 0)
    assert tune.choose("other", [(128, 4)], lambda s: 1.0, path) == (128, 4)
    d = json.load(open(path))
    assert set(d) == {"k", "other"}          # entries of other keys are kept


def test_unreadable_cache_is_rebuilt(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    monkeypatch.setenv("LBM_TUNE_CACHE", str(path))
    assert tune.cache_path() == str(path)
    assert tune.choose("k", [(32, 1)], lambda s: 1.0) == (32, 1)
    assert json.load(open(path))["k"]["shape"] == [32, 1]
