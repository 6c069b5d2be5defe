"""The seeded input recipes (host only): the batched uneven sweep, the
obstacle masks and the cavity parameters keep the invariants their
descriptions state, and a seed fixes them."""
import numpy as np
import pytest

from paper_2103_02119_gb300 import workloads as W


def test_random_obstacles_coverage_margin_and_seed():
    for seed in range(5):
        m = W.random_obstacles(200, 120, seed=seed, coverage=0.1)
        assert m.dtype == np.uint8 and m.shape == (120, 200)
        assert 0.0 < m.mean() <= 0.1
        assert not m[:2].any() and not m[-2:].any() and not m[:, :2].any() and not m[:, -2:].any()
        assert np.array_equal(m, W.random_obstacles(200, 120, seed=seed, coverage=0.1))
    assert not W.random_obstacles(5, 5, seed=0).any()  # too small for the margin


def test_stable_speed_of_sound_keeps_rest_weights_positive():
    for a in np.linspace(0.1, 0.99, 20):
        assert 0.0 < W.stable_cs2(a) < a * a
    assert W.stable_cs2(1.0) == pytest.approx(1.0 / 3.0)


def test_cavity_parameters():
    wl = W.cavity(64, 128, 0.5, 0.075, 0.05, 400.0)
    nu = 0.05 * 64 / 400.0
    tau = 1.0 / wl.omega[4]
    assert tau == pytest.approx(0.5 + nu / 0.075)
    assert wl.omega[4] == wl.omega[5] and wl.omega[3] == 1.0
    assert wl.periodic_x == 0 and wl.periodic_y == 0
    assert wl.wall_u[3] == (0.05, 0.0) and wl.wall_u[0] == (0.0, 0.0)


def test_batch_sweep_recipe():
    ws = W.batch_sweep(64, seed=0)
    assert len(ws) == 64
    kinds = [w.info["kind"] if "kind" in w.info else "cavity" for w in ws]
    assert 16 <= kinds.count("channel") <= 48
    for w in ws:
        assert 64 <= w.nx <= 1024 and 64 <= w.ny <= 1024
        assert 0.2 <= w.a <= 1.0
        assert w.cs2 == pytest.approx(W.stable_cs2(w.a))
        tau = 1.0 / w.omega[4]
        assert 0.505 - 1e-12 <= tau <= 2.0 + 1e-12
        assert w.mask is not None and w.mask.shape == (w.ny, w.nx) and w.mask.mean() <= 0.1
        if w.periodic_x:  # channel: force for a centre-line speed U
            nu, U, H = w.info["nu"], w.info["U"], w.ny * w.a
            assert w.Fx == pytest.approx(8.0 * nu * U / (H * H))
        else:             # cavity: the lid moves
            assert w.wall_u[3][0] > 0.0
    again = W.batch_sweep(64, seed=0)
    for a, b in zip(ws, again):
        assert (a.nx, a.ny, a.a, a.omega, a.Fx) == (b.nx, b.ny, b.a, b.omega, b.Fx)
        assert np.array_equal(a.mask, b.mask)
    other = W.batch_sweep(64, seed=1)
    assert any((a.nx, a.ny) != (b.nx, b.ny) for a, b in zip(ws, other))
