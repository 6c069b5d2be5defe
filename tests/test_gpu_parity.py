"""Parity of the CUDA library (through its C ABI) with the FP64 oracle.

Element by element on populations, density and velocity, after several
steps from a seeded non-equilibrium state, for every boundary type the
library supports: periodic axes, implicit half-way walls, a moving lid,
solid masks; grids that span several blocks with ragged tails, tiny grids,
a > 1, corrections switched off; FP64 and FP32 storage.  Full-size workloads
are checked in the launch configuration the benchmark uses.
"""
import math

import numpy as np
import pytest

from paper_2103_02119_gb300 import workloads as W
from gpu_common import compare, gpu_of, oracle_of, pair, rel_l2

pytestmark = pytest.mark.gpu


def _fields(wl, seed, u_amp=0.02):
    r, u, v = W.smooth_random_fields(wl.nx, wl.ny, seed, u_amp=u_amp, rho_amp=2e-3)
    return wl.with_(rho=r, ux=u, uy=v)


def configs():
    c = {}
    c["tgv_ragged"] = W.taylor_green(300, 67, 0.5, 0.075, 0.02, u0=0.03, seed=1, wavelength=60)
    c["channel_force"] = _fields(W.poiseuille(ny=40, nx=70, a=0.25, cs2=0.04, nu=0.02, U=0.03), 2)
    c["cavity_lid"] = _fields(W.cavity(45, 90, 0.5, 0.075, 0.05, 100.0), 3)
    c["obstacles_periodic"] = W.taylor_green(100, 80, 0.8, 0.2, 0.02, u0=0.02, seed=2).with_(
        mask=W.random_obstacles(100, 80, seed=3, coverage=0.1))
    c["obstacles_lid_a025"] = _fields(W.cavity(64, 128, 0.25, 0.01875, 0.03, 200.0), 4).with_(
        mask=W.random_obstacles(64, 128, seed=5, coverage=0.1))
    c["tiny_3x3"] = _fields(W.taylor_green(3, 3, 1.0, 1 / 3, 0.05, u0=0.01, seed=6), 6)
    c["tiny_4x5_lid"] = _fields(W.cavity(4, 5, 0.5, 0.075, 0.02, 10.0), 7)
    m = np.zeros((7, 5), np.uint8)
    m[3, 2] = 1
    c["tiny_5x7_mask"] = _fields(W.taylor_green(5, 7, 0.5, 0.075, 0.05, seed=8), 8).with_(mask=m)
    c["no_corrections"] = W.taylor_green(96, 50, 0.25, 0.01875, 0.02, u0=0.02, seed=9).with_(
        use_iso_corr=0, use_gi_corr=0)
    c["a2_force_xy"] = W.taylor_green(64, 40, 2.0, 1 / 3, 0.05, u0=0.02, seed=10).with_(
        Fx=2e-5, Fy=-1e-5)
    return c


CONFIGS = configs()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_parity(orc, name, precision):
    wl = CONFIGS[name]
    o, g = pair(orc, wl, precision, noise_seed=11, noise_amp=5e-4)
    compare(o, g, precision)          # the initial state itself
    o.step(7)
    g.step(7)
    compare(o, g, precision)
    o.step(13)
    g.step(13)
    compare(o, g, precision)
    # lattices of at most 4096 cells run each call's steps in one launch
    assert g.step_count == 20 and g.launch_count == (2 if wl.nx * wl.ny <= 4096 else 20)


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_fp32_setup_and_readout(orc, name):
    """FP32 storage: the equilibrium set-up, evaluated as a deviation from
    the rest state in FP32 arithmetic, against the oracle's FP64 equilibria;
    and the FP32 read-out of rho and u against the oracle's FP64 moments of
    the same stored state.  Both within a few FP32 roundings of the
    deviations (|f - w rho0| <~ 0.05), far below what a dropped term moves."""
    wl = CONFIGS[name]
    o, g = oracle_of(orc, wl), gpu_of(wl, 32)
    assert float(np.abs(g.get_f() - o.get_f()).max()) <= 1e-7
    g.step(3)
    o.set_f(g.get_f())
    ro, uo, vo = o.moments()
    rg, ug, vg = g.moments()
    assert float(np.abs(rg - ro).max()) <= 1e-7
    uscale = max(float(np.abs(uo).max()), float(np.abs(vo).max()))
    assert float(max(np.abs(ug - uo).max(), np.abs(vg - vo).max())) <= 1e-6 * uscale + 1e-9


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_parity_raw_moment_scheme(orc, name, precision):
    """The raw-moment scheme (RNR-LBM, Sec. 3) against the oracle's."""
    wl = CONFIGS[name]
    o, g = pair(orc, wl, precision, noise_seed=12, noise_amp=5e-4, scheme=1)
    o.step(9)
    g.step(9)
    compare(o, g, precision)
    o.step(11)
    g.step(11)
    compare(o, g, precision)


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("block_x,bands", [(32, 1), (32, 67), (64, 5), (256, 2), (128, 33)])
def test_tilings_are_bit_identical(precision, block_x, bands):
    """The result does not depend on how the step kernel is tiled: every cell
    computes the same arithmetic whichever block owns it or its halo."""
    wl = CONFIGS["obstacles_lid_a025"] if bands != 67 else CONFIGS["tgv_ragged"]
    ref = gpu_of(wl, precision)
    alt = gpu_of(wl, precision, block_x=block_x, bands=min(bands, wl.ny))
    ref.step(9)
    alt.step(9)
    assert ref.get_state() == alt.get_state()


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("periodic", [0, 1])
def test_narrow_tiles_with_walls(orc, precision, periodic):
    """Narrow tiles on a lattice with walls, a moving lid and a ragged last
    segment: with 64-column segments and 7-row bands most blocks see no edge
    of the lattice, the others see one or two.  The result equals the oracle
    and, bit for bit, the one-block-wide tiling (one 512-column segment,
    bands of the whole height)."""
    wl = _fields(W.cavity(300, 70, 0.5, 0.075, 0.04, 150.0), 13)
    if periodic:
        wl = wl.with_(periodic_x=1, periodic_y=1, wall_u=((0.0, 0.0),) * 4)
    o, g = pair(orc, wl, precision, noise_seed=14, noise_amp=5e-4, block_x=32, bands=10)
    ref = gpu_of(wl, precision, block_x=256, bands=1)
    ref.set_f(g.get_f())
    o.step(9)
    g.step(9)
    ref.step(9)
    compare(o, g, precision)
    assert ref.get_state() == g.get_state()


@pytest.mark.parametrize("precision", [64, 32])
def test_config1_poiseuille(orc, precision):
    """32 x 32 channel, a = 0.5, nu = 0.1, u_max = 0.01, 5000 steps from rest:
    against the oracle and against the parabola of Sec. 5.1."""
    wl = W.poiseuille()
    o, g = oracle_of(orc, wl), gpu_of(wl, precision)
    o.step(5000)
    g.step(5000)
    _, uo, vo = o.moments()
    rg, ug, vg = g.moments()
    if precision == 64:
        assert np.abs(ug - uo).max() <= 1e-12 * np.abs(uo).max()
        assert np.abs(vg).max() < 1e-14
    else:
        assert rel_l2(ug, uo) <= 1e-5
    H, U = wl.info["H"], wl.info["U"]
    y = (np.arange(wl.ny) + 0.5) * wl.a
    ua = (U * (1 - (y - H / 2) ** 2 / (H / 2) ** 2))[:, None]
    err = np.abs(ug - ua).sum() / (np.abs(ua).sum() * wl.nx)
    assert err < 3e-3


def test_tgv_decay_fp32_vs_fp64(orc):
    """Taylor-Green decay on the rectangular lattice (config 2 shape, reduced
    size): FP32 storage tracks the FP64 oracle within 1e-5 on velocity."""
    wl = W.taylor_green(128, 256, 0.5, 0.075, 0.01, u0=0.02, seed=0)
    o, g = oracle_of(orc, wl), gpu_of(wl, 32)
    o.step(1000)
    g.step(1000)
    _, uo, vo = o.moments()
    _, ug, vg = g.moments()
    assert rel_l2(np.stack([ug, vg]), np.stack([uo, vo])) <= 1e-5


@pytest.mark.parametrize("precision", [32, 64])
def test_full_size_shear_config2(orc, precision):
    """2048 x 1024 periodic Taylor-Green field at a = 0.5 with a perturbation,
    in the default launch configuration, two steps."""
    wl = W.taylor_green(2048, 1024, 0.5, 0.075, 0.01, u0=0.02, seed=1, wavelength=256)
    o, g = pair(orc, wl, precision, noise_seed=2, noise_amp=2e-4)
    o.step(2)
    g.step(2)
    compare(o, g, precision)


def test_full_size_cavity_config3(orc):
    """2048 x 8192 lid-driven cavity at a = 0.25 (the benchmark workload),
    FP32, in the benchmark's launch configuration, two steps from a smooth
    random state."""
    wl = _fields(W.cavity(2048, 8192, 0.25, 0.04, 0.05, 1000.0), 12, u_amp=0.03)
    o, g = pair(orc, wl, 32, noise_seed=13, noise_amp=2e-4)
    o.step(2)
    g.step(2)
    compare(o, g, 32)


def test_full_size_cavity_config3_200_steps(orc):
    """The benchmark workload (2048 x 8192 cavity, a = 0.25, FP32, its launch
    configuration) for 200 steps from rest, against the oracle.  A cell's
    state after n steps depends on cells at most 2n rows away (one row of
    streaming and one of the density stencil per step), so from rest
    everything more than 400 rows below the lid stays exactly at rest: the
    oracle runs the top 600 rows with a stationary wall beneath them, which
    meets only fluid at rest and so changes nothing."""
    wl = W.cavity(2048, 8192, 0.25, 0.04, 0.05, 1000.0)
    g = gpu_of(wl, 32)
    g.step(200)
    r, u, v = g.moments()
    g.close()
    top = 600
    o = oracle_of(orc, wl.with_(ny=top))
    o.step(200)
    ro, uo, vo = o.moments()
    # the window is deep enough: its bottom rows never saw the lid
    assert max(np.abs(uo[:top - 410]).max(), np.abs(vo[:top - 410]).max()) <= 1e-15
    lo = wl.ny - top
    err = rel_l2(np.stack([u[lo:], v[lo:]]), np.stack([uo, vo]))
    assert err <= 1e-5, err
    assert float(np.abs(r[lo:] - ro).max()) <= 1e-6
    # the rest of the lattice has not moved at all
    assert not np.any(u[:lo]) and not np.any(v[:lo]) and np.all(r[:lo] == 1.0)


def test_cavity_downscale_20k_steps_against_stored_oracle():
    """The benchmark cavity scaled down to 256 x 1024 cells (same a, c_s^2,
    lid speed and Re), FP32, 20,000 steps from rest, against the FP64
    oracle's values at a seeded sample of cells and its global sums (stored
    by tests/golden/make_cavity_downscale.py, which runs only the oracle)."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "cavity_256x1024_20k.json")
    with open(path) as fh:
        d = json.load(fh)
    wl = W.cavity(d["nx"], d["ny"], 0.25, 0.04, 0.05, 1000.0)
    g = gpu_of(wl, 32)
    g.step(d["steps"])
    r, u, v = g.moments()
    g.close()
    ys, xs = np.array(d["y"]), np.array(d["x"])
    got = np.stack([u[ys, xs], v[ys, xs]])
    want = np.stack([np.array(d["ux"]), np.array(d["uy"])])
    err = rel_l2(got, want)
    assert err <= 1e-5, err
    assert float(np.abs(r[ys, xs] - np.array(d["rho"])).max()) <= 1e-6
    # FP32 storage conserves the mass only to the rounding of each collision
    # (~1e-9 of a cell's density per step); over 20,000 steps the drift
    # stays below 1e-6 of the total (measured 2.7e-7)
    assert abs(math.fsum(r.ravel()) - d["mass"]) <= 1e-6 * d["mass"]
    ul2 = math.sqrt(math.fsum((u * u + v * v).ravel()))
    assert abs(ul2 - d["u_l2"]) <= 1e-5 * d["u_l2"]


@pytest.mark.parametrize("precision", [64, 32])
def test_diagnostics_match_oracle_fields(orc, precision):
    wl = CONFIGS["obstacles_lid_a025"]
    o, g = pair(orc, wl, precision, noise_seed=3, noise_amp=2e-4)
    st, d0 = g.diagnostics()
    assert st == 0 and d0[4] == -1.0 and d0[5] == 0 and d0[6] == 0 and d0[7] == -1.0
    o.step(9)
    o9 = o.moments()
    o.step(1)
    g.step(10)
    ro, uo, vo = o.moments()
    uo_prev, vo_prev = None, None
    st, d = g.diagnostics()
    assert st == 0 and d[5] == 0 and d[6] == 10
    tol = 1e-12 if precision == 64 else 1e-6
    assert abs(d[0] - math.fsum(ro.ravel())) <= tol * d[0]
    scale = math.fsum(np.abs(ro * uo).ravel()) + math.fsum(np.abs(ro * vo).ravel())
    assert abs(d[1] - math.fsum((ro * uo).ravel())) <= tol * scale
    assert abs(d[2] - math.fsum((ro * vo).ravel())) <= tol * scale
    en = math.fsum((0.5 * ro * (uo ** 2 + vo ** 2)).ravel())
    assert abs(d[3] - en) <= 10 * tol * en
    # residual between two calls 5 steps apart on the two-step means
    # ubar(n) = (u(n) + u(n-1)) / 2, and the step-to-step change, from the
    # oracle's fields
    _, u9, v9 = o9
    mb_prev = (0.5 * (uo + u9), 0.5 * (vo + v9))
    o.step(4)
    g.step(5)
    _, u14, v14 = o.moments()
    o.step(1)
    _, uo, vo = o.moments()
    st, d = g.diagnostics()
    mb = (0.5 * (uo + u14), 0.5 * (vo + v14))
    nb = math.sqrt(math.fsum((mb[0] ** 2 + mb[1] ** 2).ravel()))
    R = math.sqrt(math.fsum(((mb[0] - mb_prev[0]) ** 2 + (mb[1] - mb_prev[1]) ** 2).ravel())) / (
        5 * nb)
    assert abs(d[4] - R) <= (1e-9 if precision == 64 else 1e-4) * R
    S = math.sqrt(math.fsum(((uo - u14) ** 2 + (vo - v14) ** 2).ravel())) / nb
    assert abs(d[7] - S) <= (1e-9 if precision == 64 else 1e-4) * S


def test_streaming_is_a_permutation_mass_bit_exact():
    """With the collision switched off, a step only moves stored values (pull
    streaming and stationary bounce-back), so the exactly-summed mass keeps
    every bit, FP64 and FP32."""
    for precision in (64, 32):
        wl = _fields(W.cavity(77, 50, 0.5, 0.075, 0.0, 100.0), 14).with_(
            mask=W.random_obstacles(77, 50, seed=15))
        g = gpu_of(wl, precision, scheme=-1)
        g.set_f(g.get_f() + W.perturbation(77, 50, 16, 1e-3))
        _, d0 = g.diagnostics()
        g.step(1001)
        _, d1 = g.diagnostics()
        assert d1[0] == d0[0]


@pytest.mark.parametrize("precision", [64, 32])
def test_mass_drift_of_full_step(precision):
    """The collision conserves mass in exact arithmetic; in floating point the
    global drift per step stays at rounding level."""
    wl = CONFIGS["obstacles_lid_a025"].with_(wall_u=((0, 0),) * 4)
    g = gpu_of(wl, precision)
    _, d0 = g.diagnostics()
    g.step(200)
    _, d1 = g.diagnostics()
    eps = 2.2e-16 if precision == 64 else 1.2e-7
    assert abs(d1[0] - d0[0]) <= 200 * 0.05 * eps * wl.cells + 4 * eps * d0[0]


@pytest.mark.parametrize("precision", [64, 32])
def test_checkpoint_resume_and_determinism(precision):
    wl = CONFIGS["cavity_lid"]
    a = gpu_of(wl, precision)
    a.step(30)
    snap = a.get_state()
    a.step(25)
    end = a.get_state()
    b = gpu_of(wl, precision)
    b.set_state(snap)
    b.step(25)
    assert b.get_state() == end
    c = gpu_of(wl, precision)
    c.step(55)
    assert c.get_state() == end


def test_device_io_matches_host_io():
    import torch
    wl = CONFIGS["channel_force"]
    g = gpu_of(wl, 64)
    N = wl.cells
    rho = torch.tensor(wl.rho.ravel(), dtype=torch.float64, device="cuda")
    ux = torch.tensor(wl.ux.ravel(), dtype=torch.float64, device="cuda")
    uy = torch.tensor(wl.uy.ravel(), dtype=torch.float64, device="cuda")
    g.init_fields(rho, ux, uy)
    g.step(5)
    out = [torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3)]
    from paper_2103_02119_gb300 import lbm
    lbm.lbm_moments(g.h, N, *out)
    torch.cuda.synchronize()
    host = g.moments()
    for d_, h_ in zip(out, host):
        assert np.array_equal(d_.cpu().numpy().reshape(h_.shape), h_)
    fd = torch.empty(9 * N, dtype=torch.float64, device="cuda")
    lbm.lbm_get_f(g.h, N, fd)
    torch.cuda.synchronize()
    assert np.array_equal(fd.cpu().numpy().reshape(9, wl.ny, wl.nx), g.get_f())


def test_nonfinite_state_is_reported_and_recoverable():
    from paper_2103_02119_gb300 import lbm
    wl = CONFIGS["tgv_ragged"]
    g = gpu_of(wl, 32)
    f = g.get_f()
    bad = f.copy()
    bad[:, 10, 20] = np.nan
    g.set_f(bad)
    st, d = g.diagnostics()
    assert st == lbm.LBM_ERR_UNSTABLE and d[5] >= 1 and math.isnan(d[0])
    assert "non-finite" in lbm.lbm_last_error(g.h)
    g.set_f(f)
    st, d = g.diagnostics()
    assert st == lbm.LBM_OK and d[5] == 0


def test_state_size_mismatch_is_rejected():
    from paper_2103_02119_gb300 import lbm
    g = gpu_of(CONFIGS["tiny_3x3"], 32)
    with pytest.raises(lbm.LbmError) as e:
        g.set_state(b"\0" * 8)
    assert e.value.status == lbm.LBM_ERR_STATE


@pytest.mark.parametrize("precision", [64, 32])
@pytest.mark.parametrize("name", ["channel_force", "obstacles_lid_a025", "a2_force_xy",
                                  "tgv_ragged", "tiny_5x7_mask"])
def test_stress_output_matches_oracle(orc, name, precision):
    """Local strain rates and viscous stress (Eq. 30-40) of the same state:
    the GPU state is copied into the oracle, so that only the order of the
    FP64 arithmetic differs."""
    wl = CONFIGS[name]
    o, g = pair(orc, wl, precision, noise_seed=15, noise_amp=5e-4)
    g.step(17)
    o.set_f(g.get_f())
    sx, sy = o.strain()
    sxy, txx, tyy, txy = o.stress()
    got = g.stress()
    for ref, val in zip((sx, sy, sxy, txx, tyy, txy), got):
        scale = max(float(np.abs(ref).max()), 1e-300)
        assert float(np.abs(val - ref).max()) <= 1e-8 * scale
    solid = o.solid().astype(bool)
    for val in got:
        assert np.all(val[solid] == 0.0)
