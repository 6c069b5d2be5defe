"""The paper's remaining validation flows on the GPU (Sec. 5.2, 5.3, 5.6).

- transient Couette flow at the paper's a = 0.1, 50 x 500 setup against its
  Fourier series;
- Womersley flow at the paper's a = 0.125, 400 wall-normal cells,
  Wo = 4.25, T = 40,000, tau = 1 against the analytic solution of a channel
  driven by F_m cos(w t) (Wo read as (H/2) sqrt(w / nu));
- the shallow lid-driven cavity (H/L = 0.25, Re = 100) on the square
  lattice (400 x 100, a = 1) and on the rectangular one (100 x 125,
  a = 0.2): the centre-line velocity profiles agree with a quarter of the
  cells.
"""
import numpy as np
import pytest

from paper_2103_02119_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def lattice(wl, precision, **kw):
    from paper_2103_02119_gb300.lbm import Lattice
    return Lattice.from_workload(wl, precision=precision, **kw)


@pytest.mark.parametrize("precision", [64, 32])
def test_transient_couette_a01(precision):
    """Sec. 5.2: a = 0.1, 50 x 500 cells (H = 50), tau = 0.8, U = 0.02,
    c_s^2 = 0.005; u(y, t) against the series solution at four times."""
    a, ny, nx = 0.1, 500, 50
    wl = W.couette(ny=ny, nx=nx, a=a, cs2=0.005, tau=0.8, U=0.02)
    nu, U, H = wl.info["nu"], wl.info["U"], wl.info["H"]
    g = lattice(wl, precision)
    y = (np.arange(ny) + 0.5) * a
    n_terms = np.arange(1, 401)[:, None]
    t = 0
    for T in (0.005, 0.01, 0.02, 0.05):
        n = int(round(T * H * H / nu))
        g.step(n - t)
        t = n
        _, u, v = g.moments()
        series = U * y / H - (2 * U / np.pi) * (
            np.exp(-n_terms ** 2 * np.pi ** 2 * nu * t / H ** 2) / n_terms
            * np.sin(n_terms * np.pi * (1 - y / H))).sum(0)
        err = np.abs(u.mean(axis=1) - series).max()
        assert err < 2e-3 * U, (T, err / U)
        assert np.abs(v).max() < 1e-6 * U


@pytest.mark.parametrize("precision", [64, 32])
def test_womersley_a0125(precision):
    """Sec. 5.3: oscillating body force F_m cos(w t) between two plates,
    H = 50 over 400 cells (a = 0.125), T = 40,000, Wo = 4.25, tau = 1,
    F_m = 1e-5; from the periodic solution at t = 0, u(y) at eight phases
    of the third period."""
    a, ny, nx = 0.125, 400, 4
    H, T, Wo, tau, Fm = ny * a, 40000, 4.25, 1.0, 1e-5
    w = 2 * np.pi / T
    nu = w * (H / 2) ** 2 / Wo ** 2
    cs2 = nu / (tau - 0.5)
    wl = W.Workload("womersley", nx, ny, a, cs2, W.omega_for(nu, cs2), periodic_x=1,
                    periodic_y=0)
    yc = (np.arange(ny) + 0.5) * a - H / 2
    k = np.sqrt(1j * w / nu)
    shape = 1 - np.cosh(k * yc) / np.cosh(k * H / 2)
    amp = np.abs(Fm / (1j * w) * shape).max()
    # start on the periodic solution at t = 0: a start from rest would carry
    # a transient that decays only over H^2 / (pi^2 nu) ~ 47,000 steps
    u0 = np.real(Fm / (1j * w) * shape)[:, None] * np.ones((1, nx))
    g = lattice(wl.with_(rho=np.ones((ny, nx)), ux=u0, uy=np.zeros((ny, nx))), precision)
    checks = set(2 * T + T * np.arange(8) // 8)
    worst = 0.0
    for n in range(3 * T):
        g.set_force(Fm * np.cos(w * (n + 0.5)), 0.0)
        g.step(1)
        if n + 1 in checks:
            _, u, _ = g.moments()
            exact = np.real(Fm / (1j * w) * shape * np.exp(1j * w * (n + 1)))
            worst = max(worst, np.abs(u.mean(axis=1) - exact).max() / amp)
    assert worst < 0.02, worst


def test_shallow_cavity_square_vs_rectangular():
    """Sec. 5.6: H/L = 0.25, Re = U L / nu = 100.  Square lattice 400 x 100
    (a = 1) and rectangular 100 x 125 (a = 0.2, c_s^2 = 0.02), both run to a
    steady residual of 1e-7; u along the vertical and v along the
    horizontal centre line agree within 2 % of the lid speed."""
    from paper_2103_02119_gb300.lbm import Batch
    U, Re = 0.02, 100.0
    sq = W.cavity(400, 100, 1.0, 1.0 / 3.0, U, Re)
    rc = W.cavity(100, 125, 0.2, 0.02, U, Re)
    b = Batch([sq, rc])
    st, res = b.run(1e-7, check_every=1000, max_steps=600_000)
    assert st == 0 and np.all((res >= 0) & (res <= 1e-7)), res
    _, us, vs = b.moments(0)
    _, ur, vr = b.moments(1)
    # vertical centre line x = L/2: mean of the two middle columns
    u_sq = 0.5 * (us[:, 199] + us[:, 200]) / U
    u_rc = 0.5 * (ur[:, 49] + ur[:, 50]) / U
    y_sq = (np.arange(100) + 0.5) / 100
    y_rc = (np.arange(125) + 0.5) / 125
    assert np.abs(np.interp(y_sq, y_rc, u_rc) - u_sq).max() < 0.02
    # horizontal centre line y = H/2
    v_sq = 0.5 * (vs[49, :] + vs[50, :]) / U
    v_rc = vr[62, :] / U
    x_sq = (np.arange(400) + 0.5) / 400
    x_rc = (np.arange(100) + 0.5) / 100
    inside = (x_sq >= x_rc[0]) & (x_sq <= x_rc[-1])   # no extrapolation
    assert np.abs(np.interp(x_sq, x_rc, v_rc) - v_sq)[inside].max() < 0.02


def _amplitude(u, phase_field):
    """FP64 projection of a velocity component onto sin(phase)."""
    s = np.sin(phase_field)
    return float((u * s).sum() / (s * s).sum())


@pytest.mark.parametrize("a", [0.25, 0.5, 1.0])
@pytest.mark.parametrize("nu", [1e-3, 1e-2])
def test_config2_shear_wave_decay_rates(a, nu):
    """Config 2 at full size (2048 x 1024, periodic, lambda = 256 dx, u0 = 0.02,
    10,000 steps, FP32): the x- and the y-varying shear wave decay at the
    closed-form rate nu k^2 (within 1 % at nu = 1e-2, 3 % at nu = 1e-3) and
    at rates equal to each other (the isotropy the corrections restore)."""
    cs2 = W.stable_cs2(a)
    rates = {}
    for direction in ("y", "x"):
        wl = W.shear_wave(2048, 1024, a, cs2, nu, direction, u0=0.02, seed=3, wavelength=256)
        g = lattice(wl, 32)
        k = wl.info["k"]
        x, y = W.coords(wl.nx, wl.ny, a)
        ph = (k * y if direction == "y" else k * x) + wl.info["phase"]
        ts, amps = [], []
        for n in range(0, 10001, 2000):
            if n:
                g.step(2000)
            _, u, v = g.moments()
            amps.append(_amplitude(u if direction == "y" else v, ph))
            ts.append(n)
        rate = -np.polyfit(ts, np.log(amps), 1)[0]
        rates[direction] = rate
        tol = 0.01 if nu >= 1e-2 else 0.03
        assert abs(rate / (nu * k * k) - 1.0) < tol, (direction, rate, nu * k * k)
        g.close()
    assert abs(rates["x"] / rates["y"] - 1.0) < (0.005 if nu >= 1e-2 else 0.015), rates


def test_config2_fp32_tracks_fp64_over_10000_steps():
    """Config 2: a Taylor-Green field at a = 0.5, nu = 1e-2 over 10,000 steps;
    the FP32 deviation storage stays within 1e-5 (relative L2 on u) of the
    FP64 run, which is itself parity-tested against the FP64 oracle."""
    wl = W.taylor_green(2048, 1024, 0.5, W.stable_cs2(0.5), 1e-2, u0=0.02, seed=4,
                        wavelength=256)
    g32, g64 = lattice(wl, 32), lattice(wl, 64)
    g32.step(10000)
    g64.step(10000)
    _, u32, v32 = g32.moments()
    _, u64, v64 = g64.moments()
    err = float(np.sqrt(((u32 - u64) ** 2 + (v32 - v64) ** 2).sum() / (u64 ** 2 + v64 ** 2).sum()))
    assert err <= 1e-5, err


def test_lid_speed_sweep_small():
    """A reduced lid-speed sweep (Sec. 6, Fig. 17) through the batch: at
    tau = 0.8 on the square lattice both schemes stay stable at the low lid
    speeds for 5,000 steps, and a repeat gives the same thresholds."""
    from paper_2103_02119_gb300 import stability as S
    kw = dict(a_values=(1.0,), taus=(0.8,), u_values=[0.02, 0.04, 0.06], steps=5000, check=1000)
    t1 = S.lid_velocity_thresholds(**kw)
    assert t1 == S.lid_velocity_thresholds(**kw)
    assert t1[(1.0, 0.8, 0)] == 0.06 and t1[(1.0, 0.8, 1)] == 0.06
