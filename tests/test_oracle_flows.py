"""Physics pins of the oracle on whole flows (no GPU):

- body-force Poiseuille channel (Sec. 5.1): parabolic profile, second-order
  convergence of the global relative error the paper defines;
- viscous decay of shear waves and Taylor-Green vortices at the rate
  nu |k|^2 (Eq. 30-32), the same for every orientation at a != 1, with a
  negative control that switches the isotropy correction (Eq. 23-24) off;
- Galilean invariance of the decay rate under a uniform boost, with a
  negative control that switches the GI correction (Eq. 25-26) off;
- transient Couette flow against its Fourier series (Sec. 5.2), which pins
  the moving-wall bounce-back of Eq. 57-59;
- global mass conservation to rounding.
"""
import math

import numpy as np
import pytest

from paper_2103_02119_gb300 import workloads as W


def make(orc, wl, **kw):
    p = orc.OracleParams.make(wl.nx, wl.ny, wl.a, wl.cs2, wl.omega, Fx=wl.Fx,
                              Fy=wl.Fy, periodic_x=wl.periodic_x,
                              periodic_y=wl.periodic_y, wall_u=wl.wall_u,
                              use_iso_corr=kw.pop("iso", wl.use_iso_corr),
                              use_gi_corr=kw.pop("gi", wl.use_gi_corr), **kw)
    o = orc.Oracle(p, wl.mask)
    o.init_fields(wl.rho, wl.ux, wl.uy)
    return o


def poiseuille_error(orc, ny, steps, scheme="rc"):
    wl = W.poiseuille(ny=ny)
    o = make(orc, wl, scheme=scheme)
    o.step(steps)
    rho, ux, uy = o.moments()
    H, U = wl.info["H"], wl.info["U"]
    y = (np.arange(ny) + 0.5) * wl.a
    ua = (U * (1 - (y - H / 2) ** 2 / (H / 2) ** 2))[:, None] * np.ones((1, wl.nx))
    # Sec. 5.1: sum ||u_c - u_a|| / sum ||u_a|| over the domain
    err = np.sqrt((ux - ua) ** 2 + uy ** 2).sum() / np.abs(ua).sum()
    return err, rho, uy


@pytest.mark.parametrize("scheme", ["rc", "rnr"])
def test_poiseuille_config1(orc, scheme):
    """32 x 32, a = 0.5, nu = 0.1, u_max = 0.01, 5000 steps from rest."""
    err, rho, uy = poiseuille_error(orc, 32, 5000, scheme)
    assert err < 3e-3
    assert np.abs(uy).max() < 1e-14
    assert abs(math.fsum(rho.ravel()) / rho.size - 1.0) < 1e-13


def test_poiseuille_second_order(orc):
    e16, _, _ = poiseuille_error(orc, 16, 3000)
    e32, _, _ = poiseuille_error(orc, 32, 5000)
    assert 3.5 < e16 / e32 < 4.5


def decay_rate(orc, wl, steps, every, **kw):
    """Fit of log amplitude of the initial velocity pattern (advected with
    the background velocity) against time; returned relative to nu |k|^2 of
    the pattern (TGV: 2 nu k^2)."""
    o = make(orc, wl, **kw)
    info = wl.info
    bg = info.get("background", (0.0, 0.0))
    ux0, uy0 = wl.ux - bg[0], wl.uy - bg[1]
    x, y = W.coords(wl.nx, wl.ny, wl.a)
    k = info["k"]
    ts, amps = [], []
    for n in range(0, steps + 1, every):
        if n:
            o.step(every)
        _, u, v = o.moments()
        if bg != (0.0, 0.0):
            p1, p2 = info["phases"]
            xs, ys = x - bg[0] * n, y - bg[1] * n
            px = np.sin(k * xs + p1) * np.cos(k * ys + p2)
            py = -np.cos(k * xs + p1) * np.sin(k * ys + p2)
        else:
            px, py = ux0, uy0
        amps.append(((u - bg[0]) * px + (v - bg[1]) * py).sum() / (px * px + py * py).sum())
        ts.append(n)
    slope = np.polyfit(ts[1:], np.log(np.abs(amps[1:])), 1)[0]
    mult = 2.0 if (wl.name.startswith("tgv") or info.get("direction") == "diag") else 1.0
    return -slope / (mult * info["nu"] * k * k)


@pytest.mark.parametrize("a", [0.5, 0.25])
@pytest.mark.parametrize("direction", ["x", "y"])
def test_axis_shear_waves_decay_at_nu_k2(orc, a, direction):
    cs2 = W.stable_cs2(a)
    wl = W.shear_wave(32, int(round(32 / a)), a, cs2, 0.01, direction, u0=0.01, seed=3)
    r = decay_rate(orc, wl, 1000, 100)
    assert abs(r - 1) < 0.01


@pytest.mark.parametrize("a", [0.5, 0.25])
@pytest.mark.parametrize("kind", ["tgv", "diag"])
def test_isotropic_decay_and_negative_control(orc, a, kind):
    """Flows with normal strain (d_x u_x != 0) decay at nu |k|^2 only when the
    isotropy correction is on."""
    cs2 = W.stable_cs2(a)
    ny = int(round(32 / a))
    if kind == "tgv":
        wl = W.taylor_green(32, ny, a, cs2, 0.01, u0=0.01, seed=2)
    else:
        wl = W.shear_wave(32, ny, a, cs2, 0.01, "diag", u0=0.01, seed=2)
    assert abs(decay_rate(orc, wl, 1000, 100) - 1) < 0.02
    assert abs(decay_rate(orc, wl, 1000, 100, iso=0) - 1) > 0.2


@pytest.mark.parametrize("a,boost,gi_off_min", [(0.5, (0.05, 0.0), 0.01),
                                                (0.25, (0.0, 0.05), 0.05)])
def test_decay_rate_galilean_invariant(orc, a, boost, gi_off_min):
    cs2 = W.stable_cs2(a)
    ny = int(round(32 / a))
    rest = W.taylor_green(32, ny, a, cs2, 0.01, u0=0.005, seed=4)
    moving = W.taylor_green(32, ny, a, cs2, 0.01, u0=0.005, seed=4, background=boost)
    r0 = decay_rate(orc, rest, 2000, 200)
    r1 = decay_rate(orc, moving, 2000, 200)
    r1_off = decay_rate(orc, moving, 2000, 200, gi=0)
    assert abs(r1 / r0 - 1) < 0.008
    assert abs(r1_off / r0 - 1) > gi_off_min


@pytest.mark.parametrize("a,cs2,ny", [(0.25, 0.04, 40), (0.1, 0.005, 100)])
def test_transient_couette_series(orc, a, cs2, ny):
    wl = W.couette(ny=ny, a=a, cs2=cs2, tau=0.8, U=0.02)
    o = make(orc, wl)
    nu, U, H = wl.info["nu"], wl.info["U"], wl.info["H"]
    y = (np.arange(ny) + 0.5) * a
    n_terms = np.arange(1, 201)[:, None]
    t = 0
    for T in (0.02, 0.05, 0.1, 0.2):
        n = int(round(T * H * H / nu))
        o.step(n - t)
        t = n
        _, u, v = o.moments()
        series = U * y / H - (2 * U / np.pi) * (
            np.exp(-n_terms ** 2 * np.pi ** 2 * nu * t / H ** 2) / n_terms
            * np.sin(n_terms * np.pi * (1 - y / H))).sum(0)
        assert np.abs(u.mean(axis=1) - series).max() < 1e-3 * U
        assert np.abs(u - u.mean(axis=1, keepdims=True)).max() < 1e-15


def test_global_mass_conserved_to_rounding(orc):
    wl = W.taylor_green(24, 48, 0.5, W.stable_cs2(0.5), 0.02, u0=0.02, seed=5)
    wl = wl.with_(mask=W.random_obstacles(24, 48, seed=1, coverage=0.08),
                  periodic_y=0, wall_u=((0, 0), (0, 0), (0, 0), (0.01, 0)))
    o = make(orc, wl)
    m0 = math.fsum(o.get_f().ravel())
    o.step(300)
    m1 = math.fsum(o.get_f().ravel())
    # each of 300 steps may move the total by a few ulp per cell
    assert abs(m1 - m0) <= 300 * wl.cells * 4 * 2.2e-16


def test_solid_rows_equal_implicit_walls(orc):
    """A channel closed by rows of solid nodes (periodic y) is the same
    lattice as one closed by the implicit half-way walls."""
    wl = W.poiseuille(ny=16, nx=8)
    o = make(orc, wl)
    o.step(400)
    walled = o.moments()
    mask = np.zeros((18, 8), np.uint8)
    mask[0] = mask[17] = 1
    wl2 = wl.with_(ny=18, periodic_y=1, mask=mask)
    o2 = make(orc, wl2)
    o2.step(400)
    masked = [m[1:17] for m in o2.moments()]
    for w_, m_ in zip(walled, masked):
        np.testing.assert_allclose(m_, w_, rtol=0, atol=1e-15)


def sound_damping(orc, a, cs2, nu, ny, Uy, steps=600, every=20, delta=1e-3):
    """Damping rate of a travelling sound wave along y (4 x ny periodic box,
    background velocity (0, Uy)), relative to the closed form (nu + zeta) k^2
    / 2 of the Navier-Stokes equations of Eq. 29-33 (zeta = cs2 (1/w3 - 1/2))."""
    omega = W.omega_for(nu, cs2)
    p = orc.OracleParams.make(4, ny, a, cs2, omega)
    o = orc.Oracle(p)
    _, y = W.coords(4, ny, a)
    k = 2 * np.pi / (ny * a)
    rho = 1 + delta * np.cos(k * y)
    o.init_fields(rho, 0 * y, Uy + np.sqrt(cs2) * delta * np.cos(k * y))
    ts, amps = [], []
    for n in range(0, steps + 1, every):
        if n:
            o.step(every)
        r, _, _ = o.moments()
        prof = r.mean(axis=1) - 1
        amps.append(2 * np.abs(np.fft.fft(prof)[1]) / ny)
        ts.append(n)
    slope = np.polyfit(ts[2:], np.log(amps[2:]), 1)[0]
    zeta = cs2 * (1 / omega[3] - 0.5)
    return -slope / ((nu + zeta) * k * k / 2)


@pytest.mark.parametrize("a,tol", [(0.5, 0.002), (0.25, 0.006)])
def test_boosted_sound_wave_damping(orc, a, tol):
    """The u.grad(rho) terms of Eq. 19-20 (carried by B3/B4, C3/C4 of Eq. 40
    and by Eq. 23-24) act at first order only where a velocity meets a
    density gradient.  A sound wave in a moving fluid exercises them: its
    damping must match the closed form and not depend on the sign of the
    boost along the wave."""
    cs2 = W.stable_cs2(a)
    r0 = sound_damping(orc, a, cs2, 0.02, 64, 0.0)
    rp = sound_damping(orc, a, cs2, 0.02, 64, 0.02)
    rm = sound_damping(orc, a, cs2, 0.02, 64, -0.02)
    assert abs(r0 - 1) < 0.01
    assert abs(rp - rm) / r0 < tol


def _staggered(o, n):
    r, u, v = o.moments()
    fl = o.solid() == 0
    yy, xx = np.mgrid[0:u.shape[0], 0:u.shape[1]]
    s = (-1.0) ** n
    return (s * ((-1.0) ** xx * r * u * fl).sum(), s * ((-1.0) ** yy * r * v * fl).sum(),
            (np.abs(r * u) + np.abs(r * v))[fl].sum())


@pytest.mark.parametrize("walls", [0, 1])
def test_staggered_momenta_are_exact_invariants(orc, walls):
    """Besides the mass, the scheme keeps two staggered momenta exactly:
    G_x = sum (-1)^(x+n) rho u_x and G_y = sum (-1)^(y+n) rho u_y over the
    fluid cells (even nx, ny).  Streaming moves the populations that carry
    them one cell (or bounces them back, half-way) and flips the sign of the
    weight; the collision conserves momentum.  Checked on a periodic box and
    on a closed box with obstacles (stationary walls), from a noisy start."""
    n = 32
    wl = W.cavity(n, 24, 0.7, W.stable_cs2(0.7), 0.0, 50.0)
    mask = W.random_obstacles(n, 24, seed=7) if walls else None
    p = orc.OracleParams.make(n, 24, wl.a, wl.cs2, wl.omega, periodic_x=1 - walls,
                              periodic_y=1 - walls, nthreads=1)
    o = orc.Oracle(p, mask)
    r0, u0, v0 = W.smooth_random_fields(n, 24, seed=3, u_amp=0.03)
    rng = np.random.default_rng(1)
    o.init_fields(r0, u0 + 0.01 * rng.standard_normal(u0.shape),
                  v0 + 0.01 * rng.standard_normal(v0.shape))
    gx0, gy0, scale = _staggered(o, 0)
    assert abs(gx0) > 1e-3 * scale and abs(gy0) > 1e-3 * scale
    done = 0
    for step in (1, 2, 10, 300):
        o.step(step - done)
        done = step
        gx, gy, _ = _staggered(o, step)
        assert abs(gx - gx0) <= 1e-12 * scale and abs(gy - gy0) <= 1e-12 * scale, (step, gx, gy)


def test_longitudinal_nyquist_velocity_never_decays(orc):
    """The carrier of G_y: u_y = A (-1)^y, uniform along x, is an equilibrium
    state that streaming maps to minus itself, so it alternates forever; the
    transverse (shear) pattern u_x = A (-1)^y decays at once.  This is why
    the steady residual is taken on two-step means."""
    n, a = 32, 0.5
    cs2 = W.stable_cs2(a)
    yy, xx = np.mgrid[0:n, 0:n]
    amp = {}
    for name, (u0, v0) in {"long": (0 * yy, 0.01 * (-1.0) ** yy),
                           "shear": (0.01 * (-1.0) ** yy, 0 * yy)}.items():
        p = orc.OracleParams.make(n, n, a, cs2, W.omega_for(0.01, cs2), nthreads=1)
        o = orc.Oracle(p)
        o.init_fields(np.ones((n, n)), u0.astype(float), v0.astype(float))
        o.step(101)
        _, u, v = o.moments()
        amp[name] = (u, v)
    u, v = amp["long"]
    np.testing.assert_allclose(v, -0.01 * (-1.0) ** yy, rtol=0, atol=1e-12)
    assert np.abs(u).max() < 1e-12
    u, v = amp["shear"]
    assert max(np.abs(u).max(), np.abs(v).max()) < 1e-12
