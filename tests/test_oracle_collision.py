"""Pins of the oracle's collision against what the paper and the mathematics
fix: conservation (Sec. 4), the Maxwell-matched equilibrium in closed form,
the equilibrium fixed point, the reduction to BGK on the square lattice
(Sec. 2.2, last paragraph), the textbook second-order D2Q9 equilibrium, and
second-order convergence of the local strain rates of Eq. 37-40 to the true
velocity gradient.  No GPU.
"""
import math

import numpy as np
import pytest

from paper_2103_02119_gb300 import workloads as W

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)


def product_feq(a, cs2, rho, ux, uy):
    """Closed form: the tensor product of 1-D three-velocity distributions
    matching the Maxwellian's 0th-2nd moments (temperature cs2 along both
    axes; the y lattice spacing is a)."""
    def px(e, u):
        return 1 - cs2 - u * u if e == 0 else (cs2 + u * u + e * u) / 2
    def py(e, u):
        return 1 - (cs2 + u * u) / a ** 2 if e == 0 else (cs2 + u * u + e * a * u) / (2 * a * a)
    return np.array([rho * px(EX[i], ux) * py(EY[i], uy) for i in range(9)])


def params(orc, a, cs2, omega, Fx=0.0, Fy=0.0, iso=1, gi=1, scheme="rc"):
    return orc.OracleParams.make(8, 8, a, cs2, omega, Fx=Fx, Fy=Fy,
                                 use_iso_corr=iso, use_gi_corr=gi, scheme=scheme)


@pytest.mark.parametrize("a", [0.1, 0.25, 0.5, 1.0, 2.0])
@pytest.mark.parametrize("u", [(0.0, 0.0), (0.05, -0.03), (-0.12, 0.2)])
def test_equilibrium_is_product_form(orc, a, u):
    cs2 = min(1 / 3, 0.5 * a * a)
    rho = 1.07
    np.testing.assert_allclose(orc.feq(a, cs2, rho, *u),
                               product_feq(a, cs2, rho, *u), rtol=0, atol=1e-14)


def test_rest_weights_square_lattice(orc):
    w = orc.feq(1.0, 1 / 3, 1.0, 0.0, 0.0)
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, atol=1e-15)


@pytest.mark.parametrize("scheme", ["rc", "rnr"])
@pytest.mark.parametrize("seed", range(20))
def test_collision_conserves_mass_and_adds_force(orc, scheme, seed):
    rng = np.random.default_rng(seed)
    a = float(rng.choice([0.1, 0.25, 0.5, 0.8, 1.0, 2.0]))
    cs2 = min(1 / 3, 0.6 * a * a) * rng.uniform(0.5, 1.0)
    om = rng.uniform(0.3, 1.95, 9)
    Fx, Fy = rng.normal(0, 1e-3, 2)
    p = params(orc, a, cs2, om, Fx, Fy, *rng.integers(0, 2, 2), scheme=scheme)
    f = product_feq(a, cs2, rng.uniform(0.9, 1.1), *rng.normal(0, 0.05, 2))
    f = f * (1 + 0.05 * rng.standard_normal(9))
    ft, _ = orc.collide_cell(p, f, *rng.normal(0, 1e-2, 2))
    ey = a * EY
    assert abs(ft.sum() - f.sum()) <= 1e-14 * 9
    assert abs(ft @ EX - f @ EX - Fx) <= 1e-14 * 9
    assert abs(ft @ ey - f @ ey - Fy) <= 1e-14 * 9 * max(1, a)


@pytest.mark.parametrize("scheme", ["rc", "rnr"])
@pytest.mark.parametrize("a", [0.25, 0.5, 1.0, 2.0])
def test_equilibrium_is_a_fixed_point(orc, scheme, a):
    cs2 = min(1 / 3, 0.3 * a * a)
    om = [1, 1, 1, 0.9, 1.3, 1.3, 1, 1, 1]
    p = params(orc, a, cs2, om, scheme=scheme)
    f = product_feq(a, cs2, 1.03, 0.04, -0.02)
    ft, (sx, sy) = orc.collide_cell(p, f, 0.0, 0.0)
    np.testing.assert_allclose(ft, f, rtol=0, atol=1e-15)
    assert abs(sx) < 1e-14 and abs(sy) < 1e-14


@pytest.mark.parametrize("seed", range(10))
def test_isotropy_correction_vanishes_on_square_lattice(orc, seed):
    """Sec. 2.2: at a = 1, cs2 = 1/3 the corrections of Eq. 23-24 vanish."""
    rng = np.random.default_rng(seed)
    om = rng.uniform(0.5, 1.9, 9)
    f = product_feq(1.0, 1 / 3, 1.0, *rng.normal(0, 0.05, 2)) * (1 + 0.05 * rng.standard_normal(9))
    d = rng.normal(0, 1e-2, 2)
    on, _ = orc.collide_cell(params(orc, 1.0, 1 / 3, om, iso=1), f, *d)
    off, _ = orc.collide_cell(params(orc, 1.0, 1 / 3, om, iso=0), f, *d)
    np.testing.assert_allclose(on, off, rtol=0, atol=1e-15)
    # and they do not vanish on a rectangular lattice
    on, _ = orc.collide_cell(params(orc, 0.5, 0.075, om, iso=1), f, *d)
    off, _ = orc.collide_cell(params(orc, 0.5, 0.075, om, iso=0), f, *d)
    assert np.abs(on - off).max() > 1e-6


@pytest.mark.parametrize("seed", range(10))
def test_square_lattice_single_rate_is_bgk(orc, seed):
    """a = 1, cs2 = 1/3, one rate for every moment, no GI term, no force:
    relaxing all central moments at one rate is BGK towards f^eq."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.3, 1.9)
    f = product_feq(1.0, 1 / 3, rng.uniform(0.9, 1.1), *rng.normal(0, 0.05, 2))
    f = f * (1 + 0.1 * rng.standard_normal(9))
    ft, _ = orc.collide_cell(params(orc, 1.0, 1 / 3, [w] * 9, gi=0), f,
                             *rng.normal(0, 1e-2, 2))
    rho = f.sum()
    u = (f @ EX / rho, f @ EY / rho)
    np.testing.assert_allclose(ft, f + w * (product_feq(1.0, 1 / 3, rho, *u) - f),
                               rtol=0, atol=1e-14)


def test_square_lattice_equilibrium_matches_textbook_to_second_order(orc):
    """f^eq at a = 1 agrees with the textbook D2Q9 equilibrium
    w_i rho (1 + 3 e.u + 9/2 (e.u)^2 - 3/2 u^2) up to terms of third order."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    errs = []
    for s in (0.04, 0.02, 0.01):
        ux, uy = 1.3 * s, -0.7 * s
        eu = EX * ux + EY * uy
        text = w * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * (ux * ux + uy * uy))
        errs.append(np.abs(orc.feq(1.0, 1 / 3, 1.0, ux, uy) - text).max())
    assert errs[0] < 1e-4
    assert errs[0] / errs[1] > 7.5 and errs[1] / errs[2] > 7.5  # O(u^3)


@pytest.mark.parametrize("a", [0.5, 0.25])
def test_local_strain_rates_converge_to_velocity_gradient(orc, a):
    """Eq. 37-40 recover d_x u_x and d_y u_y from the non-equilibrium moments;
    against the spectral derivative of the velocity field of a Taylor-Green
    flow, the error falls at second order with the resolution."""
    cs2 = W.stable_cs2(a)
    errs = []
    for nx in (16, 32, 64):
        wl = W.taylor_green(nx, int(round(nx / a)), a, cs2, nu=0.05, u0=0.01, seed=1)
        o = orc.Oracle(orc.OracleParams.make(wl.nx, wl.ny, a, cs2, wl.omega))
        o.init_fields(wl.rho, wl.ux, wl.uy)
        o.step(int(50 * (nx / 16) ** 2 / 4) + 10)
        r, u, v = o.moments()
        sx, sy = o.strain()
        kx = 2 * np.pi * np.fft.fftfreq(wl.nx, 1.0)
        ky = 2 * np.pi * np.fft.fftfreq(wl.ny, a)
        dudx = np.real(np.fft.ifft2(1j * kx[None, :] * np.fft.fft2(u)))
        dvdy = np.real(np.fft.ifft2(1j * ky[:, None] * np.fft.fft2(v)))
        errs.append((np.abs(sx - dudx).max() / np.abs(dudx).max(),
                     np.abs(sy - dvdy).max() / np.abs(dvdy).max()))
    for c in range(2):
        assert errs[1][c] / errs[2][c] > 3.0, errs
        assert errs[2][c] < 0.02, errs


@pytest.mark.parametrize("a,direction", [(0.5, "x"), (0.25, "x"), (0.5, "y"), (0.25, "y")])
def test_off_diagonal_strain_converges_to_velocity_gradient(orc, a, direction):
    """Eq. 39 (left side read as d_y u_x + d_x u_y, the rate that Eq. 21 ties
    to m5) against the spectral derivatives of the velocity of a decaying
    shear wave: second-order convergence; the stress output is the
    Newtonian stress of Eq. 30-33 built from the three local rates."""
    cs2 = W.stable_cs2(a)
    errs = []
    for nx in (16, 32, 64):
        wl = W.shear_wave(nx, int(round(nx / a)), a, cs2, nu=0.05, direction=direction,
                          u0=0.01, seed=2)
        o = orc.Oracle(orc.OracleParams.make(wl.nx, wl.ny, a, cs2, wl.omega))
        o.init_fields(wl.rho, wl.ux, wl.uy)
        o.step(int(50 * (nx / 16) ** 2 / 4) + 10)
        r, u, v = o.moments()
        sxy, txx, tyy, txy = o.stress()
        kx = 2 * np.pi * np.fft.fftfreq(wl.nx, 1.0)
        ky = 2 * np.pi * np.fft.fftfreq(wl.ny, a)
        dudy = np.real(np.fft.ifft2(1j * ky[:, None] * np.fft.fft2(u)))
        dvdx = np.real(np.fft.ifft2(1j * kx[None, :] * np.fft.fft2(v)))
        ref = dudy + dvdx
        errs.append(np.abs(sxy - ref).max() / np.abs(ref).max())
        # stress from the rates: nu = cs2 (1/omega - 1/2) (Eq. 32-33)
        nu = cs2 * (1 / wl.omega[4] - 0.5)
        zeta = cs2 * (1 / wl.omega[3] - 0.5)
        sx, sy = o.strain()
        div = sx + sy
        assert np.allclose(txy, r * nu * sxy, rtol=1e-13, atol=0)
        assert np.allclose(txx, r * (nu * (2 * sx - div) + zeta * div), rtol=1e-12, atol=1e-18)
        assert np.allclose(tyy, r * (nu * (2 * sy - div) + zeta * div), rtol=1e-12, atol=1e-18)
    assert errs[1] / errs[2] > 3.0, errs
    assert errs[2] < 0.02, errs


def test_shear_stress_of_steady_channels_is_linear(orc):
    """Steady body-force channel (Sec. 5.1): the local shear stress is the
    exact linear profile tau_xy = -F (y - H/2) (momentum balance), and the
    normal stresses vanish."""
    for a in (0.5, 0.25):
        wl = W.poiseuille(ny=24, nx=4, a=a, cs2=W.stable_cs2(a), nu=0.1, U=0.01)
        o = orc.Oracle(orc.OracleParams.make(wl.nx, wl.ny, a, wl.cs2, wl.omega, Fx=wl.Fx,
                                             periodic_x=1, periodic_y=0))
        o.step(int(6 * (wl.ny * a) ** 2 / 0.1))
        sxy, txx, tyy, txy = o.stress()
        H = wl.ny * a
        y = (np.arange(wl.ny) + 0.5) * a
        exact = -wl.Fx * (y - H / 2)
        prof = txy[:, 0]
        assert np.abs(prof - exact).max() < 0.02 * np.abs(exact).max(), (a, prof, exact)
        assert np.abs(txx).max() < 1e-2 * np.abs(exact).max()
        assert np.abs(tyy).max() < 1e-2 * np.abs(exact).max()
