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


# ---- RNR-LBM (Sec. 3): raw equilibria (Eq. 12) and raw sources (Eq. 13) ----
#
# The raw-moment scheme's source and equilibrium moments must be the raw
# moments of the central-moment quantities of Sec. 4 seen from the lab frame.
# A source with central moments (0, Fx, Fy, 0, ..., 0) about u has, for each
# basis polynomial P of Eq. 3, the raw moment sum_i S_i P(e_i) =
# F . grad P(u) (Taylor-expand P(e_i) = P(u + c_i) in c_i = e_i - u: every
# term is a central basis monomial and only the first-order ones carry a
# source).  The raw equilibrium is the raw moment of the product-form f^eq.
# Both are evaluated here in exact rational arithmetic, independently of the
# oracle's typed formulas.

def _P(k, x, y):
    return [1, x, y, x * x + y * y, x * x - y * y, x * y, x * x * y, x * y * y,
            x * x * y * y][k]


def _gradP(k, x, y):
    return [(0, 0), (1, 0), (0, 1), (2 * x, 2 * y), (2 * x, -2 * y), (y, x),
            (2 * x * y, x * x), (y * y, 2 * x * y), (2 * x * y * y, 2 * x * x * y)][k]


def _exact_feq(a, cs2, rho, ux, uy):
    def px(e, u):
        return 1 - cs2 - u * u if e == 0 else (cs2 + u * u + e * u) / 2
    def py(e, u):
        return 1 - (cs2 + u * u) / (a * a) if e == 0 else (cs2 + u * u + e * a * u) / (2 * a * a)
    return [rho * px(int(EX[i]), ux) * py(int(EY[i]), uy) for i in range(9)]


def _rnr_case(seed):
    from fractions import Fraction as Q
    rng = np.random.default_rng(100 + seed)
    a = Q(int(rng.integers(2, 9)), 4)                       # 0.5 .. 2
    cs2 = min(a * a, Q(1)) * Q(int(rng.integers(1, 6)), 10)  # below min(1, a^2)
    f = [Q(int(v), 1000) for v in rng.integers(20, 300, 9)]
    Fx, Fy = (Q(int(v), 20000) for v in rng.integers(-200, 201, 2))
    rho = sum(f)
    jx = sum(fi * int(EX[i]) for i, fi in enumerate(f))
    jy = sum(fi * int(EY[i]) * a for i, fi in enumerate(f))
    ux, uy = (jx + Fx / 2) / rho, (jy + Fy / 2) / rho
    return a, cs2, f, Fx, Fy, rho, ux, uy


def _raw_after(orc, a, cs2, f, Fx, Fy, om):
    p = params(orc, float(a), float(cs2), om, float(Fx), float(Fy), iso=0, gi=0, scheme="rnr")
    ft, _ = orc.collide_cell(p, np.array([float(v) for v in f]))
    return [sum(ft[i] * float(_P(k, EX[i], EY[i] * float(a))) for i in range(9))
            for k in range(9)]


@pytest.mark.parametrize("seed", range(8))
def test_rnr_source_moments_are_the_lab_frame_central_source(orc, seed):
    """omega_5..8 = 0 leaves m~_k = m_k + Phi_k: Phi_5..8 of Eq. 13 against
    F . grad P(u); omega_3 = omega_4 = 1 (corrections off) leaves
    m~_k = m^eq_k + Phi_k / 2: Phi_3, Phi_4."""
    a, cs2, f, Fx, Fy, rho, ux, uy = _rnr_case(seed)
    om = [1, 1, 1, 1, 1, 0, 0, 0, 0]
    got = _raw_after(orc, a, cs2, f, Fx, Fy, om)
    feq = _exact_feq(a, cs2, rho, ux, uy)
    for k in range(3, 9):
        gx, gy = _gradP(k, ux, uy)
        phi = Fx * gx + Fy * gy
        m = sum(fi * _P(k, int(EX[i]), int(EY[i]) * a) for i, fi in enumerate(f))
        meq = sum(v * _P(k, int(EX[i]), int(EY[i]) * a) for i, v in enumerate(feq))
        want = m + phi if k >= 5 else meq + phi / 2
        assert abs(got[k] - float(want)) <= 1e-13 * max(1.0, abs(float(want))), (k, got[k], want)
        # the source term is far above the tolerance: a wrong coefficient shows
        assert abs(float(phi)) > 1e-7 or k == 5


@pytest.mark.parametrize("seed", range(8))
def test_rnr_raw_equilibria_are_the_product_form_moments(orc, seed):
    """Every omega = 1 (corrections off): m~_k = m^eq_k + Phi_k / 2 for every
    k, with m^eq_k the raw moments of the product-form equilibrium (Eq. 12
    with the reading of its last entry) and Phi_k = F . grad P_k(u)."""
    a, cs2, f, Fx, Fy, rho, ux, uy = _rnr_case(seed)
    got = _raw_after(orc, a, cs2, f, Fx, Fy, [1.0] * 9)
    feq = _exact_feq(a, cs2, rho, ux, uy)
    for k in range(9):
        gx, gy = _gradP(k, ux, uy)
        meq = sum(v * _P(k, int(EX[i]), int(EY[i]) * a) for i, v in enumerate(feq))
        want = meq + (Fx * gx + Fy * gy) / 2
        assert abs(got[k] - float(want)) <= 1e-13 * max(1.0, abs(float(want))), (k, got[k], want)
