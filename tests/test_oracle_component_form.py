"""The oracle's matrix-form collision (T, F(u), their inverses) against the
same collision written out component by component from the paper's
definitions, on random cells: the two are different routes to the same
numbers, so they must agree to rounding (1e-14).  No GPU.

The component form (Sec. 4, the RC-LBE and its algorithm):
- rho = sum f_i, rho u = sum f_i e_i + F/2 (Eq. 2 velocities, e_y in units
  of a);
- central moments eta^c_{x^m y^n} = sum f_i (e_ix - u_x)^m (e_iy - u_y)^n
  (Eq. 43), assembled into the basis of Eq. 46 (xx + yy and xx - yy);
- the second-order non-equilibrium raw moments of Eq. 34-35 (raw sums minus
  Eq. 12's m3, m4), the coefficients of Eq. 40, the strain rates of
  Eq. 37-38, the corrections of Eq. 23-26 (Delta t = 1), the equilibria of
  Eq. 49 and the central source (0, Fx, Fy, 0, ...);
- relaxation m~c_j = m_j + w_j (m_j^eq - m_j) + (1 - w_j/2) Phi_j;
- back to populations: the nine central moments of a 3 x 3 stencil fix its
  values, one axis at a time: along an axis with nodes (-c, 0, c) and
  central moments M0, M1, M2 about u, the raw moments are R0 = M0,
  R1 = M1 + u M0, R2 = M2 + 2 u M1 + u^2 M0, and the node values are
  R0 - R2 / c^2 at 0 and (R2 / c^2 +- R1 / c) / 2 at +-c.
The raw-moment scheme (Sec. 3) gets the same treatment below.  None of this
uses the oracle's matrices.
"""
import numpy as np
import pytest

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)


def invert_axis(M0, M1, M2, u, c):
    """Node values at (-c, 0, c) from central moments about u."""
    R0, R1, R2 = M0, M1 + u * M0, M2 + 2 * u * M1 + u * u * M0
    return ((R2 / c ** 2 - R1 / c) / 2, R0 - R2 / c ** 2, (R2 / c ** 2 + R1 / c) / 2)


def collide_component_form(f, a, cs2, w, Fx, Fy, dxr, dyr, iso=1, gi=1):
    ex, ey = EX, EY * a
    rho = f.sum()
    ux = ((f * ex).sum() + Fx / 2) / rho
    uy = ((f * ey).sum() + Fy / 2) / rho

    def eta(m, n):
        return (f * (ex - ux) ** m * (ey - uy) ** n).sum()

    k = {(m, n): eta(m, n) for m in range(3) for n in range(3)}
    mc = [k[0, 0], k[1, 0], k[0, 1], k[2, 0] + k[0, 2], k[2, 0] - k[0, 2], k[1, 1],
          k[2, 1], k[1, 2], k[2, 2]]

    # Eq. 34-35: raw second moments minus Eq. 12's equilibria
    N3 = (f * (ex ** 2 + ey ** 2)).sum() - (2 * rho * cs2 + rho * (ux ** 2 + uy ** 2))
    N4 = (f * (ex ** 2 - ey ** 2)).sum() - rho * (ux ** 2 - uy ** 2)
    # Eq. 40
    B1 = rho * (-2 * cs2 / w[3] - (-3 * cs2 + 1) / 2 + 3 * ux ** 2 / 2)
    B2 = rho * (-2 * cs2 / w[3] - (-3 * cs2 + a * a) / 2 + 3 * uy ** 2 / 2)
    C1 = rho * (-2 * cs2 / w[4] - (-3 * cs2 + 1) / 2 + 3 * ux ** 2 / 2)
    C2 = rho * (2 * cs2 / w[4] - (3 * cs2 - a * a) / 2 - 3 * uy ** 2 / 2)
    B3 = (3 * cs2 - 1) / 2 * ux
    B4 = (3 * cs2 - a * a) / 2 * uy
    C3 = (3 * cs2 - 1) / 2 * ux
    C4 = (-3 * cs2 + a * a) / 2 * uy
    R3 = N3 - B3 * dxr - B4 * dyr
    R4 = N4 - C3 * dxr - C4 * dyr
    # Eq. 37-38
    dxux = (C2 * R3 - B2 * R4) / (C2 * B1 - C1 * B2)
    dyuy = (C1 * R3 - B1 * R4) / (C1 * B2 - C2 * B1)
    # Eq. 23-26
    t3, t4 = 1 / w[3] - 0.5, 1 / w[4] - 0.5
    m3s = t3 * ((-3 * cs2 + 1) * rho * dxux + (-3 * cs2 + a * a) * rho * dyuy
                + (-3 * cs2 + 1) * ux * dxr + (-3 * cs2 + a * a) * uy * dyr)
    m4s = t4 * ((-3 * cs2 + 1) * rho * dxux + (3 * cs2 - a * a) * rho * dyuy
                + (-3 * cs2 + 1) * ux * dxr + (3 * cs2 - a * a) * uy * dyr)
    m3G = -3 * rho * t3 * (ux ** 2 * dxux + uy ** 2 * dyuy)
    m4G = -3 * rho * t4 * (ux ** 2 * dxux - uy ** 2 * dyuy)
    # Eq. 49 and the central source
    eq = [rho, 0.0, 0.0, 2 * rho * cs2 + iso * m3s + gi * m3G, iso * m4s + gi * m4G, 0.0,
          0.0, 0.0, rho * cs2 ** 2]
    phi = [0.0, Fx, Fy, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    mt = [mc[j] + w[j] * (eq[j] - mc[j]) + (1 - w[j] / 2) * phi[j] for j in range(9)]

    # back to kappa_pq, then to the 3 x 3 stencil: along x for each q, then
    # along y for each column
    kt = {(0, 0): mt[0], (1, 0): mt[1], (0, 1): mt[2], (2, 0): (mt[3] + mt[4]) / 2,
          (0, 2): (mt[3] - mt[4]) / 2, (1, 1): mt[5], (2, 1): mt[6], (1, 2): mt[7],
          (2, 2): mt[8]}
    h = {}  # h[q][X]: column X's y-moment of order q (X = -1, 0, 1)
    for q in range(3):
        lo, mid, hi = invert_axis(kt[0, q], kt[1, q], kt[2, q], ux, 1.0)
        h[q] = {-1: lo, 0: mid, 1: hi}
    out = np.zeros(9)
    for X in (-1, 0, 1):
        lo, mid, hi = invert_axis(h[0][X], h[1][X], h[2][X], uy, a)
        for Y, v in ((-1, lo), (0, mid), (1, hi)):
            i = int(np.flatnonzero((EX == X) & (EY == Y))[0])
            out[i] = v
    return out, (dxux, dyuy)


def random_cell(rng, a, cs2):
    """A population near equilibrium with a non-equilibrium part."""
    rho = 1.0 + rng.normal(0, 0.02)
    ux, uy = rng.normal(0, 0.04, 2)
    ex, ey = EX, EY * a
    f = np.empty(9)
    for i in range(9):
        px = 1 - cs2 - ux * ux if EX[i] == 0 else (cs2 + ux * ux + EX[i] * ux) / 2
        py = (1 - (cs2 + uy * uy) / a ** 2 if EY[i] == 0
              else (cs2 + uy * uy + EY[i] * a * uy) / (2 * a * a))
        f[i] = rho * px * py
    return f * (1 + rng.normal(0, 0.05, 9))


@pytest.mark.parametrize("a,cs2", [(1.0, 1 / 3), (0.5, 0.075), (0.25, 0.01875), (2.0, 1 / 3)])
@pytest.mark.parametrize("iso,gi", [(1, 1), (0, 1), (1, 0), (0, 0)])
def test_matrix_form_equals_component_form(orc, a, cs2, iso, gi):
    rng = np.random.default_rng(int(1000 * a) + 10 * iso + gi)
    for _ in range(25):
        f = random_cell(rng, a, cs2)
        w = [1.0, 1.0, 1.0, rng.uniform(0.6, 1.9), rng.uniform(0.6, 1.9),
             rng.uniform(0.6, 1.9), rng.uniform(0.5, 1.5), rng.uniform(0.5, 1.5),
             rng.uniform(0.5, 1.5)]
        Fx, Fy = rng.normal(0, 1e-3, 2)
        dxr, dyr = rng.normal(0, 1e-2, 2)
        p = orc.OracleParams.make(8, 8, a, cs2, w, Fx=Fx, Fy=Fy, use_iso_corr=iso,
                                  use_gi_corr=gi)
        got, (sx, sy) = orc.collide_cell(p, f, dxr, dyr)
        ref, (rx, ry) = collide_component_form(f, a, cs2, w, Fx, Fy, dxr, dyr, iso, gi)
        assert np.abs(got - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max()), (got - ref)
        assert abs(sx - rx) <= 1e-12 * max(1.0, abs(rx)) and abs(sy - ry) <= 1e-12 * max(1.0, abs(ry))


def collide_raw_component_form(f, a, cs2, w, Fx, Fy, dxr, dyr, iso=1, gi=1):
    """The raw-moment scheme (RNR-LBM, Sec. 3) written out: raw moments
    m_j = sum f_i P_j(e_i) of the Eq. 3 basis, the equilibria of Eq. 12 (m8
    read as rho cs2^2 + rho cs2 |u|^2 + rho ux^2 uy^2), the corrections of
    Eq. 23-26 with the strain rates of Eq. 37-38, and the source moments
    Phi_j = F . grad P_j (u) (the raw moments of a source whose central
    moments are (0, Fx, Fy, 0, ...)); back to populations as in the central
    form, about u = 0."""
    ex, ey = EX, EY * a
    rho = f.sum()
    ux = ((f * ex).sum() + Fx / 2) / rho
    uy = ((f * ey).sum() + Fy / 2) / rho
    P = [lambda x, y: 1.0 + 0 * x, lambda x, y: x, lambda x, y: y,
         lambda x, y: x * x + y * y, lambda x, y: x * x - y * y, lambda x, y: x * y,
         lambda x, y: x * x * y, lambda x, y: x * y * y, lambda x, y: x * x * y * y]
    grad = [(0.0, 0.0), (1.0, 0.0), (0.0, 1.0), (2 * ux, 2 * uy), (2 * ux, -2 * uy), (uy, ux),
            (2 * ux * uy, ux * ux), (uy * uy, 2 * ux * uy),
            (2 * ux * uy * uy, 2 * ux * ux * uy)]
    m = [(f * Pj(ex, ey)).sum() for Pj in P]
    u2 = ux * ux + uy * uy
    meq = [rho, rho * ux, rho * uy, 2 * rho * cs2 + rho * u2, rho * (ux * ux - uy * uy),
           rho * ux * uy, cs2 * rho * uy + rho * ux * ux * uy, cs2 * rho * ux + rho * ux * uy * uy,
           rho * cs2 * cs2 + rho * cs2 * u2 + rho * ux * ux * uy * uy]
    N3, N4 = m[3] - meq[3], m[4] - meq[4]
    B1 = rho * (-2 * cs2 / w[3] - (-3 * cs2 + 1) / 2 + 3 * ux ** 2 / 2)
    B2 = rho * (-2 * cs2 / w[3] - (-3 * cs2 + a * a) / 2 + 3 * uy ** 2 / 2)
    C1 = rho * (-2 * cs2 / w[4] - (-3 * cs2 + 1) / 2 + 3 * ux ** 2 / 2)
    C2 = rho * (2 * cs2 / w[4] - (3 * cs2 - a * a) / 2 - 3 * uy ** 2 / 2)
    R3 = N3 - (3 * cs2 - 1) / 2 * ux * dxr - (3 * cs2 - a * a) / 2 * uy * dyr
    R4 = N4 - (3 * cs2 - 1) / 2 * ux * dxr - (-3 * cs2 + a * a) / 2 * uy * dyr
    dxux = (C2 * R3 - B2 * R4) / (C2 * B1 - C1 * B2)
    dyuy = (C1 * R3 - B1 * R4) / (C1 * B2 - C2 * B1)
    t3, t4 = 1 / w[3] - 0.5, 1 / w[4] - 0.5
    m3s = t3 * ((-3 * cs2 + 1) * rho * dxux + (-3 * cs2 + a * a) * rho * dyuy
                + (-3 * cs2 + 1) * ux * dxr + (-3 * cs2 + a * a) * uy * dyr)
    m4s = t4 * ((-3 * cs2 + 1) * rho * dxux + (3 * cs2 - a * a) * rho * dyuy
                + (-3 * cs2 + 1) * ux * dxr + (3 * cs2 - a * a) * uy * dyr)
    m3G = -3 * rho * t3 * (ux ** 2 * dxux + uy ** 2 * dyuy)
    m4G = -3 * rho * t4 * (ux ** 2 * dxux - uy ** 2 * dyuy)
    meq[3] += iso * m3s + gi * m3G
    meq[4] += iso * m4s + gi * m4G
    phi = [gx * Fx + gy * Fy for gx, gy in grad]
    mt = [m[j] + w[j] * (meq[j] - m[j]) + (1 - w[j] / 2) * phi[j] for j in range(9)]
    kt = {(0, 0): mt[0], (1, 0): mt[1], (0, 1): mt[2], (2, 0): (mt[3] + mt[4]) / 2,
          (0, 2): (mt[3] - mt[4]) / 2, (1, 1): mt[5], (2, 1): mt[6], (1, 2): mt[7],
          (2, 2): mt[8]}
    h = {}
    for q in range(3):
        lo, mid, hi = invert_axis(kt[0, q], kt[1, q], kt[2, q], 0.0, 1.0)
        h[q] = {-1: lo, 0: mid, 1: hi}
    out = np.zeros(9)
    for X in (-1, 0, 1):
        lo, mid, hi = invert_axis(h[0][X], h[1][X], h[2][X], 0.0, a)
        for Y, v in ((-1, lo), (0, mid), (1, hi)):
            out[int(np.flatnonzero((EX == X) & (EY == Y))[0])] = v
    return out, (dxux, dyuy)


@pytest.mark.parametrize("a,cs2", [(1.0, 1 / 3), (0.5, 0.075), (0.25, 0.01875)])
@pytest.mark.parametrize("iso,gi", [(1, 1), (0, 0)])
def test_raw_moment_scheme_matrix_form_equals_component_form(orc, a, cs2, iso, gi):
    rng = np.random.default_rng(int(500 * a) + 7 * iso + gi)
    for _ in range(25):
        f = random_cell(rng, a, cs2)
        w = [1.0, 1.0, 1.0, rng.uniform(0.6, 1.9), rng.uniform(0.6, 1.9),
             rng.uniform(0.6, 1.9), rng.uniform(0.5, 1.5), rng.uniform(0.5, 1.5),
             rng.uniform(0.5, 1.5)]
        Fx, Fy = rng.normal(0, 1e-3, 2)
        dxr, dyr = rng.normal(0, 1e-2, 2)
        p = orc.OracleParams.make(8, 8, a, cs2, w, Fx=Fx, Fy=Fy, use_iso_corr=iso,
                                  use_gi_corr=gi, scheme="rnr")
        got, (sx, sy) = orc.collide_cell(p, f, dxr, dyr)
        ref, (rx, ry) = collide_raw_component_form(f, a, cs2, w, Fx, Fy, dxr, dyr, iso, gi)
        assert np.abs(got - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max()), (got - ref)
        assert abs(sx - rx) <= 1e-12 * max(1.0, abs(rx)) and abs(sy - ry) <= 1e-12 * max(1.0, abs(ry))
