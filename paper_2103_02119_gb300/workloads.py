"""Seeded synthetic workloads shaped like the paper's test flows.

This module only *describes inputs*: grid sizes, physical parameters, wall
velocities, obstacle masks and initial density/velocity fields.  It holds no
lattice Boltzmann arithmetic, so both the CUDA library and the CPU oracle can
be driven from the same inputs without sharing any of the method's code.

Lattice units throughout: dx = dt = 1, dy = a; cell (x, y) sits at the
physical point ((x + 1/2), (y + 1/2) a); arrays are indexed ``[y, x]``.
Relaxation rates follow the paper's choices: omega_4 = omega_5 = 1/tau set by
the shear viscosity nu = cs2 (tau - 1/2) (Eq. 32), every other rate is 1
(Sec. 5.1).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    a: float
    cs2: float
    omega: tuple
    Fx: float = 0.0
    Fy: float = 0.0
    periodic_x: int = 1
    periodic_y: int = 1
    # wall velocities (Ux, Uy): left, right, bottom, top
    wall_u: tuple = ((0.0, 0.0), (0.0, 0.0), (0.0, 0.0), (0.0, 0.0))
    mask: np.ndarray | None = None   # (ny, nx) uint8, 1 = solid
    rho: np.ndarray | None = None    # initial fields, (ny, nx) float64
    ux: np.ndarray | None = None
    uy: np.ndarray | None = None
    use_iso_corr: int = 1
    use_gi_corr: int = 1
    info: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def omega_for(nu: float, cs2: float, omega_bulk: float = 1.0) -> tuple:
    """Relaxation rates for shear viscosity nu: tau = nu/cs2 + 1/2."""
    tau = nu / cs2 + 0.5
    w = 1.0 / tau
    return (1.0, 1.0, 1.0, omega_bulk, w, w, 1.0, 1.0, 1.0)


def stable_cs2(a: float) -> float:
    """Speed of sound used for the decaying-flow workloads: 1/3 on the square
    lattice, 0.3 a^2 below it (c_s^2 must stay below a^2, and the scheme needs
    it well below a^2 at low viscosity)."""
    return 1.0 / 3.0 if a >= 1.0 else 0.3 * a * a


def coords(nx: int, ny: int, a: float):
    x = (np.arange(nx) + 0.5)[None, :] * np.ones((ny, 1))
    y = ((np.arange(ny) + 0.5) * a)[:, None] * np.ones((1, nx))
    return x, y


def poiseuille(ny: int = 32, nx: int = 32, a: float = 0.5, cs2: float = 0.16,
               nu: float = 0.1, U: float = 0.01) -> Workload:
    """Body-force channel of Sec. 5.1: periodic in x, walls in y, rest start.
    H = ny a; the force gives the centre-line speed U = F H^2 / (8 nu)."""
    H = ny * a
    Fx = 8.0 * nu * U / (H * H)
    return Workload(f"poiseuille_{nx}x{ny}_a{a}", nx, ny, a, cs2,
                    omega_for(nu, cs2), Fx=Fx, periodic_x=1, periodic_y=0,
                    info=dict(nu=nu, U=U, H=H))


def couette(ny: int = 40, nx: int = 4, a: float = 0.25, cs2: float = 0.04,
            tau: float = 0.8, U: float = 0.02) -> Workload:
    """Shear-driven channel of Sec. 5.2: top wall moves at (U, 0)."""
    nu = cs2 * (tau - 0.5)
    wall_u = ((0.0, 0.0), (0.0, 0.0), (0.0, 0.0), (U, 0.0))
    return Workload(f"couette_{nx}x{ny}_a{a}", nx, ny, a, cs2,
                    omega_for(nu, cs2), periodic_x=1, periodic_y=0,
                    wall_u=wall_u, info=dict(nu=nu, U=U, H=ny * a))


def cavity(nx: int, ny: int, a: float, cs2: float, U: float, Re: float) -> Workload:
    """Lid-driven cavity (Sec. 5.4): walls on all four sides, the top wall
    moves at (U, 0); Re = U L / nu with L = nx (the cavity width)."""
    L = nx
    nu = U * L / Re
    wall_u = ((0.0, 0.0), (0.0, 0.0), (0.0, 0.0), (U, 0.0))
    return Workload(f"cavity_{nx}x{ny}_a{a}_Re{Re:g}", nx, ny, a, cs2,
                    omega_for(nu, cs2), periodic_x=0, periodic_y=0,
                    wall_u=wall_u, info=dict(nu=nu, U=U, Re=Re, L=L))


def taylor_green(nx: int, ny: int, a: float, cs2: float, nu: float,
                 u0: float = 0.02, seed: int = 0, wavelength: float | None = None,
                 background=(0.0, 0.0)) -> Workload:
    """Decaying Taylor-Green vortex on a periodic box; phases from the seed.
    u_x = u0 sin(k x + p1) cos(k y + p2), u_y = -u0 cos(k x + p1) sin(k y + p2),
    rho = 1 + u0^2 / (4 cs2) [cos 2(k x + p1) + cos 2(k y + p2)]."""
    lam = float(nx if wavelength is None else wavelength)
    k = 2.0 * np.pi / lam
    rng = np.random.default_rng(seed)
    p1, p2 = 2.0 * np.pi * rng.random(2)
    x, y = coords(nx, ny, a)
    ux = u0 * np.sin(k * x + p1) * np.cos(k * y + p2) + background[0]
    uy = -u0 * np.cos(k * x + p1) * np.sin(k * y + p2) + background[1]
    rho = 1.0 + u0 * u0 / (4.0 * cs2) * (np.cos(2 * (k * x + p1)) + np.cos(2 * (k * y + p2)))
    return Workload(f"tgv_{nx}x{ny}_a{a}", nx, ny, a, cs2, omega_for(nu, cs2),
                    rho=rho, ux=ux, uy=uy,
                    info=dict(nu=nu, k=k, u0=u0, phases=(p1, p2),
                              background=tuple(background)))


def shear_wave(nx: int, ny: int, a: float, cs2: float, nu: float,
               direction: str, u0: float = 0.02, seed: int = 0,
               wavelength: float | None = None) -> Workload:
    """Decaying shear wave on a periodic box.  direction 'y': u_x varies with
    y; 'x': u_y varies with x; 'diag': wave vector (k, k), velocity normal to
    it (incompressible)."""
    lam = float(nx if wavelength is None else wavelength)
    k = 2.0 * np.pi / lam
    rng = np.random.default_rng(seed)
    ph = 2.0 * np.pi * rng.random()
    x, y = coords(nx, ny, a)
    if direction == "y":
        ux, uy = u0 * np.sin(k * y + ph), 0.0 * x
    elif direction == "x":
        ux, uy = 0.0 * x, u0 * np.sin(k * x + ph)
    elif direction == "diag":
        s = np.sin(k * x + k * y + ph) / np.sqrt(2.0)
        ux, uy = -u0 * s, u0 * s
    else:
        raise ValueError(direction)
    return Workload(f"shear_{direction}_{nx}x{ny}_a{a}", nx, ny, a, cs2,
                    omega_for(nu, cs2), rho=np.ones_like(x), ux=ux, uy=uy,
                    info=dict(nu=nu, k=k, u0=u0, phase=ph, direction=direction))


def random_obstacles(nx: int, ny: int, seed: int, coverage: float = 0.10,
                     margin: int = 2, max_side: int | None = None) -> np.ndarray:
    """Seeded axis-aligned solid rectangles, added until the next one would
    push the solid fraction above `coverage`; a `margin`-cell fluid band is
    kept along the domain edges."""
    rng = np.random.default_rng(seed)
    m = np.zeros((ny, nx), dtype=np.uint8)
    if nx <= 2 * margin + 1 or ny <= 2 * margin + 1:
        return m
    max_side = max_side or max(2, min(nx, ny) // 4)
    for _ in range(10000):
        w = int(rng.integers(1, max_side + 1))
        h = int(rng.integers(1, max_side + 1))
        x0 = int(rng.integers(margin, max(margin + 1, nx - margin - w)))
        y0 = int(rng.integers(margin, max(margin + 1, ny - margin - h)))
        trial = m.copy()
        trial[y0:y0 + h, x0:x0 + w] = 1
        if trial.mean() > coverage:
            break
        m = trial
    return m


def smooth_random_fields(nx: int, ny: int, seed: int, u_amp: float = 0.02,
                         rho_amp: float = 1e-3, modes: int = 3):
    """Smooth random periodic (rho, ux, uy): a few Fourier modes per field."""
    rng = np.random.default_rng(seed)
    X = (np.arange(nx) + 0.5)[None, :] / nx
    Y = (np.arange(ny) + 0.5)[:, None] / ny

    def field_(amp):
        out = np.zeros((ny, nx))
        for _ in range(modes):
            kx, ky = rng.integers(-3, 4, 2)
            ph = rng.random() * 2 * np.pi
            out += amp / modes * rng.normal() * np.cos(2 * np.pi * (kx * X + ky * Y) + ph)
        return out

    return 1.0 + field_(rho_amp), field_(u_amp), field_(u_amp)


def perturbation(nx: int, ny: int, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Seeded (9, ny, nx) noise added to an equilibrium state to give it a
    non-equilibrium part."""
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((9, ny, nx))


def batch_sweep(count: int, seed: int = 0, n_range=(64, 1024), a_range=(0.2, 1.0),
                re_range=(100.0, 5000.0), coverage: float = 0.10,
                tau_range=(0.505, 2.0)) -> list:
    """Uneven sweep of independent channel / cavity instances.

    Per instance (seeded): nx, ny = round(exp(U[ln n_min, ln n_max])),
    a ~ U[a_min, a_max], Re = exp(U[ln Re_min, ln Re_max]); half channels
    (periodic in x, walls in y, body force), half lid-driven cavities; seeded
    solid rectangles up to `coverage` with a 2-cell fluid margin.  c_s^2 =
    stable_cs2(a), U = min(0.05, 0.3 c_s), nu = U nx / Re.  When tau = 1/2 +
    nu / c_s^2 exceeds tau_max, U is lowered to bring tau to tau_max; when it
    falls below tau_min the instance is redrawn (the reason is kept in
    info['redrawn']).  The channel force gives a centre-line speed U in the
    empty channel (F = 8 nu U / H^2, H = ny a)."""
    rng = np.random.default_rng(seed)
    out = []
    ln = np.log
    while len(out) < count:
        nx = int(round(np.exp(rng.uniform(ln(n_range[0]), ln(n_range[1])))))
        ny = int(round(np.exp(rng.uniform(ln(n_range[0]), ln(n_range[1])))))
        a = float(rng.uniform(*a_range))
        Re = float(np.exp(rng.uniform(ln(re_range[0]), ln(re_range[1]))))
        kind = "channel" if rng.random() < 0.5 else "cavity"
        mseed = int(rng.integers(1 << 31))
        cs2 = stable_cs2(a)
        U = min(0.05, 0.3 * np.sqrt(cs2))
        nu = U * nx / Re
        tau = 0.5 + nu / cs2
        redrawn = None
        if tau > tau_range[1]:
            nu = (tau_range[1] - 0.5) * cs2
            U = nu * Re / nx
        elif tau < tau_range[0]:
            redrawn = f"tau {tau:.4f} below {tau_range[0]}"
        if redrawn:
            if out:
                out[-1].info.setdefault("redrawn", []).append(redrawn)
            continue
        mask = random_obstacles(nx, ny, seed=mseed, coverage=coverage)
        if kind == "channel":
            H = ny * a
            wl = Workload(f"channel_{nx}x{ny}_a{a:.3f}_Re{Re:.0f}", nx, ny, a, cs2,
                          omega_for(nu, cs2), Fx=8.0 * nu * U / (H * H), periodic_x=1,
                          periodic_y=0, mask=mask, info=dict(nu=nu, U=U, Re=Re, kind=kind))
        else:
            wl = cavity(nx, ny, a, cs2, U, Re).with_(mask=mask)
            wl.info["kind"] = kind
        out.append(wl)
    return out
