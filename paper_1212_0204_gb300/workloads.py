"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only input recipes: grid sizes, velocity grids, relaxation
times and initial primitive fields (density, velocity, temperature).  It holds
none of the scheme's arithmetic, so both the CUDA library's tests/benchmark and
the CPU oracle can take their inputs from it.  Conversions to conserved
moments are done by each side on its own.

Workloads (analytic initial data, no dataset):
  * ``sod_1d``          1D-1V Riemann tube (Section 5.1 shape).
  * ``sod_1d_300x100``  Section 5.1's Sod tube itself: 300 cells, 100 velocities.
  * ``quadrant_2d``     2D-2V four-quadrant Riemann problem with a 1 % seeded
                        density perturbation (counter-based SplitMix64).
  * ``density_wave_3d`` 3D-3V periodic smooth density wave.
  * ``batched_tubes``   many independent 1D-1V tubes of uneven size.
  * ``shear_layer_2d``  2D-2V shear layer with a smooth random tau field.
  * ``entropy_wave_1d`` smooth advected density wave (uniform pressure).
  * ``isentropic_vortex_2d`` Section 5.2's advected isentropic vortex (convergence study).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1212

PERIODIC, OUTFLOW = 0, 1
FKS, HOFKS, HOFKS_UNLIMITED, HOFKS_WENO, FKS_STRANG = 0, 1, 2, 3, 4


@dataclass
class Case:
    """One scheme configuration plus its initial primitive fields.

    Arrays are flattened with x fastest: ``rho[c]``, ``u[i][c]``, ``T[c]``,
    ``tau`` is a scalar or a per-cell array.
    """
    name: str
    d: int
    nx: tuple
    dx: float
    nv: tuple
    kmin: tuple
    dv: float
    p: int
    bc: tuple
    tau: object
    rho: np.ndarray
    u: np.ndarray
    T: np.ndarray
    steps: int
    scheme: int = HOFKS
    subcycles: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return int(np.prod(self.nx))

    @property
    def nvel(self) -> int:
        return int(np.prod(self.nv))

    @property
    def points(self) -> int:
        return self.ncells * self.nvel

    @property
    def dt(self) -> float:
        return self.dx / (self.p * self.dv)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea & Flood 2014) on uint64 inputs."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def counter_uniform(seed: int, n: int) -> np.ndarray:
    """Uniform(-1, 1) per counter 0..n-1: SplitMix64 of (seed << 32) + counter."""
    ctr = (np.uint64(seed) << np.uint64(32)) + np.arange(n, dtype=np.uint64)
    bits = splitmix64(ctr) >> np.uint64(11)
    return bits.astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0


def _centres(n: int, dx: float, x0: float = 0.0) -> np.ndarray:
    return x0 + (np.arange(n) + 0.5) * dx


def sod_1d(nx: int = 200, nv: int = 32, tau: float = 1e-4, steps: int | None = None,
           dv: float = 0.4, p: int = 1, t_final: float = 0.15,
           left=(1.0, 1.0), right=(0.125, 0.8), scheme: int = HOFKS) -> Case:
    """1D-1V Riemann tube on [0,1], outflow ends; left/right = (rho, T), u = 0.

    Velocities v_k = k dv with k = -nv/2 .. nv/2-1; with p = 1 every shift is an
    integer number of cells (dt = dx/dv).
    """
    dx = 1.0 / nx
    x = _centres(nx, dx)
    rho = np.where(x < 0.5, left[0], right[0])
    T = np.where(x < 0.5, left[1], right[1])
    dt = dx / (p * dv)
    if steps is None:
        steps = int(round(t_final / dt))
    return Case("sod_1d", 1, (nx,), dx, (nv,), (-(nv // 2),), dv, p, (OUTFLOW,), tau,
                rho, np.zeros((1, nx)), T, steps, scheme)


def quadrant_2d(n: int = 256, nv: int = 32, tau: float = 1e-3, steps: int = 500,
                dv: float = 0.4, seed: int = SEED_BASE, scheme: int = HOFKS) -> Case:
    """2D-2V four-quadrant Riemann problem, periodic, 1 % seeded density noise.

    (x >= 1/2, y >= 1/2): rho 1, T 1; (x < 1/2, y >= 1/2) and (x >= 1/2, y < 1/2):
    rho 0.5, T 0.8; (x < 1/2, y < 1/2): rho 0.125, T 0.8; u = 0.
    """
    dx = 1.0 / n
    xc = _centres(n, dx)
    X, Y = np.meshgrid(xc, xc, indexing="xy")  # X varies fastest in flattening
    X, Y = X.ravel(), Y.ravel()
    hi_x, hi_y = X >= 0.5, Y >= 0.5
    rho = np.where(hi_x & hi_y, 1.0, np.where(~hi_x & ~hi_y, 0.125, 0.5))
    T = np.where(hi_x & hi_y, 1.0, 0.8)
    rho = rho * (1.0 + 0.01 * counter_uniform(seed, n * n))
    return Case("quadrant_2d", 2, (n, n), dx, (nv, nv), (-(nv // 2),) * 2, dv, 1,
                (PERIODIC, PERIODIC), tau, rho, np.zeros((2, n * n)), T, steps, scheme)


def density_wave_3d(n: int = 96, nv: int = 24, tau: float = 1e-4, steps: int = 100,
                    dv: float = 0.5, amp: float = 0.2, ux: float = 0.5,
                    scheme: int = HOFKS) -> Case:
    """3D-3V periodic box: rho = 1 + amp sin(2 pi x) sin(2 pi y) sin(2 pi z), T = 1,
    u = (ux, 0, 0)."""
    dx = 1.0 / n
    xc = _centres(n, dx)
    Z, Y, X = np.meshgrid(xc, xc, xc, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    rho = 1.0 + amp * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(2 * np.pi * Z)
    u = np.zeros((3, n ** 3))
    u[0] = ux
    return Case("density_wave_3d", 3, (n, n, n), dx, (nv,) * 3, (-(nv // 2),) * 3, dv, 1,
                (PERIODIC,) * 3, tau, rho, u, np.ones(n ** 3), steps, scheme)


def entropy_wave_1d(nx: int, nv: int = 32, tau: float = 1e-4, dv: float = 0.4,
                    amp: float = 0.2, ux: float = 0.5, t_final: float = 0.25,
                    scheme: int = HOFKS, subcycles: int = 0) -> Case:
    """Smooth advected density wave with uniform pressure p = 1 (T = 1/rho): in the
    fluid limit its exact solution is rho(x - ux t)."""
    dx = 1.0 / nx
    x = _centres(nx, dx)
    rho = 1.0 + amp * np.sin(2 * np.pi * x)
    steps = int(round(t_final / (dx / dv)))
    return Case("entropy_wave_1d", 1, (nx,), dx, (nv,), (-(nv // 2),), dv, 1, (PERIODIC,),
                tau, rho, np.full((1, nx), ux), 1.0 / rho, steps, scheme, subcycles,
                extra={"amp": amp, "ux": ux, "t_final": steps * dx / dv})


def implosion_2d(n: int = 100, nv: int = 30, tau: float = 1e-3, scheme: int = HOFKS,
                 t_final: float = 0.07) -> Case:
    """Section 5.4's 2D implosion: [0, 2]^2, a disk of radius 0.2 centred at (1, 1)
    with rho = 0.125, u = 0, T = 4 inside a gas with rho = 1, T = 4, u_x = +1 for
    x < 1 and -1 for x > 1, u_y = +1 for y < 1 and -1 for y > 1 (the flow converges
    on the disk); nv^2 velocities on [-20, 20)^2 (the printed 30 per direction);
    zero-gradient outflow boundaries (not stated).  The shift denominator p is the
    smallest one for which t_final is a whole number of exact-transport steps
    dt = dx / (p dv); the Euler part sub-steps inside each step (Eq. Time2)."""
    dx = 2.0 / n
    dv = 40.0 / nv
    xc = _centres(n, dx)
    Y, X = np.meshgrid(xc, xc, indexing="ij")
    X, Y = X.ravel(), Y.ravel()
    disk = (X - 1.0) ** 2 + (Y - 1.0) ** 2 < 0.2 ** 2
    rho = np.where(disk, 0.125, 1.0)
    u = np.stack([np.where(X < 1.0, 1.0, -1.0), np.where(Y < 1.0, 1.0, -1.0)])
    u[:, disk] = 0.0
    # dt = dx / (p dv): t_final / dt = p (t_final n dv / 2) must be whole
    from fractions import Fraction
    per = Fraction(t_final).limit_denominator(10 ** 6) * n * Fraction(dv).limit_denominator(10 ** 6) / 2
    p, steps = per.denominator, per.numerator
    return Case("implosion_2d", 2, (n, n), dx, (nv, nv), (-(nv // 2),) * 2, dv, p, (OUTFLOW, OUTFLOW), tau,
                rho, u, np.full(n * n, 4.0), steps, scheme, extra={"t_final": steps * dx / (p * dv)})


def sod_1d_300x100(tau: float, scheme: int = HOFKS) -> Case:
    """Section 5.1's Sod tube: 300 cells on [0, 1], 100 velocities on [-15, 15)
    (dv = 0.3), left (rho, u, T) = (1, 0, 5), right (0.125, 0, 4), outflow, up to
    t = 0.05, for the relaxation times 1e-2, 1e-3, 5e-4 and 1e-4 of the paper.
    The paper gives no time step; dt = dx / v_max (p = v_max / dv = 50, 225 steps)
    is the one at which these four tau run from the kinetic (dt / tau = 0.02) to
    the fluid regime (2.2)."""
    return sod_1d(nx=300, nv=100, tau=tau, dv=0.3, p=50, t_final=0.05,
                  left=(1.0, 5.0), right=(0.125, 4.0), scheme=scheme)


def isentropic_vortex_2d(n: int, nv: int = 40, vmax: float = 8.0, tau: float = 1e-4,
                         t_final: float = 1.0, beta: float = 5.0, scheme: int = HOFKS,
                         subcycles: int | None = None) -> Case:
    """Section 5.2's advected isentropic vortex on the periodic square of side 10
    (centred, i.e. the paper's vortex at the origin of [-5, 5]^2): background
    rho = u = v = T = 1, perturbations du = -y' b e^{(1-r^2)/2}, dv = x' b e^{(1-r^2)/2}
    with b = beta / (2 pi), dT = -(g - 1) beta^2 / (8 g pi^2) e^{1-r^2},
    rho = T^{1/(g-1)}, for the ratio g = 1 + 2/d = 2 of the 2D-2V kinetic model
    (reading R4; the printed 5/3 is not the model's) and beta^2 in dT (the radial
    balance of the exact vortex; the printed beta is read as garbled).  nv^2
    velocities on [-vmax, vmax), p = 1: by default 40^2 on [-8, 8) (dv = 0.4)
    instead of the paper's 20^2 on [-15, 15] (dv = 1.5, under two points per
    thermal width sqrt(T_min) ~ 0.75, on which FKS leaves the physical states at
    50^2); dv = 0.4 also makes t = 1 a whole number of steps dx / dv on each of the
    paper's meshes 25^2 .. 400^2.  The Euler sub-steps are forced to n per kinetic
    step, so that their length is of order dx^2 as the paper makes the time error
    negligible.  The exact density at t_final, which must be a whole number of
    steps, is the initial one translated by (1, 1) t: extra["rho_exact"]."""
    L = 10.0
    dx = L / n
    dv = 2.0 * vmax / nv
    g = 2.0
    steps = int(round(t_final / (dx / dv)))
    t = steps * dx / dv
    if steps < 1 or abs(t - t_final) > 1e-9 * t_final:
        raise ValueError("t_final %g is not a whole number of steps dx/dv = %g" % (t_final, dx / dv))
    xc = _centres(n, dx)
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    X, Y = X.ravel(), Y.ravel()

    def fields(shift):
        xp = (X - L / 2 - shift + L / 2) % L - L / 2
        yp = (Y - L / 2 - shift + L / 2) % L - L / 2
        r2 = xp * xp + yp * yp
        b = beta / (2.0 * np.pi)
        e = np.exp(0.5 * (1.0 - r2))
        T = 1.0 - (g - 1.0) * beta * beta / (8.0 * g * np.pi * np.pi) * e * e
        return T ** (1.0 / (g - 1.0)), 1.0 - yp * b * e, 1.0 + xp * b * e, T

    rho, ux, uy, T = fields(0.0)
    return Case("isentropic_vortex_2d", 2, (n, n), dx, (nv, nv), (-(nv // 2),) * 2, dv, 1,
                (PERIODIC, PERIODIC), tau, rho, np.stack([ux, uy]), T, steps, scheme,
                n if subcycles is None else subcycles,
                extra={"t_final": t, "rho_exact": fields(t)[0]})


def batched_tubes(ncases: int = 512, seed: int = SEED_BASE, steps: int = 100,
                  nx_range=(100, 2000), nv_choices=(32, 64, 128)) -> list:
    """Independent 1D-1V Riemann tubes of uneven size.

    Nx ~ U{100..2000}, Nv in {32, 64, 128}, tau = 10^U(-5, 0), left/right rho and T
    ~ U(0.1, 1), u = 0, outflow.  The velocity grid is centred on 0 with half-width
    min(6.4, 5 sqrt(1.5 T_max)), T_max the hotter side: dv = 2 * halfwidth / Nv.  (A
    fixed [-6.4, 6.4) grid leaves dv = 0.4 at Nv = 32, coarser than the thermal speed
    of a T = 0.1 side, and the discrete Maxwellian of such a cell is under-resolved.)
    If the drawn Nv leaves fewer than two velocities per thermal width sqrt(T_min)
    of the colder side, the next larger size of the set is taken (with 1.3 points
    per width the cold state of a tube loses its temperature within ~140 steps, in
    the FP64 oracle as on the GPU).  Case i draws from seed + i.
    """
    cases = []
    for i in range(ncases):
        rng = np.random.default_rng(seed + i)
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        nv = int(rng.choice(nv_choices))
        tau = float(10.0 ** rng.uniform(-5.0, 0.0))
        rl, rr, tl, tr = rng.uniform(0.1, 1.0, size=4)
        half = min(6.4, 5.0 * np.sqrt(1.5 * max(tl, tr)))
        larger = [n for n in sorted(nv_choices) if n > nv]
        while np.sqrt(min(tl, tr)) < 2.0 * (2.0 * half / nv) and larger:
            nv = larger.pop(0)
        c = sod_1d(nx=nx, nv=nv, tau=tau, steps=steps, dv=2.0 * half / nv, left=(rl, tl),
                   right=(rr, tr))
        c.name = f"tube_{i}"
        cases.append(c)
    return cases


def smooth_field_2d(n: int, seed: int, modes: int = 4) -> np.ndarray:
    """Seeded smooth periodic field on the n x n cell centres, min-max scaled to [0, 1]:
    sum over |m|,|l| <= modes of a_ml cos(2 pi (m x + l y) + phi_ml),
    a_ml ~ N(0,1)/(1 + m^2 + l^2), phi_ml ~ U(0, 2 pi)."""
    rng = np.random.default_rng(seed)
    xc = _centres(n, 1.0 / n)
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    r = np.zeros_like(X)
    for m in range(-modes, modes + 1):
        for l in range(-modes, modes + 1):
            a = rng.standard_normal() / (1.0 + m * m + l * l)
            phi = rng.uniform(0.0, 2.0 * np.pi)
            r += a * np.cos(2.0 * np.pi * (m * X + l * Y) + phi)
    r = (r - r.min()) / (r.max() - r.min())
    return r.ravel()


def shear_layer_2d(n: int = 512, nv: int = 32, steps: int = 200, dv: float = 0.4,
                   seed: int = SEED_BASE, width: float = 0.02) -> Case:
    """2D-2V shear layer u_x = 0.5 tanh((y - 1/2)/width), rho = T = 1, periodic, with
    tau(x, y) = 1e-5 * 10^(5 r(x, y)), r a seeded smooth field in [0, 1]."""
    dx = 1.0 / n
    xc = _centres(n, dx)
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    u = np.zeros((2, n * n))
    u[0] = 0.5 * np.tanh((Y.ravel() - 0.5) / width)
    r = smooth_field_2d(n, seed)
    tau = 1e-5 * 10.0 ** (5.0 * r)
    return Case("shear_layer_2d", 2, (n, n), dx, (nv, nv), (-(nv // 2),) * 2, dv, 1,
                (PERIODIC, PERIODIC), tau, np.ones(n * n), u, np.ones(n * n), steps)
