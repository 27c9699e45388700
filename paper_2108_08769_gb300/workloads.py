"""Seeded synthetic workloads shaped like the paper's test problems.

This module is the one place that both the CUDA path and the oracle take
their inputs from.  It holds no arithmetic of the numerical method: it only
builds grids, parameters and initial states (densities sampled at cell
centres, fluid at rest, hydrostatic pressure columns).

Conventions shared by every consumer:

* A problem is a :class:`Case`.  Fields are ``numpy.float64`` arrays of shape
  ``(ny, nx)``, row-major with x fastest, interior cells only.
* ``beta`` is in pressure units (Pa): the paper's artificial sound speed is
  ``c = sqrt(u^2 + 4 beta / rho)`` (Sec. 2.1.3).  Workloads that are specified
  by an artificial sound speed ``c0`` of the heavy fluid use
  ``beta = rho_heavy * c0**2`` (:func:`beta_from_speed`).
* Boundary kinds are the strings ``slip``, ``noslip``, ``transmissive`` and
  ``periodic``, given for the x-lo, x-hi, y-lo and y-hi sides.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np

SEED = 2108

BC_KINDS = ("slip", "noslip", "transmissive", "periodic")
RIEMANN = ("osher", "bassi", "roe")
GRADP = ("new", "minmod", "superbee", "split_minmod", "split_superbee")


@dataclasses.dataclass
class Options:
    s_max: int = 3
    riemann: str = "osher"
    gradp: str = "new"
    limiter_k: int = 1
    local_dtau: bool = True
    realtime: bool = True
    bdf_order: int = 1
    alpha_pi_p_row: bool = True
    cfl_tau: float = 0.45
    abs_tol: Tuple[float, float, float, float] = (0.0, 0.0, 0.0, 0.0)


@dataclasses.dataclass
class Case:
    name: str
    nx: int
    ny: int
    lx: float
    ly: float
    gx: float
    gy: float
    beta: float
    bc: Tuple[str, str, str, str]
    rho: np.ndarray
    rhou: np.ndarray
    rhov: np.ndarray
    p: np.ndarray
    dt: float = 1e-3
    steps: int = 1
    tol: float = 1e-8
    max_iters: int = 500
    options: Options = dataclasses.field(default_factory=Options)

    @property
    def dx(self) -> float:
        return self.lx / self.nx

    @property
    def dy(self) -> float:
        return self.ly / self.ny

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def state(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
        return (self.rho.copy(), self.rhou.copy(), self.rhov.copy(), self.p.copy())


def beta_from_speed(c0: float, rho_ref: float) -> float:
    """Artificial compressibility (Pa) for an artificial sound speed c0 (m/s)."""
    return rho_ref * c0 * c0


def cell_centres(nx: int, ny: int, lx: float, ly: float) -> Tuple[np.ndarray, np.ndarray]:
    x = (np.arange(nx) + 0.5) * (lx / nx)
    y = (np.arange(ny) + 0.5) * (ly / ny)
    X, Y = np.meshgrid(x, y)
    return X, Y


def hydrostatic_columns(rho: np.ndarray, dy: float, gy: float, p_top: float = 0.0) -> np.ndarray:
    """Discrete hydrostatic pressure per column (initial condition).

    The lid (top face) holds ``p_top``.  The top cell is half a cell below it,
    and each step down between cell centres adds the mean weight of the two
    half cells: p[j] = p[j+1] - (rho[j] + rho[j+1]) gy dy / 2.  At a density
    interface that lies on a face this is the exact piecewise-linear profile
    sampled at cell centres.
    """
    ny = rho.shape[0]
    p = np.empty_like(rho)
    p[ny - 1] = p_top - rho[ny - 1] * gy * dy / 2.0
    for j in range(ny - 2, -1, -1):
        p[j] = p[j + 1] - (rho[j] + rho[j + 1]) * gy * dy / 2.0
    return p


def hydrostatic_rows(rho: np.ndarray, dx: float, gx: float, p_right: float = 0.0) -> np.ndarray:
    """As :func:`hydrostatic_columns` for gravity along x (rows, x-hi face held)."""
    return hydrostatic_columns(rho.T.copy(), dx, gx, p_right).T.copy()


# --------------------------------------------------------------------------
# The five workloads (sizes and parameters as specified for this library)
# --------------------------------------------------------------------------

def riemann_tank(nx: int = 200, ny: int = 4) -> Case:
    """1D density-discontinuity Riemann problem, 200x4, FP64.

    [0,1] m split at x = 0.5: rho 1000 | 1, p 1e5 | 0, at rest, no gravity,
    c0 = 10 m/s of the heavy fluid, pseudo CFL 0.5, dt = 1e-4 s, 20 physical
    steps, 1e-8 residual drop or 500 iterations.  Transmissive in x, periodic
    in y.
    """
    lx, ly = 1.0, ny * (1.0 / nx)
    X, _ = cell_centres(nx, ny, lx, ly)
    left = X < 0.5
    rho = np.where(left, 1000.0, 1.0)
    p = np.where(left, 1e5, 0.0)
    z = np.zeros_like(rho)
    return Case("riemann_200x4", nx, ny, lx, ly, 0.0, 0.0, beta_from_speed(10.0, 1000.0),
                ("transmissive", "transmissive", "periodic", "periodic"),
                rho, z.copy(), z.copy(), p, dt=1e-4, steps=20, tol=1e-8, max_iters=500,
                options=Options(cfl_tau=0.5))


def hydrostatic_tank(n: int = 256) -> Case:
    """Hydrostatic two-fluid tank, n x n cells on a closed 1x1 m box.

    Water (1000) below y = 0.5, air (1) above, at rest, discrete hydrostatic
    pressure, g = -9.81, c0 = 20 m/s, dt = 1e-3 s, 100 physical steps.
    """
    lx = ly = 1.0
    _, Y = cell_centres(n, n, lx, ly)
    rho = np.where(Y < 0.5, 1000.0, 1.0)
    p = hydrostatic_columns(rho, ly / n, -9.81)
    z = np.zeros_like(rho)
    return Case(f"hydrostatic_{n}x{n}", n, n, lx, ly, 0.0, -9.81, beta_from_speed(20.0, 1000.0),
                ("slip",) * 4, rho, z.copy(), z.copy(), p, dt=1e-3, steps=100, tol=1e-8,
                max_iters=500)


def water_column(nx: int = 1024, ny: int = 512) -> Case:
    """Collapsing water column, nx x ny cells on a closed 4x2 m tank.

    Water (1000) in [0,1]x[0,2] m, air (1) elsewhere, at rest, hydrostatic p,
    g = -9.81, c0 = 30 m/s, dt = 2e-4 s, 500 physical steps.
    """
    lx, ly = 4.0, 2.0
    X, Y = cell_centres(nx, ny, lx, ly)
    rho = np.where((X < 1.0) & (Y < 2.0), 1000.0, 1.0)
    p = hydrostatic_columns(rho, ly / ny, -9.81)
    z = np.zeros_like(rho)
    return Case(f"water_column_{nx}x{ny}", nx, ny, lx, ly, 0.0, -9.81, beta_from_speed(30.0, 1000.0),
                ("slip",) * 4, rho, z.copy(), z.copy(), p, dt=2e-4, steps=500, tol=1e-8,
                max_iters=500)


def rayleigh_taylor(nx: int = 2048, ny: int = 8192) -> Case:
    """Rayleigh-Taylor-type set-up, nx x ny cells on a 1x4 m slip-walled box.

    rho = 3 above y = 2 + 0.05 cos(2 pi x), 1 below, at rest, hydrostatic p,
    g = -9.81, c0 = 10 m/s, dt = 5e-4 s, 200 physical steps.
    """
    lx, ly = 1.0, 4.0
    X, Y = cell_centres(nx, ny, lx, ly)
    rho = np.where(Y > 2.0 + 0.05 * np.cos(2.0 * math.pi * X), 3.0, 1.0)
    p = hydrostatic_columns(rho, ly / ny, -9.81)
    z = np.zeros_like(rho)
    return Case(f"rayleigh_taylor_{nx}x{ny}", nx, ny, lx, ly, 0.0, -9.81, beta_from_speed(10.0, 3.0),
                ("slip",) * 4, rho, z.copy(), z.copy(), p, dt=5e-4, steps=200, tol=1e-8,
                max_iters=500)


def batched_tanks(count: int = 64, nmin: int = 64, nmax: int = 1024, seed: int = SEED,
                  sizes: Optional[List[int]] = None) -> List[Case]:
    """Many closed 1x1 m tanks of uneven size and density ratio.

    Sizes uniform in [nmin, nmax] (square), density ratio log-uniform in
    [2, 1000] (light fluid 1), water-column width and height uniform in
    [0.2, 0.6] of the box, c0 = 10 sqrt(g H) with H the column height.
    """
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(count):
        n = int(sizes[k]) if sizes is not None else int(rng.integers(nmin, nmax + 1))
        ratio = float(math.exp(rng.uniform(math.log(2.0), math.log(1000.0))))
        w = float(rng.uniform(0.2, 0.6))
        h = float(rng.uniform(0.2, 0.6))
        X, Y = cell_centres(n, n, 1.0, 1.0)
        rho = np.where((X < w) & (Y < h), ratio, 1.0)
        p = hydrostatic_columns(rho, 1.0 / n, -9.81)
        z = np.zeros_like(rho)
        c0 = 10.0 * math.sqrt(9.81 * h)
        cases.append(Case(f"tank{k}_{n}x{n}", n, n, 1.0, 1.0, 0.0, -9.81, beta_from_speed(c0, ratio),
                          ("slip",) * 4, rho, z.copy(), z.copy(), p, dt=1e-3, steps=1, tol=1e-8,
                          max_iters=500))
    return cases


# --------------------------------------------------------------------------
# The paper's own benchmark set-ups (Sec. 3), as synthetic initial states
# --------------------------------------------------------------------------

# Table "riemann_problems" (Sec. 3.1): rho_L, rho_R, u_L, u_R, p_L, p_R, beta, tau
RIEMANN_TABLE: Dict[int, Tuple[float, ...]] = {
    1: (1.0, 1.0, 1.0, 1.0, 0.1, 1.0, 0.81, 0.1),
    2: (1.0, 1.0, 0.0, 0.0, 1000.0, 0.01, 1000.0, 0.005),
    3: (1.4, 1.0, 0.0, 0.0, 1.0, 1.0, 1.0, 2.0),
    4: (1.4, 1.0, 0.1, 0.1, 1.0, 1.0, 1.0, 2.0),
    5: (0.00125, 1.0, 1.0, 1.0, 0.1, 1.0, 1.0, 0.005),
}


def riemann_problem(k: int, nx: int = 100, half_width: Optional[float] = None,
                    along: str = "x") -> Case:
    """Riemann problem RPk on nx x 1 cells (or 1 x nx with along='y').

    Pure pseudo-time evolution: real-time term off, global pseudo-time step,
    3 stages, CFL 0.98, minmod on rho, u, v and p, no gravity, zero-gradient
    boundaries (Sec. 3.1).  The domain [-X, X] is wide enough that no wave
    reaches a boundary by the output pseudo-time.
    """
    rL, rR, uL, uR, pL, pR, beta, tau = RIEMANN_TABLE[k]
    if half_width is None:
        smax = 0.0
        for r, u in ((rL, uL), (rR, uR)):
            c = math.sqrt(u * u + 4.0 * beta / r)
            smax = max(smax, abs(0.5 * (u - c)), abs(0.5 * (u + c)))
        half_width = 1.25 * smax * tau
    L = 2.0 * half_width
    x = -half_width + (np.arange(nx) + 0.5) * (L / nx)
    left = x < 0.0
    rho = np.where(left, rL, rR)
    u = np.where(left, uL, uR)
    p = np.where(left, pL, pR)
    opts = Options(s_max=3, gradp="minmod", local_dtau=False, realtime=False, cfl_tau=0.98)
    if along == "x":
        shape = (1, nx)
        case = Case(f"RP{k}_{nx}", nx, 1, L, L / nx, 0.0, 0.0, beta, ("transmissive",) * 4,
                    rho.reshape(shape), (rho * u).reshape(shape), np.zeros(shape), p.reshape(shape),
                    dt=1.0, steps=1, tol=-1.0, max_iters=100000, options=opts)
    else:
        shape = (nx, 1)
        case = Case(f"RP{k}_{nx}_y", 1, nx, L / nx, L, 0.0, 0.0, beta, ("transmissive",) * 4,
                    rho.reshape(shape), np.zeros(shape), (rho * u).reshape(shape), p.reshape(shape),
                    dt=1.0, steps=1, tol=-1.0, max_iters=100000, options=opts)
    case.tau_end = tau  # type: ignore[attr-defined]
    case.x = x  # type: ignore[attr-defined]
    return case


def hydrostatic_column_1d(n: int = 20) -> Case:
    """Sec. 3.2: 20x1 cells, air over water with g = (9.81, 0), p = 0 initially,
    walls on all sides, beta = 2000, one real-time step dt = 0.05, CFL 0.98
    local, until the rho u residual is below 1e-5.  Gravity points along +x,
    so the water (rho 1000) lies at the x-hi end."""
    L = 1.0
    x = (np.arange(n) + 0.5) * (L / n)
    rho = np.where(x > 0.5, 1000.0, 1.0).reshape(1, n)
    z = np.zeros((1, n))
    opts = Options(s_max=3, cfl_tau=0.98, abs_tol=(math.inf, 1e-5, math.inf, math.inf))
    return Case("hydrostatic_column_20x1", n, 1, L, L / n, 9.81, 0.0, 2000.0, ("slip",) * 4,
                rho, z.copy(), z.copy(), z.copy(), dt=0.05, steps=1, tol=0.0, max_iters=200000,
                options=opts)


def dam_break_small(n: int = 20) -> Case:
    """Sec. 3.3.1: 20x20 cells, water (1000) left of x = 0.4 (domain read as
    1x1 m, column height the full domain), air (1) elsewhere, p = 0, g = (0, -9.81),
    walls, beta = 1100, dt = 0.01, CFL 0.48 local, until the rho u and rho v
    residuals are below 1e-3."""
    X, _ = cell_centres(n, n, 1.0, 1.0)
    rho = np.where(X < 0.4, 1000.0, 1.0)
    z = np.zeros_like(rho)
    opts = Options(s_max=3, cfl_tau=0.48, abs_tol=(math.inf, 1e-3, 1e-3, math.inf))
    return Case("dam_break_20x20", n, n, 1.0, 1.0, 0.0, -9.81, 1100.0, ("slip",) * 4,
                rho, z.copy(), z.copy(), z.copy(), dt=0.01, steps=1, tol=0.0, max_iters=200000,
                options=opts)


# --------------------------------------------------------------------------
# Random states for parity tests
# --------------------------------------------------------------------------

def random_two_fluid(nx: int, ny: int, seed: int = SEED, ratio: float = 1000.0,
                     bc: Tuple[str, str, str, str] = ("slip",) * 4, c0: float = 20.0,
                     velocity: float = 0.05, gy: float = -9.81, gx: float = 0.0,
                     options: Optional[Options] = None) -> Case:
    """A perturbed two-fluid state on an nx x ny box of 1 x (ny/nx) m.

    A heavy blob (ratio) with a wavy interface over light fluid (1), small
    random velocities and a hydrostatic pressure with a small random
    perturbation.  Used where a parity test wants every branch of the
    limiter and the flux to be exercised."""
    rng = np.random.default_rng(seed)
    lx, ly = 1.0, ny / nx
    X, Y = cell_centres(nx, ny, lx, ly)
    iface = 0.5 * ly + 0.1 * ly * np.sin(2 * math.pi * X * 1.5 + 0.3)
    rho = np.where(Y < iface, ratio, 1.0) * (1.0 + 0.01 * rng.standard_normal((ny, nx)))
    u = velocity * rng.standard_normal((ny, nx))
    v = velocity * rng.standard_normal((ny, nx))
    p = hydrostatic_columns(rho, ly / ny, gy) if gy != 0.0 else np.zeros_like(rho)
    p = p + 0.5 * ratio * velocity ** 2 * rng.standard_normal((ny, nx))
    return Case(f"random_{nx}x{ny}", nx, ny, lx, ly, gx, gy, beta_from_speed(c0, ratio), bc,
                rho, rho * u, rho * v, p, dt=1e-3, steps=1, tol=1e-8, max_iters=500,
                options=options or Options())
