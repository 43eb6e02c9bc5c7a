"""Seeded synthetic workloads shared by the CUDA library's tests/bench and the oracle.

This module only describes inputs: grid sizes, boundary kinds, physical
parameters, the initial/inflow velocity profile and leaf-area-density (LAD)
profiles.  It holds none of the lattice Boltzmann arithmetic; the random
initial perturbation is drawn inside each implementation from the published
SplitMix64 generator, keyed by (seed, cell, component).

Shapes follow the paper's domains as scaled for one B300: the channel of the
validation case (aspect and driving, Sec. 4, Eq. Body_force) and the forest
atmospheric boundary layer (Sec. 5, Table tab:forest_cases, Eq. af_theory).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence, Tuple

import numpy as np

PERIODIC, BOUNCEBACK, FREESLIP, EQUILIBRIUM, INFLOW, OUTFLOW = range(6)

SEED_BASE = 20220630
KAPPA = 0.41  # von Karman constant of the log-law initial profile


@dataclasses.dataclass
class Case:
    name: str
    nx: int
    ny: int
    nz: int
    bc_x: Tuple[int, int] = (PERIODIC, PERIODIC)
    bc_y: Tuple[int, int] = (BOUNCEBACK, BOUNCEBACK)
    bc_z: Tuple[int, int] = (PERIODIC, PERIODIC)
    tau0: float = 0.8
    cs: float = 0.0
    g: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    cd: float = 0.0
    canopy_x: Tuple[int, int] = (0, 0)
    u_bulk_target: float = 0.0
    ctrl_gain: float = 0.0
    u_top: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    stats_xbins: int = 1
    seed: int = SEED_BASE
    init_perturb: float = 0.0
    lad: Optional[np.ndarray] = None
    u_profile: Optional[np.ndarray] = None
    # model variants (0 = default): canopy drag on u_x only; forcing scheme
    # (0 Guo, 1 exact difference); tau_total with Q^1/2 / rho^p, p = 1 (0) or 2
    drag_streamwise_only: int = 0
    forcing_scheme: int = 0
    sgs_rho_power: int = 0

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def replace(self, **kw) -> "Case":
        return dataclasses.replace(self, **kw)


# ---- profiles ---------------------------------------------------------------

def cell_heights(ny: int) -> np.ndarray:
    """Cell-centre heights above a halfway bounce-back ground at y = 0."""
    return np.arange(ny, dtype=np.float64) + 0.5


def log_law_profile(ny: int, u_tau: float, nu: float, u_bulk: float) -> np.ndarray:
    """Log-law shape (u_tau/kappa) ln(1 + y+) at cell centres, rescaled so that
    its mean equals u_bulk (initial condition of the channel)."""
    yp = cell_heights(ny) * u_tau / nu
    shape = (u_tau / KAPPA) * np.log1p(yp)
    return shape * (u_bulk / shape.mean())


def log_law_inflow(ny: int, u_inf: float, z0: float = 0.1) -> np.ndarray:
    """Log-law inflow ln(1 + y/z0), normalised to u_inf at the top cell."""
    s = np.log1p(cell_heights(ny) / z0)
    return u_inf * s / s[-1]


def lad_constant(ny: int, a: float, h: float) -> np.ndarray:
    """Constant LAD a below the forest height h (case 1 of Table tab:forest_cases)."""
    y = cell_heights(ny)
    return np.where(y < h, a, 0.0)


def lad_gaussian(ny: int, a0: float, h: float) -> np.ndarray:
    """a(y) = a0 exp(-((y - 0.7h)/(0.3h))^2) below h (ensemble workload)."""
    y = cell_heights(ny)
    return np.where(y < h, a0 * np.exp(-(((y - 0.7 * h) / (0.3 * h)) ** 2)), 0.0)


def lad_lalic(y: np.ndarray, a_m: float, y_m: float, h: float) -> np.ndarray:
    """Eq. af_theory (Lalic & Mihailovic form): a_m ((h-y_m)/(h-y))^n
    exp[n (1 - (h-y_m)/(h-y))], n = 6 below y_m and 1/2 from y_m to h; zero
    at and above h (the limit of the expression at y -> h is 0)."""
    y = np.asarray(y, dtype=np.float64)
    out = np.zeros_like(y)
    inside = (y >= 0) & (y < h)
    r = (h - y_m) / (h - y[inside])
    n = np.where(y[inside] < y_m, 6.0, 0.5)
    out[inside] = a_m * r ** n * np.exp(n * (1.0 - r))
    return out


def lad_lalic_cells(ny: int, a_m: float, y_m: float, h: float) -> np.ndarray:
    return lad_lalic(cell_heights(ny), a_m, y_m, h)


# ---- the workloads ----------------------------------------------------------

def poiseuille(nx=32, ny=32, nz=32, g=1e-6, tau=0.8) -> Case:
    """Laminar channel: periodic x/z, halfway bounce-back at y = -1/2 and
    y = ny - 1/2, uniform body force, rho0 = 1, fluid at rest."""
    return Case("poiseuille", nx, ny, nz, bc_y=(BOUNCEBACK, BOUNCEBACK), tau0=tau, cs=0.0,
                g=(g, 0.0, 0.0), seed=SEED_BASE + 1)


def channel_params(ny=128, u_bulk=0.05, re_bulk=2800.0, re_tau=180.0):
    nu = u_bulk * ny / re_bulk
    tau0 = 3.0 * nu + 0.5
    u_tau = re_tau * nu / ny
    return nu, tau0, u_tau


def channel_les(nx=256, ny=128, nz=128) -> Case:
    """Turbulent open-channel LES: periodic x/z, bounce-back bottom, free-slip
    top, C_s = 0.1, bulk velocity driven to 0.05 by a proportional controller on
    the body force; initial log-law mean plus seeded +-5 % perturbations."""
    u_bulk = 0.05
    nu, tau0, u_tau = channel_params(ny, u_bulk)
    return Case("channel_les", nx, ny, nz, bc_y=(BOUNCEBACK, FREESLIP), tau0=tau0, cs=0.1,
                g=(u_tau ** 2 / ny, 0.0, 0.0), u_bulk_target=u_bulk, ctrl_gain=1e-2,
                seed=SEED_BASE + 2, init_perturb=0.05 * u_bulk,
                u_profile=log_law_profile(ny, u_tau, nu, u_bulk))


def canopy_abl(nx=512, ny=128, nz=256, h=10.0, a=0.2, cd=0.15, canopy_x0=128,
               u_inf=0.05, tau0=0.501, xbin=64) -> Case:
    """Forest-canopy boundary layer: constant LAD below h over x in [canopy_x0, nx),
    inflow/outflow in x, periodic z, free-slip top, bounce-back ground."""
    return Case("canopy_abl", nx, ny, nz, bc_x=(INFLOW, OUTFLOW), bc_y=(BOUNCEBACK, FREESLIP),
                tau0=tau0, cs=0.1, cd=cd, canopy_x=(canopy_x0, nx),
                stats_xbins=max(1, nx // xbin), seed=SEED_BASE + 3,
                init_perturb=0.05 * u_inf, lad=lad_constant(ny, a, h),
                u_profile=log_law_inflow(ny, u_inf))


def canopy_turbulent(nx=96, ny=24, nz=96, h=8.0, a=0.5, g=3e-5, cd=0.15, tau0=0.5005,
                     u0=0.03, perturb=0.3, seed=SEED_BASE + 5) -> Case:
    """A turbulent canopy flow cheap enough for the FP64 oracle: periodic in x,
    y and z, a dense canopy (LAD a below height h) in the lower third driven by a
    uniform body force, so shear layers form at both canopy edges (the
    inflection point of canopy flows, Sec. 5) and turn turbulent; initial
    uniform streamwise velocity u0 with seeded perturbations of perturb * 0.05
    per component.  Two runs that differ by rounding decorrelate within about
    8000 steps."""
    return Case("canopy_turbulent", nx, ny, nz, bc_y=(PERIODIC, PERIODIC), tau0=tau0, cs=0.1,
                g=(g, 0.0, 0.0), cd=cd, canopy_x=(0, nx), seed=seed,
                init_perturb=perturb * 0.05, lad=lad_constant(ny, a, h),
                u_profile=np.full(ny, u0))


def abl_forest(case: int = 1, nx: int = 160, ny: int = 64, nz: int = 128,
               u_top: float = 0.05, tau0: float = 0.501, xbin: int = 1) -> Case:
    """The paper's atmospheric boundary layer over a forest (Sec. 5): a
    1000 x 400 x 800 m domain (nx, ny, nz cells, dx = 400 m / ny), periodic in x
    and z, no-slip (bounce-back) ground, forced-equilibrium top moving with the
    free stream u_top, a forest of height 20 m over the whole ground, driven by a
    uniform body force.  Forest cases of Table tab:forest_cases: 1 = constant
    LAD 0.215 per m, 2 = Eq. af_theory with a_m = 0.38 per m at y_m = 0.7 h,
    3 = no forest.  LAD per lattice length = LAD per m * dx.  The body force
    balances a friction velocity u_* = 0.1 u_top over the domain height
    (g = u_*^2 / ny): the paper's non-dimensional force value is not used
    (its normalisation is ambiguous as printed)."""
    dx = 400.0 / ny
    h = 20.0 / dx
    if case == 1:
        lad = lad_constant(ny, 0.215 * dx, h)
    elif case == 2:
        lad = lad_lalic_cells(ny, 0.38 * dx, 0.7 * h, h)
    elif case == 3:
        lad = None
    else:
        raise ValueError("forest case is 1, 2 or 3")
    u_star = 0.1 * u_top
    return Case(f"abl_forest{case}", nx, ny, nz, bc_y=(BOUNCEBACK, EQUILIBRIUM), tau0=tau0,
                cs=0.1, g=(u_star ** 2 / ny, 0.0, 0.0), cd=0.15 if lad is not None else 0.0,
                canopy_x=(0, nx) if lad is not None else (0, 0), u_top=(u_top, 0.0, 0.0),
                stats_xbins=max(1, nx // max(1, xbin)) if xbin > 1 else 1,
                seed=SEED_BASE + 10 + case, init_perturb=0.05 * u_top,
                lad=lad, u_profile=log_law_inflow(ny, u_top))


def ensemble_boxes(n_boxes=64, ny=64, nz=64, nx_range=(96, 160), seed=SEED_BASE + 4,
                   u_tau=0.003, tau0=0.501) -> Sequence[Case]:
    """Independent canopy boxes of uneven x-length with seeded Gaussian LAD."""
    rng = np.random.default_rng(seed)
    nxs = rng.integers(nx_range[0], nx_range[1] + 1, size=n_boxes)
    a0s = rng.uniform(0.1, 0.4, size=n_boxes)
    hs = rng.choice(np.array([6.0, 8.0, 10.0, 12.0]), size=n_boxes)
    g = u_tau ** 2 / ny
    out = []
    for b in range(n_boxes):
        nx = int(nxs[b])
        out.append(Case(f"box{b}", nx, ny, nz, bc_y=(BOUNCEBACK, FREESLIP), tau0=tau0, cs=0.1,
                        g=(g, 0.0, 0.0), cd=0.15, canopy_x=(0, nx), seed=seed * 1000 + b,
                        init_perturb=0.05 * 0.05, lad=lad_gaussian(ny, float(a0s[b]), float(hs[b])),
                        u_profile=log_law_inflow(ny, 0.05)))
    return out


def taylor_green_profile(n: int, u0: float):
    """2-D Taylor-Green initial velocity on an n x n periodic x-y grid (z = 1)."""
    k = 2.0 * math.pi / n
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")  # [y][x]
    u = u0 * np.sin(k * X) * np.cos(k * Y)
    v = -u0 * np.cos(k * X) * np.sin(k * Y)
    return u, v


def small_cases():
    """Small seeded cases spanning every boundary combination, ragged sizes
    included (sizes the oracle finishes in seconds)."""
    ch = channel_les(48, 24, 20)
    cases = [
        poiseuille(32, 32, 32),
        ch,
        canopy_abl(64, 24, 16, h=6.0, canopy_x0=16, xbin=16),
        # ragged: nothing a multiple of a warp or a tile
        channel_les(37, 19, 11).replace(name="ragged_channel", lad=lad_constant(19, 0.3, 5.0),
                                        cd=0.15, canopy_x=(5, 30)),
        canopy_abl(45, 13, 7, h=4.0, canopy_x0=9, xbin=9).replace(name="ragged_canopy"),
        poiseuille(33, 17, 3).replace(name="eq_top", bc_y=(BOUNCEBACK, EQUILIBRIUM),
                                      u_top=(0.04, 0.0, 0.01), init_perturb=0.01, seed=77),
        Case("periodic_box", 24, 16, 8, bc_y=(PERIODIC, PERIODIC), tau0=0.55, cs=0.1,
             g=(1e-5, 2e-6, -1e-6), init_perturb=0.02, seed=5,
             lad=lad_gaussian(16, 0.3, 10.0), cd=0.15, canopy_x=(3, 20)),
    ]
    return cases
