"""Training data and training for the learned first-layer correction.

The plain method (no wall function, no correction) is run on the coarse grid
and on the same physical set-up at twice the resolution; the fine run's mean
profiles, coarsened, are the reference for the coarse run.  The network learns, from
the coarse run's instantaneous column features, the time-averaged deficits of
the coarse first cell (one cell high, wall half a cell below its centre) at
that x-position:

    du_x, du_z     = <u>_fine->coarse(first cell) - <u>_coarse(first cell)
    dtau_x, dtau_z = R_fine - R_coarse,   R = tau_wall - tau_top

where R is the net retarding shear stress on the first cell: the wall stress
nu <u>_0 / (1/2) minus the stress through its top face, nu d<u>/dy - <u'v'>
(viscous plus resolved turbulent flux, from the time-averaged profiles).
Applied as the extra acceleration lam * du - dtau of the first cells, the
stress term supplies the momentum flux the coarse grid misses and the velocity
term relaxes the first cell towards the fine-grid mean at rate lam.

Everything here is orchestration (which runs, what to average, how to pair
features with targets); the steps, the features, the network and its training
all run in the CUDA library.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import LBM_F32, CorrectionNet, Domain


def refine(case, factor: int = 2):
    """The same physical set-up on a grid `factor` times finer in every
    direction, at equal lattice velocity (dt_fine = dt / factor): viscosity in
    lattice units grows by `factor`, accelerations shrink by it, leaf-area
    density per cell length shrinks by it, heights and x-ranges scale by it."""
    f = factor
    ny = case.ny * f

    yf = (np.arange(ny) + 0.5) / f  # fine cell centres in coarse cell units

    def cellwise(profile):  # piecewise constant per coarse cell (leaf-area density)
        return np.asarray(profile, dtype=np.float64)[np.minimum(yf.astype(int), case.ny - 1)]

    def smooth(profile):    # interpolated between coarse cell centres (velocity)
        return np.interp(yf, np.arange(case.ny) + 0.5, np.asarray(profile, dtype=np.float64))

    lad = None if case.lad is None else cellwise(case.lad) / f
    nu = (case.tau0 - 0.5) / 3.0
    return dataclasses.replace(
        case, name=case.name + f"_x{f}", nx=case.nx * f, ny=ny, nz=case.nz * f,
        tau0=0.5 + 3.0 * nu * f, g=tuple(v / f for v in case.g),
        canopy_x=(case.canopy_x[0] * f, case.canopy_x[1] * f), lad=lad,
        u_profile=None if case.u_profile is None else smooth(case.u_profile),
        seed=case.seed + 7919)


def _first_cell(stats, nu: float, fine: bool):
    """Per x-bin: mean (u, w) of the first coarse cell and its net retarding
    shear stress (x, z) R = tau_wall - tau_top, in coarse lattice units (the
    same numbers on both grids at equal lattice velocity).  A fine run's first
    coarse cell is its two lowest rows; its top face lies between rows 1 and 2."""
    u, w, uv, vw = stats[0], stats[2], stats[6], stats[8]
    if fine:
        mu, mw = 0.5 * (u[:, 0] + u[:, 1]), 0.5 * (w[:, 0] + w[:, 1])
        wall_x, wall_z = nu * u[:, 0] / 0.5, nu * w[:, 0] / 0.5       # fine cell units
        top_x = nu * (u[:, 2] - u[:, 1]) - 0.5 * (uv[:, 1] + uv[:, 2])
        top_z = nu * (w[:, 2] - w[:, 1]) - 0.5 * (vw[:, 1] + vw[:, 2])
    else:
        mu, mw = u[:, 0], w[:, 0]
        wall_x, wall_z = nu * u[:, 0] / 0.5, nu * w[:, 0] / 0.5
        top_x = nu * (u[:, 1] - u[:, 0]) - 0.5 * (uv[:, 0] + uv[:, 1])
        top_z = nu * (w[:, 1] - w[:, 0]) - 0.5 * (vw[:, 0] + vw[:, 1])
    return mu, mw, wall_x - top_x, wall_z - top_z


@dataclasses.dataclass
class Reference:
    """Time-averaged profiles of the plain coarse and fine runs (per x-bin)."""
    coarse: np.ndarray          # [9][xbins][ny] statistics of the coarse run
    fine_coarsened: np.ndarray  # [3][xbins][ny] mean velocity of the fine run on coarse cells
    targets: np.ndarray         # [xbins][4]: du_x, du_z, dtau_x, dtau_z
    features: np.ndarray        # [samples][9] coarse-run features
    labels: np.ndarray          # [samples][4]


def coarsen_means(fine_stats):
    """Mean velocity of a fine run averaged onto coarse cells (pairs of rows;
    the x-bins already cover whole coarse columns, z is averaged)."""
    m = fine_stats[:3]
    return 0.5 * (m[:, :, 0::2] + m[:, :, 1::2])


def reference_runs(case, spinup: int, average: int, sample_every: int = 20,
                   storage=LBM_F32, fine_storage=None) -> Reference:
    """Run the plain method on `case` (coarse) and on refine(case) for the same
    physical time, average their profiles per x-bin, and collect the coarse
    run's column features every `sample_every` steps of the averaging window,
    each paired with the deficits of its x-bin.  The fine run may use another
    storage (fine_storage; e.g. the in-place AA layout, which halves the
    memory of a grid with eight times the cells)."""
    fine_case = refine(case)
    nb = case.stats_xbins
    assert fine_case.stats_xbins == nb and case.nx % nb == 0
    fine = Domain(fine_case, storage if fine_storage is None else fine_storage)
    fine.step(2 * spinup)
    fine.stats_reset(True)
    fine.step(2 * average)
    fs, _ = fine.stats()
    fine.close()

    coarse = Domain(case, storage)
    coarse.step(spinup)
    coarse.stats_reset(True)
    feats, bins = [], []
    col_bin = (np.arange(case.nx) * nb) // case.nx
    for k in range(average // sample_every):
        coarse.step(sample_every)
        X = coarse.features()
        feats.append(X)
        bins.append(np.tile(col_bin, case.nz))
    cs, _ = coarse.stats()
    coarse.close()

    nu_c = (case.tau0 - 0.5) / 3.0
    nu_f = (fine_case.tau0 - 0.5) / 3.0
    uf, wf, rfx, rfz = _first_cell(fs, nu_f, fine=True)
    uc, wc, rcx, rcz = _first_cell(cs, nu_c, fine=False)
    targets = np.stack([uf - uc, wf - wc, rfx - rcx, rfz - rcz], axis=1)
    X = np.concatenate(feats).astype(np.float32)
    Y = targets[np.concatenate(bins)].astype(np.float32)
    return Reference(coarse=cs, fine_coarsened=coarsen_means(fs), targets=targets,
                     features=X, labels=Y)


def train_correction(ref: Reference, epochs: int = 40, batch: int = 1024, lr: float = 2e-3,
                     seed: int = 1) -> tuple:
    """A CorrectionNet fitted to the reference's (features, labels); returns
    (net, first-epoch loss, last-epoch loss)."""
    net = CorrectionNet(seed=seed)
    l0, l1 = net.train(ref.features, ref.labels, epochs=epochs, batch=batch, lr=lr, seed=seed)
    return net, l0, l1


def corrected_run(case, net, lam: float, spinup: int, average: int, storage=LBM_F32,
                  plain=None):
    """Statistics of the coarse run with the correction on (from the start of
    the averaging window), and of the same run without it (`plain`: those
    statistics already taken, e.g. Reference.coarse of the same case, window and
    storage, which the deterministic step reproduces)."""
    out = [] if plain is None else [plain]
    for use in ((False, True) if plain is None else (True,)):
        d = Domain(case, storage)
        d.step(spinup)
        if use:
            d.set_correction(net, lam)
        d.stats_reset(True)
        d.step(average)
        s, _ = d.stats()
        d.close()
        out.append(s)
    return out[0], out[1]


def profile_error(stats, fine_coarsened, rows: int) -> float:
    """Relative L2 error of the mean streamwise velocity over the lowest `rows`
    cells of every x-bin against the coarsened fine run."""
    a = stats[0][:, :rows]
    b = fine_coarsened[0][:, :rows]
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
