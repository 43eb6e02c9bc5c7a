"""ctypes wrapper of the FP64 CPU oracle (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It mirrors the oracle's C API in
``oracle/lbm_oracle.h``; nothing here imports the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

Q = 19

PERIODIC, BOUNCEBACK, FREESLIP, EQUILIBRIUM, INFLOW, OUTFLOW = range(6)


class OlbmParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("bc_x_lo", C.c_int32), ("bc_x_hi", C.c_int32),
        ("bc_y_lo", C.c_int32), ("bc_y_hi", C.c_int32),
        ("bc_z_lo", C.c_int32), ("bc_z_hi", C.c_int32),
        ("tau0", C.c_double), ("cs", C.c_double),
        ("g", C.c_double * 3), ("cd", C.c_double),
        ("canopy_x0", C.c_int32), ("canopy_x1", C.c_int32),
        ("u_bulk_target", C.c_double), ("ctrl_gain", C.c_double),
        ("u_top", C.c_double * 3),
        ("stats_xbins", C.c_int32), ("pad0", C.c_int32),
        ("seed", C.c_uint64), ("init_perturb", C.c_double),
        ("drag_streamwise_only", C.c_int32), ("forcing_scheme", C.c_int32),
        ("sgs_rho_power", C.c_int32), ("pad1", C.c_int32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        _lib.olbm_create.restype = C.c_void_p
        _lib.olbm_create.argtypes = [C.POINTER(OlbmParams), dp, dp]
        _lib.olbm_destroy.argtypes = [C.c_void_p]
        _lib.olbm_step.argtypes = [C.c_void_p, C.c_int]
        _lib.olbm_get_f.argtypes = [C.c_void_p, dp]
        _lib.olbm_set_f.argtypes = [C.c_void_p, dp]
        _lib.olbm_macro.argtypes = [C.c_void_p, dp, dp]
        _lib.olbm_mass.restype = C.c_double
        _lib.olbm_mass.argtypes = [C.c_void_p]
        _lib.olbm_stats_reset.argtypes = [C.c_void_p, C.c_int]
        _lib.olbm_stats.restype = C.c_int64
        _lib.olbm_stats.argtypes = [C.c_void_p, dp]
        _lib.olbm_drive.argtypes = [C.c_void_p, dp, dp]
        _lib.olbm_fields.argtypes = [C.c_void_p, dp, dp, dp]
        _lib.olbm_set_layer0_accel.restype = C.c_int
        _lib.olbm_set_layer0_accel.argtypes = [C.c_void_p, dp]
        _lib.olbm_steps_done.restype = C.c_int64
        _lib.olbm_steps_done.argtypes = [C.c_void_p]
        _lib.olbm_lattice.argtypes = [C.POINTER(C.c_int32), dp]
        _lib.olbm_feq.argtypes = [C.c_double, dp, dp]
        _lib.olbm_guo.argtypes = [C.c_double, dp, dp, dp]
        _lib.olbm_tau_total.restype = C.c_double
        _lib.olbm_tau_total.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        _lib.olbm_canopy_velocity.argtypes = [dp, C.c_double, dp]
        _lib.olbm_collide_cell.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double, dp,
                                           dp, dp]
        _lib.olbm_canopy_velocity_x.argtypes = [dp, C.c_double, dp]
        _lib.olbm_tau_total_p.restype = C.c_double
        _lib.olbm_tau_total_p.argtypes = [C.c_double, C.c_double, C.c_double, dp, C.c_int]
        _lib.olbm_edm_force.argtypes = [C.c_double, dp, dp, dp]
        _lib.olbm_collide_cell_model.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double,
                                                 C.c_int, C.c_int, C.c_int, dp, dp, dp]
        _lib.olbm_splitmix64.restype = C.c_uint64
        _lib.olbm_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        _lib.olbm_uniform.restype = C.c_double
        _lib.olbm_uniform.argtypes = [C.c_uint64, C.c_uint64]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(x, n) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(n))


# ---- building blocks -------------------------------------------------------

def lattice():
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19, dtype=np.float64)
    lib().olbm_lattice(c.ctypes.data_as(C.POINTER(C.c_int32)), _dp(w))
    return c.reshape(19, 3), w


def feq(rho, u):
    u = _vec(u, 3)
    out = np.zeros(19)
    lib().olbm_feq(float(rho), _dp(u), _dp(out))
    return out


def guo(tau, u, F):
    u, F = _vec(u, 3), _vec(F, 3)
    out = np.zeros(19)
    lib().olbm_guo(float(tau), _dp(u), _dp(F), _dp(out))
    return out


def tau_total(tau0, cs, rho, pineq6):
    p = _vec(pineq6, 6)
    return lib().olbm_tau_total(float(tau0), float(cs), float(rho), _dp(p))


def canopy_velocity(v, k):
    v = _vec(v, 3)
    u = np.zeros(3)
    lib().olbm_canopy_velocity(_dp(v), float(k), _dp(u))
    return u


def canopy_velocity_x(v, k):
    v = _vec(v, 3)
    u = np.zeros(3)
    lib().olbm_canopy_velocity_x(_dp(v), float(k), _dp(u))
    return u


def tau_total_p(tau0, cs, rho, pineq6, p):
    q = _vec(pineq6, 6)
    return lib().olbm_tau_total_p(float(tau0), float(cs), float(rho), _dp(q), int(p))


def edm_force(rho, u, g):
    u, g = _vec(u, 3), _vec(g, 3)
    out = np.zeros(19)
    lib().olbm_edm_force(float(rho), _dp(u), _dp(g), _dp(out))
    return out


def collide_cell_model(fin, g_drive, k, tau0, cs, drag_x_only=0, scheme=0, rho_power=1):
    fin, g = _vec(fin, 19), _vec(g_drive, 3)
    fout, rho, u = np.zeros(19), np.zeros(1), np.zeros(3)
    lib().olbm_collide_cell_model(_dp(fin), _dp(g), float(k), float(tau0), float(cs),
                                  int(drag_x_only), int(scheme), int(rho_power), _dp(fout),
                                  _dp(rho), _dp(u))
    return fout, float(rho[0]), u


def collide_cell(fin, g_drive, k, tau0, cs):
    fin, g = _vec(fin, 19), _vec(g_drive, 3)
    fout, rho, u = np.zeros(19), np.zeros(1), np.zeros(3)
    lib().olbm_collide_cell(_dp(fin), _dp(g), float(k), float(tau0), float(cs), _dp(fout),
                            _dp(rho), _dp(u))
    return fout, float(rho[0]), u


def splitmix64(seed, n):
    return int(lib().olbm_splitmix64(int(seed), int(n)))


def uniform(seed, n):
    return lib().olbm_uniform(int(seed), int(n))


# ---- a domain --------------------------------------------------------------

class Oracle:
    """One FP64 domain; argument names follow ``workloads.Case``."""

    def __init__(self, case):
        p = OlbmParams()
        p.nx, p.ny, p.nz = case.nx, case.ny, case.nz
        p.bc_x_lo, p.bc_x_hi = case.bc_x
        p.bc_y_lo, p.bc_y_hi = case.bc_y
        p.bc_z_lo, p.bc_z_hi = case.bc_z
        p.tau0, p.cs = case.tau0, case.cs
        p.g[:] = list(case.g)
        p.cd = case.cd
        p.canopy_x0, p.canopy_x1 = case.canopy_x
        p.u_bulk_target, p.ctrl_gain = case.u_bulk_target, case.ctrl_gain
        p.u_top[:] = list(case.u_top)
        p.stats_xbins = case.stats_xbins
        p.seed, p.init_perturb = case.seed, case.init_perturb
        p.drag_streamwise_only = case.drag_streamwise_only
        p.forcing_scheme = case.forcing_scheme
        p.sgs_rho_power = case.sgs_rho_power
        self.case = case
        self.shape = (case.nz, case.ny, case.nx)
        self.n = case.nx * case.ny * case.nz
        self._lad = None if case.lad is None else _vec(case.lad, case.ny)
        self._uprof = None if case.u_profile is None else _vec(case.u_profile, case.ny)
        nullp = C.POINTER(C.c_double)()
        h = lib().olbm_create(C.byref(p),
                              nullp if self._lad is None else _dp(self._lad),
                              nullp if self._uprof is None else _dp(self._uprof))
        if not h:
            raise ValueError("olbm_create rejected the parameters")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().olbm_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def step(self, n=1):
        lib().olbm_step(self._h, int(n))

    def get_f(self):
        f = np.zeros((Q,) + self.shape)
        lib().olbm_get_f(self._h, _dp(f))
        return f

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((Q,) + self.shape)
        lib().olbm_set_f(self._h, _dp(f))

    def macro(self):
        rho = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        lib().olbm_macro(self._h, _dp(rho), _dp(u))
        return rho, u

    def mass(self):
        return lib().olbm_mass(self._h)

    def stats_reset(self, enable=True):
        lib().olbm_stats_reset(self._h, int(bool(enable)))

    def stats(self):
        out = np.zeros((9, self.case.stats_xbins, self.case.ny))
        n = lib().olbm_stats(self._h, _dp(out))
        return out, int(n)

    def drive(self):
        g, ub = np.zeros(3), np.zeros(1)
        lib().olbm_drive(self._h, _dp(g), _dp(ub))
        return g, float(ub[0])

    def steps_done(self):
        return int(lib().olbm_steps_done(self._h))

    # ---- learned first-layer correction (inputs and application) ----------------

    def fields(self):
        """rho, u and |S| that the next step computes (no layer-0 correction)."""
        rho = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        strain = np.zeros(self.shape)
        lib().olbm_fields(self._h, _dp(rho), _dp(u), _dp(strain))
        return rho, u, strain

    def features(self):
        """Correction inputs per first-cell column, rows in (z, x) order:
        u_x at y = 0, 1, 2, |S| at y = 0, 1, 2, leaf-area density at y = 0, 1, 2
        (zero outside the canopy's x-range)."""
        _, u, strain = self.fields()
        c = self.case
        nz, nx = c.nz, c.nx
        lad = np.zeros((3, nx))
        if c.lad is not None:
            x = np.arange(nx)
            inside = (x >= c.canopy_x[0]) & (x < c.canopy_x[1])
            for y in range(3):
                lad[y] = np.where(inside, c.lad[y], 0.0)
        X = np.zeros((nz, nx, 9))
        for y in range(3):
            X[:, :, y] = u[0, :, y, :]
            X[:, :, 3 + y] = strain[:, y, :]
            X[:, :, 6 + y] = lad[y][None, :]
        return X.reshape(nz * nx, 9)

    def set_layer0_accel(self, a):
        """Extra (x, z) acceleration of the cells at y = 0, shape (nz, nx, 2),
        applied by every following step; None switches it off."""
        if a is None:
            lib().olbm_set_layer0_accel(self._h, C.POINTER(C.c_double)())
            return
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(self.case.nz, self.case.nx, 2)
        self._accel0 = a
        if lib().olbm_set_layer0_accel(self._h, _dp(a)) != 0:
            raise MemoryError("olbm_set_layer0_accel")


def omp_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
