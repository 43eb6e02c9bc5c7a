"""B300 (sm_103a) D3Q19 LBM-LES library for forest-canopy boundary layers.

Thin ctypes binding of the C ABI in ``include/lbm.h`` (same function names,
argument marshalling only).  Every step of the method runs in the CUDA
kernels of ``csrc/``; PyTorch only supplies device memory (the workspace) and
the stream.  There is no CPU fallback: if the shared library is missing the
import of any entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblbm_b300.so")

Q = 19
LBM_OK, LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_NAN, LBM_ERR_TIMEOUT, \
    LBM_ERR_STATE, LBM_ERR_IO, LBM_ERR_BOUNDS = range(9)
LBM_BC_PERIODIC, LBM_BC_BOUNCEBACK, LBM_BC_FREESLIP, LBM_BC_EQUILIBRIUM, LBM_BC_INFLOW, \
    LBM_BC_OUTFLOW, LBM_BC_HALO = range(7)
LBM_FORCE_GUO, LBM_FORCE_EXACT_DIFFERENCE = range(2)
LBM_F32, LBM_F16_SHIFTED, LBM_BF16_SHIFTED = range(3)
LBM_STORAGE_AA = 0x100  # or-ed into a storage type: AA-pattern in-place storage (one set)
STORAGE_NAMES = {"f32": LBM_F32, "f16s": LBM_F16_SHIFTED, "bf16s": LBM_BF16_SHIFTED,
                 "f32-aa": LBM_F32 | LBM_STORAGE_AA, "f16s-aa": LBM_F16_SHIFTED | LBM_STORAGE_AA,
                 "bf16s-aa": LBM_BF16_SHIFTED | LBM_STORAGE_AA}
_BYTES = {LBM_F32: 152, LBM_F16_SHIFTED: 76, LBM_BF16_SHIFTED: 76}
BYTES_PER_LUP = {k: _BYTES[k & 0xFF] for k in STORAGE_NAMES.values()}


class LbmGrid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("x_lo", C.c_int32), ("x_hi", C.c_int32), ("y_lo", C.c_int32),
                ("y_hi", C.c_int32), ("z_lo", C.c_int32), ("z_hi", C.c_int32)]


class LbmForcing(C.Structure):
    _fields_ = [("g", C.c_double * 3), ("cd", C.c_double),
                ("x_canopy_begin", C.c_int32), ("x_canopy_end", C.c_int32),
                ("u_bulk_target", C.c_double), ("ctrl_gain", C.c_double),
                ("u_top", C.c_double * 3), ("u_in_profile", C.POINTER(C.c_double)),
                ("drag_streamwise_only", C.c_int32), ("scheme", C.c_int32),
                ("sgs_rho_power", C.c_int32), ("reserved", C.c_int32)]


class LbmBox(C.Structure):
    _fields_ = [("grid", LbmGrid), ("tau0", C.c_double), ("cs", C.c_double),
                ("lad", C.POINTER(C.c_double)), ("forcing", LbmForcing), ("seed", C.c_uint64)]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None
_DP = C.POINTER(C.c_double)


def lib():
    """Load the in-tree CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LbmError(LBM_ERR_CUDA, f"CUDA library missing: {LIB_PATH} (build it with python -m paper_2206_15454_b300.build)")
        L = C.CDLL(LIB_PATH)
        vp, st = C.c_void_p, C.c_int32
        L.lbm_workspace_bytes.restype = C.c_size_t
        L.lbm_workspace_bytes.argtypes = [C.POINTER(LbmGrid), C.c_int32, C.c_int32]
        L.lbm_create.restype = st
        L.lbm_create.argtypes = [C.POINTER(LbmGrid), C.c_double, C.c_double, _DP,
                                 C.POINTER(LbmForcing), C.c_int32, C.c_int32, C.c_uint64,
                                 C.c_double, vp, C.c_size_t, C.POINTER(vp)]
        for name, args in [("lbm_set_stream", [vp, vp]), ("lbm_step", [vp, C.c_int32]),
                           ("lbm_sync", [vp]), ("lbm_stats_reset", [vp, C.c_int32]),
                           ("lbm_stats", [vp, _DP, C.c_size_t, C.POINTER(C.c_int64)]),
                           ("lbm_stats_begin", [vp]),
                           ("lbm_stats_end", [vp, _DP, C.c_size_t, C.POINTER(C.c_int64)]),
                           ("lbm_mass", [vp, _DP]), ("lbm_get_f", [vp, _DP, C.c_size_t]),
                           ("lbm_set_f", [vp, _DP, C.c_size_t]),
                           ("lbm_get_macro", [vp, _DP, _DP, C.c_size_t]),
                           ("lbm_get_macro_noalloc", [vp, _DP, _DP, C.c_size_t]),
                           ("lbm_get_q", [vp, _DP, C.c_size_t]),
                           ("lbm_test_withhold_fill", [vp, C.c_int32]),
                           ("lbm_halo_pack", [vp, vp, vp]), ("lbm_halo_unpack", [vp, vp, vp]),
                           ("lbm_drive", [vp, _DP, _DP]), ("lbm_save", [vp, C.c_char_p]),
                           ("lbm_load", [vp, C.c_char_p])]:
            fn = getattr(L, name)
            fn.restype = st
            fn.argtypes = args
        bp = C.POINTER(LbmBox)
        L.lbm_batch_workspace_bytes.restype = C.c_size_t
        L.lbm_batch_workspace_bytes.argtypes = [C.c_int32, bp, C.c_int32, C.c_int32]
        L.lbm_batch_create.restype = st
        L.lbm_batch_create.argtypes = [C.c_int32, bp, C.c_int32, C.c_int32, C.c_double, C.c_int32,
                                       vp, vp, C.c_size_t, C.POINTER(vp)]
        for name, args in [("lbm_batch_step", [vp, C.c_int32]), ("lbm_batch_sync", [vp]),
                           ("lbm_batch_stats_reset", [vp, C.c_int32]),
                           ("lbm_batch_tuning", [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                                 _DP])]:
            fn = getattr(L, name)
            fn.restype = st
            fn.argtypes = args
        FP = C.POINTER(C.c_float)
        L.lbm_mlp_create.restype = st
        L.lbm_mlp_create.argtypes = [C.c_uint64, vp, C.POINTER(vp)]
        for name, args in [("lbm_mlp_params", [vp, FP, C.c_size_t]),
                           ("lbm_mlp_set_params", [vp, FP, C.c_size_t]),
                           ("lbm_mlp_forward", [vp, FP, C.c_int64, FP]),
                           ("lbm_mlp_gradient", [vp, FP, FP, C.c_int64, FP, C.c_size_t, FP]),
                           ("lbm_mlp_train", [vp, FP, FP, C.c_int64, C.c_int32, C.c_int32,
                                              C.c_float, C.c_uint64, FP, FP]),
                           ("lbm_set_correction", [vp, vp, C.c_double]),
                           ("lbm_features", [vp, FP, C.c_size_t]),
                           ("lbm_correction_field", [vp, FP, C.c_size_t])]:
            fn = getattr(L, name)
            fn.restype = st
            fn.argtypes = args
        L.lbm_mlp_destroy.restype = None
        L.lbm_mlp_destroy.argtypes = [vp]
        L.lbm_mlp_last_error.restype = C.c_char_p
        L.lbm_mlp_last_error.argtypes = [vp]
        L.lbm_batch_candidates.restype = C.c_int32
        L.lbm_batch_candidates.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _DP,
                                           C.c_int32]
        L.lbm_batch_box.restype = vp
        L.lbm_batch_box.argtypes = [vp, C.c_int32]
        L.lbm_batch_destroy.restype = None
        L.lbm_batch_destroy.argtypes = [vp]
        L.lbm_batch_last_error.restype = C.c_char_p
        L.lbm_batch_last_error.argtypes = [vp]
        L.lbm_halo_bytes.restype = C.c_size_t
        L.lbm_halo_bytes.argtypes = [vp]
        L.lbm_steps_done.restype = C.c_int64
        L.lbm_steps_done.argtypes = [vp]
        L.lbm_destroy.restype = None
        L.lbm_destroy.argtypes = [vp]
        L.lbm_last_error.restype = C.c_char_p
        L.lbm_last_error.argtypes = [vp]
        L.lbm_status_string.restype = C.c_char_p
        L.lbm_status_string.argtypes = [C.c_int32]
        _lib = L
    return _lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _check(status, ctx=None, what=""):
    if status != LBM_OK:
        msg = lib().lbm_last_error(ctx).decode() if ctx else ""
        base = lib().lbm_status_string(status).decode()
        raise LbmError(status, f"{what}: {base}{(' - ' + msg) if msg else ''}")


# ---- the C entry points, one to one -------------------------------------------------

def lbm_workspace_bytes(grid: LbmGrid, storage: int, stats_xbins: int) -> int:
    return int(lib().lbm_workspace_bytes(C.byref(grid), storage, stats_xbins))


def lbm_create(grid, tau0, cs, lad, forcing, storage, stats_xbins, seed, init_perturb,
               workspace=0, workspace_bytes=0):
    ctx = C.c_void_p()
    lad_p = _dp(lad) if lad is not None else _DP()
    s = lib().lbm_create(C.byref(grid), tau0, cs, lad_p, C.byref(forcing), storage,
                         stats_xbins, seed, init_perturb, C.c_void_p(workspace or None),
                         workspace_bytes, C.byref(ctx))
    _check(s, None, "lbm_create")
    return ctx


def lbm_set_stream(ctx, stream_ptr):
    _check(lib().lbm_set_stream(ctx, C.c_void_p(stream_ptr or None)), ctx, "lbm_set_stream")


def lbm_step(ctx, n):
    _check(lib().lbm_step(ctx, int(n)), ctx, "lbm_step")


def lbm_sync(ctx):
    _check(lib().lbm_sync(ctx), ctx, "lbm_sync")


def lbm_stats_reset(ctx, enable=True):
    _check(lib().lbm_stats_reset(ctx, int(bool(enable))), ctx, "lbm_stats_reset")


def lbm_stats(ctx, out: np.ndarray):
    n = C.c_int64()
    _check(lib().lbm_stats(ctx, _dp(out), out.size, C.byref(n)), ctx, "lbm_stats")
    return int(n.value)


def lbm_stats_begin(ctx):
    _check(lib().lbm_stats_begin(ctx), ctx, "lbm_stats_begin")


def lbm_stats_end(ctx, out: np.ndarray):
    n = C.c_int64()
    _check(lib().lbm_stats_end(ctx, _dp(out), out.size, C.byref(n)), ctx, "lbm_stats_end")
    return int(n.value)


def lbm_get_q(ctx, q: np.ndarray):
    _check(lib().lbm_get_q(ctx, _dp(q), q.size), ctx, "lbm_get_q")


def lbm_test_withhold_fill(ctx, fill):
    _check(lib().lbm_test_withhold_fill(ctx, fill), ctx, "lbm_test_withhold_fill")


def lbm_mass(ctx):
    out = np.zeros(1)
    _check(lib().lbm_mass(ctx, _dp(out)), ctx, "lbm_mass")
    return float(out[0])


def lbm_get_f(ctx, out: np.ndarray):
    _check(lib().lbm_get_f(ctx, _dp(out), out.size), ctx, "lbm_get_f")


def lbm_set_f(ctx, f: np.ndarray):
    _check(lib().lbm_set_f(ctx, _dp(f), f.size), ctx, "lbm_set_f")


def lbm_get_macro(ctx, rho: np.ndarray, u: np.ndarray):
    _check(lib().lbm_get_macro(ctx, _dp(rho), _dp(u), rho.size), ctx, "lbm_get_macro")


def lbm_get_macro_noalloc(ctx, rho: np.ndarray, u: np.ndarray):
    """lbm_get_macro without device allocation (static field buffer, <= 262144 cells)."""
    _check(lib().lbm_get_macro_noalloc(ctx, _dp(rho), _dp(u), rho.size), ctx,
           "lbm_get_macro_noalloc")


def lbm_halo_bytes(ctx) -> int:
    return int(lib().lbm_halo_bytes(ctx))


def lbm_halo_pack(ctx, to_lo: int, to_hi: int):
    """Pack the slab's outgoing faces into two device buffers (pointers)."""
    _check(lib().lbm_halo_pack(ctx, C.c_void_p(to_lo), C.c_void_p(to_hi)), ctx, "lbm_halo_pack")


def lbm_halo_unpack(ctx, from_lo: int, from_hi: int):
    """Write received faces (device buffers) into the slab's halo ghost slots."""
    _check(lib().lbm_halo_unpack(ctx, C.c_void_p(from_lo), C.c_void_p(from_hi)), ctx,
           "lbm_halo_unpack")


def lbm_drive(ctx):
    g, ub = np.zeros(3), np.zeros(1)
    _check(lib().lbm_drive(ctx, _dp(g), _dp(ub)), ctx, "lbm_drive")
    return g, float(ub[0])


def lbm_save(ctx, path):
    _check(lib().lbm_save(ctx, str(path).encode()), ctx, "lbm_save")


def lbm_load(ctx, path):
    _check(lib().lbm_load(ctx, str(path).encode()), ctx, "lbm_load")


def lbm_steps_done(ctx):
    return int(lib().lbm_steps_done(ctx))


def lbm_destroy(ctx):
    lib().lbm_destroy(ctx)


# ---- learned first-layer correction ---------------------------------------------------

MLP_PARAMS, MLP_WEIGHTS, MLP_IN, MLP_OUT = 9246, 9220, 9, 4
_FP = C.POINTER(C.c_float)


def _fp(a):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(_FP)


def _mlp_check(status, m, what):
    if status != LBM_OK:
        msg = lib().lbm_mlp_last_error(m).decode() if m else ""
        base = lib().lbm_status_string(status).decode()
        raise LbmError(status, f"{what}: {base}{(' - ' + msg) if msg else ''}")


def lbm_mlp_create(seed, stream_ptr=0):
    m = C.c_void_p()
    _mlp_check(lib().lbm_mlp_create(seed, C.c_void_p(stream_ptr or None), C.byref(m)), None,
               "lbm_mlp_create")
    return m


def lbm_mlp_params(m):
    th = np.zeros(MLP_PARAMS, dtype=np.float32)
    _mlp_check(lib().lbm_mlp_params(m, _fp(th), th.size), m, "lbm_mlp_params")
    return th


def lbm_mlp_set_params(m, theta):
    th = np.ascontiguousarray(theta, dtype=np.float32)
    _mlp_check(lib().lbm_mlp_set_params(m, _fp(th), th.size), m, "lbm_mlp_set_params")


def lbm_mlp_forward(m, X):
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, MLP_IN)
    Y = np.zeros((X.shape[0], MLP_OUT), dtype=np.float32)
    _mlp_check(lib().lbm_mlp_forward(m, _fp(X), X.shape[0], _fp(Y)), m, "lbm_mlp_forward")
    return Y


def lbm_mlp_gradient(m, X, Y):
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, MLP_IN)
    Y = np.ascontiguousarray(Y, dtype=np.float32).reshape(-1, MLP_OUT)
    g = np.zeros(MLP_WEIGHTS, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _mlp_check(lib().lbm_mlp_gradient(m, _fp(X), _fp(Y), X.shape[0], _fp(g), g.size, _fp(loss)),
               m, "lbm_mlp_gradient")
    return g, float(loss[0])


def lbm_mlp_train(m, X, Y, epochs, batch, lr, seed=1):
    X = np.ascontiguousarray(X, dtype=np.float32).reshape(-1, MLP_IN)
    Y = np.ascontiguousarray(Y, dtype=np.float32).reshape(-1, MLP_OUT)
    l0, l1 = np.zeros(1, dtype=np.float32), np.zeros(1, dtype=np.float32)
    _mlp_check(lib().lbm_mlp_train(m, _fp(X), _fp(Y), X.shape[0], epochs, batch, lr, seed,
                                   _fp(l0), _fp(l1)), m, "lbm_mlp_train")
    return float(l0[0]), float(l1[0])


def lbm_mlp_destroy(m):
    lib().lbm_mlp_destroy(m)


def lbm_set_correction(ctx, m, lam):
    _check(lib().lbm_set_correction(ctx, m, float(lam)), ctx, "lbm_set_correction")


def lbm_features(ctx, n_columns):
    X = np.zeros((n_columns, MLP_IN), dtype=np.float32)
    _check(lib().lbm_features(ctx, _fp(X), X.size), ctx, "lbm_features")
    return X


def lbm_correction_field(ctx, n_columns):
    a = np.zeros((n_columns, 2), dtype=np.float32)
    _check(lib().lbm_correction_field(ctx, _fp(a), a.size), ctx, "lbm_correction_field")
    return a


class CorrectionNet:
    """The learned first-layer correction network (see include/lbm.h)."""

    def __init__(self, seed=1, stream=None):
        import torch

        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.m = lbm_mlp_create(seed, self.stream.cuda_stream)

    def params(self):
        return lbm_mlp_params(self.m)

    def set_params(self, theta):
        lbm_mlp_set_params(self.m, theta)

    def forward(self, X):
        return lbm_mlp_forward(self.m, X)

    def gradient(self, X, Y):
        return lbm_mlp_gradient(self.m, X, Y)

    def train(self, X, Y, epochs=20, batch=1024, lr=1e-3, seed=1):
        return lbm_mlp_train(self.m, X, Y, epochs, batch, lr, seed)

    def close(self):
        if getattr(self, "m", None) is not None:
            lbm_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- ensembles ----------------------------------------------------------------------

def _batch_check(status, b, what):
    if status != LBM_OK:
        msg = lib().lbm_batch_last_error(b).decode() if b else ""
        base = lib().lbm_status_string(status).decode()
        raise LbmError(status, f"{what}: {base}{(' - ' + msg) if msg else ''}")


def lbm_batch_workspace_bytes(boxes, storage: int, stats_xbins: int) -> int:
    return int(lib().lbm_batch_workspace_bytes(len(boxes), boxes, storage, stats_xbins))


def lbm_batch_create(boxes, storage, stats_xbins, init_perturb, tune_steps=0, stream_ptr=0,
                     workspace=0, workspace_bytes=0):
    b = C.c_void_p()
    s = lib().lbm_batch_create(len(boxes), boxes, storage, stats_xbins, init_perturb, tune_steps,
                               C.c_void_p(stream_ptr or None), C.c_void_p(workspace or None),
                               workspace_bytes, C.byref(b))
    _batch_check(s, None, "lbm_batch_create")
    return b


def lbm_batch_step(b, n):
    _batch_check(lib().lbm_batch_step(b, int(n)), b, "lbm_batch_step")


def lbm_batch_sync(b):
    _batch_check(lib().lbm_batch_sync(b), b, "lbm_batch_sync")


def lbm_batch_stats_reset(b, enable=True):
    _batch_check(lib().lbm_batch_stats_reset(b, int(bool(enable))), b, "lbm_batch_stats_reset")


def lbm_batch_box(b, i):
    return C.c_void_p(lib().lbm_batch_box(b, int(i)))


def lbm_batch_tuning(b):
    xt, nb, ms = C.c_int32(), C.c_int32(), np.zeros(1)
    _batch_check(lib().lbm_batch_tuning(b, C.byref(xt), C.byref(nb), _dp(ms)), b,
                 "lbm_batch_tuning")
    return int(xt.value), int(nb.value), float(ms[0])


def lbm_batch_candidates(b, cap=64):
    """[(chunk width, blocks per launch, ms per step)] for every candidate the tuner timed."""
    xt, nb, ms = (C.c_int32 * cap)(), (C.c_int32 * cap)(), np.zeros(cap)
    n = int(lib().lbm_batch_candidates(b, xt, nb, _dp(ms), cap))
    return [(int(xt[k]), int(nb[k]), float(ms[k])) for k in range(min(max(n, 0), cap))]


def lbm_batch_destroy(b):
    lib().lbm_batch_destroy(b)


# ---- convenience: one domain with a PyTorch-owned workspace and stream ---------------

class Domain:
    """A simulation domain.  ``case`` is any object with the attributes of
    ``workloads.Case`` (nx, ny, nz, bc_x/bc_y/bc_z pairs, tau0, cs, g, cd,
    canopy_x, u_bulk_target, ctrl_gain, u_top, stats_xbins, seed,
    init_perturb, lad, u_profile)."""

    _owned = True

    def __init__(self, case, storage=LBM_F32, use_torch_workspace=True, stream=None):
        import torch

        if isinstance(storage, str):
            storage = STORAGE_NAMES[storage]
        self.case, self.storage = case, storage
        self.shape = (case.nz, case.ny, case.nx)
        self.cells = case.nx * case.ny * case.nz
        g, fo, lad, keep = _case_inputs(case)
        self._keep = keep
        self.workspace = None
        ws_ptr, ws_bytes = 0, 0
        if use_torch_workspace:
            ws_bytes = lbm_workspace_bytes(g, storage, case.stats_xbins)
            if ws_bytes == 0:
                raise LbmError(LBM_ERR_ARG, "lbm_workspace_bytes: invalid grid/storage/bins")
            self.workspace = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
            ws_ptr = self.workspace.data_ptr()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        torch.cuda.synchronize()
        self.ctx = lbm_create(g, case.tau0, case.cs, lad, fo, storage, case.stats_xbins,
                              case.seed, case.init_perturb, ws_ptr, ws_bytes)
        lbm_set_stream(self.ctx, self.stream.cuda_stream)

    @classmethod
    def _view(cls, ctx, case, storage, stream, owner):
        """A box of an ensemble: same readouts, owned (and freed) by the ensemble."""
        d = cls.__new__(cls)
        d.case, d.storage, d.ctx, d.stream, d.workspace = case, storage, ctx, stream, None
        d.shape = (case.nz, case.ny, case.nx)
        d.cells = case.nx * case.ny * case.nz
        d._owned, d._owner = False, owner
        return d

    def close(self):
        if getattr(self, "ctx", None) is not None and self._owned:
            lbm_destroy(self.ctx)
        self.ctx = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def sync(self):
        lbm_sync(self.ctx)

    def get_f(self):
        f = np.zeros((Q,) + self.shape)
        lbm_get_f(self.ctx, f)
        return f

    def set_f(self, f):
        lbm_set_f(self.ctx, np.ascontiguousarray(f, dtype=np.float64))

    def macro(self):
        rho, u = np.zeros(self.shape), np.zeros((3,) + self.shape)
        lbm_get_macro(self.ctx, rho, u)
        return rho, u

    def q_criterion(self):
        """Q-criterion [z][y][x] of the velocity field the next step computes."""
        q = np.zeros(self.shape)
        lbm_get_q(self.ctx, q)
        return q

    def mass(self):
        return lbm_mass(self.ctx)

    def stats_reset(self, enable=True):
        lbm_stats_reset(self.ctx, enable)

    def stats(self):
        out = np.zeros((9, self.case.stats_xbins, self.case.ny))
        n = lbm_stats(self.ctx, out)
        return out, n

    def stats_begin(self):
        """Enqueue a read-out of the statistics after the work enqueued so far
        (at most two pending)."""
        lbm_stats_begin(self.ctx)

    def stats_end(self, out=None):
        """The oldest pending read-out, as stats() would have returned it at
        the matching stats_begin()."""
        if out is None:
            out = np.zeros((9, self.case.stats_xbins, self.case.ny))
        n = lbm_stats_end(self.ctx, out)
        return out, n

    def drive(self):
        return lbm_drive(self.ctx)

    def save(self, path):
        lbm_save(self.ctx, path)

    def load(self, path):
        lbm_load(self.ctx, path)

    def steps_done(self):
        return lbm_steps_done(self.ctx)

    def features(self):
        """Correction-network inputs of the current state, (nz*nx, 9)."""
        return lbm_features(self.ctx, self.case.nx * self.case.nz)

    def set_correction(self, net, lam=0.0):
        """Apply `net` (a CorrectionNet, or None) as the first-layer correction."""
        self._net = net
        lbm_set_correction(self.ctx, net.m if net is not None else None, lam)

    def correction_field(self):
        return lbm_correction_field(self.ctx, self.case.nx * self.case.nz)


def _case_inputs(case):
    """lbm_grid, lbm_forcing and the LAD array of a case (plus arrays to keep alive)."""
    g = LbmGrid(case.nx, case.ny, case.nz, *case.bc_x, *case.bc_y, *case.bc_z)
    uprof = (None if case.u_profile is None
             else np.ascontiguousarray(case.u_profile, dtype=np.float64))
    fo = LbmForcing()
    fo.g[:] = [float(v) for v in case.g]
    fo.cd = case.cd
    fo.x_canopy_begin, fo.x_canopy_end = case.canopy_x
    fo.u_bulk_target, fo.ctrl_gain = case.u_bulk_target, case.ctrl_gain
    fo.u_top[:] = [float(v) for v in case.u_top]
    fo.u_in_profile = _dp(uprof) if uprof is not None else _DP()
    fo.drag_streamwise_only = getattr(case, "drag_streamwise_only", 0)
    fo.scheme = getattr(case, "forcing_scheme", 0)
    fo.sgs_rho_power = getattr(case, "sgs_rho_power", 0)
    lad = None if case.lad is None else np.ascontiguousarray(case.lad, dtype=np.float64)
    return g, fo, lad, (uprof, lad)


class Batch:
    """An ensemble of independent boxes (cases with the same storage, statistics
    bins and perturbation amplitude) advanced together, all steps replayed as
    one CUDA graph.  ``tune_steps`` as in lbm_batch_create (> 0: timed
    candidates; 0: one chunk width for all; -1: each box its own).
    ``box(i)`` gives a Domain view of box i."""

    def __init__(self, cases, storage=LBM_F16_SHIFTED, tune_steps=0, use_torch_workspace=True,
                 stream=None):
        import torch

        if isinstance(storage, str):
            storage = STORAGE_NAMES[storage]
        self.cases, self.storage = list(cases), storage
        bins = {c.stats_xbins for c in self.cases}
        amps = {c.init_perturb for c in self.cases}
        if len(bins) != 1 or len(amps) != 1:
            raise LbmError(LBM_ERR_ARG, "Batch: all boxes need the same stats_xbins and init_perturb")
        self._keep = []
        arr = (LbmBox * len(self.cases))()
        for i, c in enumerate(self.cases):
            g, fo, lad, keep = _case_inputs(c)
            self._keep.append(keep)
            arr[i].grid, arr[i].forcing = g, fo
            arr[i].tau0, arr[i].cs, arr[i].seed = c.tau0, c.cs, c.seed
            arr[i].lad = _dp(lad) if lad is not None else _DP()
        self._boxes = arr
        nbins, amp = bins.pop(), amps.pop()
        self.workspace = None
        ws_ptr, ws_bytes = 0, 0
        if use_torch_workspace:
            ws_bytes = lbm_batch_workspace_bytes(arr, storage, nbins)
            if ws_bytes == 0:
                raise LbmError(LBM_ERR_ARG, "lbm_batch_workspace_bytes: invalid boxes")
            self.workspace = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
            ws_ptr = self.workspace.data_ptr()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        torch.cuda.synchronize()
        self.b = lbm_batch_create(arr, storage, nbins, amp, tune_steps, self.stream.cuda_stream,
                                  ws_ptr, ws_bytes)
        self.boxes = [Domain._view(lbm_batch_box(self.b, i), c, storage, self.stream, self)
                      for i, c in enumerate(self.cases)]

    def step(self, n=1):
        lbm_batch_step(self.b, n)

    def sync(self):
        lbm_batch_sync(self.b)

    def stats_reset(self, enable=True):
        lbm_batch_stats_reset(self.b, enable)

    def box(self, i):
        return self.boxes[i]

    def tuning(self):
        return lbm_batch_tuning(self.b)

    def candidates(self):
        return lbm_batch_candidates(self.b)

    @property
    def cells(self):
        return sum(c.nx * c.ny * c.nz for c in self.cases)

    def close(self):
        if getattr(self, "b", None) is not None:
            for d in self.boxes:
                d.ctx = None
            lbm_batch_destroy(self.b)
            self.b = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
