"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/lbm.h, sizes its workspace as documented and rejects
invalid arguments before touching the device."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2206_15454_b300 as P
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    P.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lbm_[a-z_0-9]+)", out))
    declared = header_functions()
    assert len(declared) >= 18
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    for n in declared:
        assert hasattr(P.lib(), n)
        assert hasattr(P, n) or n in ("lbm_last_error", "lbm_status_string", "lbm_batch_last_error",
                                      "lbm_mlp_last_error")


def _grid(nx=64, ny=32, nz=16, bc=(0, 0, 1, 2, 0, 0)):
    return P.LbmGrid(nx, ny, nz, *bc)


def test_workspace_bytes():
    g = _grid()
    n32 = P.lbm_workspace_bytes(g, P.LBM_F32, 1)
    n16 = P.lbm_workspace_bytes(g, P.LBM_F16_SHIFTED, 1)
    pops32 = 2 * 19 * 64 * 32 * 16 * 4
    # rows of 64 cells carry 128 bytes of ghost/alignment slots on each side
    assert pops32 <= n32 < pops32 * 128 // 64 + 128 * 1024
    assert n32 - n16 >= pops32 // 2 - 4096
    # rows are cut into chunks of 64, 128 or 256 cells
    assert P.lbm_workspace_bytes(_grid(nx=65), P.LBM_F32, 1) >= 2 * 19 * 128 * 32 * 16 * 4


@pytest.mark.parametrize("grid,storage,bins", [
    (dict(nx=0), 0, 1),
    (dict(bc=(4, 0, 1, 2, 0, 0)), 0, 1),        # inflow without outflow
    (dict(bc=(0, 0, 2, 2, 0, 0)), 0, 1),        # free-slip bottom unsupported
    (dict(bc=(0, 0, 1, 2, 1, 1)), 0, 1),        # walls in z unsupported
    (dict(), 3, 1),                              # unknown storage
    (dict(), 0, 0),                              # no statistics bin
    (dict(nx=8), 0, 9),                          # more bins than columns
    (dict(nx=4096, ny=4096, nz=256), 0, 1),      # beyond 2^31 cells
])
def test_invalid_grids_rejected(grid, storage, bins):
    assert P.lbm_workspace_bytes(_grid(**grid), storage, bins) == 0


def test_create_rejects_bad_arguments_without_a_device():
    g = _grid()
    fo = P.LbmForcing()
    ctx = C.c_void_p()
    L = P.lib()
    # tau0 <= 1/2 is unstable by construction (negative viscosity)
    s = L.lbm_create(C.byref(g), 0.5, 0.1, P._DP(), C.byref(fo), 0, 1, 1, 0.0, None, 0,
                     C.byref(ctx))
    assert s == P.LBM_ERR_ARG and not ctx.value
    s = L.lbm_create(C.byref(g), float("nan"), 0.1, P._DP(), C.byref(fo), 0, 1, 1, 0.0, None, 0,
                     C.byref(ctx))
    assert s == P.LBM_ERR_ARG
    # inflow needs a profile
    gi = _grid(bc=(4, 5, 1, 2, 0, 0))
    s = L.lbm_create(C.byref(gi), 0.6, 0.1, P._DP(), C.byref(fo), 0, 1, 1, 0.0, None, 0,
                     C.byref(ctx))
    assert s == P.LBM_ERR_ARG
    # a workspace smaller than lbm_workspace_bytes
    s = L.lbm_create(C.byref(g), 0.6, 0.1, P._DP(), C.byref(fo), 0, 1, 1, 0.0,
                     C.c_void_p(4096), 16, C.byref(ctx))
    assert s == P.LBM_ERR_OOM
    assert L.lbm_create(C.byref(g), 0.6, 0.1, P._DP(), C.byref(fo), 0, 1, 1, 0.0, None, 0,
                        None) == P.LBM_ERR_ARG


def test_model_variants_and_halo_checked_without_a_device():
    L = P.lib()
    ctx = C.c_void_p()
    g = _grid()
    for field, bad in (("drag_streamwise_only", 2), ("scheme", 2), ("sgs_rho_power", 3),
                       ("reserved", 1)):
        fo = P.LbmForcing()
        setattr(fo, field, bad)
        s = L.lbm_create(C.byref(g), 0.6, 0.1, P._DP(), C.byref(fo), 0, 1, 1, 0.0, None, 0,
                         C.byref(ctx))
        assert s == P.LBM_ERR_ARG, field
    # halo faces come in pairs; a slab cannot run the bulk-velocity controller
    assert P.lbm_workspace_bytes(_grid(bc=(P.LBM_BC_HALO, 0, 1, 2, 0, 0)), 0, 1) == 0
    gh = _grid(bc=(P.LBM_BC_HALO, P.LBM_BC_HALO, 1, 2, 0, 0))
    assert P.lbm_workspace_bytes(gh, 0, 1) > 0
    fo = P.LbmForcing()
    fo.u_bulk_target, fo.ctrl_gain = 0.05, 0.01
    s = L.lbm_create(C.byref(gh), 0.6, 0.1, P._DP(), C.byref(fo), 0, 1, 1, 0.0, None, 0,
                     C.byref(ctx))
    assert s == P.LBM_ERR_ARG
    assert L.lbm_halo_bytes(None) == 0
    assert L.lbm_halo_pack(None, None, None) == P.LBM_ERR_ARG
    assert L.lbm_halo_unpack(None, None, None) == P.LBM_ERR_ARG
    # the ensemble runs the default model on whole boxes
    cases = W.ensemble_boxes(n_boxes=2, ny=16, nz=8, nx_range=(40, 90), seed=3)
    for kw in ({"forcing_scheme": 1}, {"drag_streamwise_only": 1}, {"sgs_rho_power": 2}):
        arr = (P.LbmBox * 2)()
        keep = []
        for i, c in enumerate(cases):
            gg, ff, lad, k = P._case_inputs(c.replace(**kw) if i == 1 else c)
            keep.append((k, lad))
            arr[i].grid, arr[i].forcing, arr[i].tau0, arr[i].cs = gg, ff, c.tau0, c.cs
            arr[i].lad = P._dp(lad) if lad is not None else P._DP()
        assert P.lbm_batch_workspace_bytes(arr, P.LBM_F16_SHIFTED, 1) == 0, kw


def test_aa_storage_argument_without_a_device():
    g = _grid()
    aa = P.LBM_STORAGE_AA
    pull = P.lbm_workspace_bytes(g, P.LBM_F32, 1)
    one = P.lbm_workspace_bytes(g, P.LBM_F32 | aa, 1)
    # one set with a one-cell ghost layer: (64 + 2 -> 96) x 34 x 18 cells, 19 directions
    assert 19 * 96 * 34 * 18 * 4 <= one < pull
    assert P.lbm_workspace_bytes(g, P.LBM_F16_SHIFTED | aa, 1) < one
    assert P.lbm_workspace_bytes(g, 0x200, 1) == 0          # unknown flag
    assert P.lbm_workspace_bytes(g, 3 | aa, 1) == 0         # unknown type
    halo = _grid(bc=(P.LBM_BC_HALO, P.LBM_BC_HALO, 1, 2, 0, 0))
    assert P.lbm_workspace_bytes(halo, P.LBM_F32 | aa, 1) == 0  # slabs use two sets


def test_null_context_calls_fail_cleanly():
    L = P.lib()
    assert L.lbm_step(None, 1) == P.LBM_ERR_ARG
    assert L.lbm_sync(None) == P.LBM_ERR_ARG
    assert L.lbm_steps_done(None) == -1
    L.lbm_destroy(None)
    assert L.lbm_status_string(P.LBM_ERR_NAN).decode().startswith("non-finite")
    assert L.lbm_last_error(None).decode() == "no context"


def test_structs_match_the_header():
    # lbm_grid: 9 int32; lbm_forcing: 3+1 doubles, 2 int32, 2+3 doubles, 1 pointer,
    # 4 int32 (model variants)
    assert C.sizeof(P.LbmGrid) == 36
    assert C.sizeof(P.LbmForcing) == 8 * 4 + 8 + 8 * 5 + 8 + 16


def test_ensemble_arguments_checked_without_a_device():
    cases = W.ensemble_boxes(n_boxes=3, ny=16, nz=8, nx_range=(40, 90), seed=3)
    arr = (P.LbmBox * 3)()
    keep = []
    for i, c in enumerate(cases):
        g, fo, lad, k = P._case_inputs(c)
        keep.append(k)
        arr[i].grid, arr[i].forcing, arr[i].tau0, arr[i].cs, arr[i].seed = g, fo, c.tau0, c.cs, 1
        arr[i].lad = P._dp(lad)
    n = P.lbm_batch_workspace_bytes(arr, P.LBM_F16_SHIFTED, 1)
    # at least the sum of the boxes alone (the tuner may pick another chunk width)
    alone = sum(P.lbm_workspace_bytes(arr[i].grid, P.LBM_F16_SHIFTED, 1) for i in range(3))
    assert n >= alone > 0
    assert P.lbm_batch_workspace_bytes(arr, 7, 1) == 0
    arr[1].forcing.u_bulk_target = 0.05  # no controller inside an ensemble
    assert P.lbm_batch_workspace_bytes(arr, P.LBM_F16_SHIFTED, 1) == 0
    b = C.c_void_p()
    assert P.lib().lbm_batch_create(3, arr, 1, 1, 0.0, 0, None, None, 0, C.byref(b)) == P.LBM_ERR_ARG
    arr[1].forcing.u_bulk_target = 0.0
    assert P.lib().lbm_batch_create(0, arr, 1, 1, 0.0, 0, None, None, 0, C.byref(b)) == P.LBM_ERR_ARG
    assert P.lib().lbm_batch_create(3, arr, 1, 1, 0.0, -2, None, None, 0, C.byref(b)) == P.LBM_ERR_ARG
    assert P.lib().lbm_batch_create(3, arr, 1, 1, 0.0, 0, None, C.c_void_p(4096), 16,
                                    C.byref(b)) == P.LBM_ERR_OOM
    assert P.lib().lbm_batch_step(None, 1) == P.LBM_ERR_ARG
    assert P.lib().lbm_batch_box(None, 0) is None
    P.lib().lbm_batch_destroy(None)
    assert P.lib().lbm_batch_candidates(None, None, None, None, 0) == -1


def test_box_struct_matches_the_header():
    # lbm_box: lbm_grid (36 B, padded to 40), 2 doubles, 1 pointer, lbm_forcing, uint64
    assert C.sizeof(P.LbmBox) == 40 + 16 + 8 + C.sizeof(P.LbmForcing) + 8
