"""The library's x-slab data path on one GPU: one periodic-in-x domain cut
into 2 or 3 slabs, each an lbm_ctx with halo faces (LBM_BC_HALO), stepped with
a face exchange after every step (lbm_halo_pack, device-to-device copies,
lbm_halo_unpack).  The joined state must equal the library's own undivided run
bit for bit (same per-cell arithmetic on the same inputs) and the FP64 oracle
within the FP32 parity bounds."""
import numpy as np
import pytest

import oracle
import paper_2206_15454_b300 as P
from paper_2206_15454_b300 import slabs as S
import workloads as W
from parity_util import assert_population_parity

pytestmark = pytest.mark.gpu


def _no_controller(case):
    return case.replace(u_bulk_target=0.0, ctrl_gain=0.0)


CASES = [
    _no_controller(W.channel_les(48, 24, 20)).replace(name="channel"),
    W.abl_forest(1, nx=40, ny=16, nz=12).replace(name="forest_abl_eq_top"),
    # a canopy that starts and ends inside slabs, ragged sizes, periodic y
    W.small_cases()[6].replace(nx=37, canopy_x=(5, 29), name="periodic_box_ragged"),
    # slabs wider than one 64-cell chunk (chunk ghosts inside a slab too)
    _no_controller(W.channel_les(150, 9, 6)).replace(name="two_chunk_slabs"),
]


@pytest.mark.parametrize("storage", [P.LBM_F32, P.LBM_F16_SHIFTED], ids=["f32", "f16s"])
@pytest.mark.parametrize("nslabs", [2, 3])
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_slabs_equal_the_undivided_run(case, nslabs, storage):
    whole = P.Domain(case, storage)
    f0 = whole.get_f()
    whole.set_f(f0)          # both start from the same rounded state
    sl = S.DeviceSlabs(case, nslabs, storage)
    sl.set_f(f0)
    assert np.array_equal(sl.get_f(), whole.get_f())
    whole.stats_reset(True)
    sl.stats_reset(True)
    whole.step(100)
    sl.step(100)
    fs, fw = sl.get_f(), whole.get_f()
    assert np.array_equal(fs, fw), np.abs(fs - fw).max()
    # plane statistics recombined from the slabs (summed in another order)
    ss, ns = sl.stats()
    sw, nw = whole.stats()
    assert ns == nw == 100
    assert np.max(np.abs(ss[:3] - sw[:3])) <= 1e-6 * max(np.abs(sw[:3]).max(), 1e-12)
    if storage == P.LBM_F32:
        o = oracle.Oracle(case)
        o.set_f(f0)
        o.step(100)
        assert_population_parity(fs, o.get_f(), 1e-6, label=f"{case.name} in {nslabs} slabs")
    sl.close()
    whole.close()


def test_halo_calls_check_their_arguments():
    d = P.Domain(_no_controller(W.channel_les(32, 8, 4)))   # periodic x: no halo faces
    assert P.lbm_halo_bytes(d.ctx) == 0
    with pytest.raises(P.LbmError) as e:
        P.lbm_halo_pack(d.ctx, 256, 256)
    assert e.value.status == P.LBM_ERR_ARG
    sl = S.DeviceSlabs(_no_controller(W.channel_les(32, 8, 4)), 2)
    h = sl.doms[0]
    assert P.lbm_halo_bytes(h.ctx) == 5 * 8 * 4 * 4
    buf = sl.send[0][0]
    with pytest.raises(P.LbmError) as e:
        P.lbm_halo_pack(h.ctx, buf.data_ptr() + 4, buf.data_ptr())   # not 16-byte aligned
    assert e.value.status == P.LBM_ERR_ARG
    with pytest.raises(P.LbmError) as e:
        P.lbm_halo_unpack(h.ctx, 0, buf.data_ptr())
    assert e.value.status == P.LBM_ERR_ARG
    sl.step(2)   # argument errors are not sticky
    sl.doms[0].sync()
