"""The timeout path of the bounded device waits, made to run out on purpose
without faulting or hanging anything: block 0 of one step does not issue one
of its tile fills (lbm_test_withhold_fill), so its waits on that stage can
only give up after their poll limit (about a second).  The context must report
LBM_ERR_TIMEOUT (and keep reporting it), and the device must stay usable."""
import numpy as np
import pytest

import paper_2206_15454_b300 as P
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", [P.LBM_F32, P.LBM_F16_SHIFTED])
@pytest.mark.parametrize("fill", [0, 1, 5])
def test_a_withheld_fill_times_out_and_is_reported(storage, fill):
    # 8192 tiles (FP16: two rows per tile) or 16384 (FP32) over at most
    # 148 x 3 blocks: every block's static run is at least 16 tiles long, so
    # the withheld fill is always one of block 0's static fills
    case = W.channel_les(256, 128, 128)
    d = P.Domain(case, storage)
    d.step(2)
    d.sync()
    P.lbm_test_withhold_fill(d.ctx, fill)
    d.step(1)
    with pytest.raises(P.LbmError) as e:
        d.sync()
    assert e.value.status == P.LBM_ERR_TIMEOUT
    with pytest.raises(P.LbmError) as e:  # sticky
        d.step(1)
    d.close()
    # the device is fine: a fresh domain steps and matches a second fresh one
    a, b = P.Domain(case, storage), P.Domain(case, storage)
    a.step(5)
    b.step(5)
    assert np.array_equal(a.get_f(), b.get_f())
    a.close()
    b.close()


def test_withhold_arguments_are_checked_and_act_on_one_step():
    d = P.Domain(W.channel_les(64, 32, 16))
    with pytest.raises(P.LbmError) as e:
        P.lbm_test_withhold_fill(d.ctx, -1)
    assert e.value.status == P.LBM_ERR_ARG
    # a fill index past the block's fills withholds nothing
    P.lbm_test_withhold_fill(d.ctx, 1 << 30)
    d.step(3)
    d.sync()
    d.close()
