"""lbm_stats_begin / lbm_stats_end: the pipelined read-out returns, step by
step, what the synchronous lbm_stats returns at the same point, through the C
ABI; misuse is an argument error that leaves the context usable."""
import numpy as np
import pytest

import paper_2206_15454_b300 as P
import workloads as W

pytestmark = pytest.mark.gpu


def test_pipelined_readout_matches_synchronous_stats():
    case = W.channel_les(64, 32, 16)
    a, b = P.Domain(case), P.Domain(case)
    a.stats_reset(True)
    b.stats_reset(True)
    got = []
    a.step(1)
    a.stats_begin()
    for _ in range(5):  # step k+1 is enqueued before step k's read-out is taken
        a.step(1)
        a.stats_begin()
        got.append(a.stats_end())
    got.append(a.stats_end())
    for k in range(6):
        b.step(1)
        ref, n = b.stats()
        out, m = got[k]
        assert m == n == k + 1
        # FP64 plane sums of two runs differ only in the order of their atomic adds
        np.testing.assert_allclose(out, ref, rtol=1e-9, atol=1e-15)
    a.close()
    b.close()


def test_pipelined_readout_misuse_is_not_sticky():
    d = P.Domain(W.poiseuille(32, 16, 8))
    d.stats_reset(True)
    with pytest.raises(P.LbmError) as e:
        d.stats_end()
    assert e.value.status == P.LBM_ERR_ARG
    d.step(2)
    d.stats_begin()
    d.stats_begin()
    with pytest.raises(P.LbmError) as e:
        d.stats_begin()  # two pending already
    assert e.value.status == P.LBM_ERR_ARG
    first, n1 = d.stats_end()
    second, n2 = d.stats_end()
    assert n1 == n2 == 2 and np.array_equal(first, second)
    d.step(1)
    assert d.stats()[1] == 3
    d.close()
