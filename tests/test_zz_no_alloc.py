"""lbm_get_macro_noalloc: the field readout for callers that must not allocate
device memory (a fixed memory budget or pre-reserved pool, or code running
while other work on the device is captured or timed).  It must return what
lbm_get_macro returns, call after call, through the C ABI.

This file is collected last on purpose: a run that stops at the first failure
has run every other test before reaching it.
"""
import numpy as np
import pytest

import paper_2206_15454_b300 as P
import workloads as W

pytestmark = pytest.mark.gpu


def fields(d, fn):
    rho = np.zeros(d.shape)
    u = np.zeros((3,) + d.shape)
    fn(d.ctx, rho, u)
    return rho, u


def test_noalloc_readout_matches_get_macro_on_consecutive_calls():
    a = P.Domain(W.channel_les(48, 24, 20))
    b = P.Domain(W.canopy_abl(64, 24, 16, h=6.0, canopy_x0=16, xbin=16), P.LBM_F16_SHIFTED)
    for _ in range(2):  # two calls in a row on each domain, interleaved (shared buffer)
        for d in (a, b):
            d.step(7)
            r1, u1 = fields(d, P.lbm_get_macro_noalloc)
            r0, u0 = fields(d, P.lbm_get_macro)
            # same kernel arithmetic; the tolerance is the one the parity tests use
            assert np.allclose(r1, r0, rtol=0, atol=1e-12)
            assert np.allclose(u1, u0, rtol=0, atol=1e-12)
            assert np.isfinite(r1).all() and np.abs(u1).max() > 0


def test_noalloc_readout_rejects_grids_above_its_buffer():
    d = P.Domain(W.channel_les(80, 64, 64))  # 327680 cells > 262144
    with pytest.raises(P.LbmError) as e:
        fields(d, P.lbm_get_macro_noalloc)
    assert e.value.status == P.LBM_ERR_ARG
    d.step(1)  # argument errors are not sticky
    d.sync()
