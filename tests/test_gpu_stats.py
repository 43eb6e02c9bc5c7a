"""Statistics parity with the FP64 oracle where the benchmark spec states it:

* on a flow that is really turbulent: the GPU and the oracle decorrelate
  (population difference of order one after the spin-up) and only their
  statistics can agree.  Mean velocity and Reynolds-stress profiles (Sec. 4:
  averaged in time and over x-z planes) are compared as the largest deviation
  over y relative to the largest magnitude of the profile.  <u> and <u'v'>,
  which the mean momentum balance of the driven canopy flow fixes, must agree
  within 2 %.  The normal stresses and <u'w'>, <v'w'> carry a sampling spread
  of 2-4 % over any window the oracle can run in minutes (measured between two
  GPU runs that differ by 1e-7 in the initial populations); they must agree
  within 2 % or within twice that spread, measured here on the same window;
* with 16-bit storage: FP16- and BF16-shifted populations (FP32 arithmetic) on
  the forest-canopy boundary layer against the FP64 oracle, mean-velocity
  profiles per x-bin within 2 %.
"""
import numpy as np
import pytest

import oracle
import paper_2206_15454_b300 as P
import workloads as W

pytestmark = pytest.mark.gpu

NAMES = ["u", "v", "w", "uu", "vv", "ww", "uv", "uw", "vw"]
W_LAT = np.array([1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12)[:, None, None, None]


def profile_errors(s, ref):
    """Largest deviation over the profile, relative to the largest magnitude of
    the reference profile (<v>, <w> on the <u> scale; <u'w'>, <v'w'>, which
    vanish by symmetry, on the <u'v'> scale)."""
    out = {}
    for k, name in enumerate(NAMES):
        scale = ref[0] if k < 3 else (ref[6] if k in (7, 8) else ref[k])
        out[name] = float(np.abs(s[k] - ref[k]).max() / np.abs(scale).max())
    return out


def test_turbulent_canopy_statistics_within_2_percent():
    case = W.canopy_turbulent()
    spin, window = 8000, 16000
    d, o, d2 = P.Domain(case), oracle.Oracle(case), P.Domain(case)
    f0 = d.get_f()
    d2.set_f(f0 * (1.0 + 1e-7 * np.random.default_rng(5).standard_normal(f0.shape)))
    for x in (d, o, d2):
        x.step(spin)
    fd, fo = d.get_f(), o.get_f()
    decor = float(np.linalg.norm(fd - fo) / np.linalg.norm(fo - W_LAT))
    for x in (d, o, d2):
        x.stats_reset(True)
        x.step(window)
    sd, nd = d.stats()
    so, no = o.stats()
    s2, _ = d2.stats()
    assert nd == no == window
    err = profile_errors(sd, so)
    spread = profile_errors(sd, s2)
    print(f"GPU vs oracle after {spin} steps: population difference {decor:.2f} of |f - w| "
          f"(decorrelated); over {window} steps:")
    for k in NAMES:
        print(f"  {k:>2}: GPU vs oracle {err[k]:.4f}, GPU vs GPU (1e-7 apart) {spread[k]:.4f}")
    assert decor > 0.1, decor
    for k in ("u", "v", "w", "uv"):
        assert err[k] < 0.02, (k, err[k])
    for k in ("uu", "vv", "ww", "uw", "vw"):
        assert err[k] < max(0.02, 2.0 * spread[k]), (k, err[k], spread[k])


@pytest.mark.parametrize("storage", [P.LBM_F16_SHIFTED, P.LBM_BF16_SHIFTED], ids=["f16s", "bf16s"])
def test_half_storage_canopy_profiles_against_fp64_oracle(storage):
    """The canopy boundary layer (inflow/outflow, canopy over the last 3/4 of
    the domain, statistics per x-bin of 32 cells): mean-velocity profile of
    every x-bin within 2 % of the oracle's."""
    case = W.canopy_abl(128, 32, 32, h=8.0, canopy_x0=32, xbin=32)
    spin, window = 1000, 2000
    o = oracle.Oracle(case)
    o.step(spin)
    o.stats_reset(True)
    o.step(window)
    so, _ = o.stats()
    res = {}
    for st in (P.LBM_F32, storage):
        d = P.Domain(case, st)
        d.step(spin)
        d.stats_reset(True)
        d.step(window)
        s, _ = d.stats()
        res[st] = profile_errors(s, so)
        d.close()
    print(f"storage {storage}: mean-velocity error {res[storage]['u']:.2e} of max <u> "
          f"(FP32: {res[P.LBM_F32]['u']:.2e}); <u'v'> {res[storage]['uv']:.2e}")
    assert res[storage]["u"] < 0.02
    assert res[P.LBM_F32]["u"] < 1e-3
