"""Statistics parity with the FP64 oracle where the benchmark spec states it:

* on a flow that is really turbulent, two runs agree only statistically.  The
  GPU runs K realizations of the turbulent canopy flow that differ only in the
  seed of their initial perturbations (independent samples of the same flow);
  their spread per height is the sampling spread of one run's statistics over
  the window (Sec. 4: averaged in time and over x-z planes).  One run over a
  window the oracle finishes in minutes has a spread of about 4 % in <u>, 1.5 %
  in <u'v'> and 10-25 % in the normal stresses (B300, 16 realizations), so a 2 %
  bound on one realization is below the noise.  The oracle's run (the base
  seed) must be a sample of the same distribution: for every statistic and
  height its deviation from the GPU ensemble mean, in units of the spread of
  that difference, stays below 5 (largest over the heights) and below 3 (root
  mean square over the heights; the heights are strongly correlated, a
  realization with a low bulk velocity is low at every height, so this acts
  like one z-score, and a bias at several heights raises it).
  Inside the canopy the spread of <u> is 0.1-0.4 %, so there the check is far
  tighter than 2 %.  A GPU run from the oracle's own initial state shows the
  decorrelation (population difference of order one after the spin-up);
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


def test_turbulent_canopy_statistics_match_oracle():
    base = W.canopy_turbulent()
    spin, window, K = 8000, 16000, 32
    o, d = oracle.Oracle(base), P.Domain(base)
    for x in (d, o):
        x.step(spin)
    fd, fo = d.get_f(), o.get_f()
    decor = float(np.linalg.norm(fd - fo) / np.linalg.norm(fo - W_LAT))
    for x in (d, o):
        x.stats_reset(True)
        x.step(window)
    so, no = o.stats()
    sd, nd = d.stats()
    d.close()
    assert nd == no == window
    ens = []
    for k in range(1, K + 1):
        e = P.Domain(base.replace(seed=base.seed + 1000 + k))
        e.step(spin)
        e.stats_reset(True)
        e.step(window)
        ens.append(e.stats()[0])
        e.close()
    S = np.stack(ens)
    mu = S.mean(axis=0)
    # spread of (one sample - mean of K samples), per statistic and height
    spread = S.std(axis=0, ddof=1) * np.sqrt(1.0 + 1.0 / K)
    print(f"GPU run from the oracle's initial state: population difference {decor:.2f} of "
          f"|f - w| after {spin} steps; oracle vs {K} independent GPU realizations over "
          f"{window} steps:")
    worst = {}
    for k, name in enumerate(NAMES):
        scale = np.abs(so[0] if k < 3 else (so[6] if k in (7, 8) else so[k])).max()
        sig = np.maximum(spread[k], 1e-3 * scale)
        z = (so[k] - mu[k]) / sig
        worst[name] = (float(np.abs(z).max()), float(np.sqrt(np.mean(z ** 2))))
        print(f"  {name:>2}: oracle - GPU mean {np.abs(so[k] - mu[k]).max() / scale:.4f} of scale, "
              f"one run's spread up to {spread[k].max() / scale:.4f}; |z| max {worst[name][0]:.2f}, "
              f"rms {worst[name][1]:.2f}; same-seed GPU run vs oracle "
              f"{np.abs(sd[k] - so[k]).max() / scale:.4f}")
    assert decor > 0.1, decor
    for name, (zmax, zrms) in worst.items():
        assert zmax < 5.0 and zrms < 3.0, (name, zmax, zrms)


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
