"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances: FP32 compute with FP32 storage must keep the relative L2 error of
the populations within 1e-6 over the first 100 steps, and every single
population within ELEM_TOL of the largest offset max |f - w| (parity_util
derives the bound); FP16/BF16 shifted storage errors are measured and bounded
loosely (they are stated, not pinned).
"""
import math

import numpy as np
import pytest

import oracle
import paper_2206_15454_b300 as P
from paper_2206_15454_b300 import post
import workloads as W
from parity_util import assert_population_parity

pytestmark = pytest.mark.gpu

F32_TOL = 1e-6


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def pair(case, storage=P.LBM_F32):
    return P.Domain(case, storage), oracle.Oracle(case)


CASES = W.small_cases() + [
    W.Case("tiny_periodic", 1, 1, 1, bc_y=(W.PERIODIC, W.PERIODIC), tau0=0.7, init_perturb=0.03,
           seed=9),
    W.Case("one_row_walls", 3, 1, 2, bc_y=(W.BOUNCEBACK, W.FREESLIP), tau0=0.9, g=(1e-5, 0, 0),
           init_perturb=0.01, seed=11),
    W.poiseuille(1, 32, 1).replace(name="column"),
    W.channel_les(300, 9, 5).replace(name="two_x_chunks"),  # nx > 256: two tiles per row
    # inflow/outflow with a one-cell last chunk: that cell feeds both the
    # previous chunk's ghost and its own outflow ghost
    W.canopy_abl(257, 9, 5, h=3.0, canopy_x0=60, xbin=64).replace(name="outflow_one_cell_chunk"),
]


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_initial_state_matches(case):
    d, o = pair(case)
    # the FP64 initial state rounded once to FP32: half an ulp of each offset
    assert_population_parity(d.get_f(), o.get_f(), 1e-7, 1e-6, label=f"{case.name} initial")


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_first_100_steps_f32(case):
    d, o = pair(case)
    done = 0
    for k in (1, 9, 90):
        d.step(k)
        o.step(k)
        done += k
        assert_population_parity(d.get_f(), o.get_f(), F32_TOL, label=f"{case.name} step {done}")
    rho_d, u_d = d.macro()
    rho_o, u_o = o.macro()
    assert np.max(np.abs(rho_d - rho_o)) < 1e-6
    umax = max(np.max(np.abs(u_o)), 1e-12)
    assert np.max(np.abs(u_d - u_o)) / umax < 1e-4 + 1e-7 / umax


# FP16 keeps 11 significant bits of f_i - w_i, BF16 8 bits: one rounding per
# step of offsets ~1e-2 gives ~1e-5 (FP16) and ~1e-4 (BF16) of |f| per step,
# a random walk over 100 steps ~1e-4 and ~1e-3.  Measured (B300): FP16 0.7-1.0e-4,
# BF16 5.8-8.2e-4; the bounds leave 3x headroom to catch a real defect.
@pytest.mark.parametrize("storage,bound", [(P.LBM_F16_SHIFTED, 3e-4), (P.LBM_BF16_SHIFTED, 2.5e-3)],
                         ids=["f16s", "bf16s"])
@pytest.mark.parametrize("case", CASES[:5], ids=[c.name for c in CASES[:5]])
def test_first_100_steps_half_storage(case, storage, bound):
    d, o = pair(case, storage)
    d.step(100)
    o.step(100)
    err = rel_l2(d.get_f(), o.get_f())
    print(f"{case.name} storage={storage}: population rel L2 after 100 steps = {err:.3e}")
    assert err < bound


def test_poiseuille_32cube_2000_steps_against_series_and_oracle():
    """Laminar channel case: 32^3, g = 1e-6, tau = 0.8, 2000 steps."""
    case = W.poiseuille(32, 32, 32)
    d = P.Domain(case)
    d.step(2000)
    u = d.macro()[1][0]
    assert np.ptp(u, axis=(0, 2)).max() < 1e-9  # x,z-uniform
    prof = u.mean(axis=(0, 2))
    H, g, nu, lam, t = 32, 1e-6, 0.1, 0.09, 2000
    eta = np.arange(H) + 0.5
    ser = g / (2 * nu) * eta * (H - eta) + g * (16 * lam - 3) / (24 * nu)
    for n in range(1, 400, 2):
        ser -= (4 * g * H * H / (nu * n ** 3 * math.pi ** 3) * np.sin(n * math.pi * eta / H)
                * math.exp(-n * n * math.pi ** 2 * nu * t / H ** 2))
    assert np.linalg.norm(prof - ser) / np.linalg.norm(ser) < 1e-2
    o = oracle.Oracle(W.poiseuille(1, 32, 1))
    o.step(2000)
    uo = o.macro()[1][0, 0, :, 0]
    # FP32: each step adds a Guo increment ~2e-7 to offsets ~1e-4 whose ulp is
    # ~7e-12, so 2000 steps accumulate up to ~1e-8 on u ~ 1e-3
    assert np.max(np.abs(prof - uo)) / uo.max() < 5e-5


@pytest.mark.parametrize("storage", [P.LBM_F32, P.LBM_F16_SHIFTED, P.LBM_BF16_SHIFTED])
def test_mass_conservation(storage):
    case = W.channel_les(64, 32, 16)
    d = P.Domain(case, storage)
    m0 = d.mass()
    o = oracle.Oracle(case)
    assert abs(m0 - o.mass()) / o.mass() < 1e-7
    d.step(1000)
    drift = abs(d.mass() - m0) / m0
    print(f"storage={storage}: relative mass drift over 1000 steps = {drift:.3e}")
    assert drift < {P.LBM_F32: 1e-6, P.LBM_F16_SHIFTED: 1e-4, P.LBM_BF16_SHIFTED: 1e-3}[storage]


def test_statistics_and_controller_match_oracle():
    case = W.canopy_abl(64, 24, 16, h=6.0, canopy_x0=16, xbin=16)
    d, o = pair(case)
    d.step(20)
    o.step(20)
    d.stats_reset(True)
    o.stats_reset(True)
    d.step(30)
    o.step(30)
    sd, nd = d.stats()
    so, no = o.stats()
    assert nd == no == 30
    assert np.max(np.abs(sd[:3] - so[:3])) < 1e-6 * max(1.0, np.abs(so[:3]).max())
    # covariances come from <ab> - <a><b>; FP32 products of u ~ 0.05 carry
    # ~1.5e-10 absolute rounding, here against covariances ~1e-6
    assert np.max(np.abs(sd[3:] - so[3:])) < 1e-3 * np.abs(so[3:]).max()

    ch = W.channel_les(48, 24, 20)
    d, o = pair(ch)
    d.step(50)
    o.step(50)
    gd, ubd = d.drive()
    go, ubo = o.drive()
    # FP32 cell velocities carry ~1e-7..1e-6 relative error after 50 steps
    assert abs(ubd - ubo) < 2e-6 * abs(ubo)
    assert abs(gd[0] - go[0]) < ch.ctrl_gain * 2e-6 * abs(ubo) + 1e-15


def test_full_size_channel_step_matches_oracle():
    """256 x 128 x 128 turbulent channel in the benchmark's launch shape: two
    full steps against the oracle, every population compared."""
    case = W.channel_les()
    d, o = pair(case)
    d.step(2)
    o.step(2)
    assert_population_parity(d.get_f(), o.get_f(), F32_TOL, label="channel 256x128x128, 2 steps")
    gd, ubd = d.drive()
    go, ubo = o.drive()
    assert abs(ubd - ubo) < 2e-6 * abs(ubo)


def test_nan_is_detected_and_sticky(tmp_path):
    case = W.channel_les(32, 16, 8)
    d = P.Domain(case)
    f = d.get_f()
    f[3, 2, 5, 7] = np.nan
    d.set_f(f)
    d.step(1)
    with pytest.raises(P.LbmError) as e:
        d.sync()
    assert e.value.status == P.LBM_ERR_NAN
    with pytest.raises(P.LbmError) as e:
        d.step(1)
    assert e.value.status == P.LBM_ERR_STATE


def test_checkpoint_resume_is_bitwise(tmp_path):
    case = W.channel_les(48, 24, 20)
    a = P.Domain(case, P.LBM_F16_SHIFTED)
    a.step(10)
    a.stats_reset(True)
    a.step(5)
    path = tmp_path / "ck.lbm"
    a.save(path)
    a.step(20)
    fa, sa = a.get_f(), a.stats()
    b = P.Domain(case, P.LBM_F16_SHIFTED)
    b.load(path)
    assert b.steps_done() == 15
    b.step(20)
    assert np.array_equal(b.get_f(), fa)
    # statistics are summed with atomics (order-dependent rounding)
    sb = b.stats()[0]
    assert np.allclose(sb, sa[0], rtol=1e-6, atol=1e-6 * np.abs(sa[0]).max())
    raw = bytearray(path.read_bytes())
    raw[-100] ^= 0xFF
    path.write_bytes(bytes(raw))
    with pytest.raises(P.LbmError) as e:
        b.load(path)
    assert e.value.status == P.LBM_ERR_IO


def test_library_allocated_workspace_and_default_stream():
    case = W.channel_les(40, 16, 8)
    d1 = P.Domain(case, use_torch_workspace=False)
    d2 = P.Domain(case)
    d1.step(7)
    d2.step(7)
    assert np.array_equal(d1.get_f(), d2.get_f())


def _profile_errors(sd, so):
    """Largest deviation of each statistic, relative to the largest magnitude of
    that statistic over the profile (means: <u>, <v>, <w> share the <u> scale)."""
    out = {}
    scale_mean = np.abs(so[0]).max()
    for k, name in enumerate(["u", "v", "w", "uu", "vv", "ww", "uv", "uw", "vw"]):
        scale = scale_mean if k < 3 else np.abs(so[k]).max()
        out[name] = float(np.abs(sd[k] - so[k]).max() / scale)
    return out


# The statistics path over a long run: mean velocity and Reynolds-stress
# profiles (time, x and z averaged; per x-bin for the canopy) must agree within
# 2 % of their profile scale; u'w' and v'w' average to zero by symmetry, so
# they are compared against the u'v' scale.  At these sizes the seeded
# perturbations do not grow into decorrelated turbulence within the run (the
# printed population difference after the spin-up stays near 1e-6), so this
# checks the statistics path (per-thread sums, warp reduction, FP64
# accumulation, x-bins) over thousands of steps; tests/test_gpu_stats.py
# compares statistics on a flow that does decorrelate.
TURB_STEPS = (1500, 2500)  # spin-up, averaging window


@pytest.mark.parametrize("name,case", [
    ("channel", W.channel_les(64, 32, 32)),
    ("canopy", W.canopy_abl(96, 32, 32, h=6.0, canopy_x0=32, xbin=32)),
], ids=["channel", "canopy"])
def test_long_run_statistics_within_2_percent(name, case):
    d, o = pair(case)
    spin, avg = TURB_STEPS
    d.step(spin)
    o.step(spin)
    diverged = rel_l2(d.get_f(), o.get_f())
    d.stats_reset(True)
    o.stats_reset(True)
    d.step(avg)
    o.step(avg)
    sd, nd = d.stats()
    so, no = o.stats()
    assert nd == no == avg
    err = _profile_errors(sd, so)
    uv = np.abs(so[6]).max()
    err["uw"] = float(np.abs(sd[7] - so[7]).max() / uv)
    err["vw"] = float(np.abs(sd[8] - so[8]).max() / uv)
    print(f"{name}: population rel L2 after spin-up {diverged:.2e}; profile errors "
          + " ".join(f"{k}={v:.2e}" for k, v in err.items()))
    for k, v in err.items():
        assert v < 0.02, (k, v)


@pytest.mark.parametrize("forest", [1, 2, 3])
def test_paper_abl_forest_cases_match_oracle(forest):
    """The paper's ABL set-up (periodic x/z, forced-equilibrium top, body force)
    with the three forest cases of Table tab:forest_cases, 100 steps."""
    case = W.abl_forest(forest, nx=40, ny=16, nz=12)
    d, o = pair(case)
    d.step(60)
    o.step(60)
    d.stats_reset(True)
    o.stats_reset(True)
    d.step(40)
    o.step(40)
    assert_population_parity(d.get_f(), o.get_f(), F32_TOL, label=f"forest case {forest}")
    # the forest friction velocity of Sec. 5 (Reynolds stresses at y/h = 2)
    h = 20.0 / (400.0 / case.ny)
    us_d = post.friction_velocity(d.stats()[0], 2 * h)
    us_o = post.friction_velocity(o.stats()[0], 2 * h)
    assert us_o > 0 and abs(us_d - us_o) <= 0.02 * us_o, (forest, us_d, us_o)


def test_paper_abl_forest_profiles_are_ordered():
    """Profile comparison of the three forest cases (same seed and driving):
    inside the forest the modelled drag slows the flow, so after the same time
    the no-forest case is fastest there, and the two forest cases (equal total
    obstruction by design, close as implemented) stay close to each other."""
    means = {}
    for forest in (1, 2, 3):
        case = W.abl_forest(forest, nx=80, ny=32, nz=64)
        d = P.Domain(case)
        d.step(1500)
        d.stats_reset(True)
        d.step(500)
        s, _ = d.stats()
        h = int(round(20.0 / (400.0 / case.ny)))
        means[forest] = (s[0, 0, :h].mean(), s[0, 0, 2 * h:4 * h].mean())
    print({k: tuple(round(float(x), 5) for x in v) for k, v in means.items()})
    assert means[3][0] > 1.2 * max(means[1][0], means[2][0])
    assert abs(means[1][0] - means[2][0]) < 0.5 * means[3][0]


def test_full_size_canopy_step_matches_oracle():
    """The 512 x 128 x 256 forest-canopy boundary layer (inflow/outflow, 16.8 M
    cells) in the benchmark's launch shape: two full steps against the oracle,
    every population compared."""
    case = W.canopy_abl()
    d, o = pair(case)
    d.step(2)
    o.step(2)
    fo = o.get_f()
    o.close()
    assert_population_parity(d.get_f(), fo, F32_TOL, label="canopy 512x128x256, 2 steps")
