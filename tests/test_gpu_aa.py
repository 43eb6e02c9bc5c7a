"""AA-pattern in-place storage (one population set) against the FP64 oracle
and against the pull scheme with two sets.  Both run the same per-cell
arithmetic on the same inputs, so the AA state must equal the pull state bit
for bit after any number of steps (odd: streamed layout, even: swapped
layout), and the oracle within the FP32 parity bounds, on every boundary
combination."""
import numpy as np
import pytest

import oracle
import paper_2206_15454_b300 as P
import workloads as W
from parity_util import assert_population_parity

pytestmark = pytest.mark.gpu

AA = P.LBM_STORAGE_AA
CASES = W.small_cases() + [
    W.Case("tiny_periodic", 1, 1, 1, bc_y=(W.PERIODIC, W.PERIODIC), tau0=0.7, init_perturb=0.03,
           seed=9),
    W.poiseuille(1, 32, 1).replace(name="column"),
    W.channel_les(300, 9, 5).replace(name="wide_rows"),
    W.canopy_abl(257, 9, 5, h=3.0, canopy_x0=60, xbin=64).replace(name="outflow_257"),
    W.small_cases()[2].replace(name="canopy_variants", drag_streamwise_only=1, forcing_scheme=1,
                               sgs_rho_power=2),
    # faces of 70,000 rows, more than the boundary fill's grid has block rows
    # (65,535): the fill's grid-stride loop over a face's slow coordinate
    W.poiseuille(2, 3, 70000).replace(name="tall_z", init_perturb=0.03, seed=11),
]


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_aa_matches_oracle_and_pull_scheme(case):
    aa, pull, o = P.Domain(case, P.LBM_F32 | AA), P.Domain(case, P.LBM_F32), oracle.Oracle(case)
    assert np.array_equal(aa.get_f(), pull.get_f())
    aa.stats_reset(True)
    pull.stats_reset(True)
    done = 0
    for k in (1, 1, 98, 1):   # odd, even, even, odd step counts
        for x in (aa, pull, o):
            x.step(k)
        done += k
        fa = aa.get_f()
        assert np.array_equal(fa, pull.get_f()), (case.name, done)
        assert_population_parity(fa, o.get_f(), 1e-6, label=f"{case.name} AA step {done}")
    ra, ua = aa.macro()
    rp, up = pull.macro()
    assert np.array_equal(ra, rp) and np.array_equal(ua, up)
    sa, na = aa.stats()
    sp, npl = pull.stats()
    assert na == npl == done
    assert np.max(np.abs(sa[:3] - sp[:3])) <= 1e-6 * max(np.abs(sp[:3]).max(), 1e-12)
    assert abs(aa.mass() - pull.mass()) <= 1e-9 * pull.mass()
    (ga, uba), (gp, ubp) = aa.drive(), pull.drive()
    assert uba == ubp and np.array_equal(ga, gp)


# 16-bit storage: two cells per thread in both layouts (odd x-lengths leave a
# lone last cell; 300-cell rows take two 256-cell units).  The equilibrium top
# is left out: the AA fill stores its constant rounded to the storage type,
# the pull scheme uses it in FP32.
HALF_CASES = [c for c in W.small_cases() if c.name != "eq_top"] + [
    W.channel_les(300, 9, 5).replace(name="wide_rows"),
    W.canopy_abl(257, 9, 5, h=3.0, canopy_x0=60, xbin=64).replace(name="outflow_257")]


@pytest.mark.parametrize("storage", [P.LBM_F16_SHIFTED, P.LBM_BF16_SHIFTED], ids=["f16s", "bf16s"])
@pytest.mark.parametrize("case", HALF_CASES, ids=[c.name for c in HALF_CASES])
def test_aa_half_storage_equals_pull(storage, case):
    aa, pull = P.Domain(case, storage | AA), P.Domain(case, storage)
    aa.stats_reset(True)
    pull.stats_reset(True)
    for k in (1, 50, 49):
        aa.step(k)
        pull.step(k)
        assert np.array_equal(aa.get_f(), pull.get_f()), (case.name, k)
    (ga, uba), (gp, ubp) = aa.drive(), pull.drive()
    assert uba == ubp and np.array_equal(ga, gp)
    sa, _ = aa.stats()
    sp, _ = pull.stats()
    assert np.max(np.abs(sa[:3] - sp[:3])) <= 1e-6 * max(np.abs(sp[:3]).max(), 1e-12)


def test_aa_set_f_checkpoint_and_readouts_at_odd_parity(tmp_path):
    case = W.canopy_abl(64, 24, 16, h=6.0, canopy_x0=16, xbin=16)
    a = P.Domain(case, P.LBM_F32 | AA)
    a.step(7)                      # streamed layout
    f = a.get_f()
    b = P.Domain(case, P.LBM_F32 | AA)
    b.step(3)                      # also odd: set_f writes in the current layout
    b.set_f(f)
    a.step(5)
    b.step(5)
    assert np.array_equal(a.get_f(), b.get_f())
    path = tmp_path / "aa.lbm"
    a.save(path)
    a.step(9)
    c = P.Domain(case, P.LBM_F32 | AA)
    c.load(path)
    assert c.steps_done() == 12
    c.step(9)
    assert np.array_equal(a.get_f(), c.get_f())
    # a checkpoint of the AA layout does not load into a two-set context
    d = P.Domain(case, P.LBM_F32)
    with pytest.raises(P.LbmError):
        d.load(path)
    q = a.q_criterion()
    assert np.isfinite(q).all()
    r1, u1 = np.zeros(a.shape), np.zeros((3,) + a.shape)
    P.lbm_get_macro_noalloc(a.ctx, r1, u1)
    r0, u0 = a.macro()
    assert np.allclose(r1, r0, rtol=0, atol=1e-12) and np.allclose(u1, u0, rtol=0, atol=1e-12)


def test_aa_full_size_channel_and_footprint():
    """The 256 x 128 x 128 channel in AA storage: two steps against the
    oracle, 40 steps bit-identical to the pull scheme, about half the memory."""
    case = W.channel_les()
    g = P._case_inputs(case)[0]
    pull_bytes = P.lbm_workspace_bytes(g, P.LBM_F32, 1)
    aa_bytes = P.lbm_workspace_bytes(g, P.LBM_F32 | AA, 1)
    print(f"workspace: pull {pull_bytes / 2**20:.0f} MiB, AA {aa_bytes / 2**20:.0f} MiB")
    assert aa_bytes < 0.55 * pull_bytes
    aa, o = P.Domain(case, P.LBM_F32 | AA), oracle.Oracle(case)
    aa.step(2)
    o.step(2)
    assert_population_parity(aa.get_f(), o.get_f(), 1e-6, label="channel 256x128x128 AA, 2 steps")
    o.close()
    pull = P.Domain(case, P.LBM_F32)
    pull.step(2)
    aa.step(39)
    pull.step(39)
    assert np.array_equal(aa.get_f(), pull.get_f())


def test_aa_rejects_what_it_does_not_support():
    d = P.Domain(W.small_cases()[2], P.LBM_F32 | AA)
    net = P.CorrectionNet(seed=1)
    with pytest.raises(P.LbmError) as e:
        d.set_correction(net, 0.01)
    assert e.value.status == P.LBM_ERR_ARG
    with pytest.raises(P.LbmError) as e:
        P.lbm_test_withhold_fill(d.ctx, 0)
    assert e.value.status == P.LBM_ERR_ARG
    d.step(1)
    d.sync()
