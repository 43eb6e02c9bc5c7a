"""The model variants on the GPU against the FP64 oracle: canopy drag on the
streamwise component only (Eq. forestForce read as a streamwise force),
exact-difference forcing (Kupershtokh) in place of Guo's (Eq. bodyforce), and
Q^1/2 / rho^2 under the root of tau_total (the tau_total equation as printed
in Sec. 2.2), alone and together, over the first 100 steps (FP32 parity
bounds), plus the read-outs that follow the model (velocity, strain rate) and
the bulk-velocity controller."""
import numpy as np
import pytest

import oracle
import paper_2206_15454_b300 as P
import workloads as W
from parity_util import assert_population_parity

pytestmark = pytest.mark.gpu

SMALL = W.small_cases()
VARIANTS = {
    "drag_x": dict(drag_streamwise_only=1),
    "edm": dict(forcing_scheme=1),
    "rho2": dict(sgs_rho_power=2),
    "all": dict(drag_streamwise_only=1, forcing_scheme=1, sgs_rho_power=2),
}


def strong_forcing_box():
    """A periodic box with strong driving, very dense Gaussian canopy (C_D a up to
    3 per cell), C_s = 0.3 and 10 % velocity perturbations: accelerations of
    1e-3..1e-2 per step and density varying by about 1 %, where each variant
    changes the state by more than 1e-5 within 100 steps (exact-difference and
    Guo forcing differ at O(g^2); the rho power matters through rho - 1)."""
    ny = 8
    return W.Case("strong_forcing_box", 16, ny, 8, bc_y=(W.PERIODIC, W.PERIODIC), tau0=0.51,
                  cs=0.3, g=(2e-3, 5e-4, -3e-4), cd=0.15, canopy_x=(2, 14),
                  lad=W.lad_gaussian(ny, 20.0, 8.0), seed=21, init_perturb=0.1,
                  u_profile=np.full(ny, 0.08))


CASES = [
    strong_forcing_box(),
    SMALL[2],                                             # canopy, inflow/outflow, x-bins
    SMALL[3],                                             # ragged channel + canopy, controller
    SMALL[6],                                             # periodic box, 3-component driving, Gaussian LAD
    W.canopy_abl(300, 9, 5, h=3.0, canopy_x0=40, xbin=60).replace(name="two_chunk_canopy"),
]


@pytest.mark.parametrize("variant", list(VARIANTS), ids=list(VARIANTS))
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_variant_first_100_steps_f32(case, variant):
    c = case.replace(**VARIANTS[variant])
    d, o = P.Domain(c), oracle.Oracle(c)
    for k in (1, 99):
        d.step(k)
        o.step(k)
    assert_population_parity(d.get_f(), o.get_f(), 1e-6, label=f"{c.name} {variant}")
    rho_d, u_d = d.macro()
    rho_o, u_o = o.macro()
    assert np.max(np.abs(rho_d - rho_o)) < 1e-6
    assert np.max(np.abs(u_d - u_o)) <= 1e-4 * np.abs(u_o).max() + 1e-9
    if c.u_bulk_target > 0:
        (gd, ubd), (go, ubo) = d.drive(), o.drive()
        assert abs(ubd - ubo) < 2e-6 * abs(ubo)


def test_variants_change_the_flow():
    """Each variant is a different model: after 100 steps its state differs
    from the default one by more than twice the FP32 parity bound (1e-6), so a
    kernel that ignored the flag would fail the variant parity test above
    (the measured FP32 error is about 1e-7)."""
    base = strong_forcing_box()
    d0 = P.Domain(base)
    d0.step(100)
    f0 = d0.get_f()
    for name, kw in VARIANTS.items():
        d = P.Domain(base.replace(**kw))
        d.step(100)
        diff = np.linalg.norm(d.get_f() - f0) / np.linalg.norm(f0)
        print(f"{name}: rel L2 difference from the default model after 100 steps {diff:.2e}")
        assert diff > 2e-6, name


@pytest.mark.parametrize("variant", ["drag_x", "edm", "all"])
def test_variant_features_match_oracle(variant):
    """The correction network's inputs (u_x and the strain rate of the three
    lowest cells) follow the model: the strain rate from Pi_neq against the
    equilibrium the collision relaxes towards, with its tau_total."""
    c = W.canopy_abl(40, 12, 6, h=4.0, canopy_x0=12, xbin=8).replace(**VARIANTS[variant])
    d, o = P.Domain(c), oracle.Oracle(c)
    d.step(30)
    o.step(30)
    Xg, Xo = d.features(), o.features()
    scale = np.abs(Xo).max(axis=0)
    scale[scale == 0] = 1.0
    err = (np.abs(Xg - Xo) / scale).max(axis=0)
    assert np.all(err[:3] < 1e-5) and np.all(err[3:6] < 1e-3) and np.all(err[6:] < 1e-6), err


def test_variant_half_storage_error_is_stated():
    c = SMALL[2].replace(**VARIANTS["all"])
    o = oracle.Oracle(c)
    o.step(100)
    for st, bound in ((P.LBM_F16_SHIFTED, 3e-4), (P.LBM_BF16_SHIFTED, 2.5e-3)):
        d = P.Domain(c, st)
        d.step(100)
        err = np.linalg.norm(d.get_f() - o.get_f()) / np.linalg.norm(o.get_f())
        print(f"all variants, storage {st}: population rel L2 after 100 steps {err:.2e}")
        assert err < bound
