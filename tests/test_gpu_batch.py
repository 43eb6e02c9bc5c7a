"""Ensembles of independent boxes (all boxes' steps in one CUDA graph, a
launch per chain of boxes and step) against the FP64 oracle and against the
same boxes run one at a time."""
import numpy as np
import pytest

import oracle
import paper_2206_15454_b300 as P
import workloads as W
from parity_util import assert_population_parity

pytestmark = pytest.mark.gpu


def small_boxes():
    # uneven x-lengths spanning one to three 64-cell chunks and a ragged tail
    return W.ensemble_boxes(n_boxes=5, ny=16, nz=12, nx_range=(40, 150), seed=77)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_batch_boxes_match_oracle_first_100_steps():
    cases = small_boxes()
    b = P.Batch(cases, P.LBM_F32)
    b.step(100)
    for i, c in enumerate(cases):
        o = oracle.Oracle(c)
        o.step(100)
        assert_population_parity(b.box(i).get_f(), o.get_f(), 1e-6, label=f"{c.name} nx={c.nx}")


@pytest.mark.parametrize("storage", [P.LBM_F32, P.LBM_F16_SHIFTED])
@pytest.mark.parametrize("widths", [0, -1])
def test_batch_equals_boxes_run_alone_bitwise(storage, widths):
    """Same per-cell arithmetic whatever the launch: a box advanced inside the
    ensemble is bit-identical to the box advanced on its own.  x-lengths 49,
    166, 142, 128, 168: widths 0 puts every box at 256 cells (two chains of
    alternate boxes), -1 each box in its own width, 64, 128 and 256 (three
    chains)."""
    cases = W.ensemble_boxes(n_boxes=5, ny=16, nz=12, nx_range=(40, 200), seed=77)
    assert sorted(c.nx for c in cases) == [49, 128, 142, 166, 168]
    b = P.Batch(cases, storage, tune_steps=widths)
    assert b.tuning()[0] == (256 if widths == 0 else 0)
    b.step(7)
    b.step(7)   # the graph for 7 steps is built once, then replayed from the other parity
    b.step(20)
    for i, c in enumerate(cases):
        d = P.Domain(c, storage)
        d.step(34)
        assert b.box(i).steps_done() == 34
        assert np.array_equal(b.box(i).get_f(), d.get_f()), c.name


def test_tuned_batch_reports_its_choice_and_stays_exact():
    cases = small_boxes()
    b = P.Batch(cases, P.LBM_F16_SHIFTED, tune_steps=4)
    xt, blocks, ms = b.tuning()
    assert xt in (0, 64, 128, 256) and blocks >= len(cases) and ms > 0  # 0: each box its own width
    tried = b.candidates()
    assert len(tried) >= 3 and min(t[2] for t in tried if t[2] > 0) == ms
    assert all(b.box(i).steps_done() == 0 for i in range(len(cases)))  # re-initialised
    b.step(10)
    for i, c in enumerate(cases):
        d = P.Domain(c, P.LBM_F16_SHIFTED)
        d.step(10)
        assert np.array_equal(b.box(i).get_f(), d.get_f())


def test_batch_statistics_and_errors():
    cases = small_boxes()
    b = P.Batch(cases, P.LBM_F32)
    b.step(5)
    b.stats_reset(True)
    b.step(12)
    for i, c in enumerate(cases):
        d = P.Domain(c, P.LBM_F32)
        d.step(5)
        d.stats_reset(True)
        d.step(12)
        sb, nb = b.box(i).stats()
        sd, nd = d.stats()
        assert nb == nd == 12
        # the same cells summed in other groupings (FP32 per-thread partial sums)
        assert np.max(np.abs(sb[:3] - sd[:3])) < 1e-6 * np.abs(sd[:3]).max()
        assert np.max(np.abs(sb[3:] - sd[3:])) < 1e-3 * np.abs(sd[3:]).max()
    # statistics on for some boxes only is refused (argument error, not sticky)
    P.lbm_stats_reset(b.box(0).ctx, False)
    with pytest.raises(P.LbmError) as e:
        b.step(1)
    assert e.value.status == P.LBM_ERR_ARG
    b.stats_reset(False)
    b.step(1)
    b.sync()
    # a box is owned by its ensemble: lbm_destroy on it does nothing
    P.lbm_destroy(b.box(1).ctx)
    assert b.box(1).steps_done() == 18


def test_full_size_ensemble_64_boxes_fp16():
    """64 canopy boxes of 96..160 x 64 x 64 cells in FP16-shifted storage."""
    cases = W.ensemble_boxes()
    b = P.Batch(cases, P.LBM_F16_SHIFTED)
    m0 = [b.box(i).mass() for i in (0, 31, 63)]
    b.step(20)
    b.sync()
    for k, i in enumerate((0, 31, 63)):
        assert abs(b.box(i).mass() - m0[k]) / m0[k] < 1e-4
    # spot check one box against the oracle after 20 steps
    o = oracle.Oracle(cases[5])
    o.step(20)
    assert rel_l2(b.box(5).get_f(), o.get_f()) < 5e-4
