"""The checked build (LBM_CHECK_BOUNDS: every bulk copy and global store of
the step, and every access of the AA-pattern kernels, verified against its
buffer) on every small boundary combination, ragged rows, chunked rows, a
one-cell outflow chunk, 16-bit storage, an ensemble, x-binned statistics, the
model variants, halo slabs and AA-pattern storage: no index leaves its buffer
and the results still match the FP64 oracle.  Runs in a child process, which loads the checked
library instead of the default one."""
import os
import subprocess
import sys

import pytest

from paper_2206_15454_b300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
import paper_2206_15454_b300 as P
import workloads as W
import oracle
P.LIB_PATH = sys.argv[1]
cases = W.small_cases() + [
    W.Case("tiny_periodic", 1, 1, 1, bc_y=(W.PERIODIC, W.PERIODIC), tau0=0.7, init_perturb=0.03, seed=9),
    W.poiseuille(1, 32, 1).replace(name="column"),
    W.channel_les(300, 9, 5).replace(name="two_x_chunks"),
    W.canopy_abl(257, 9, 5, h=3.0, canopy_x0=60, xbin=64).replace(name="outflow_one_cell_chunk"),
    W.canopy_abl(600, 12, 6, h=4.0, canopy_x0=100, xbin=60).replace(name="xbinned_three_chunks"),
]
worst = 0.0
for c in cases:
    for st in (P.LBM_F32, P.LBM_F16_SHIFTED):
        d, o = P.Domain(c, st), oracle.Oracle(c)
        d.stats_reset(True)
        o.stats_reset(True)
        d.step(12)
        o.step(12)
        d.stats()
        a, b = d.get_f(), o.get_f()
        err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        bound = 1e-6 if st == P.LBM_F32 else 5e-3
        assert err <= bound, (c.name, st, err)
        worst = max(worst, err) if st == P.LBM_F32 else worst
        d.close()
        o.close()
boxes = W.ensemble_boxes(n_boxes=5, ny=16, nz=12, nx_range=(40, 150), seed=77)
bt = P.Batch(boxes, P.LBM_F16_SHIFTED)
bt.step(6)
bt.sync()
for i, c in enumerate(boxes):
    alone = P.Domain(c, P.LBM_F16_SHIFTED)
    alone.step(6)
    assert np.array_equal(bt.box(i).get_f(), alone.get_f()), c.name
    alone.close()
bt.close()
# the model variants and the halo data path under the same checks
for c in (cases[2].replace(drag_streamwise_only=1, forcing_scheme=1, sgs_rho_power=2),
          cases[6].replace(forcing_scheme=1)):
    d, o = P.Domain(c), oracle.Oracle(c)
    d.step(12)
    o.step(12)
    a, b = d.get_f(), o.get_f()
    err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert err <= 1e-6, (c.name, "variant", err)
    d.close()
# AA-pattern storage: every load and store of the fill and step kernels checked
for c in cases:
    for st in (P.LBM_F32 | P.LBM_STORAGE_AA, P.LBM_F16_SHIFTED | P.LBM_STORAGE_AA):
        d, o = P.Domain(c, st), oracle.Oracle(c)
        d.stats_reset(True)
        d.step(11)
        o.step(11)
        d.stats()
        a, b = d.get_f(), o.get_f()
        err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        assert err <= (1e-6 if st == P.LBM_F32 | P.LBM_STORAGE_AA else 5e-3), (c.name, "AA", st, err)
        d.close()
        o.close()
# ... and on faces longer than the fill grid's 65,535 block rows (its
# grid-stride loop)
c = W.poiseuille(2, 3, 70000).replace(name="tall_z", init_perturb=0.03, seed=11)
d, o = P.Domain(c, P.LBM_F32 | P.LBM_STORAGE_AA), oracle.Oracle(c)
d.step(11)
o.step(11)
a, b = d.get_f(), o.get_f()
err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
assert err <= 1e-6, (c.name, "AA", err)
d.close()
o.close()
from paper_2206_15454_b300 import slabs as S
c = W.channel_les(150, 9, 6).replace(u_bulk_target=0.0, ctrl_gain=0.0)
whole = P.Domain(c)
f0 = whole.get_f()
whole.set_f(f0)
sl = S.DeviceSlabs(c, 3)
sl.set_f(f0)
whole.step(12)
sl.step(12)
assert np.array_equal(sl.get_f(), whole.get_f()), "halo slabs differ"
sl.doms[0].sync()
print("checked build ok; worst FP32 rel L2", worst)
'''


def test_checked_build_keeps_every_index_in_its_buffer():
    lib = B.build(checked=True)
    r = subprocess.run([sys.executable, "-c", CHILD, lib], cwd=ROOT, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout
