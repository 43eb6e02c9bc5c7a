"""Q-criterion read-out (lbm_get_q) against the FP64 oracle: the same steps on
both sides, then Q of the velocity field the next step computes, cell by
cell.  The GPU differentiates FP32 velocities, so the bound is relative to the
largest |Q| of the field."""
import numpy as np
import pytest

import oracle
import paper_2206_15454_b300 as P
import workloads as W
from oracle.qcrit import q_criterion

pytestmark = pytest.mark.gpu

CASES = [
    W.channel_les(48, 24, 20).replace(init_perturb=0.01),                 # walls in y, periodic x, z
    W.canopy_abl(64, 24, 16, h=6.0, canopy_x0=16, xbin=16),                # inflow/outflow in x
    W.abl_forest(2, nx=40, ny=16, nz=12),                                  # equilibrium top
    W.poiseuille(1, 16, 5).replace(name="one_cell_x"),                     # nx = 1
]


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_q_matches_oracle(case):
    d = P.Domain(case, P.LBM_F32)
    o = oracle.Oracle(case)
    d.step(20)
    o.step(20)
    q = d.q_criterion()
    _, u = o.macro()
    periodic = (case.bc_x[0] == 0, case.bc_y[0] == 0, True)
    ref = q_criterion(u, periodic)
    scale = np.abs(ref).max()
    assert scale > 0 or case.nx == 1
    assert np.abs(q - ref).max() <= 1e-4 * max(scale, 1e-30) + 1e-18
    d.close()
    o.close()


def test_q_of_a_taylor_green_field_marks_the_vortex_cores():
    # equilibrium populations of a Taylor-Green velocity field, set through
    # the C ABI on both sides
    case = W.poiseuille(16, 16, 4).replace(bc_y=(0, 0))  # fully periodic box
    d = P.Domain(case, P.LBM_F32)
    o = oracle.Oracle(case)
    f = o.get_f()
    nz, ny, nx = o.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    k = 2 * np.pi / nx
    ux = 0.01 * np.sin(k * x) * np.cos(k * y)
    uy = -0.01 * np.cos(k * x) * np.sin(k * y)
    c = np.array(oracle.lattice()[0])
    w = np.array(oracle.lattice()[1])
    for i in range(19):
        cu = c[i, 0] * ux + c[i, 1] * uy
        f[i] = w[i] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))
    d.set_f(f)
    o.set_f(f)
    q = d.q_criterion()
    ref = q_criterion(o.macro()[1], (True, True, True))
    assert np.abs(q - ref).max() <= 1e-4 * np.abs(ref).max()
    # Taylor-Green cells: rotation dominates in a cell's core, strain at the
    # stagnation point between cells
    assert q[0, 0, 0] < 0 < q[0, nx // 4, nx // 4]
    d.close()
    o.close()
