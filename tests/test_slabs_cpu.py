"""x-slab decomposition on the CPU: gloo ranks on 127.0.0.1 each step the FP64
oracle on their slab and exchange the five c_x = +-1 populations of each face
per step (paper_2206_15454_b300.slabs).  The owned columns must equal the
undivided oracle bit for bit, and the all-reduced plane sums must equal the
undivided plane sums up to FP64 summation order."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W
from paper_2206_15454_b300 import slabs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cases():
    return {
        # constant driving force (the controller needs a global sum every step)
        "channel": W.channel_les(23, 10, 6).replace(u_bulk_target=0.0, g=(2e-5, 0.0, 0.0),
                                                    init_perturb=0.01),
        # the paper's forest ABL: canopy over all x, equilibrium top
        "forest": W.abl_forest(1, nx=17, ny=12, nz=5),
        # a canopy over part of x, so slabs see both sides of its edge
        "canopy_edge": W.channel_les(20, 9, 4).replace(
            u_bulk_target=0.0, g=(2e-5, 0.0, 0.0), cd=0.15, canopy_x=(5, 13),
            lad=W.lad_constant(9, 0.3, 4.0), init_perturb=0.01),
    }


def _plane_sums(rho, u):
    """Sum over (z, x) per y of u, v, w and their products (the statistics'
    per-plane sums) from fields [z][y][x]."""
    q = [u[0], u[1], u[2], u[0] * u[0], u[1] * u[1], u[2] * u[2], u[0] * u[1], u[0] * u[2],
         u[1] * u[2]]
    return np.stack([a.sum(axis=(0, 2)) for a in q])


def _rank(rank, world, port, name, steps, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    import oracle

    dist.init_process_group("gloo", rank=rank, world_size=world)
    case = _cases()[name]
    x0, x1 = slabs.slab_bounds(case.nx, world, rank)
    full = oracle.Oracle(case)  # the initial state of the whole domain
    f0 = full.get_f()
    full.close()
    o = oracle.Oracle(slabs.slab_case(case, x0, x1))
    f = slabs.extract(f0, x0, x1)
    for _ in range(steps):
        o.set_f(f)
        o.step(1)
        f = o.get_f()
        slabs.exchange(f, rank, world)
    o.set_f(f)
    rho, u = o.macro()
    sums = slabs.allreduce_sum(_plane_sums(slabs.owned(rho), slabs.owned(u)))
    out[rank] = (x0, x1, slabs.owned(f).copy(), sums)
    o.close()
    dist.destroy_process_group()


def test_slab_bounds_cover_the_row():
    for nx, world in ((23, 2), (23, 3), (7, 7), (64, 4)):
        b = [slabs.slab_bounds(nx, world, r) for r in range(world)]
        assert b[0][0] == 0 and b[-1][1] == nx
        assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
        assert max(x1 - x0 for x0, x1 in b) - min(x1 - x0 for x0, x1 in b) <= 1
    with pytest.raises(ValueError):
        slabs.slab_bounds(3, 4, 0)


def test_faces_and_halos_move_the_streaming_populations():
    # a face carries exactly the populations that cross it in one pull
    f = np.arange(19 * 2 * 3 * 6, dtype=np.float64).reshape(19, 2, 3, 6)
    to_left, to_right = slabs.faces(f)
    assert np.array_equal(to_left, f[[2, 8, 10, 12, 14], :, :, 1])
    assert np.array_equal(to_right, f[[1, 7, 9, 11, 13], :, :, 4])
    g = f.copy()
    slabs.fill_halos(g, to_right + 0.5, to_left + 0.25)
    assert np.array_equal(g[[1, 7, 9, 11, 13], :, :, 0], to_right + 0.5)
    assert np.array_equal(g[[2, 8, 10, 12, 14], :, :, 5], to_left + 0.25)
    rest = np.ones(g.shape, bool)
    rest[[1, 7, 9, 11, 13], :, :, 0] = False
    rest[[2, 8, 10, 12, 14], :, :, 5] = False
    assert np.array_equal(g[rest], f[rest])


def test_slab_case_rejects_what_does_not_decompose():
    with pytest.raises(ValueError):
        slabs.slab_case(W.canopy_abl(64, 16, 8), 0, 32)       # inflow/outflow in x
    with pytest.raises(ValueError):
        slabs.slab_case(W.channel_les(32, 16, 8), 0, 16)      # bulk-velocity controller


@pytest.mark.parametrize("name,world", [("channel", 2), ("forest", 3), ("canopy_edge", 2)])
def test_slabs_match_the_undivided_oracle(name, world):
    import oracle

    steps = 12
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, name, steps, out), nprocs=world, join=True)
        res = dict(out)
    case = _cases()[name]
    ref = oracle.Oracle(case)
    ref.step(steps)
    f_ref = ref.get_f()
    rho, u = ref.macro()
    ref.close()
    got = np.concatenate([res[r][2] for r in range(world)], axis=-1)
    assert [res[r][:2] for r in range(world)] == \
        [slabs.slab_bounds(case.nx, world, r) for r in range(world)]
    # the same FP64 operations on the same inputs: bit for bit
    assert np.array_equal(got, f_ref)
    sums = _plane_sums(rho, u)
    for r in range(world):
        np.testing.assert_allclose(res[r][3], sums, rtol=1e-12, atol=1e-15)
