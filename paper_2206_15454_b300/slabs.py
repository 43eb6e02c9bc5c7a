"""x-slab decomposition of one domain over several ranks: the host-side logic.

A periodic-in-x domain of nx columns is cut into contiguous slabs, one per
rank.  Each rank keeps its slab with one halo column on each side.  Per time
step a face exchanges only what streams across it (Sec. 2.1, Eq. lbe: the pull
f_i(x) <- f*_i(x - c_i) reaches one column across a slab face, and only for
the five directions with c_x = +1 or -1):

* the last owned column's c_x = +1 populations go to the right neighbour,
  which keeps them in its left halo;
* the first owned column's c_x = -1 populations go to the left neighbour,
  which keeps them in its right halo.

The per-plane statistics (Sec. 4: mean velocity and Reynolds-stress
profiles) are sums over cells, so they need one all-reduce of the plane sums
per read-out.

Arrays use the public population layout f[q][z][y][x] (FP64).  The exchange
runs over torch.distributed point-to-point calls (gloo on the host); this
module holds no arithmetic of the method.
"""
from __future__ import annotations

import numpy as np

# directions with c_x = +1 and c_x = -1 (public direction order)
PLUS_X = (1, 7, 9, 11, 13)
MINUS_X = (2, 8, 10, 12, 14)


def slab_bounds(nx: int, world: int, rank: int) -> tuple:
    """Owned columns [x0, x1) of `rank`: contiguous, sizes differing by at
    most one, the larger slabs first."""
    if not 0 <= rank < world or nx < world:
        raise ValueError("need 0 <= rank < world <= nx")
    base, extra = divmod(nx, world)
    x0 = rank * base + min(rank, extra)
    return x0, x0 + base + (1 if rank < extra else 0)


def slab_case(case, x0: int, x1: int):
    """The slab [x0, x1) of a periodic-in-x case as a domain of its own,
    x1 - x0 + 2 columns wide (a halo column on each side, the slab periodic in
    itself until the halos are overwritten).  The canopy's x-range moves with
    the slab; statistics are kept per plane."""
    if tuple(case.bc_x) != (0, 0):
        raise ValueError("the x-slab decomposition needs a periodic x direction")
    if case.u_bulk_target > 0:
        raise ValueError("a bulk-velocity controller needs a global sum every step")
    c0, c1 = case.canopy_x
    lo, hi = max(c0, x0 - 1), min(c1, x1 + 1)
    canopy = (lo - x0 + 1, hi - x0 + 1) if lo < hi else (0, 0)
    return case.replace(name=f"{case.name}_slab{x0}_{x1}", nx=x1 - x0 + 2, canopy_x=canopy,
                        stats_xbins=1)


def extract(f_global: np.ndarray, x0: int, x1: int) -> np.ndarray:
    """Slab [x0, x1) with its two halo columns from a global population array
    (periodic wrap)."""
    nx = f_global.shape[-1]
    cols = [(x0 - 1) % nx] + list(range(x0, x1)) + [x1 % nx]
    return np.ascontiguousarray(f_global[..., cols])


def owned(f_slab: np.ndarray) -> np.ndarray:
    """The owned columns of a slab array (halos dropped)."""
    return f_slab[..., 1:-1]


def faces(f_slab: np.ndarray) -> tuple:
    """What this slab sends: (to the left neighbour: the c_x = -1 populations
    of its first owned column, to the right neighbour: the c_x = +1
    populations of its last owned column), each [5][z][y]."""
    return (np.ascontiguousarray(f_slab[list(MINUS_X), :, :, 1]),
            np.ascontiguousarray(f_slab[list(PLUS_X), :, :, -2]))


def fill_halos(f_slab: np.ndarray, from_left: np.ndarray, from_right: np.ndarray) -> None:
    """Write the received faces into the halo columns: the left neighbour's
    c_x = +1 populations into the left halo, the right neighbour's c_x = -1
    populations into the right halo (the only halo values a step reads)."""
    f_slab[list(PLUS_X), :, :, 0] = from_left
    f_slab[list(MINUS_X), :, :, -1] = from_right


def exchange(f_slab: np.ndarray, rank: int, world: int) -> None:
    """One halo exchange around the periodic ring of slabs (torch.distributed
    point-to-point; tag 0 travels left, tag 1 travels right)."""
    import torch
    import torch.distributed as dist

    to_left, to_right = faces(f_slab)
    if world == 1:
        fill_halos(f_slab, to_right, to_left)
        return
    left, right = (rank - 1) % world, (rank + 1) % world
    recv_from_right = torch.empty(to_left.shape, dtype=torch.float64)
    recv_from_left = torch.empty(to_right.shape, dtype=torch.float64)
    reqs = [dist.isend(torch.from_numpy(to_left), left, tag=0),
            dist.isend(torch.from_numpy(to_right), right, tag=1),
            dist.irecv(recv_from_right, right, tag=0),
            dist.irecv(recv_from_left, left, tag=1)]
    for r in reqs:
        r.wait()
    fill_halos(f_slab, recv_from_left.numpy(), recv_from_right.numpy())


def allreduce_sum(a: np.ndarray) -> np.ndarray:
    """Sum of an FP64 array over all ranks (the plane sums of the statistics)."""
    import torch
    import torch.distributed as dist

    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


# ---- the library's x-slab data path ------------------------------------------------

def slab_case_halo(case, x0: int, x1: int):
    """The slab [x0, x1) of a periodic-in-x case as a library domain whose x
    faces are halos (LBM_BC_HALO): x1 - x0 columns, the neighbours' columns
    living in the ghost slots that lbm_halo_unpack fills.  The canopy's
    x-range moves with the slab; statistics are kept per plane."""
    from . import LBM_BC_HALO

    if tuple(case.bc_x) != (0, 0):
        raise ValueError("the x-slab decomposition needs a periodic x direction")
    if case.u_bulk_target > 0:
        raise ValueError("a bulk-velocity controller needs a global sum every step")
    c0, c1 = case.canopy_x
    lo, hi = max(c0, x0), min(c1, x1)
    canopy = (lo - x0, hi - x0) if lo < hi else (0, 0)
    return case.replace(name=f"{case.name}_halo{x0}_{x1}", nx=x1 - x0, canopy_x=canopy,
                        bc_x=(LBM_BC_HALO, LBM_BC_HALO), stats_xbins=1)


class DeviceSlabs:
    """One periodic-in-x domain cut into `nslabs` x-slabs, each an lbm_ctx with
    halo faces, all on this GPU and stream.  Per step every slab steps, packs
    its two outgoing faces into device buffers, the buffers are copied
    device-to-device to the neighbours' receive buffers (the exchange a
    multi-GPU run does with NCCL send/receive or peer copies into local
    memory), and every slab unpacks what it received.  The state is set from a
    global population array (public layout) and read back as one."""

    def __init__(self, case, nslabs, storage=0):
        import torch

        from . import Domain, lbm_halo_bytes

        self.case, self.storage = case, storage
        self.bounds = [slab_bounds(case.nx, nslabs, r) for r in range(nslabs)]
        self.doms = [Domain(slab_case_halo(case, x0, x1), storage) for x0, x1 in self.bounds]
        nb = lbm_halo_bytes(self.doms[0].ctx)
        mk = lambda: torch.empty(nb, dtype=torch.uint8, device="cuda")
        self.send = [(mk(), mk()) for _ in self.doms]   # (to the left, to the right)
        self.recv = [(mk(), mk()) for _ in self.doms]   # (from the left, from the right)

    def exchange(self):
        from . import lbm_halo_pack, lbm_halo_unpack

        n = len(self.doms)
        for d, (lo, hi) in zip(self.doms, self.send):
            lbm_halo_pack(d.ctx, lo.data_ptr(), hi.data_ptr())
        for r in range(n):
            self.recv[r][0].copy_(self.send[(r - 1) % n][1])  # left neighbour's last column
            self.recv[r][1].copy_(self.send[(r + 1) % n][0])  # right neighbour's first column
        for d, (lo, hi) in zip(self.doms, self.recv):
            lbm_halo_unpack(d.ctx, lo.data_ptr(), hi.data_ptr())

    def set_f(self, f_global):
        for d, (x0, x1) in zip(self.doms, self.bounds):
            d.set_f(np.ascontiguousarray(f_global[..., x0:x1]))
        self.exchange()

    def step(self, n=1):
        for _ in range(n):
            for d in self.doms:
                d.step(1)
            self.exchange()

    def get_f(self):
        return np.concatenate([d.get_f() for d in self.doms], axis=-1)

    def stats_reset(self, enable=True):
        for d in self.doms:
            d.stats_reset(enable)

    def stats(self):
        """Plane statistics of the whole domain from the slabs' (the plane sums
        add up; the covariances are recombined from the slabs' raw moments)."""
        out = [d.stats() for d in self.doms]
        n = out[0][1]
        w = np.array([x1 - x0 for x0, x1 in self.bounds], dtype=np.float64) / self.case.nx
        mean = sum(wi * s[:3] for wi, (s, _) in zip(w, out))
        pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
        res = np.zeros_like(out[0][0])
        res[:3] = mean
        for k, (a, b) in enumerate(pairs):
            raw = sum(wi * (s[3 + k] + s[a] * s[b]) for wi, (s, _) in zip(w, out))
            res[3 + k] = raw - mean[a] * mean[b]
        return res, n

    def close(self):
        for d in self.doms:
            d.close()
