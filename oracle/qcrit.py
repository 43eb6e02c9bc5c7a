"""FP64 reference of the Q-criterion diagnostic (test infrastructure; only the
tests, the smoke check and the benchmark's baseline leg may import it).

The paper shows vortical structures as iso-surfaces of the Q-criterion
(Sec. 4, the turbulent-channel figure): Q = (|Omega|^2 - |S|^2) / 2 with the velocity
gradient G_ab = d u_a / d x_b split into its symmetric part S = (G + G^T)/2
and its antisymmetric part Omega = (G - G^T)/2, |A|^2 = sum_ab A_ab^2.  The
paper gives no discretisation; this one differentiates the cell velocities
(the velocity the next step computes) with central differences,
(u(x+1) - u(x-1)) / 2, wrapping around periodic directions and taking the
one-sided difference u(1) - u(0) (or u(n-1) - u(n-2)) at the first and last
cell of a non-periodic direction; a direction one cell wide has zero
derivative.  Written out with S and Omega as defined, nothing fused.
"""
from __future__ import annotations

import numpy as np


def gradient(u, periodic):
    """G[a][b] = d u_a / d x_b for u[3][z][y][x]; periodic = (x, y, z) flags."""
    u = np.asarray(u, dtype=np.float64)
    axes = {0: 3, 1: 2, 2: 1}  # x, y, z -> array axis of u[a]
    G = np.zeros((3, 3) + u.shape[1:])
    for a in range(3):
        for b in range(3):
            f = u[a]
            ax = axes[b] - 1  # axis within f = u[a] ([z][y][x])
            n = f.shape[ax]
            if n == 1:
                continue
            if periodic[b]:
                d = (np.roll(f, -1, axis=ax) - np.roll(f, 1, axis=ax)) / 2.0
            else:
                d = np.empty_like(f)
                sl = lambda i: tuple(slice(None) if k != ax else i for k in range(3))
                d[sl(slice(1, n - 1))] = (f[sl(slice(2, n))] - f[sl(slice(0, n - 2))]) / 2.0
                d[sl(0)] = f[sl(1)] - f[sl(0)]
                d[sl(n - 1)] = f[sl(n - 1)] - f[sl(n - 2)]
            G[a, b] = d
    return G


def q_criterion(u, periodic):
    """Q[z][y][x] from u[3][z][y][x] (see the module docstring)."""
    G = gradient(u, periodic)
    S = 0.5 * (G + G.transpose(1, 0, 2, 3, 4))
    Om = 0.5 * (G - G.transpose(1, 0, 2, 3, 4))
    return 0.5 * ((Om ** 2).sum(axis=(0, 1)) - (S ** 2).sum(axis=(0, 1)))
