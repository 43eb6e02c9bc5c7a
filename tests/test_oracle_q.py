"""Pins of the Q-criterion oracle (oracle/qcrit.py) against closed forms: on
linear velocity fields every difference is exact, so solid-body rotation,
pure strain and simple shear give omega^2, -(a^2 + b^2 + c^2)/2 and 0; on a
periodic Taylor-Green field the central difference of sin(kx) is sin(k)
cos(kx), so the discrete Q is the continuum Q with each derivative scaled by
sin(k)/k."""
import numpy as np
import pytest

from oracle.qcrit import gradient, q_criterion


def grid(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(float), y.astype(float), z.astype(float)


NP = (False, False, False)


def test_solid_body_rotation_q_is_omega_squared():
    x, y, z = grid(7, 6, 5)
    for w in (0.3, -1.7):
        u = np.stack([-w * (y - 2.5), w * (x - 3.0), np.zeros_like(x)])
        assert np.allclose(q_criterion(u, NP), w * w, rtol=0, atol=1e-13)


def test_pure_strain_q_is_minus_rate_squared():
    x, y, z = grid(6, 7, 5)
    a, b = 0.4, -0.25  # u = (a x, b y, -(a + b) z), divergence free
    u = np.stack([a * x, b * y, -(a + b) * z])
    assert np.allclose(q_criterion(u, NP), -0.5 * (a * a + b * b + (a + b) ** 2), atol=1e-13)


def test_simple_shear_has_zero_q_and_equal_strain_and_rotation():
    x, y, z = grid(5, 6, 4)
    u = np.stack([0.8 * y, np.zeros_like(x), np.zeros_like(x)])
    G = gradient(u, NP)
    assert np.allclose(G[0, 1], 0.8) and np.allclose(np.delete(G.reshape(9, -1), 1, 0), 0)
    assert np.allclose(q_criterion(u, NP), 0.0, atol=1e-15)


def test_general_linear_field_matches_the_invariant():
    rng = np.random.default_rng(5)
    A = rng.normal(size=(3, 3))
    x, y, z = grid(5, 4, 6)
    r = np.stack([x, y, z])
    u = np.einsum("ab,b...->a...", A, r)
    # Q = -(1/2) sum_ab A_ab A_ba for a constant gradient A
    assert np.allclose(q_criterion(u, NP), -0.5 * np.trace(A @ A), atol=1e-12)


@pytest.mark.parametrize("n", [8, 16, 24])
def test_periodic_taylor_green_is_the_scaled_continuum_q(n):
    x, y, z = grid(n, n, 3)
    k = 2 * np.pi / n
    u = np.stack([np.sin(k * x) * np.cos(k * y), -np.cos(k * x) * np.sin(k * y), np.zeros_like(x)])
    s = np.sin(k)  # central difference of sin(k x) = sin(k) cos(k x)
    q_exact = s * s * (np.sin(k * x) ** 2 * np.sin(k * y) ** 2 - np.cos(k * x) ** 2 * np.cos(k * y) ** 2)
    assert np.allclose(q_criterion(u, (True, True, True)), q_exact, atol=1e-14)


def test_one_cell_direction_and_planted_transpose_error():
    x, y, z = grid(6, 1, 5)  # ny = 1: no y derivative
    u = np.stack([0.5 * z, 0.2 * x, np.zeros_like(x)])
    G = gradient(u, (True, False, False))
    assert np.all(G[:, 1] == 0)
    # a Q written with Omega and S swapped, or with G G instead of G G^T, fails the rotation pin
    x, y, z = grid(7, 6, 5)
    u = np.stack([-(y - 2.5), (x - 3.0), np.zeros_like(x)])
    G = gradient(u, NP)
    wrong = -0.5 * np.einsum("ab...,ab...->...", G, G)  # sum G_ab G_ab
    assert not np.allclose(wrong, 1.0) and np.allclose(q_criterion(u, NP), 1.0)
