"""Pins of the oracle's model variants against what the mathematics fixes.

* Streamwise-only canopy drag (Eq. forestForce read as a force on u_x alone):
  the implicit velocity solves its scalar equation (checked against an
  independent root finder and the vector-drag special case), and in a uniform
  periodic box the momentum follows the recurrence m_{n+1} = m_n + rho g_c(u_n)
  with only the streamwise component changing.
* Exact-difference forcing (Kupershtokh): the moments of
  f_eq(rho, u + g) - f_eq(rho, u) are (0, rho g, rho (ug + gu + gg)); in a
  uniform box with drag the momentum follows the same recurrence as with Guo's
  forcing; the steady Poiseuille channel is the same closed form as with Guo's
  forcing (both schemes put the same odd-in-c forcing 3 w rho c.g into the
  populations per step; they differ at O(g^2) only).
* tau_total with Q^1/2 / rho^2 (the tau_total equation of Sec. 2.2 as
  printed): the root of its quadratic, equal to the 1/rho form at rho = 1.
"""
import math

import numpy as np
import pytest
from scipy.optimize import brentq

import oracle
import workloads as W


def rng(seed):
    return np.random.default_rng(seed)


# ------------------------------------------------------ streamwise-only drag ---

def _ux_by_brentq(v, k):
    s2 = v[1] ** 2 + v[2] ** 2
    if v[0] == 0.0:
        return 0.0
    f = lambda u: u * (1.0 + 0.5 * k * math.sqrt(u * u + s2)) - abs(v[0])
    return math.copysign(brentq(f, 0.0, abs(v[0]), xtol=1e-300, rtol=4 * np.finfo(float).eps,
                                maxiter=500), v[0])


@pytest.mark.parametrize("seed", range(8))
def test_streamwise_drag_velocity_solves_its_equation(seed):
    r = rng(900 + seed)
    v = 0.1 * r.standard_normal(3)
    k = r.choice([0.0, 0.03, 0.15 * 0.4, 1.0, 50.0])
    u = oracle.canopy_velocity_x(v, k)
    assert u[1] == v[1] and u[2] == v[2]            # no drag across the stream
    un = np.linalg.norm(u)
    assert abs(u[0] * (1 + 0.5 * k * un) - v[0]) <= 1e-15 * max(abs(v[0]), 1e-300)
    assert abs(u[0] - _ux_by_brentq(v, k)) <= 1e-15 * abs(v[0]) + 1e-300
    # with no cross-stream velocity the vector and streamwise drags coincide
    v1 = np.array([v[0], 0.0, 0.0])
    assert abs(oracle.canopy_velocity_x(v1, k)[0] - oracle.canopy_velocity(v1, k)[0]) \
        <= 1e-15 * abs(v[0])


def _uniform_box(scheme=0, drag_x=0, g=(0.0, 0.0, 0.0), u0=(0.03, 0.01, -0.02), a=0.4):
    ny = 3
    case = W.Case("box", 4, ny, 2, bc_y=(W.PERIODIC, W.PERIODIC), tau0=0.7, cs=0.1, cd=0.15,
                  lad=np.full(ny, a), canopy_x=(0, 4), g=g, drag_streamwise_only=drag_x,
                  forcing_scheme=scheme)
    o = oracle.Oracle(case)
    f = np.stack([np.full((2, ny, 4), v) for v in oracle.feq(1.0, np.array(u0))])
    o.set_f(f)
    return o, 0.15 * a


def _momentum(o):
    c, _ = oracle.lattice()
    mom = np.einsum("iq,qzyx->izyx", c.T.astype(float), o.get_f())
    assert np.ptp(mom, axis=(1, 2, 3)).max() < 1e-16  # stays uniform
    return mom[:, 0, 0, 0]


@pytest.mark.parametrize("scheme", [0, 1], ids=["guo", "exact_difference"])
def test_streamwise_drag_momentum_recurrence(scheme):
    """Uniform periodic box, no driving: with the drag on u_x alone only the
    streamwise momentum decays, m_x <- m_x - k |u| u_x, with u the implicit
    velocity of m (root found here by brentq); m_y and m_z stay."""
    o, k = _uniform_box(scheme=scheme, drag_x=1)
    m = np.array([0.03, 0.01, -0.02])
    for n in range(150):
        o.step(1)
        u = np.array([_ux_by_brentq(m, k), m[1], m[2]])
        m = m - np.array([k * np.linalg.norm(u) * u[0], 0.0, 0.0])
    mo = _momentum(o)
    assert np.max(np.abs(mo - m)) < 1e-15
    # (exact-difference forcing rounds rho (m / rho) once per step)
    assert mo[1] == pytest.approx(0.01, abs=1e-15) and mo[2] == pytest.approx(-0.02, abs=1e-15)
    assert mo[0] < 0.03  # decayed


# ---------------------------------------------------- exact-difference forcing ---

@pytest.mark.parametrize("seed", range(6))
def test_exact_difference_force_moments(seed):
    r = rng(950 + seed)
    rho = 1.0 + 0.05 * r.standard_normal()
    u = 0.05 * r.standard_normal(3)
    g = 1e-3 * r.standard_normal(3)
    F = oracle.edm_force(rho, u, g)
    c, _ = oracle.lattice()
    c = c.astype(float)
    # F is a difference of equilibria of size ~ w rho: rounding ~1e-16 rho,
    # against moments of size |g| ~ 1e-3
    assert abs(F.sum()) < 1e-15
    assert np.max(np.abs(F @ c - rho * g)) < 1e-15
    pi = np.einsum("i,ia,ib->ab", F, c, c)
    exact = rho * (np.outer(u, g) + np.outer(g, u) + np.outer(g, g))
    assert np.max(np.abs(pi - exact)) < 1e-15


def test_exact_difference_momentum_recurrence_with_drag_and_driving():
    """Uniform periodic box with a driving acceleration and vector drag: the
    collision conserves the momentum it relaxes (rho u_b = m), so per step
    m <- m + rho (g_drive - k |u| u), u the implicit velocity of
    v = m + g_drive/2 (rho = 1) -- the same recurrence as with Guo's forcing."""
    gd = np.array([2e-5, 0.0, -1e-5])
    o, k = _uniform_box(scheme=1, g=tuple(gd))
    m = np.array([0.03, 0.01, -0.02])
    for n in range(150):
        o.step(1)
        v = m + 0.5 * gd
        vn = np.linalg.norm(v)
        s = 2.0 * vn / (1.0 + math.sqrt(1.0 + 2.0 * k * vn))
        u = v * (s / vn)
        m = m + gd - k * s * u
    assert np.max(np.abs(_momentum(o) - m)) < 1e-15
    # the reported velocity is the physical one, m/rho + g_total/2
    rho, u = o.macro()
    v = m + 0.5 * gd
    vn = np.linalg.norm(v)
    uu = v * (2.0 / (1.0 + math.sqrt(1.0 + 2.0 * k * vn)))
    assert np.max(np.abs(u[:, 0, 0, 0] - uu)) < 1e-15


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_exact_difference_poiseuille_closed_form(tau):
    """The steady bounce-back channel under exact-difference forcing is the
    closed form of Guo's forcing, parabola g/(2nu) eta (H - eta) plus the slip
    g (16 L - 3) / (24 nu), L = (tau - 1/2)^2: in a steady x-uniform flow only
    the odd-in-c parts of the populations carry x-momentum, and both schemes
    add 3 w rho c.g to them per step."""
    H, g = 16, 1e-6
    nu, lam = (tau - 0.5) / 3, (tau - 0.5) ** 2
    o = oracle.Oracle(W.poiseuille(1, H, 1, g=g, tau=tau).replace(forcing_scheme=1))
    o.step(20000)
    u = o.macro()[1][0, 0, :, 0]
    eta = np.arange(H) + 0.5
    exact = g / (2 * nu) * eta * (H - eta) + g * (16 * lam - 3) / (24 * nu)
    assert np.max(np.abs(u - exact)) / exact.max() < 1e-8


# ------------------------------------------------------- tau_total with rho^2 ---

@pytest.mark.parametrize("seed", range(6))
def test_tau_total_rho2_is_the_root_of_its_quadratic(seed):
    r = rng(980 + seed)
    tau0 = 0.5 + r.uniform(1e-3, 0.5)
    cs = r.uniform(0.05, 0.3)
    rho = 1.0 + 0.05 * r.standard_normal()
    pineq = 1e-3 * r.standard_normal(6)
    q = math.sqrt(sum(p * p for p in pineq[:3]) + 2 * sum(p * p for p in pineq[3:]))
    t2 = oracle.tau_total_p(tau0, cs, rho, pineq, 2)
    # tau^2 - tau0 tau - 9 sqrt(2) C_s^2 Q^(1/2) / (2 rho^2) = 0, the positive root
    assert abs(t2 * t2 - tau0 * t2 - 9 * math.sqrt(2) * cs * cs * q / (2 * rho * rho)) < 1e-15
    assert t2 > tau0
    assert oracle.tau_total_p(tau0, cs, rho, pineq, 1) == oracle.tau_total(tau0, cs, rho, pineq)
    assert oracle.tau_total_p(tau0, cs, 1.0, pineq, 2) == oracle.tau_total_p(tau0, cs, 1.0, pineq, 1)
    assert oracle.tau_total_p(tau0, 0.0, rho, pineq, 2) == tau0


def test_variant_parameters_are_checked():
    for kw in ({"drag_streamwise_only": 2}, {"forcing_scheme": 2}, {"sgs_rho_power": 3}):
        with pytest.raises(ValueError):
            oracle.Oracle(W.poiseuille(4, 4, 4).replace(**kw))
