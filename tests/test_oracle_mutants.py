"""The pins catch plausible mistakes: each case plants one mistake in a copy of
the oracle's C source (on the CPU, in a temporary directory), builds it, and
checks that the pin aimed at that part of the method now fails."""
import ctypes as C
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import workloads as W

SRC = os.path.join(os.path.dirname(oracle.__file__), "lbm_oracle.c")


def _build_mutant(old, new, tmp):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    path = os.path.join(tmp, "m.c")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    lib = os.path.join(tmp, "libm.so")
    subprocess.run(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-I",
                    os.path.dirname(SRC), "-o", lib, path, "-lm"], check=True)
    return lib


def _with_lib(path, fn):
    saved = oracle._lib
    oracle._lib = None
    real = oracle._build.build
    oracle._build.build = lambda force=False: path
    try:
        return fn()
    finally:
        oracle._build.build = real
        oracle._lib = saved


def _poiseuille_error():
    H, g, tau = 16, 1e-6, 0.8
    nu, lam = (tau - 0.5) / 3, (tau - 0.5) ** 2
    o = oracle.Oracle(W.poiseuille(1, H, 1, g=g, tau=tau))
    o.step(12000)
    u = o.macro()[1][0, 0, :, 0]
    eta = np.arange(H) + 0.5
    exact = g / (2 * nu) * eta * (H - eta) + g * (16 * lam - 3) / (24 * nu)
    return np.nan_to_num(np.max(np.abs(u - exact)) / exact.max(), nan=1e9)


def _freeslip_error():
    H, g, tau = 8, 1e-6, 0.8
    nu, lam = (tau - 0.5) / 3, (tau - 0.5) ** 2
    o = oracle.Oracle(W.Case("fs", 1, H, 1, bc_y=(W.BOUNCEBACK, W.FREESLIP), tau0=tau,
                             g=(g, 0, 0)))
    o.step(12000)
    u = o.macro()[1][0, 0, :, 0]
    eta = np.arange(H) + 0.5
    exact = g / (2 * nu) * eta * (2 * H - eta) + g * (16 * lam - 3) / (24 * nu)
    return np.max(np.abs(u - exact)) / exact.max()


def _feq_error():
    c, _ = oracle.lattice()
    u = np.array([0.03, -0.02, 0.01])
    f = oracle.feq(1.1, u)
    pi = np.einsum("i,ia,ib->ab", f, c, c)
    return np.max(np.abs(pi - 1.1 * (np.eye(3) / 3 + np.outer(u, u))))


def _smag_error():
    from test_oracle_pins import test_smagorinsky_channel_matches_semi_analytic as t
    try:
        t()
        return 0.0
    except AssertionError:
        return 1.0


def _shear_wave_error():
    from test_oracle_pins import test_advected_shear_wave_moves_downstream as t
    try:
        t()
        return 0.0
    except AssertionError:
        return 1.0


def _drag_error():
    from test_oracle_pins import test_canopy_momentum_recurrence as t
    try:
        t()
        return 0.0
    except AssertionError:
        return 1.0


def _stats_error():
    from test_oracle_pins import test_stats_are_pooled_time_plane_moments as t
    try:
        t()
        return 0.0
    except AssertionError:
        return 1.0


def _fails(fn, *args):
    """1.0 if the pin `fn` fails (AssertionError) on the loaded oracle, else 0.0."""
    try:
        fn(*args)
        return 0.0
    except AssertionError:
        return 1.0


def _edm_moments_error():
    from test_oracle_variants import test_exact_difference_force_moments as t
    return _fails(t, 0)


def _edm_recurrence_error():
    from test_oracle_variants import test_exact_difference_momentum_recurrence_with_drag_and_driving as t
    return _fails(t)


def _streamwise_drag_error():
    from test_oracle_variants import test_streamwise_drag_momentum_recurrence as t
    return _fails(t, 0)


def _tau_rho2_error():
    from test_oracle_variants import test_tau_total_rho2_is_the_root_of_its_quadratic as t
    return _fails(t, 0)


MUTANTS = [
    ("guo_prefactor", "Fi[i] = (1.0 - 1.0 / (2.0 * tau))", "Fi[i] = (1.0 - 1.0 / tau)",
     _poiseuille_error, 1e-6),
    ("collision_sign", "fout[i] = fin[i] - (fin[i] - feq[i]) / tau",
     "fout[i] = fin[i] + (fin[i] - feq[i]) / tau", _poiseuille_error, 1e-6),
    ("half_force_dropped", "v[a] = (m[a] + 0.5 * rho * g_drive[a]) / rho",
     "v[a] = (m[a] + rho * g_drive[a]) / rho", _poiseuille_error, 1e-6),
    ("bounceback_not_reversed", "return src[(size_t)opposite(i) * s->n + cell_index(s, x, y, z)];",
     "return src[(size_t)i * s->n + cell_index(s, x, y, z)];", _poiseuille_error, 1e-6),
    ("freeslip_as_bounceback", "return post_value(s, src, mirror_y(i), x - CV[i][0], y, z - CV[i][2]);",
     "return post_value(s, src, opposite(i), x, y, z);", _freeslip_error, 1e-6),
    ("feq_dropped_u2", "- uu / (2.0 * CS2));", ");", _feq_error, 1e-12),
    ("smag_sqrt2_dropped", "18.0 * sqrt(2.0) * csmag", "18.0 * csmag", _smag_error, 0.5),
    ("smag_offdiag_once", "2.0 * (pineq[3] * pineq[3]", "1.0 * (pineq[3] * pineq[3]",
     _smag_error, 0.5),
    ("stream_reversed", "return post_value(s, src, i, x - CV[i][0], ys, z - CV[i][2]);",
     "return post_value(s, src, i, x + CV[i][0], ys, z + CV[i][2]);", _shear_wave_error, 0.5),
    ("drag_root", "2.0 / (1.0 + sqrt(1.0 + 2.0 * k * vn))", "2.0 / (1.0 + sqrt(1.0 + k * vn))",
     _drag_error, 0.5),
    ("cov_sign", "out[6 * nb + k] = s->acc[6 * nb + k] / n - mu * mv;",
     "out[6 * nb + k] = s->acc[6 * nb + k] / n + mu * mv;", _stats_error, 0.5),
    # model variants
    ("edm_half_step", "double ug[3] = {u[0] + g[0], u[1] + g[1], u[2] + g[2]};",
     "double ug[3] = {u[0] + 0.5 * g[0], u[1] + 0.5 * g[1], u[2] + 0.5 * g[2]};",
     _edm_moments_error, 0.5),
    ("edm_relaxes_to_physical_u",
     "urel[a] = (scheme == OLBM_EXACT_DIFFERENCE) ? m[a] / rho : u[a];", "urel[a] = u[a];",
     _edm_recurrence_error, 0.5),
    ("streamwise_drag_on_all_components", "if (drag_x_only) g[0] -= k * un * u[0];",
     "if (0) g[0] -= k * un * u[0];", _streamwise_drag_error, 0.5),
    ("tau_rho_power_ignored", "double rp = (p == 2) ? rho * rho : rho;", "double rp = rho;",
     _tau_rho2_error, 0.5),
]


def test_unmutated_oracle_passes_the_probes():
    assert _poiseuille_error() < 1e-9
    assert _freeslip_error() < 1e-9
    assert _feq_error() < 1e-15


@pytest.mark.parametrize("name,old,new,probe,threshold", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, probe, threshold):
    with tempfile.TemporaryDirectory() as tmp:
        path = _build_mutant(old, new, tmp)
        err = _with_lib(path, probe)
    assert err > threshold, f"{name}: pin did not notice the planted mistake ({err})"
