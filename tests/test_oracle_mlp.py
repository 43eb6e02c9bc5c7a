"""Pins of the oracle's learned-correction parts (CPU, FP64): the network's
forward pass against a closed form, its gradient against central differences,
Adam's first step, BF16 rounding, the strain-rate feature against the
Chapman-Enskog closed form, and the layer-0 acceleration against the exact
momentum balance of the Guo step."""
import numpy as np
import pytest

import oracle
import oracle.mlp as M
import workloads as W


def identity_net(x_mean=0.0, x_std=1.0):
    layers = []
    W1 = np.zeros((64, 9))
    W1[np.arange(9), np.arange(9)] = 1.0
    layers.append((W1, np.zeros(64)))
    layers.append((np.eye(64), np.zeros(64)))
    layers.append((np.eye(64), np.zeros(64)))
    W4 = np.zeros((4, 64))
    W4[0, 0], W4[1, 1], W4[2, 2], W4[3, 8] = 2.0, -1.0, 0.5, 1.0
    layers.append((W4, np.array([0.1, 0.0, 0.0, 0.0])))
    norm = (np.full(9, x_mean), np.full(9, x_std), np.array([1.0, 0.0, 0.0, 0.0]),
            np.array([2.0, 1.0, 1.0, 1.0]))
    return M.pack(layers, norm)


def test_forward_matches_closed_form():
    rng = np.random.default_rng(1)
    X = rng.uniform(-2, 2, size=(5, 9))
    th = identity_net(x_mean=0.5, x_std=2.0)
    z = (X - 0.5) / 2.0
    t3 = np.tanh(np.tanh(np.tanh(z)))
    want = np.stack([1.0 + 2.0 * (2.0 * t3[:, 0] + 0.1), -t3[:, 1], 0.5 * t3[:, 2], t3[:, 8]],
                    axis=1)
    assert np.allclose(M.forward(th, X), want, rtol=0, atol=1e-15)
    assert M.N_PARAMS == len(th)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    th = np.concatenate([rng.normal(0, 0.3, M.N_WEIGHTS), rng.normal(0, 0.1, 9),
                         rng.uniform(0.5, 2, 9), rng.normal(0, 0.1, 4), rng.uniform(0.5, 2, 4)])
    X = rng.normal(size=(11, 9))
    Y = rng.normal(size=(11, 4))
    g = M.gradient(th, X, Y)
    assert g.shape == (M.N_WEIGHTS,)
    # every bias and a sample of weights of every layer
    idx = list(rng.choice(M.N_WEIGHTS, 60, replace=False)) + [9 * 64 + 3, M.N_WEIGHTS - 1]
    eps = 1e-6
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += eps
        tm[k] -= eps
        num = (M.loss(tp, X, Y) - M.loss(tm, X, Y)) / (2 * eps)
        assert abs(num - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3), (k, num, g[k])


def test_gradient_catches_a_planted_sign_error():
    """The central-difference check would see a wrong sign in tanh' (mutant)."""
    rng = np.random.default_rng(3)
    th = rng.normal(0, 0.3, M.N_PARAMS)
    th[M.N_WEIGHTS:] = np.concatenate([np.zeros(9), np.ones(9), np.zeros(4), np.ones(4)])
    X, Y = rng.normal(size=(6, 9)), rng.normal(size=(6, 4))
    orig = M.gradient

    def mutant(theta, X, Y):
        layers, (xm, xs, ym, ys) = M.unpack(theta)
        _, acts = M.forward(theta, X, keep=True)
        t = (Y - ym) / ys
        delta = 2.0 * (acts[-1] - t) / (X.shape[0] * 4)
        out = []
        for l in range(3, -1, -1):
            Wl, _ = layers[l]
            out = [np.ravel(delta.T @ acts[l]), delta.sum(axis=0)] + out
            if l > 0:
                delta = (delta @ Wl) * (1.0 + acts[l] ** 2)  # planted: wrong sign
        return np.concatenate(out)

    k = 9 * 64 + 64 + 5  # a weight of layer 2
    eps = 1e-6
    tp, tm = th.copy(), th.copy()
    tp[k] += eps
    tm[k] -= eps
    num = (M.loss(tp, X, Y) - M.loss(tm, X, Y)) / (2 * eps)
    assert abs(num - orig(th, X, Y)[k]) < 1e-6 * max(1e-3, abs(num))
    assert abs(num - mutant(th, X, Y)[k]) > 1e-3 * max(1e-3, abs(num))


def test_adam_first_step_is_a_signed_step_of_lr():
    w, g = np.array([1.0, -2.0, 0.5]), np.array([0.3, -4.0, 1e-3])
    w1, m, v = M.adam_update(w, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(w1, w - 0.01 * np.sign(g), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.0e-3, 65504.0, 1.0 + 2 ** -7 + 2 ** -8])
    r = M.round_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # tie to even (down)
    assert r[2] == 1.0 + 2 ** -7            # above the half-way point: up
    assert abs(r[3] + 3.0e-3) < 3.0e-3 * 2 ** -8
    assert r[5] == 1.0 + 2 ** -6            # tie to even (up)


def _shear_box(s, tau0=0.8, u0=(0.02, -0.01, 0.005)):
    """Uniform periodic box whose populations are f_eq(1, u0) plus the first-order
    Chapman-Enskog non-equilibrium part of a pure shear S_xy = S_yx = s."""
    case = W.Case("shear", 4, 3, 2, bc_y=(W.PERIODIC, W.PERIODIC), tau0=tau0, cs=0.0,
                  init_perturb=0.0, u_profile=np.full(3, u0[0]))
    o = oracle.Oracle(case)
    c, w = oracle.lattice()
    feq = oracle.feq(1.0, np.array(u0))
    fneq = -w * 1.0 * tau0 / (1.0 / 3.0) * 2.0 * c[:, 0] * c[:, 1] * s
    f = np.broadcast_to((feq + fneq)[:, None, None, None], (19, 2, 3, 4)).copy()
    o.set_f(f)
    return o


@pytest.mark.parametrize("s", [1e-4, -3e-3])
def test_strain_feature_matches_chapman_enskog(s):
    o = _shear_box(s)
    rho, u, strain = o.fields()
    # |S| = sqrt(2 S:S) = 2 |s| for a pure shear, whatever the velocity
    assert np.allclose(strain, 2 * abs(s), rtol=1e-12, atol=0)
    assert np.allclose(rho, 1.0, atol=1e-14)


def test_features_are_the_fields_of_the_three_lowest_cells():
    case = W.canopy_abl(24, 8, 4, h=3.0, canopy_x0=10, xbin=8)
    o = oracle.Oracle(case)
    o.step(3)
    X = o.features()
    _, u, strain = o.fields()
    assert X.shape == (4 * 24, 9)
    Xr = X.reshape(4, 24, 9)
    for y in range(3):
        assert np.array_equal(Xr[:, :, y], u[0, :, y, :])
        assert np.array_equal(Xr[:, :, 3 + y], strain[:, y, :])
    assert np.all(Xr[:, :10, 6:] == 0.0)
    assert np.allclose(Xr[:, 10:, 6], case.lad[0]) and np.allclose(Xr[:, 10:, 8], case.lad[2])


def test_layer0_acceleration_adds_exactly_rho_a_of_momentum():
    case = W.channel_les(12, 6, 5)
    a = np.random.default_rng(4).uniform(-1e-4, 1e-4, size=(5, 12, 2))
    o1, o2 = oracle.Oracle(case), oracle.Oracle(case)
    rho, _, _ = o1.fields()
    o2.set_layer0_accel(a)
    o1.step(1)
    o2.step(1)
    f1, f2 = o1.get_f(), o2.get_f()
    c, _ = oracle.lattice()
    dm = np.einsum("i,izyx->zyx", c[:, 0], f2 - f1)
    dmz = np.einsum("i,izyx->zyx", c[:, 2], f2 - f1)
    assert np.allclose(dm[:, 0, :], rho[:, 0, :] * a[:, :, 0], rtol=1e-9, atol=1e-15)
    assert np.allclose(dmz[:, 0, :], rho[:, 0, :] * a[:, :, 1], rtol=1e-9, atol=1e-15)
    assert np.all(dm[:, 1:, :] == 0.0)           # other layers untouched in this step
    assert abs(o1.mass() - o2.mass()) < 1e-12 * o1.mass()
    o2.set_layer0_accel(None)


def _bias_net(b4):
    """A network whose last layer has zero weights: every row outputs its bias
    b4 (y_mean = 0, y_std = 1)."""
    layers = [(np.zeros((64, 9)), np.zeros(64)), (np.zeros((64, 64)), np.zeros(64)),
              (np.zeros((64, 64)), np.zeros(64)), (np.zeros((4, 64)), np.asarray(b4, float))]
    norm = (np.zeros(9), np.ones(9), np.zeros(4), np.ones(4))
    return M.pack(layers, norm)


def _check_correction_accel(mod):
    """The outputs are (du_x, du_z, dtau_x, dtau_z): velocity deficits of the
    first cell (fine minus coarse) and net retarding-stress deficits.  The
    acceleration relaxes the velocity deficit at rate lam and adds the missing
    retardation with a minus sign, per direction: for outputs (3, 5, 7, 11) and
    lam = 0.5 that is (0.5*3 - 7, 0.5*5 - 11) = (-5.5, -8.5)."""
    X = np.random.default_rng(3).normal(size=(5, 9))
    a = mod.correction_accel(_bias_net([3.0, 5.0, 7.0, 11.0]), X, 0.5)
    assert a.shape == (5, 2)
    assert np.all(a[:, 0] == -5.5) and np.all(a[:, 1] == -8.5)
    # meanings one output at a time: a faster fine run (du_x > 0) accelerates
    # the coarse cell in x only; a larger fine-run stress deficit (dtau_z > 0)
    # decelerates in z only
    a = mod.correction_accel(_bias_net([2.0, 0.0, 0.0, 0.0]), X, 0.25)
    assert np.all(a[:, 0] == 0.5) and np.all(a[:, 1] == 0.0)
    a = mod.correction_accel(_bias_net([0.0, 0.0, 0.0, 4.0]), X, 0.25)
    assert np.all(a[:, 0] == 0.0) and np.all(a[:, 1] == -4.0)


def test_correction_accel_on_hand_set_outputs():
    _check_correction_accel(M)


def test_correction_accel_pin_catches_swapped_stress_outputs(tmp_path):
    """Plant the mistake (dtau_x and dtau_z swapped) in a copy of the oracle's
    network module, on the CPU: the pin above must fail."""
    import importlib.util

    src = open(M.__file__).read()
    old = "lam * y[:, 0] - y[:, 2], lam * y[:, 1] - y[:, 3]"
    assert src.count(old) == 1
    path = tmp_path / "mlp_mutant.py"
    path.write_text(src.replace(old, "lam * y[:, 0] - y[:, 3], lam * y[:, 1] - y[:, 2]"))
    spec = importlib.util.spec_from_file_location("mlp_mutant", path)
    mutant = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mutant)
    with pytest.raises(AssertionError):
        _check_correction_accel(mutant)
