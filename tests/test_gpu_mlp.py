"""The learned first-layer correction on the GPU against the FP64 oracle:
network forward (tensor cores) and gradient (training path) with the same
BF16-rounded weights, the column features, the correction field, the step that
applies it, and training."""
import numpy as np
import pytest

import oracle
import oracle.mlp as M
import paper_2206_15454_b300 as P
import workloads as W

pytestmark = pytest.mark.gpu


def random_theta(seed, scale=0.25):
    rng = np.random.default_rng(seed)
    th = np.concatenate([rng.normal(0, scale, M.N_WEIGHTS), rng.normal(0, 0.5, 9),
                         rng.uniform(0.5, 2.0, 9), rng.normal(0, 0.1, 4), rng.uniform(0.5, 2.0, 4)])
    return th.astype(np.float32)


def as_bf16_weights(theta):
    """The parameters the GPU computes with: weights rounded to BF16; biases and
    the normalisation stay FP32 values."""
    th = np.asarray(theta, dtype=np.float64).copy()
    layers, norm = M.unpack(th)
    layers = [(M.round_bf16(Wl), bl) for Wl, bl in layers]
    return M.pack(layers, norm)


def test_forward_matches_oracle_with_bf16_weights():
    net = P.CorrectionNet(seed=3)
    th = random_theta(1)
    net.set_params(th)
    assert np.array_equal(net.params(), th)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, size=(1000, 9)).astype(np.float32)   # ragged last tile of 16
    Yg = net.forward(X)
    Yo = M.forward(as_bf16_weights(th), X.astype(np.float64))
    err = np.abs(Yg - Yo).max() / np.abs(Yo).max()
    print(f"forward: max error / max output = {err:.2e}")
    # BF16 activations (8 significant bits) through four layers
    assert err < 2e-2


def test_gradient_matches_oracle_with_bf16_weights():
    net = P.CorrectionNet(seed=4)
    th = random_theta(5)
    net.set_params(th)
    rng = np.random.default_rng(6)
    X = rng.normal(0, 1, size=(300, 9)).astype(np.float32)
    Y = rng.normal(0, 1, size=(300, 4)).astype(np.float32)
    g, loss = net.gradient(X, Y)
    tho = as_bf16_weights(th)
    go = M.gradient(tho, X.astype(np.float64), Y.astype(np.float64))
    lo = M.loss(tho, X.astype(np.float64), Y.astype(np.float64))
    rel = np.linalg.norm(g - go) / np.linalg.norm(go)
    print(f"gradient rel L2 = {rel:.2e}, loss {loss:.6f} vs {lo:.6f}")
    assert rel < 1e-2
    assert abs(loss - lo) < 1e-2 * lo


def test_training_fits_a_smooth_map():
    rng = np.random.default_rng(7)
    X = rng.normal(0, 1, size=(20000, 9)).astype(np.float32)
    A = rng.normal(0, 0.5, size=(9, 4))
    Y = (np.tanh(X @ A) + 0.3 * X[:, :4] ** 2).astype(np.float32)
    net = P.CorrectionNet(seed=8)
    l0, l1 = net.train(X, Y, epochs=25, batch=512, lr=2e-3, seed=9)
    th = net.params()
    # the normalisation was set from the data
    assert np.allclose(th[9220:9229], X.mean(axis=0), atol=1e-3)
    Yp = net.forward(X[:2000])
    r2 = 1 - np.mean((Yp - Y[:2000]) ** 2) / np.var(Y[:2000])
    print(f"training loss {l0:.4f} -> {l1:.4f}, R^2 = {r2:.4f}")
    assert l1 < 0.1 * l0 and r2 > 0.9


CASE = W.canopy_abl(40, 12, 6, h=4.0, canopy_x0=12, xbin=8)


def test_features_match_oracle():
    d, o = P.Domain(CASE), oracle.Oracle(CASE)
    d.step(30)
    o.step(30)
    Xg, Xo = d.features(), o.features()
    scale = np.abs(Xo).max(axis=0)
    scale[scale == 0] = 1.0
    err = (np.abs(Xg - Xo) / scale).max(axis=0)
    print("feature errors / scale:", " ".join(f"{e:.1e}" for e in err))
    assert np.all(err[:3] < 1e-5)   # velocities
    assert np.all(err[3:6] < 1e-3)  # strain rates (differences of populations)
    assert np.all(err[6:] < 1e-6)   # leaf-area densities


def test_fused_correction_equals_network_on_features():
    """After a step the correction kernel gathers each 16-column tile's features
    and runs the network in one pass.  Its field must be the network's forward
    pass (lbm_mlp_forward: the same tensor-core arithmetic) on lbm_features'
    output, combined by the correction rule a = (lam dux - dtx, lam duz - dtz),
    on every column: 70 x 19 = 1330 columns are 83 full warp tiles and a ragged
    one, over a canopy edge, inflow and outflow."""
    case = W.canopy_abl(70, 24, 19, h=6.0, canopy_x0=10, xbin=10)
    th = random_theta(21, scale=0.1)
    th[M.N_WEIGHTS + 18:M.N_WEIGHTS + 22] = 0.0        # y_mean
    th[M.N_WEIGHTS + 22:] = 2e-4                       # y_std
    net = P.CorrectionNet(seed=3)
    net.set_params(th)
    d = P.Domain(case)
    d.step(7)
    X = d.features()
    d.set_correction(net, lam=0.05)                    # the field of the current state
    a = d.correction_field().reshape(-1, 2)
    Y = net.forward(X)
    lam = np.float32(0.05)
    ref = np.stack([lam * Y[:, 0] - Y[:, 2], lam * Y[:, 1] - Y[:, 3]], axis=1)
    err = np.abs(a - ref).max() / np.abs(ref).max()
    print(f"fused correction vs network on features: max error / max = {err:.1e}")
    assert a.shape == ref.shape and err < 1e-6


def test_corrected_steps_match_oracle_given_the_same_field():
    th = random_theta(10, scale=0.1)
    th[M.N_WEIGHTS + 18:M.N_WEIGHTS + 22] = 0.0        # y_mean
    th[M.N_WEIGHTS + 22:] = 2e-4                       # y_std: outputs ~1e-4
    net = P.CorrectionNet(seed=11)
    net.set_params(th)
    d, o = P.Domain(CASE), oracle.Oracle(CASE)
    d.step(5)
    o.step(5)
    d.set_correction(net, lam=0.05)
    a = d.correction_field()
    # the field the GPU computed from its state against the oracle's network
    ao = M.correction_accel(as_bf16_weights(th), o.features(), 0.05)
    err = np.abs(a - ao).max() / np.abs(ao).max()
    print(f"correction field: max error / max = {err:.2e}, max |a| = {np.abs(ao).max():.2e}")
    assert err < 2e-2 and np.abs(ao).max() > 1e-6
    # the step that applies it: the oracle takes the GPU's field, step by step
    for k in range(20):
        o.set_layer0_accel(d.correction_field().astype(np.float64).reshape(CASE.nz, CASE.nx, 2))
        d.step(1)
        o.step(1)
    rel = np.linalg.norm(d.get_f() - o.get_f()) / np.linalg.norm(o.get_f())
    print(f"corrected steps: population rel L2 after 20 steps = {rel:.2e}")
    assert rel < 1e-6
    # switching it off restores the plain step
    d.set_correction(None)
    o.set_layer0_accel(None)
    d.step(3)
    o.step(3)
    assert np.linalg.norm(d.get_f() - o.get_f()) / np.linalg.norm(o.get_f()) < 1e-6


def test_corrected_run_statistics_match_oracle_within_2_percent():
    """The learned form against the FP64 oracle running the same correction
    (its own features, the network in FP64 with the same BF16 weights), over a
    statistics window: mean-velocity profiles within 2 %."""
    th = random_theta(12, scale=0.1)
    th[M.N_WEIGHTS + 18:M.N_WEIGHTS + 22] = 0.0
    th[M.N_WEIGHTS + 22:] = 2e-4
    net = P.CorrectionNet(seed=13)
    net.set_params(th)
    tho = as_bf16_weights(th)
    d, o = P.Domain(CASE), oracle.Oracle(CASE)
    d.set_correction(net, lam=0.01)
    d.stats_reset(True)
    o.stats_reset(True)
    for k in range(300):
        o.set_layer0_accel(M.correction_accel(tho, o.features(), 0.01).reshape(CASE.nz, CASE.nx, 2))
        o.step(1)
    d.step(300)
    sd, _ = d.stats()
    so, _ = o.stats()
    err = np.abs(sd[:3] - so[:3]).max() / np.abs(so[0]).max()
    print(f"corrected run: mean-velocity profile error = {err:.2e} of max <u>")
    assert err < 0.02


def test_trained_correction_gains_over_the_plain_coarse_run():
    """Gain test: a canopy boundary layer (64 x 32 x 32, h = 6, a = 0.25,
    C_D = 0.15, inflow/outflow) run plain on the coarse grid and on the 2x finer
    grid; the network is trained on the coarse run's features against the
    coarsened fine run's first-cell deficits; the corrected coarse run's mean
    streamwise velocity must be closer to the coarsened fine profile than the
    plain coarse run's, in the first cell and over the canopy layer."""
    from paper_2206_15454_b300 import learned as L

    case = W.canopy_abl(64, 32, 32, h=6.0, a=0.25, cd=0.15, canopy_x0=16, xbin=1)
    spin, avg = 2000, 2000
    ref = L.reference_runs(case, spin, avg, sample_every=20)
    net, l0, l1 = L.train_correction(ref, epochs=30)
    plain, corr = L.corrected_run(case, net, 0.01, spin, avg)
    out = {}
    for rows in (1, 6, 12):
        out[rows] = (L.profile_error(plain, ref.fine_coarsened, rows),
                     L.profile_error(corr, ref.fine_coarsened, rows))
    print("training loss %.3f -> %.3f; " % (l0, l1) + "; ".join(
        f"rows {r}: plain {a:.4f} corrected {b:.4f}" for r, (a, b) in out.items()))
    assert l1 < 0.6 * l0
    assert out[1][1] < 0.8 * out[1][0]   # first cell
    assert out[6][1] < 0.85 * out[6][0]  # the canopy layer
    assert out[12][1] < out[12][0]
