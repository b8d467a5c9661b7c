"""Pins of the oracle predictors (GPR of §3.3.1, the MLP) against closed
forms, finite differences and published reference values."""
import math

import numpy as np
import pytest

from oracle import predict as OP


def test_splitmix64_reference_outputs():
    # the first outputs of SplitMix64 from state 0, as published with the generator
    got = OP.splitmix64(0, 3)
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = OP.uniform01(12345, 1000)
    assert (u >= 0).all() and (u < 1).all() and abs(u.mean() - 0.5) < 0.05


@pytest.mark.parametrize("ell,sn", [(0.5, 1e-3), (1.0, 1e-2), (2.0, 1e-1)])
def test_gpr_two_point_closed_form(ell, sn):
    X = np.array([[0.0, 3.0], [1.0, 3.0]])
    Y = np.array([[2.0, -1.0], [5.0, 4.0]])
    m = OP.gpr_fit(X, Y, ells=(ell,), noises=(sn,))
    # standardised inputs -1, +1; k12 = exp(-2/ell^2); alpha = [-1, 1]/(1 + sn^2 - k12)
    k12 = math.exp(-2.0 / ell ** 2)
    mid = OP.gpr_predict(m, [[0.5, 3.0]])[0]
    assert np.allclose(mid, Y.mean(axis=0), atol=1e-12)
    at1 = OP.gpr_predict(m, [[0.0, 3.0]])[0]
    z = -(1.0 - k12) / (1.0 - k12 + sn * sn)          # standardised prediction at x1
    want = Y.mean(axis=0) + z * Y.std(axis=0)
    assert np.allclose(at1, want, rtol=1e-12, atol=1e-12)


def test_gpr_interpolates_with_small_noise():
    rng = np.random.default_rng(3)
    X = rng.uniform(-2, 2, size=(12, 2))
    Y = np.stack([np.sin(X[:, 0]) + X[:, 1], np.cos(X[:, 1])], axis=1)
    m = OP.gpr_fit(X, Y, ells=(1.0,), noises=(1e-6,))
    assert np.allclose(OP.gpr_predict(m, X), Y, atol=1e-5)


def test_gpr_hyperparameters_maximise_marginal_likelihood():
    rng = np.random.default_rng(5)
    X = rng.uniform(-2, 2, size=(20, 2))
    Y = np.stack([np.sin(2 * X[:, 0]), X[:, 1] ** 2], axis=1)
    m = OP.gpr_fit(X, Y)
    Xs, _, _ = OP.standardize(X)
    Ys, _, _ = OP.standardize(Y)
    for j, c in enumerate(m["cols"]):
        best = OP.gpr_log_marginal(Xs, Ys[:, j], c["ell"], c["sn"])
        for e in OP.GPR_ELLS:
            for s in OP.GPR_NOISES:
                assert OP.gpr_log_marginal(Xs, Ys[:, j], e, s) <= best + 1e-9


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((9, 2))
    T = rng.standard_normal((9, 2))
    p = OP.mlp_init(11)
    for k in p:
        p[k] = p[k] + 0.1 * rng.standard_normal(p[k].shape)   # nonzero biases too
    g = OP.mlp_grads(p, X, T)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = OP.mlp_loss(p, X, T)
            flat[idx] = old - h
            lm = OP.mlp_loss(p, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[idx] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_mlp_init_bounds_and_adam_first_step():
    p = OP.mlp_init(3)
    assert np.abs(p["W2"]).max() <= math.sqrt(6.0 / 128) and np.abs(p["W1"]).max() <= math.sqrt(6.0 / 66)
    X = np.array([[0.0, 1.0], [1.0, 0.0], [2.0, 2.0], [3.0, -1.0]])
    Y = np.array([[1.0, 0.0], [0.0, 1.0], [2.0, 1.0], [0.5, 0.5]])
    m0, _ = OP.mlp_train(X, Y, epochs=0, seed=3)
    m1, _ = OP.mlp_train(X, Y, epochs=1, lr=1e-3, seed=3)
    # Adam's first step moves a coordinate by lr g / (|g| + eps): by lr wherever |g| >> eps
    d = np.abs(m1["params"]["W2"] - m0["params"]["W2"])
    Xs, _, _ = OP.standardize(X)
    Ys, _, _ = OP.standardize(Y)
    g = np.abs(OP.mlp_grads(m0["params"], Xs, Ys)["W2"])
    big = g > 1e-4
    assert big.mean() > 0.5
    assert np.allclose(d[big], 1e-3, rtol=1e-3)
    assert (d <= 1e-3 * (1 + 1e-12)).all()


def test_mlp_training_fits_a_smooth_map():
    rng = np.random.default_rng(1)
    X = rng.uniform(-2, 2, size=(64, 2))
    Y = np.stack([np.tanh(X[:, 0]) + 0.3 * X[:, 1], 0.5 * X[:, 0] * X[:, 1]], axis=1)
    model, hist = OP.mlp_train(X, Y, epochs=1500, lr=1e-2, seed=2)
    assert hist[-1] < 0.02 * hist[0]
    assert np.abs(OP.mlp_predict(model, X) - Y).max() < 0.2
