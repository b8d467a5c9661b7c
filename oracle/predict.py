"""CPU oracle of the parameter predictors -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy, written from the definitions:

* GPR (§3.3.1): Gaussian-process regression with a squared-exponential
  kernel k(x, x') = sf^2 exp(-|x - x'|^2 / (2 ell^2)) and noise sn^2,
  posterior mean m(x*) = k*^T (K + sn^2 I)^-1 y, hyperparameters chosen on a
  grid by the log marginal likelihood
  -1/2 y^T (K + sn^2 I)^-1 y - 1/2 log|K + sn^2 I| - m/2 log(2 pi).
* MLP 2 -> 64 -> 64 -> 2 with tanh hidden layers and a linear output,
  mean-squared-error loss L = 1/(2m) sum (y - t)^2, gradients by the chain
  rule written out layer by layer, Adam updates.

Features and targets are standardised (zero mean, unit variance per column)
before fitting; predictions are mapped back. Weights start from a
SplitMix64 stream (the published 64-bit mixing function), uniform in
+-sqrt(6 / (fan_in + fan_out)), the same stream the library uses.
"""
from __future__ import annotations

import math

import numpy as np

HIDDEN = 64
GPR_ELLS = (0.25, 0.5, 1.0, 2.0, 4.0)
GPR_NOISES = (1e-3, 1e-2, 1e-1)

_M64 = (1 << 64) - 1


def splitmix64(seed: int, count: int) -> np.ndarray:
    """count outputs of SplitMix64 started at state seed, as uint64."""
    out = np.empty(count, dtype=np.uint64)
    s = seed & _M64
    for i in range(count):
        s = (s + 0x9E3779B97F4A7C15) & _M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        out[i] = z ^ (z >> 31)
    return out


def uniform01(seed: int, count: int) -> np.ndarray:
    """(x >> 11) * 2^-53 for SplitMix64 outputs x: doubles in [0, 1)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def standardize(A):
    A = np.asarray(A, dtype=np.float64)
    mu = A.mean(axis=0)
    sd = A.std(axis=0)
    sd = np.where(sd > 0, sd, 1.0)
    return (A - mu) / sd, mu, sd


# ---------------------------------------------------------------------------
# GPR
# ---------------------------------------------------------------------------

def se_kernel(X1, X2, ell, sf=1.0):
    d2 = ((X1[:, None, :] - X2[None, :, :]) ** 2).sum(axis=2)
    return sf * sf * np.exp(-d2 / (2.0 * ell * ell))


def gpr_log_marginal(X, y, ell, sn, sf=1.0):
    K = se_kernel(X, X, ell, sf) + sn * sn * np.eye(len(X))
    sign, logdet = np.linalg.slogdet(K)
    a = np.linalg.solve(K, y)
    return -0.5 * float(y @ a) - 0.5 * logdet - 0.5 * len(X) * math.log(2 * math.pi)


def gpr_fit(X, Y, ells=GPR_ELLS, noises=GPR_NOISES):
    """One GP per target column; (ell, sn) by the largest log marginal
    likelihood on the grid (sf = 1 on standardised targets)."""
    Xs, xmu, xsd = standardize(X)
    Ys, ymu, ysd = standardize(Y)
    cols = []
    for j in range(Ys.shape[1]):
        y = Ys[:, j]
        best = max(((gpr_log_marginal(Xs, y, e, s), e, s) for e in ells for s in noises))
        _, e, s = best
        K = se_kernel(Xs, Xs, e) + s * s * np.eye(len(Xs))
        cols.append({"ell": e, "sn": s, "alpha": np.linalg.solve(K, y)})
    return {"X": Xs, "xmu": xmu, "xsd": xsd, "ymu": ymu, "ysd": ysd, "cols": cols}


def gpr_predict(model, Xq):
    Xq = (np.asarray(Xq, dtype=np.float64) - model["xmu"]) / model["xsd"]
    out = np.empty((len(Xq), len(model["cols"])))
    for j, c in enumerate(model["cols"]):
        out[:, j] = se_kernel(Xq, model["X"], c["ell"]) @ c["alpha"]
    return out * model["ysd"] + model["ymu"]


# ---------------------------------------------------------------------------
# MLP
# ---------------------------------------------------------------------------

def mlp_init(seed: int, n_in=2, hidden=HIDDEN, n_out=2):
    """Glorot-uniform weights from one SplitMix64 stream in the order W1, W2,
    W3 (row-major, W[out][in]); zero biases."""
    sizes = [(hidden, n_in), (hidden, hidden), (n_out, hidden)]
    total = sum(a * b for a, b in sizes)
    u = uniform01(seed, total)
    params, k = {}, 0
    for li, (fo, fi) in enumerate(sizes, start=1):
        a = math.sqrt(6.0 / (fi + fo))
        params[f"W{li}"] = ((2.0 * u[k:k + fo * fi] - 1.0) * a).reshape(fo, fi)
        params[f"b{li}"] = np.zeros(fo)
        k += fo * fi
    return params


def mlp_forward(p, X):
    Z1 = X @ p["W1"].T + p["b1"]
    H1 = np.tanh(Z1)
    Z2 = H1 @ p["W2"].T + p["b2"]
    H2 = np.tanh(Z2)
    Y = H2 @ p["W3"].T + p["b3"]
    return Y, (H1, H2)


def mlp_loss(p, X, T):
    Y, _ = mlp_forward(p, X)
    return 0.5 * float(((Y - T) ** 2).sum()) / len(X)


def mlp_grads(p, X, T):
    """Gradients of L = 1/(2m) sum (Y - T)^2, layer by layer."""
    m = len(X)
    Y, (H1, H2) = mlp_forward(p, X)
    dY = (Y - T) / m
    g = {"W3": dY.T @ H2, "b3": dY.sum(axis=0)}
    dZ2 = (dY @ p["W3"]) * (1.0 - H2 * H2)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * (1.0 - H1 * H1)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    return g


def mlp_train(X, Y, epochs=2000, lr=1e-2, seed=1, beta1=0.9, beta2=0.999, eps=1e-8):
    """Full-batch Adam on standardised data. Returns the model and the loss
    history."""
    Xs, xmu, xsd = standardize(X)
    Ys, ymu, ysd = standardize(Y)
    p = mlp_init(seed)
    mom = {k: np.zeros_like(v) for k, v in p.items()}
    vel = {k: np.zeros_like(v) for k, v in p.items()}
    hist = []
    for t in range(1, epochs + 1):
        g = mlp_grads(p, Xs, Ys)
        for k in p:
            mom[k] = beta1 * mom[k] + (1 - beta1) * g[k]
            vel[k] = beta2 * vel[k] + (1 - beta2) * g[k] * g[k]
            mh = mom[k] / (1 - beta1 ** t)
            vh = vel[k] / (1 - beta2 ** t)
            p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
        hist.append(mlp_loss(p, Xs, Ys))
    return {"params": p, "xmu": xmu, "xsd": xsd, "ymu": ymu, "ysd": ysd}, hist


def mlp_predict(model, Xq):
    Xq = (np.asarray(Xq, dtype=np.float64) - model["xmu"]) / model["xsd"]
    Y, _ = mlp_forward(model["params"], Xq)
    return Y * model["ysd"] + model["ymu"]
