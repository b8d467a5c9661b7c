"""Parameter predictors (§3.3): MLP trained on the GPU by the library's own
kernels, GPR in FP32, grid search -- against the oracle, and against solving
without a predictor."""
import math

import numpy as np
import pytest

import oracle
from oracle import predict as OP
from paper_2501_04229_gb300 import gadi as G
from paper_2501_04229_gb300 import problems as P
from paper_2501_04229_gb300 import sweep as SW

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2501_04229_gb300 import build
    build.build()
    oracle.build()
    G.load()


def _flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]])


def test_mlp_gradient_matches_oracle_backprop():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((77, 2))            # ragged against the 32-sample blocks
    T = rng.standard_normal((77, 2))
    p = OP.mlp_init(9)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.05 * rng.standard_normal(p[k].shape)
    want = _flat(OP.mlp_grads(p, X, T))
    got = G.gadi_mlp_gradient(_flat(p), X, T)
    assert got.shape == want.shape == (G.gadi_mlp_param_count(),)
    # BF16 operands with FP32 accumulation against FP64
    assert np.linalg.norm(got - want) <= 2e-2 * np.linalg.norm(want)
    sl = {"W1": slice(0, 128), "W2": slice(192, 4288), "W3": slice(4352, 4480)}
    for name, s in sl.items():
        cos = got[s] @ want[s] / (np.linalg.norm(got[s]) * np.linalg.norm(want[s]))
        assert cos > 0.999, name


def test_mlp_training_on_gpu_fits_like_the_oracle():
    rng = np.random.default_rng(1)
    X = rng.uniform(-2, 2, size=(96, 2))
    Y = np.stack([np.tanh(X[:, 0]) + 0.3 * X[:, 1], 0.5 * X[:, 0] * X[:, 1]], axis=1)
    m = G.gadi_model_fit(G.GADI_MODEL_MLP, X, Y, hyper=[1500, 1e-2, 2])
    try:
        loss = G.gadi_model_loss(m)
        assert len(loss) == 1500 and loss[-1] < 0.02 * loss[0]
        _, hist = OP.mlp_train(X, Y, epochs=1500, lr=1e-2, seed=2)
        assert loss[-1] < 5 * hist[-1] + 1e-3
        pred = G.gadi_model_predict(m, X)
        assert np.abs(pred - Y).max() < 0.25
    finally:
        G.gadi_model_destroy(m)


def test_mlp_initial_loss_matches_oracle():
    rng = np.random.default_rng(6)
    X = rng.uniform(-1, 1, size=(40, 2))
    Y = rng.uniform(-1, 1, size=(40, 2))
    m = G.gadi_model_fit(G.GADI_MODEL_MLP, X, Y, hyper=[1, 1e-3, 5])
    try:
        Xs, _, _ = OP.standardize(X)
        Ys, _, _ = OP.standardize(Y)
        want = OP.mlp_loss(OP.mlp_init(5), Xs, Ys)     # loss at the SplitMix64 initial weights
        assert G.gadi_model_loss(m)[0] == pytest.approx(want, rel=2e-2)
    finally:
        G.gadi_model_destroy(m)


@pytest.mark.parametrize("hyper", [[0.5, 1e-2], [0.5, 1e-3], [1.0, 3e-2], None])
def test_gpr_matches_oracle(hyper):
    rng = np.random.default_rng(2)
    X = np.stack([rng.uniform(5, 14, 30), rng.uniform(-2, 7, 30)], axis=1)
    Y = np.stack([0.3 * np.sin(X[:, 0]) - 0.1 * X[:, 1], 0.5 + 0.1 * np.cos(X[:, 1])], axis=1)
    Xq = np.stack([rng.uniform(5, 14, 12), rng.uniform(-2, 7, 12)], axis=1)
    if hyper is None:
        om = OP.gpr_fit(X, Y)
    else:
        om = OP.gpr_fit(X, Y, ells=(hyper[0],), noises=(hyper[1],))
    m = G.gadi_model_fit(G.GADI_MODEL_GPR, X, Y, hyper=hyper)
    try:
        got, want = G.gadi_model_predict(m, Xq), OP.gpr_predict(om, Xq)
        # FP32 solves with K + sn^2 I lose about cond(K) * 2^-24 (relative)
        kappa = max(np.linalg.cond(OP.se_kernel(om["X"], om["X"], c["ell"]) + c["sn"] ** 2 * np.eye(len(X)))
                    for c in om["cols"])
        tol = max(2e-3, 20 * kappa * 2.0 ** -24) if hyper is not None else 5e-2
        assert np.abs(got - want).max() <= tol * max(1.0, np.abs(want).max())
    finally:
        G.gadi_model_destroy(m)


def _stencil_handle(p):
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt, device="cuda")
    return G.gadi_create(t(p.A.row_ptr, torch.int32), t(p.A.col_idx, torch.int32), t(p.A.val),
                         stencil=(p.dim, p.N, p.beta, 0))


def _cost(p, alpha, omega):
    h = _stencil_handle(p)
    try:
        G.gadi_set_params(h, alpha, omega)
        G.gadi_set_inner(h, 0.1, 200, 20000)
        b = torch.as_tensor(p.b).cuda()
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st, info = G.gadi_solve(h, b, x, 1e-13)
        assert st == G.GADI_OK
        assert oracle.backward_error(p.A, p.b, x.cpu().numpy()) <= 1e-13
        return info["spmv_count"]
    finally:
        G.gadi_destroy(h)


def test_predict_params_kinds_and_grid_search():
    p = P.make_problem(2, 16, 20.0, rhs="ones")
    h = _stencil_handle(p)
    try:
        st, _, _ = G.gadi_predict_params(h, [math.log(p.n), math.log(20.0)], G.GADI_MODEL_MLP)
        assert st == G.GADI_ERR_NO_MODEL
        X = np.array([[math.log(256), 1.0], [math.log(1024), 2.0], [math.log(4096), 3.0]])
        Y = np.array([[0.0, 0.5], [0.5, 0.0], [1.0, 1.0]])
        gm = G.gadi_model_fit(G.GADI_MODEL_GPR, X, Y)
        try:
            G.gadi_set_model(h, G.GADI_MODEL_GPR, gm)
            st, a, w = G.gadi_predict_params(h, [math.log(1024), 2.0], G.GADI_MODEL_GPR)
            y = G.gadi_model_predict(gm, [[math.log(1024), 2.0]])[0]
            assert st == G.GADI_OK and a == pytest.approx(math.exp(y[0])) and w == pytest.approx(min(1.999, max(0, y[1])))
        finally:
            G.gadi_set_model(h, G.GADI_MODEL_GPR, None)
            G.gadi_model_destroy(gm)
        st, a, w = G.gadi_predict_params(h, None, G.GADI_MODEL_GRID)
        assert st == G.GADI_OK and a > 0 and 0 <= w < 2
    finally:
        G.gadi_destroy(h)
    best = _cost(p, a, w)
    for a2, w2 in ((1.0, 1.0), (0.1, 0.0), (10.0, 0.5)):
        assert best <= _cost(p, a2, w2) * 1.05


def test_trained_mlp_beats_default_parameters():
    """Train the MLP on sweep records of small 2D systems (§3.3's training set
    from small systems of the same structure), then solve held-out systems
    with the predicted (alpha, omega) and with the default alpha = omega = 1:
    the predictor must need fewer operator applications."""
    train = SW.random_instances(24, seed=11, dim=2, side=(16, 48), beta=(0.5, 200.0))
    recs = SW.run(train, cands=SW.candidates(n_alpha=10, omegas=(0.0, 1.0), lo=-1.5, hi=1.5), max_outer=8000)
    X = np.array([[r["log_n"], r["log_beta"]] for r in recs if r["best"]])
    Y = np.array([[math.log(r["best"]["alpha"]), r["best"]["omega"]] for r in recs if r["best"]])
    assert len(X) >= 20
    m = G.gadi_model_fit(G.GADI_MODEL_MLP, X, Y, hyper=[2000, 1e-2, 3])
    try:
        held = SW.random_instances(6, seed=99, dim=2, side=(16, 48), beta=(0.5, 200.0))
        gain = []
        for d, N, b in held:
            p = P.make_problem(d, N, b, rhs="ones")
            y = G.gadi_model_predict(m, [[math.log(p.n), math.log(b)]])[0]
            a, w = math.exp(y[0]), min(1.999, max(0.0, y[1]))
            gain.append(_cost(p, 1.0, 1.0) / _cost(p, a, w))
        assert np.mean(gain) > 1.2, gain
    finally:
        G.gadi_model_destroy(m)
