"""GADI-AB for the Sylvester equation on the GPU (gadi_sylv_* through the C
ABI) against the oracle: every outer step is the same sequence of IEEE
operations (FP64 residual chains, direct tridiagonal solves in the inner
precision, power-of-two scalings, FP64 update), so the iterates agree bit
for bit; the converged solution also matches a Bartels-Stewart solve."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_2501_04229_gb300 import problems as P
from paper_2501_04229_gb300 import gadi as G

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


PRECS = [(G.GADI_F64, oracle.PREC_DOUBLE), (G.GADI_F32, oracle.PREC_SINGLE), (G.GADI_F16, oracle.PREC_HALF),
         (G.GADI_BF16, oracle.PREC_BF16)]


def _case(m, n, r, seed=0):
    a = P.sylvester_matrices(m, r)
    b = P.sylvester_matrices(n, r)
    A, B = P.tri_dense(*a), P.tri_dense(*b)
    Xs = np.random.default_rng(seed).standard_normal((m, n))
    return a, b, A, B, A @ Xs + Xs @ B


def _gpu(a, b, Cm, alpha, omega, u_r, tol, max_outer, x0=None):
    s = G.gadi_sylv_create(a, b)
    try:
        G.gadi_sylv_set_params(s, alpha, omega, u_r)
        Cd = torch.from_numpy(np.ascontiguousarray(Cm)).cuda()
        Xd = torch.zeros_like(Cd) if x0 is None else torch.from_numpy(np.ascontiguousarray(x0)).cuda()
        st, info = G.gadi_sylv_solve(s, Cd, Xd, tol, max_outer)
        return st, info, Xd.cpu().numpy()
    finally:
        G.gadi_sylv_destroy(s)


@pytest.mark.parametrize("u_r,prec", PRECS)
@pytest.mark.parametrize("steps", [1, 4, 17])
def test_iterates_bit_exact(u_r, prec, steps):
    a, b, A, B, Cm = _case(45, 37, 0.1, seed=2)                 # ragged against the 32 x 32 tiles
    want, oinfo, _ = oracle.sylv_gadi_ab(a, b, Cm, 0.8, 0.6, prec=prec, tol=0.0, max_outer=steps)
    st, info, got = _gpu(a, b, Cm, 0.8, 0.6, u_r, 0.0, steps)
    assert st == G.GADI_ERR_NOT_CONVERGED and info["outer_iters"] == oinfo["outer_iters"] == steps
    assert np.array_equal(got, want), np.abs(got - want).max()
    assert (info["scale_exp_M"], info["scale_exp_N"]) == (oinfo["scale_exp_M"], oinfo["scale_exp_N"])


@pytest.mark.parametrize("u_r,prec", PRECS)
@pytest.mark.parametrize("r", [0.01, 1.0])
def test_solution_matches_oracle_and_bartels_stewart(u_r, prec, r):
    a, b, A, B, Cm = _case(64, 48, r, seed=4)
    want, oinfo, _ = oracle.sylv_gadi_ab(a, b, Cm, 1.0, 1.0, prec=prec, tol=1e-13)
    st, info, got = _gpu(a, b, Cm, 1.0, 1.0, u_r, 1e-13, 100000)
    assert st == G.GADI_OK and oinfo["status"] == oracle.OK
    assert info["outer_iters"] == oinfo["outer_iters"] and info["eta_inf"] <= 1e-13
    assert np.array_equal(got, want)
    ref = sl.solve_sylvester(A, B, Cm)
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


def test_larger_system_matches_oracle():
    a, b, A, B, Cm = _case(384, 512, 0.1, seed=7)
    want, oinfo, _ = oracle.sylv_gadi_ab(a, b, Cm, 1.5, 0.5, prec=oracle.PREC_HALF, tol=1e-13)
    st, info, got = _gpu(a, b, Cm, 1.5, 0.5, G.GADI_F16, 1e-13, 100000)
    assert st == G.GADI_OK and info["outer_iters"] == oinfo["outer_iters"]
    assert np.array_equal(got, want)


def test_one_by_one_and_invalid_arguments():
    a = (np.zeros(1), np.array([3.0]), np.zeros(1))
    st, info, got = _gpu(a, a, np.array([[12.0]]), 1.0, 1.0, G.GADI_F16, 1e-13, 1000)
    assert st == G.GADI_OK and abs(got[0, 0] - 2.0) <= 24 * 1e-13 / 6     # |r| <= eta (||L|| |x| + |c|), |x - 2| <= |r| / 6
    with pytest.raises(G.GadiError):
        G.gadi_sylv_create((np.zeros(0), np.zeros(0), np.zeros(0)), a)
    with pytest.raises(G.GadiError):
        G.gadi_sylv_create((np.zeros(2), np.array([1.0, np.nan]), np.zeros(2)), a)
    s = G.gadi_sylv_create(a, a)
    try:
        for alpha, omega in ((0.0, 1.0), (1.0, 2.0)):
            with pytest.raises(G.GadiError):
                G.gadi_sylv_set_params(s, alpha, omega)
        with pytest.raises(G.GadiError) as e:
            G.gadi_sylv_set_params(s, 1.0, 1.0, G.GADI_E4M3)            # no FP8 Sylvester path
        assert e.value.status == G.GADI_ERR_UNSUPPORTED
        with pytest.raises(G.GadiError):
            G.gadi_sylv_solve(s, np.ones((1, 1)), np.zeros((1, 1)))       # host arrays are rejected
    finally:
        G.gadi_sylv_destroy(s)
