"""Pins of the oracle's GADI-AB for the Sylvester equation A X + X B = C
(§4.3): the solution of a library Sylvester solver (Bartels-Stewart), one
outer step against dense solves of eq. (gadi)'s form, the observed
contraction against Thm 1's iteration matrix for commuting splittings, and
the (r, alpha) cases of Table 'sylvester-results'."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_2501_04229_gb300 import problems as P


def _case(m, n, r, seed=0):
    a = P.sylvester_matrices(m, r)
    b = P.sylvester_matrices(n, r)
    A, B = P.tri_dense(*a), P.tri_dense(*b)
    Xs = np.random.default_rng(seed).standard_normal((m, n))
    return a, b, A, B, A @ Xs + Xs @ B


def test_matrices_follow_section_4_3():
    lo, dg, up = P.sylvester_matrices(5, 0.1)
    T = P.tri_dense(lo, dg, up)
    M = 2 * np.eye(5) - np.eye(5, k=1) - np.eye(5, k=-1)
    N = 0.5 * np.eye(5, k=-1) - 0.5 * np.eye(5, k=1)
    assert np.array_equal(T, M + 2 * 0.1 * N + 100.0 / 36 * np.eye(5))


@pytest.mark.parametrize("r", [0.01, 0.1, 1.0])
@pytest.mark.parametrize("prec", ["PREC_DOUBLE", "PREC_HALF", "PREC_BF16"])
def test_solution_matches_bartels_stewart(r, prec):
    a, b, A, B, Cm = _case(24, 20, r)
    want = sl.solve_sylvester(A, B, Cm)
    X, info, _ = oracle.sylv_gadi_ab(a, b, Cm, 1.0, 1.0, prec=getattr(oracle, prec))
    assert info["status"] == oracle.OK and info["eta_inf"] <= 1e-13
    L = np.kron(np.eye(20), A) + np.kron(B.T, np.eye(24))
    kappa = np.linalg.cond(L)
    assert np.abs(X - want).max() <= 10 * kappa * 1e-13 * np.abs(want).max()


def test_one_step_is_the_gadi_step():
    """From X0 the step is X0 + (2 - w) a (aI + A)^-1 R0 (aI + B)^-1, R0 = C - A X0 - X0 B
    (the two half steps of eq. (gadi) with M, N replaced by A, B)."""
    a, b, A, B, Cm = _case(16, 12, 0.1, seed=3)
    X0 = np.random.default_rng(5).standard_normal((16, 12))
    alpha, omega = 0.7, 0.4
    X1, info, _ = oracle.sylv_gadi_ab(a, b, Cm, alpha, omega, prec=oracle.PREC_DOUBLE, max_outer=1, tol=0.0, x0=X0)
    R0 = Cm - A @ X0 - X0 @ B
    Y = np.linalg.solve(alpha * np.eye(16) + A, R0) @ np.linalg.inv(alpha * np.eye(12) + B)
    want = X0 + (2 - omega) * alpha * Y
    assert info["outer_iters"] == 1
    assert np.abs(X1 - want).max() <= 1e-13 * np.abs(want).max()
    # and the half-step form: (aI + A) X+ = (aI - B) X0 ... as eq. (gadi), on vec(X)
    Lh = np.kron(np.eye(12), A)
    Ls = np.kron(B.T, np.eye(16))
    x0 = X0.T.reshape(-1)
    c = Cm.T.reshape(-1)
    I = np.eye(16 * 12)
    xh = np.linalg.solve(alpha * I + Lh, (alpha * I - Ls) @ x0 + c)
    x1 = np.linalg.solve(alpha * I + Ls, (Ls - (1 - omega) * alpha * I) @ x0 + (2 - omega) * alpha * xh)
    assert np.abs(x1.reshape(12, 16).T - want).max() <= 1e-12 * np.abs(want).max()


@pytest.mark.parametrize("r,alpha,omega", [(0.1, 1.0, 1.0), (0.01, 0.3, 0.5)])
def test_contraction_matches_iteration_matrix(r, alpha, omega):
    """Thm 1 with commuting A-part and B-part: T has eigenvalues
    (a^2 + lm mu - (1 - w) a (lm + mu)) / ((a + lm)(a + mu)) over the
    eigenvalues lm of A and mu of B; the error contracts by rho(T)."""
    m, n = 20, 16
    a, b, A, B, Cm = _case(m, n, r)
    lam, mu = np.linalg.eigvals(A), np.linalg.eigvals(B)
    t = (alpha ** 2 + np.outer(lam, mu) - (1 - omega) * alpha * (lam[:, None] + mu[None, :])) / \
        ((alpha + lam)[:, None] * (alpha + mu)[None, :])
    rho = np.abs(t).max()
    _, info, hist = oracle.sylv_gadi_ab(a, b, Cm, alpha, omega, prec=oracle.PREC_DOUBLE, tol=1e-15,
                                        max_outer=400)
    h = hist[np.isfinite(hist) & (hist > 1e-12)]
    k = len(h)
    rate = (h[k - 1] / h[k // 2]) ** (1.0 / (k - 1 - k // 2))
    assert rho < 1 and abs(rate - rho) <= 0.05 * rho


@pytest.mark.parametrize("r", [0.01, 0.1, 1.0])
@pytest.mark.parametrize("alpha", [0.02, 10.0])
def test_table_cases_converge(r, alpha):
    """Table 'sylvester-results': alpha = 0.02 and 10 converge for r = 0.01,
    0.1, 1 (the table's residuals 1e-8..1e-10 are its FP16 stall; with the
    power-of-two scaling the FP16-inner method reaches 1e-13)."""
    a, b, A, B, Cm = _case(32, 32, r, seed=1)
    X, info, _ = oracle.sylv_gadi_ab(a, b, Cm, alpha, 1.0, prec=oracle.PREC_HALF, max_outer=20000)
    assert info["status"] == oracle.OK and info["eta_inf"] <= 1e-13
