"""Pins of the CPU oracle against facts that do not come from the oracle:
dense LU, closed-form spectra of the Kronecker-sum operator, Thm 1's
iteration matrix, IEEE 754 binary16 rounding, manufactured solutions and the
qualitative results of the paper's tables.

Each test names the passage of arXiv 2501.04229 it follows.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2501_04229_gb300 import problems as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense_MN(oracle, A):
    m, nv = oracle.hss_split(A)
    Md = P.Csr(A.n, A.row_ptr, A.col_idx, m).to_dense()
    Nd = P.Csr(A.n, A.row_ptr, A.col_idx, nv).to_dense()
    return Md, Nd


# ---------------------------------------------------------------------------
# Generator and HSS splitting (§4.1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim,N", [(2, 7), (3, 5)])
def test_generator_nnz_and_row_sums(dim, N):
    A = P.convdiff_csr(dim, N, beta=3.0)
    nnz = (2 * dim + 1) * N ** dim - 2 * dim * N ** (dim - 1)
    assert A.nnz == nnz
    Ad = A.to_dense()
    # interior rows of the k = 1 operator sum to zero (diffusion + centred convection)
    idx = np.arange(A.n)
    coords = [(idx // N ** d) % N for d in range(dim)]
    interior = np.all([(c > 0) & (c < N - 1) for c in coords], axis=0)
    assert np.abs(Ad[interior].sum(axis=1)).max() < 1e-13
    # §4.1: beta = 1 and 3D gives diagonal 6 and off-diagonals -1 -/+ r, r = 1/(2N+2)
    if dim == 3:
        B = P.convdiff_csr(3, N, beta=1.0).to_dense()
        r = 1.0 / (2 * N + 2)
        assert np.allclose(np.diag(B), 6.0)
        assert np.allclose(np.diag(B, -1)[np.diag(B, -1) != 0], -1 - r)
        assert np.allclose(np.diag(B, 1)[np.diag(B, 1) != 0], -1 + r)


def test_hss_split_exact_symmetry(oracle_lib):
    A = P.convdiff_csr(3, 6, beta=7.0, faces=P.grf_faces(6, seed=11))
    Md, Nd = _dense_MN(oracle_lib, A)
    Ad = A.to_dense()
    assert np.array_equal(Md, Md.T)
    assert np.array_equal(Nd, -Nd.T)
    assert np.allclose(Md + Nd, Ad, rtol=0, atol=1e-15)
    assert np.array_equal(np.diag(Nd), np.zeros(A.n))


@pytest.mark.parametrize("dim,N,beta", [(2, 9, 10.0), (3, 6, 25.0)])
def test_hss_spectra_closed_form(oracle_lib, dim, N, beta):
    """Kronecker-sum spectra (§4.1): lambda(M) = sum_d (2 - 2 cos(j_d pi h)),
    lambda(N) = i beta h sum_d cos(j_d pi h)."""
    A = P.convdiff_csr(dim, N, beta)
    Md, Nd = _dense_MN(oracle_lib, A)
    h = 1.0 / (N + 1)
    j = np.arange(1, N + 1)
    grids = np.meshgrid(*([j] * dim), indexing="ij")
    lam_M = sum(2 - 2 * np.cos(g * math.pi * h) for g in grids).ravel()
    lam_N = (beta * h * sum(np.cos(g * math.pi * h) for g in grids)).ravel()
    assert np.allclose(np.sort(np.linalg.eigvalsh(Md)), np.sort(lam_M), atol=1e-11)
    ev = np.linalg.eigvals(Nd)
    assert np.abs(ev.real).max() < 1e-10
    assert np.allclose(np.sort(ev.imag), np.sort(lam_N), atol=1e-10)


def test_hss_rejects_unsymmetric_pattern(oracle_lib):
    A = P.Csr(2, np.array([0, 2, 3], np.int32), np.array([0, 1, 1], np.int32),
              np.array([1.0, 2.0, 3.0]))
    with pytest.raises(ValueError):
        oracle_lib.hss_split(A)


# ---------------------------------------------------------------------------
# Operator products, norms, backward error
# ---------------------------------------------------------------------------

def test_spmv_and_residual_match_dense(oracle_lib):
    A = P.convdiff_csr(3, 5, beta=4.0, faces=P.grf_faces(5, seed=2))
    x = P.random_vector(A.n, 1)
    b = P.random_vector(A.n, 2)
    Ad = A.to_dense()
    y = oracle_lib.spmv_shift(A.n, A.row_ptr, A.col_idx, A.val, 0.75, x)
    assert np.allclose(y, 0.75 * x + Ad @ x, rtol=1e-14, atol=1e-13)
    r = oracle_lib.residual(A, b, x)
    assert np.allclose(r, b - Ad @ x, rtol=1e-14, atol=1e-13)
    assert oracle_lib.matrix_norm_inf(A) == pytest.approx(np.abs(Ad).sum(axis=1).max(), rel=1e-15)


def test_backward_error_hand_example(oracle_lib):
    # A = [[2, -1], [-1, 3]], x = [1, 1], b = [2, 1]: r = [1, -1]
    A = P.Csr(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32),
              np.array([2.0, -1.0, -1.0, 3.0]))
    eta = oracle_lib.backward_error(A, np.array([2.0, 1.0]), np.array([1.0, 1.0]))
    # ||r||_inf = 1, ||A||_inf = 4, ||x||_inf = 1, ||b||_inf = 2
    assert eta == pytest.approx(1.0 / 6.0, rel=1e-15)


# ---------------------------------------------------------------------------
# Inner solvers against dense LU
# ---------------------------------------------------------------------------

def test_cg_and_cgnr_match_lu(oracle_lib):
    A = P.convdiff_csr(3, 5, beta=30.0)
    m, nv = oracle_lib.hss_split(A)
    Md, Nd = _dense_MN(oracle_lib, A)
    rhs = P.random_vector(A.n, 3)
    a = 0.3
    v, it = oracle_lib.cg_solve(A, m, a, rhs, eps=1e-13, maxit=2000)
    ref = np.linalg.solve(a * np.eye(A.n) + Md, rhs)
    assert it > 0 and np.linalg.norm(v - ref) <= 1e-11 * np.linalg.norm(ref)
    v, it = oracle_lib.cgnr_solve(A, nv, a, rhs, eps=1e-13, maxit=4000)
    ref = np.linalg.solve(a * np.eye(A.n) + Nd, rhs)
    assert it > 0 and np.linalg.norm(v - ref) <= 1e-10 * np.linalg.norm(ref)


# ---------------------------------------------------------------------------
# GADI and GADI-IR (eq. (gadi), Algorithm 1, Thm 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("alpha,omega", [(0.05, 0.0), (0.7, 1.0), (4.0, 1.5), (20.0, 1.9)])
def test_thm1_spectral_radius_below_one(oracle_lib, alpha, omega):
    A = P.convdiff_csr(3, 5, beta=20.0, faces=P.grf_faces(5, seed=4))
    Md, Nd = _dense_MN(oracle_lib, A)
    T = oracle_lib.iteration_matrix(Md, Nd, alpha, omega)
    rho = np.abs(np.linalg.eigvals(T)).max()
    assert rho < 1.0
    # the same T written as I - (2-w) a S^-1 H^-1 A (§2.1 notation p = (2-w) a)
    n = A.n
    T2 = np.eye(n) - (2 - omega) * alpha * np.linalg.solve(
        alpha * np.eye(n) + Nd, np.linalg.solve(alpha * np.eye(n) + Md, Md + Nd))
    assert np.allclose(T, T2, atol=1e-11)


@pytest.mark.parametrize("form", ["gadi", "gadi_ir"])
@pytest.mark.parametrize("alpha,omega", [(0.4, 1.0), (2.0, 0.3), (0.1, 1.8)])
def test_one_step_is_iteration_matrix(oracle_lib, form, alpha, omega):
    """With b = 0 one outer step maps x0 to T(alpha, omega) x0 (Thm 1), for
    both the two-half-step form and Algorithm 1 with exact inner solves."""
    A = P.convdiff_csr(2, 6, beta=15.0, faces=None)
    Md, Nd = _dense_MN(oracle_lib, A)
    T = oracle_lib.iteration_matrix(Md, Nd, alpha, omega)
    x0 = P.random_vector(A.n, 5)
    b = np.zeros(A.n)
    if form == "gadi":
        x1, info, _ = oracle_lib.gadi(A, b, alpha, omega, tol=0.0, eps_inner=1e-15,
                                      max_inner=400, max_outer=1, x0=x0)
    else:
        x1, info, _ = oracle_lib.gadi_ir(A, b, alpha, omega, tol=0.0, eps_inner=1e-15,
                                         max_inner=400, max_outer=1, x0=x0,
                                         prec=oracle_lib.PREC_DOUBLE)
    assert info["outer_iters"] == 1
    assert np.linalg.norm(x1 - T @ x0) <= 1e-11 * np.linalg.norm(x0)


def test_two_forms_give_the_same_iterates(oracle_lib):
    """eq. (gadi) with inner solves started at x^k equals Algorithm 1 with
    u_r = u = u_f = double (x^{k+1/2} = x^k + H^-1 r^k)."""
    A = P.convdiff_csr(3, 5, beta=8.0, faces=P.grf_faces(5, seed=9))
    b = P.rhs_from_solution(A, P.manufactured_solution(3, 5))
    for k in (1, 2, 5):
        x1, _, _ = oracle_lib.gadi(A, b, 0.6, 1.2, tol=0.0, eps_inner=1e-15, max_inner=500,
                                   max_outer=k)
        x2, _, _ = oracle_lib.gadi_ir(A, b, 0.6, 1.2, tol=0.0, eps_inner=1e-15, max_inner=500,
                                      max_outer=k, prec=oracle_lib.PREC_DOUBLE)
        assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)


def test_fixed_point(oracle_lib):
    """x* = A^-1 b is a fixed point of eq. (gadi)."""
    A = P.convdiff_csr(3, 5, beta=12.0)
    b = P.random_vector(A.n, 6)
    xs = np.linalg.solve(A.to_dense(), b)
    x1, _, _ = oracle_lib.gadi(A, b, 0.9, 0.8, tol=0.0, eps_inner=1e-12, max_inner=300,
                               max_outer=1, x0=xs)
    assert np.linalg.norm(x1 - xs) <= 1e-12 * np.linalg.norm(xs)


@pytest.mark.parametrize("form", ["gadi", "gadi_ir64", "gadi_ir16", "gadi_ir32"])
def test_solution_matches_dense_lu(oracle_lib, form):
    A = P.convdiff_csr(3, 6, beta=40.0, faces=P.grf_faces(6, seed=21))
    b = P.random_vector(A.n, 7)
    xs = np.linalg.solve(A.to_dense(), b)
    kw = dict(tol=1e-14, max_outer=5000)
    if form == "gadi":
        x, info, _ = oracle_lib.gadi(A, b, 1.5, 1.0, eps_inner=1e-10, **kw)
    else:
        prec = {"gadi_ir64": oracle_lib.PREC_DOUBLE, "gadi_ir16": oracle_lib.PREC_HALF,
                "gadi_ir32": oracle_lib.PREC_SINGLE}[form]
        x, info, _ = oracle_lib.gadi_ir(A, b, 1.5, 1.0, eps_inner=1e-2, prec=prec, **kw)
    assert info["status"] == oracle_lib.OK
    assert info["eta_inf"] <= 1e-14
    cond = np.linalg.cond(A.to_dense(), np.inf)
    assert np.abs(x - xs).max() <= 4 * cond * 1e-14 * np.abs(xs).max()


def test_manufactured_solution_config_2d(oracle_lib):
    """2D 32x32, beta = 10, b = A*1, alpha = 0.5, omega = 1, inner eps 1e-10,
    RES <= 1e-12 (§4.1's RES). Forward error bound ||x - 1||_2 <= ||r||_2 /
    lambda_min(M), since A is positive real with symmetric part M."""
    p = P.workload("convdiff2d_32_b10")
    x, info, _ = oracle_lib.gadi(p.A, p.b, 0.5, 1.0, tol=1e-12, eps_inner=1e-10,
                                 stop=oracle_lib.STOP_RES)
    assert info["status"] == oracle_lib.OK and info["res_rel"] <= 1e-12
    h = 1.0 / 33
    lam_min = 2 * (2 - 2 * math.cos(math.pi * h))
    rnorm = np.linalg.norm(oracle_lib.residual(p.A, p.b, x))
    assert np.linalg.norm(x - 1.0) <= rnorm / lam_min * (1 + 1e-6) + 1e-14


@pytest.mark.parametrize("prec", ["PREC_HALF", "PREC_BF16", "PREC_SINGLE"])
def test_low_precision_inner_reaches_fp64_floor(oracle_lib, prec):
    """Cor. 1: the limiting accuracy depends on u and u_f only. With scaling,
    FP16 (and bfloat16, FP32) inner solves reach the same eta as FP64 inner
    solves, in the same number of outer steps up to a few."""
    p = P.workload("convdiff2d_32_b10")
    x16, i16, _ = oracle_lib.gadi_ir(p.A, p.b, 0.5, 1.0, tol=1e-13, eps_inner=1e-2,
                                     prec=getattr(oracle_lib, prec))
    x64, i64, _ = oracle_lib.gadi_ir(p.A, p.b, 0.5, 1.0, tol=1e-13, eps_inner=1e-2,
                                     prec=oracle_lib.PREC_DOUBLE)
    assert i16["status"] == oracle_lib.OK and i64["status"] == oracle_lib.OK
    assert i16["eta_inf"] <= 1e-13
    assert abs(i16["outer_iters"] - i64["outer_iters"]) <= max(3, 0.05 * i64["outer_iters"])
    assert np.abs(x16 - 1).max() < 1e-10


def test_naive_fp16_stalls_scaled_fp16_does_not(oracle_lib):
    """Table '3d' (§4.1): with u_r = half the unscaled method fails or stalls
    far above double-precision accuracy; here the scaled method reaches
    RES 1e-13 where the naive one (alpha rounded into the FP16 diagonal, no
    residual scaling) does not."""
    p = P.make_problem(3, 8, 1.0, rhs="ones")
    kw = dict(tol=1e-13, stop=oracle_lib.STOP_RES, eps_inner=1e-2, max_outer=1500,
              max_inner=300)
    for alpha in (0.5, 10.0):
        _, good, _ = oracle_lib.gadi_ir(p.A, p.b, alpha, 1.0, prec=oracle_lib.PREC_HALF, **kw)
        _, bad, _ = oracle_lib.gadi_ir(p.A, p.b, alpha, 1.0,
                                       prec=oracle_lib.PREC_HALF_NAIVE, **kw)
        assert good["status"] == oracle_lib.OK and good["res_rel"] <= 1e-13
        assert bad["status"] != oracle_lib.OK and bad["res_rel"] > 1e-9


@pytest.mark.parametrize("alpha,shift_m,shift_n", [(0.5, 0.5, 0.5), (0.01, 0.01171875, 0.01000213623046875)])
def test_naive_apply_is_exact_product_with_rounded_diagonal(oracle_lib, alpha, shift_m, shift_n):
    """Unscaled FP16 operators (alpha rounded into the stored FP16 diagonal,
    §4.1's FP16 runs): with beta h / 2 = 1/4 and 2D diagonal 4, every stored
    value is exact in FP16 except the shifted diagonals: fl16(4 + alpha) = 4 +
    shift_m (FP16 spacing 2^-8 at 4: 0.01 becomes 3 * 2^-8) and fl16(0 +
    alpha) = shift_n. With small integer x the FP32 row sums are exact, so the
    applications equal the exact products (shift_m I + M)x, (shift_n I + N)x
    and (shift_n I + N)^T x, rounded once to FP16 where they are stored."""
    p = P.make_problem(2, 7, 4.0, rhs="ones")            # h = 1/8, beta h / 2 = 1/4
    rng = np.random.default_rng(3)
    x = rng.integers(-8, 9, p.n).astype(np.float64)
    A = p.A.to_dense()
    Md, Nd = (A + A.T) / 2, (A - A.T) / 2
    I = np.eye(p.n)
    assert float(np.float16(4 + alpha)) - 4 == shift_m and float(np.float16(alpha)) == shift_n
    for which, K in ((1, Md + shift_m * I), (2, Nd + shift_n * I), (3, (Nd + shift_n * I).T)):
        y, sM, sN = oracle_lib.lp_apply(p.A, alpha, which, oracle_lib.PREC_HALF_NAIVE, x)
        assert (sM, sN) == (0, 0)
        assert np.array_equal(y, (K @ x).astype(np.float16).astype(np.float64)), which


def test_outer_steps_u_shaped_in_alpha(oracle_lib):
    """Table 'alpha-effects' (§4.1): small and large alpha both need many more
    outer steps than a moderate alpha."""
    golden = json.load(open(os.path.join(GOLDEN, "alpha_effects.json")))
    steps = {r[0]: r[2] for r in golden["rows"] if r[2] is not None}
    best_paper = min(steps, key=steps.get)
    assert steps[0.02] > steps[best_paper] < steps[100.0]
    p = P.make_problem(3, 8, 1.0, rhs="ones")
    counts = {}
    for alpha in (0.1, 0.5, 10.0):
        _, info, _ = oracle_lib.gadi_ir(p.A, p.b, alpha, 1.0, tol=1e-13, stop=oracle_lib.STOP_RES,
                                        eps_inner=1e-2, prec=oracle_lib.PREC_HALF,
                                        max_outer=3000)
        assert info["status"] == oracle_lib.OK
        counts[alpha] = info["outer_iters"]
    assert counts[0.1] > counts[0.5] < counts[10.0]


def test_invalid_parameters_rejected(oracle_lib):
    A = P.convdiff_csr(2, 4, beta=1.0)
    b = np.ones(A.n)
    for a, w in ((0.0, 1.0), (-1.0, 1.0), (1.0, 2.0), (1.0, -0.1)):
        _, info, _ = oracle_lib.gadi_ir(A, b, a, w)
        assert info["status"] == oracle_lib.INVALID
        _, info, _ = oracle_lib.gadi(A, b, a, w)
        assert info["status"] == oracle_lib.INVALID


# ---------------------------------------------------------------------------
# FP16 emulation against IEEE 754 binary16 (Table 1)
# ---------------------------------------------------------------------------

def _half_bits_ref(x: float) -> int:
    """binary16 encoding of x, round to nearest, ties to even, computed with
    exact rational arithmetic from IEEE 754's definition."""
    if math.isnan(x):
        return 0x7E00
    sign = 0x8000 if math.copysign(1.0, x) < 0 else 0
    a = abs(x)
    if a == 0.0:
        return sign
    if math.isinf(a):
        return sign | 0x7C00
    e = math.frexp(a)[1] - 1
    e = max(e, -14)
    q = Fraction(2) ** (e - 10)
    m = Fraction(a) / q
    mi = math.floor(m)
    rem = m - mi
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and mi % 2 == 1):
        mi += 1
    if mi == 2048:
        mi, e = 1024, e + 1
    if e > 15:
        return sign | 0x7C00
    if mi < 1024:
        return sign | mi
    return sign | ((e + 15) << 10) | (mi - 1024)


def test_fp16_rounding_is_ieee_rne(oracle_lib):
    rng = np.random.default_rng(123)
    mags = np.exp2(rng.uniform(-27, 17, 4000))
    vals = mags * rng.choice([-1.0, 1.0], 4000)
    # exact ties between neighbouring halves, subnormal ties, overflow edge
    ties = [(k + 0.5) * 2.0 ** -10 for k in range(1024, 1040)]
    ties += [(k + 0.5) * 2.0 ** -24 for k in range(0, 20)]
    special = [0.0, -0.0, 65504.0, 65519.99, 65520.0, 1e6, -1e6, 2.0 ** -25, 2.0 ** -26,
               6.1e-5, 5.96e-8, 1.0 / 3.0]
    x = np.concatenate([vals, ties, special])
    got = oracle_lib.to_half_bits(x)
    want = np.array([_half_bits_ref(float(v)) for v in x], dtype=np.uint16)
    assert np.array_equal(got, want)
    with np.errstate(over="ignore"):
        assert np.array_equal(got, x.astype(np.float16).view(np.uint16))


def _bf16_bits_ref(x: float) -> int:
    """bfloat16 encoding of x (8 significant bits, exponent range of IEEE
    binary32: normal down to 2^-126, subnormal steps 2^-133), round to
    nearest, ties to even, with exact rational arithmetic."""
    if math.isnan(x):
        return 0x7FC0
    sign = 0x8000 if math.copysign(1.0, x) < 0 else 0
    a = abs(x)
    if a == 0.0:
        return sign
    if math.isinf(a):
        return sign | 0x7F80
    e = math.frexp(a)[1] - 1
    e = max(e, -126)
    q = Fraction(2) ** (e - 7)
    m = Fraction(a) / q
    mi = math.floor(m)
    rem = m - mi
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and mi % 2 == 1):
        mi += 1
    if mi == 256:
        mi, e = 128, e + 1
    if e > 127:
        return sign | 0x7F80
    if mi < 128:
        return sign | mi
    return sign | ((e + 127) << 7) | (mi - 128)


def test_bf16_rounding_is_rne_with_one_rounding(oracle_lib):
    """The bfloat16 inner-precision variant rounds FP64 values once to 8
    significant bits (not through an intermediate FP32 rounding)."""
    rng = np.random.default_rng(321)
    vals = np.exp2(rng.uniform(-140, 130, 4000)) * rng.choice([-1.0, 1.0], 4000)
    ties = [(k + 0.5) * 2.0 ** -7 for k in range(128, 150)]            # halfway in the normal range
    ties += [(k + 0.5) * 2.0 ** -133 for k in range(0, 20)]            # halfway between subnormals
    # just above a tie by less than FP32's resolution: rounding through FP32 would create the tie
    ties += [(129 + 0.5) * 2.0 ** -7 * (1 + 2.0 ** -40), (130 + 0.5) * 2.0 ** -7 * (1 - 2.0 ** -40)]
    special = [0.0, -0.0, 3.3895313892515355e38, 3.4e38, 1e39, 2.0 ** -134, 2.0 ** -135, 1.0 / 3.0]
    x = np.concatenate([vals, ties, special])
    got = oracle_lib.to_bf16_bits(x)
    want = np.array([_bf16_bits_ref(float(v)) for v in x], dtype=np.uint16)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]


def test_fp16_parameters_of_table1(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "ieee_precisions.json")))["half"]
    u = 2.0 ** g["unit_roundoff_log2"]
    rng = np.random.default_rng(7)
    x = np.exp2(rng.uniform(-14, 15, 20000))        # normal range
    h = oracle_lib.to_half_bits(x).view(np.float16).astype(np.float64)
    relerr = np.abs(h - x) / x
    assert relerr.max() <= u and relerr.max() > 0.9 * u
    big = oracle_lib.to_half_bits(np.array([65504.0])).view(np.float16)[0]
    assert math.floor(math.log10(float(big))) + 1 == g["range_exp10"]     # 6.5e4 ~ 10^5
    tiny = 2.0 ** -14
    assert oracle_lib.to_half_bits(np.array([tiny])).view(np.float16)[0] == np.float16(tiny)
    assert round(math.log10(tiny)) == -g["range_exp10"] + 1 or round(math.log10(tiny)) == -g["range_exp10"]
