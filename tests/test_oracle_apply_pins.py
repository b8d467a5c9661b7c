"""Pins of the oracle's single operator applications in the scaled inner
precisions (FP16 and bfloat16 storage with the power-of-two scaling, and
FP32), the reference of every bit-exact GPU application test.

The scaled inner operators of Algorithm 1 steps 2 and 3 are
H' = 2^-sM (aI + M) and S' = 2^-sN (aI + N) (and S'^T), with M, N the HSS
parts of §4.1, the stored entries rounded to u_r (§2.2: values rounded to
the inner precision, Table 1's formats), alpha kept in FP32 and every row
summed in FP32. The scale exponent makes the largest absolute row sum of the
scaled operator fall in (1, 2].

Two kinds of pin, both computed here from the definition without the
oracle:
  * exact cases: every stored value, 2^-s alpha and every FP32 row sum is
    exact, so an application must equal the exact product K x rounded once
    to the storage format (the rounding written out below from the format's
    significand width). Planted mistakes (alpha dropped, the scale off by
    one, 2^-s alpha rounded to the storage format instead of FP32) change
    the expected outputs, which the tests check as well.
  * an error bound on a case with inexact coefficients.
"""
import math

import numpy as np
import pytest

from paper_2501_04229_gb300 import problems as P


def _round_sig(v, bits):
    """Round to nearest even with `bits` significant bits (normal range)."""
    out = np.empty_like(v)
    for i, t in enumerate(v):
        if t == 0.0:
            out[i] = 0.0
            continue
        m, e = math.frexp(t)                 # t = m 2^e, 0.5 <= |m| < 1
        q = m * 2.0 ** bits                  # exact
        out[i] = math.ldexp(float(np.round(q)), e - bits)   # np.round: half to even
    return out


SIG_BITS = {"PREC_HALF": 11, "PREC_BF16": 8}


def _scale_exp(rowsum):
    """s with rowsum 2^-s in (1, 2]."""
    m, e = math.frexp(rowsum)                # rowsum = m 2^e, m in [0.5, 1)
    return e - 1 if m > 0.5 else e - 2


def _exact_case():
    # 2D N = 7: h = 1/8, beta h / 2 = 1/4; A has diagonal 4, off-diagonals
    # -1 -+ 1/4, so M = 4 on the diagonal and -1 off it, N = +-1/4
    p = P.make_problem(2, 7, 4.0, rhs="ones")
    A = p.A.to_dense()
    Md, Nd = (A + A.T) / 2, (A - A.T) / 2
    return p, Md, Nd


ALPHA = 0.5 + 3 * 2.0 ** -12      # exact in FP32; alpha / 8 is not an FP16 value


def _x(n):
    rng = np.random.default_rng(11)
    x = rng.integers(-8, 9, n).astype(np.float64)
    x[: n // 3] = 3.0                 # constant patches: the M part cancels there
    return x


@pytest.mark.parametrize("prec", ["PREC_HALF", "PREC_BF16"])
def test_scaled_application_is_exact_product_rounded_once(oracle_lib, prec):
    p, Md, Nd = _exact_case()
    n = p.n
    I = np.eye(n)
    x = _x(n)
    bits = SIG_BITS[prec]
    sM = _scale_exp(np.abs(Md).sum(axis=1).max() + ALPHA)
    sN = _scale_exp(max(np.abs(Nd).sum(axis=1).max(), np.abs(Nd.T).sum(axis=1).max()) + ALPHA)
    assert (sM, sN) == (3, 0)
    for which, V, s in ((1, Md, sM), (2, Nd, sN), (3, Nd.T, sN)):
        K = np.ldexp(ALPHA * I + V, -s)
        # the stored entries 2^-s v are exact in both formats here
        assert np.array_equal(_round_sig(np.ldexp(V[V != 0], -s), bits), np.ldexp(V[V != 0], -s))
        want = _round_sig(K @ x, bits)
        y, gM, gN = oracle_lib.lp_apply(p.A, ALPHA, which, getattr(oracle_lib, prec), x)
        assert (gM, gN) == (sM, sN)
        assert np.array_equal(y, want), which
        # planted mistakes change the result, so the equality above pins them
        wrong = {
            "alpha dropped": _round_sig(np.ldexp(V, -s) @ x, bits),
            "scale off by one": _round_sig(np.ldexp(ALPHA * I + V, -(s + 1)) @ x, bits),
            "2^-s alpha in the storage format": _round_sig(
                (_round_sig(np.array([math.ldexp(ALPHA, -s)]), bits)[0] * I + np.ldexp(V, -s)) @ x, bits),
        }
        for name, w in wrong.items():
            assert not np.array_equal(w, want), (which, name)


def test_fp32_application_is_exact_unscaled_product(oracle_lib):
    p, Md, Nd = _exact_case()
    I = np.eye(p.n)
    x = _x(p.n)
    for which, V in ((1, Md), (2, Nd), (3, Nd.T)):
        y, gM, gN = oracle_lib.lp_apply(p.A, ALPHA, which, oracle_lib.PREC_SINGLE, x)
        assert (gM, gN) == (0, 0)            # FP32 inner operators are not scaled
        assert np.array_equal(y, (ALPHA * I + V) @ x), which
        assert not np.array_equal(y, V @ x)


@pytest.mark.parametrize("prec", ["PREC_HALF", "PREC_BF16"])
@pytest.mark.parametrize("which", [1, 2, 3])
def test_scaled_application_error_bound(oracle_lib, prec, which):
    """Inexact coefficients (beta h / 2 = 40/14): with K the exactly scaled
    operator, stored entries off by at most u |K_ij| (u = 2^-bits), 2^-s alpha
    exact in FP32 to 2^-24, at most 7 FP32 fused multiply-adds per row and one
    rounding of the result to the format,
        |y - K x| <= u |K x| + (1 + u) ((u + 2^-24) + 8 2^-24) |K| |x|."""
    A = P.convdiff_csr(3, 6, beta=40.0)
    alpha = 0.7
    bits = SIG_BITS[prec]
    u = 2.0 ** -bits
    rng = np.random.default_rng(100 + which)
    x = _round_sig(rng.uniform(-2, 2, A.n), bits)
    y, sM, sN = oracle_lib.lp_apply(A, alpha, which, getattr(oracle_lib, prec), x)
    Ad = A.to_dense()
    V = (Ad + Ad.T) / 2 if which == 1 else (Ad - Ad.T) / 2
    if which == 3:
        V = V.T
    s = sM if which == 1 else sN
    K = np.ldexp(alpha * np.eye(A.n) + V, -s)
    exact = K @ x
    bound = u * np.abs(exact) + (1 + u) * ((u + 2.0 ** -24) + 8 * 2.0 ** -24) * (np.abs(K) @ np.abs(x))
    assert np.all(np.abs(y - exact) <= bound)
    # every output is a value of the format, and the scale is the one stated
    assert np.array_equal(_round_sig(y, bits), y)
    assert 1.0 < np.abs(K).sum(axis=1).max() <= 2.0
