"""Pins of the oracle's FP8 E4M3 inner precision (a storage format below the
paper's FP16, the direction its conclusion leaves open) against facts that do
not come from the oracle: the value set of the format enumerated from its
bit layout, nearest-even rounding found by exhaustive search, PyTorch's own
float8_e4m3fn conversion, the error bound of one rounded operator
application, and Cor. 1 (the limiting accuracy of GADI-IR depends on u and
u_f only).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2501_04229_gb300 import problems as P


def _e4m3_value(code: int):
    """Value of an 8-bit E4M3 code: sign bit, 4 exponent bits (bias 7), 3
    fraction bits; exponent field 0 is subnormal (f 2^-9); S.1111.111 is NaN."""
    s = -1 if code & 0x80 else 1
    e = (code >> 3) & 0xF
    f = code & 0x7
    if e == 0xF and f == 0x7:
        return None
    if e == 0:
        return s * Fraction(f, 512)
    return s * Fraction(8 + f, 8) * Fraction(2) ** (e - 7)


_FINITE = [(c, _e4m3_value(c)) for c in range(256) if _e4m3_value(c) is not None]


def _nearest_code(x: float) -> int:
    """Code of the representable value nearest to x (ties: even fraction
    bit), magnitudes beyond 448 saturated; zero keeps the sign of x."""
    if math.isnan(x):
        return 0x7F
    neg = math.copysign(1.0, x) < 0
    a = Fraction(abs(x)) if math.isfinite(x) else Fraction(10 ** 6)
    if a >= 448:
        return 0xFE if neg else 0x7E
    best = None
    for c, v in _FINITE:
        if c & 0x80:
            continue
        d = abs(v - a)
        key = (d, c & 1)               # nearer first, then the even fraction
        if best is None or key < best[0]:
            best = (key, c)
    c = best[1]
    return c | 0x80 if neg else c


def test_value_set_of_the_format():
    vals = sorted(v for c, v in _FINITE if not c & 0x80)
    assert len(_FINITE) == 254                  # 256 codes minus the two NaNs
    assert vals[-1] == 448 and vals[1] == Fraction(1, 512)
    assert Fraction(1, 64) in vals              # smallest normal 2^-6


def test_e4m3_rounding_is_nearest_even_and_saturating(oracle_lib):
    rng = np.random.default_rng(77)
    vals = np.exp2(rng.uniform(-12, 10, 3000)) * rng.choice([-1.0, 1.0], 3000)
    pos = sorted(float(v) for c, v in _FINITE if not c & 0x80)
    ties = [(a + b) / 2 for a, b in zip(pos[:-1], pos[1:])]       # every halfway point
    near = [t * (1 + 2.0 ** -30) for t in ties[::7]] + [t * (1 - 2.0 ** -30) for t in ties[3::7]]
    special = [0.0, -0.0, 448.0, 449.0, 464.0, 480.0, 1e9, -1e9, 2.0 ** -10, 2.0 ** -10 * 1.0001,
               -(2.0 ** -11), 3 * 2.0 ** -10, 1.0 / 3.0]
    x = np.concatenate([vals, ties, near, special])
    got = oracle_lib.to_e4m3_bits(x)
    want = np.array([_nearest_code(float(v)) for v in x], dtype=np.uint8)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]


def test_e4m3_rounding_agrees_with_torch_float8(oracle_lib):
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8_e4m3fn in this PyTorch")
    rng = np.random.default_rng(5)
    x = (np.exp2(rng.uniform(-11, 8.8, 20000)) * rng.choice([-1.0, 1.0], 20000)).astype(np.float32)
    x = x[np.abs(x) < 448]
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = oracle_lib.to_e4m3_bits(x.astype(np.float64))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("which", [1, 2, 3])
def test_e4m3_operator_application_error_bound(oracle_lib, which):
    """One application of H' (or S', S'^T) in E4M3: entries and result are
    rounded to 4 significant bits (unit roundoff u8 = 2^-4), the sums are
    FP32, so |y - K x| <= u8 |K x| + (1 + u8) u8 |K| |x| + 2^-10 + FP32
    terms, with K the exactly scaled operator of the returned scales."""
    A = P.convdiff_csr(3, 6, beta=40.0)
    alpha = 0.7
    rng = np.random.default_rng(which)
    xv = rng.uniform(-2, 2, A.n)
    codes = oracle_lib.to_e4m3_bits(xv)
    x = np.array([float(_e4m3_value(int(c))) for c in codes])
    y, sM, sN = oracle_lib.lp_apply(A, alpha, which, oracle_lib.PREC_E4M3, x)
    m, nv = oracle_lib.hss_split(A)
    V = P.Csr(A.n, A.row_ptr, A.col_idx, m if which == 1 else nv).to_dense()
    if which == 3:
        V = V.T
    s = sM if which == 1 else sN
    K = np.ldexp(alpha * np.eye(A.n) + V, -s)
    exact = K @ x
    u8 = 2.0 ** -4
    bound = u8 * np.abs(exact) + (1 + u8) * u8 * (np.abs(K) @ np.abs(x)) + 2.0 ** -10 + 1e-5
    assert np.all(np.abs(y - exact) <= bound)
    # every output is an E4M3 value
    back = np.array([float(_e4m3_value(int(c))) for c in oracle_lib.to_e4m3_bits(y)])
    assert np.array_equal(back, y)
    # the scaled operator's largest row sum lies in (1, 2]
    assert 1.0 < np.abs(K).sum(axis=1).max() <= 2.0


def test_e4m3_inner_reaches_fp64_floor(oracle_lib):
    """Cor. 1: the limiting accuracy depends on u and u_f only, so with the
    power-of-two scaling even 4-significant-bit inner storage reaches the
    accuracy of FP64 inner solves; the weaker inner solves cost outer steps."""
    p = P.workload("convdiff2d_32_b10")
    kw = dict(tol=1e-13, eps_inner=0.1, max_outer=3000)
    x8, i8, _ = oracle_lib.gadi_ir(p.A, p.b, 0.5, 1.0, prec=oracle_lib.PREC_E4M3, **kw)
    x64, i64, _ = oracle_lib.gadi_ir(p.A, p.b, 0.5, 1.0, prec=oracle_lib.PREC_DOUBLE, **kw)
    assert i8["status"] == oracle_lib.OK and i8["eta_inf"] <= 1e-13
    assert np.abs(x8 - 1).max() < 1e-10
    assert i64["outer_iters"] <= i8["outer_iters"] <= 1.25 * i64["outer_iters"]
