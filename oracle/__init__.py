"""CPU oracle for GADI / GADI-IR (arXiv 2501.04229) -- TEST INFRASTRUCTURE.

Only the tests, the smoke check and the bench's CPU-baseline leg may import
this package. The library path never does; it shares no code with it.

The arithmetic lives in gadi_oracle.c (plain C, FP64, OpenMP); this module
builds it with gcc and wraps it with ctypes. Dense helpers for tiny systems
(`iteration_matrix`, `dense_split`) are plain numpy, written from Thm 1 and
the HSS definition.

Parity pins: every function here is pinned by a CPU test against something
other than itself (dense LU, closed-form spectra, Thm 1's iteration matrix,
IEEE-754 FP16 rounding, manufactured solutions); see tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gadi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PREC_DOUBLE, PREC_SINGLE, PREC_HALF, PREC_HALF_NAIVE, PREC_BF16, PREC_E4M3 = 0, 1, 2, 3, 4, 5
STOP_ETA, STOP_RES = 0, 1
OK, INVALID, OOM, NOT_CONVERGED, DIVERGED = 0, 1, 2, 5, 6


class Params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("omega", C.c_double), ("tol", C.c_double),
                ("eps_inner", C.c_double), ("max_inner", C.c_int32), ("max_outer", C.c_int32),
                ("stop_kind", C.c_int32), ("inner_prec", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("outer_iters", C.c_int32),
                ("inner_iters_H", C.c_int64), ("inner_iters_S", C.c_int64),
                ("spmv_count", C.c_int64), ("eta_inf", C.c_double), ("res_rel", C.c_double),
                ("res0", C.c_double), ("scale_exp_M", C.c_int32), ("scale_exp_N", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile gadi_oracle.c into liboracle.so (gcc, OpenMP, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB_PATH)
    p_i32, p_f64, p_u16 = C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(C.c_uint16)
    p_u8 = C.POINTER(C.c_uint8)
    i64, f64 = C.c_int64, C.c_double
    sig = {
        "or_set_threads": (None, [C.c_int]),
        "or_get_threads": (C.c_int, []),
        "or_spmv_shift": (None, [i64, p_i32, p_i32, p_f64, f64, p_f64, p_f64]),
        "or_residual": (None, [i64, p_i32, p_i32, p_f64, p_f64, p_f64, p_f64]),
        "or_matrix_norm_inf": (f64, [i64, p_i32, p_f64]),
        "or_backward_error": (f64, [i64, p_i32, p_i32, p_f64, p_f64, p_f64]),
        "or_hss_split": (C.c_int, [i64, p_i32, p_i32, p_f64, p_f64, p_f64]),
        "or_cg_solve": (i64, [i64, p_i32, p_i32, p_f64, f64, p_f64, p_f64, f64, C.c_int32]),
        "or_cgnr_solve": (i64, [i64, p_i32, p_i32, p_f64, f64, p_f64, p_f64, f64, C.c_int32]),
        "or_gadi": (C.c_int, [i64, p_i32, p_i32, p_f64, p_f64, p_f64, C.POINTER(Params),
                              C.POINTER(Info), p_f64, p_i32, p_i32]),
        "or_gadi_ir": (C.c_int, [i64, p_i32, p_i32, p_f64, p_f64, p_f64, C.POINTER(Params),
                                 C.POINTER(Info), p_f64, p_i32, p_i32]),
        "or_gadi_ir_split": (C.c_int, [i64, p_i32, p_i32, p_f64, p_f64, p_f64, p_f64,
                                       C.POINTER(Params), C.POINTER(Info), p_f64, p_i32, p_i32]),
        "or_lp_apply": (C.c_int, [i64, p_i32, p_i32, p_f64, p_f64, f64, C.c_int, C.c_int,
                                  p_f64, p_f64, p_i32, p_i32]),
        "or_to_half_bits": (None, [i64, p_f64, p_u16]),
        "or_to_bf16_bits": (None, [i64, p_f64, p_u16]),
        "or_to_e4m3_bits": (None, [i64, p_f64, p_u8]),
        "or_sylv_norm_inf": (f64, [i64, i64, p_f64, p_f64, p_f64, p_f64, p_f64, p_f64]),
        "or_sylv_gadi_ab": (C.c_int, [i64, i64, p_f64, p_f64, p_f64, p_f64, p_f64, p_f64, p_f64, p_f64,
                                  f64, f64, C.c_int32, f64, C.c_int32, C.POINTER(Info), p_f64]),
        "or_wtime": (f64, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _csr(A):
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    v = np.ascontiguousarray(A.val, dtype=np.float64)
    return int(A.n), rp, ci, v


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def set_threads(t: int) -> None:
    _load().or_set_threads(int(t))


def get_threads() -> int:
    return int(_load().or_get_threads())


def wtime() -> float:
    return float(_load().or_wtime())


def spmv_shift(n, row_ptr, col_idx, val, sigma, x):
    """y = (sigma I + V) x."""
    lib = _load()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    v, x = _f64(val), _f64(x)
    y = np.empty(n)
    lib.or_spmv_shift(n, _p(rp, C.c_int32), _p(ci, C.c_int32), _p(v, C.c_double), float(sigma),
                      _p(x, C.c_double), _p(y, C.c_double))
    return y


def residual(A, b, x):
    lib = _load()
    n, rp, ci, v = _csr(A)
    b, x = _f64(b), _f64(x)
    r = np.empty(n)
    lib.or_residual(n, _p(rp, C.c_int32), _p(ci, C.c_int32), _p(v, C.c_double),
                    _p(b, C.c_double), _p(x, C.c_double), _p(r, C.c_double))
    return r


def matrix_norm_inf(A) -> float:
    n, rp, ci, v = _csr(A)
    return float(_load().or_matrix_norm_inf(n, _p(rp, C.c_int32), _p(v, C.c_double)))


def backward_error(A, b, x) -> float:
    """eta_inf = ||b - Ax||_inf / (||A||_inf ||x||_inf + ||b||_inf), FP64."""
    n, rp, ci, v = _csr(A)
    b, x = _f64(b), _f64(x)
    return float(_load().or_backward_error(n, _p(rp, C.c_int32), _p(ci, C.c_int32),
                                           _p(v, C.c_double), _p(b, C.c_double), _p(x, C.c_double)))


def hss_split(A):
    """(M values, N values) on A's pattern: M = (A+A^T)/2, N = (A-A^T)/2."""
    n, rp, ci, v = _csr(A)
    m = np.empty_like(v)
    nv = np.empty_like(v)
    st = _load().or_hss_split(n, _p(rp, C.c_int32), _p(ci, C.c_int32), _p(v, C.c_double),
                              _p(m, C.c_double), _p(nv, C.c_double))
    if st != OK:
        raise ValueError("matrix pattern is not structurally symmetric (or rows unsorted)")
    return m, nv


def cg_solve(A_pattern, mval, sigma, rhs, x0=None, eps=1e-10, maxit=1000):
    """CG on (sigma I + M) v = rhs (M symmetric, values on A's pattern)."""
    n, rp, ci, _ = _csr(A_pattern)
    m = _f64(mval)
    rhs = _f64(rhs)
    v = np.zeros(n) if x0 is None else _f64(x0).copy()
    it = _load().or_cg_solve(n, _p(rp, C.c_int32), _p(ci, C.c_int32), _p(m, C.c_double),
                             float(sigma), _p(rhs, C.c_double), _p(v, C.c_double), float(eps),
                             int(maxit))
    return v, int(it)


def cgnr_solve(A_pattern, nval, sigma, rhs, x0=None, eps=1e-10, maxit=1000):
    """CGNR on (sigma I + N) v = rhs."""
    n, rp, ci, _ = _csr(A_pattern)
    nv = _f64(nval)
    rhs = _f64(rhs)
    v = np.zeros(n) if x0 is None else _f64(x0).copy()
    it = _load().or_cgnr_solve(n, _p(rp, C.c_int32), _p(ci, C.c_int32), _p(nv, C.c_double),
                               float(sigma), _p(rhs, C.c_double), _p(v, C.c_double), float(eps),
                               int(maxit))
    return v, int(it)


def _run(fn_name, A, b, x0, alpha, omega, tol, eps_inner, max_inner, max_outer, stop, prec,
         m_user=None):
    lib = _load()
    n, rp, ci, v = _csr(A)
    b = _f64(b)
    x = np.zeros(n) if x0 is None else _f64(x0).copy()
    P = Params(alpha=alpha, omega=omega, tol=tol, eps_inner=eps_inner, max_inner=max_inner,
               max_outer=max_outer, stop_kind=stop, inner_prec=prec)
    I = Info()
    eta = np.full(max_outer + 1, np.nan)
    itH = np.zeros(max(max_outer, 1), dtype=np.int32)
    itS = np.zeros(max(max_outer, 1), dtype=np.int32)
    tail = (_p(b, C.c_double), _p(x, C.c_double), C.byref(P), C.byref(I),
            _p(eta, C.c_double), _p(itH, C.c_int32), _p(itS, C.c_int32))
    if fn_name == "or_gadi_ir_split":
        mu = _f64(m_user)
        getattr(lib, fn_name)(n, _p(rp, C.c_int32), _p(ci, C.c_int32), _p(v, C.c_double),
                              _p(mu, C.c_double), *tail)
    else:
        getattr(lib, fn_name)(n, _p(rp, C.c_int32), _p(ci, C.c_int32), _p(v, C.c_double), *tail)
    k = I.outer_iters
    hist = {"eta": eta[:k + 1].copy(), "itH": itH[:k].copy(), "itS": itS[:k].copy()}
    return x, I.as_dict(), hist


def gadi(A, b, alpha, omega, tol=1e-13, eps_inner=1e-10, max_inner=10000, max_outer=10000,
         stop=STOP_ETA, x0=None):
    """Plain FP64 GADI in the two-half-step form of eq. (gadi)."""
    return _run("or_gadi", A, b, x0, alpha, omega, tol, eps_inner, max_inner, max_outer, stop,
                PREC_DOUBLE)


def gadi_ir(A, b, alpha, omega, tol=1e-13, eps_inner=1e-2, max_inner=200, max_outer=10000,
            stop=STOP_ETA, prec=PREC_HALF, x0=None, m_user=None):
    """GADI-IR, Algorithm 1, u = u_f = FP64, u_r = prec. m_user: None for the
    HSS splitting, else M's values on A's pattern (N = A - M)."""
    if m_user is not None:
        return _run("or_gadi_ir_split", A, b, x0, alpha, omega, tol, eps_inner, max_inner,
                    max_outer, stop, prec, m_user=m_user)
    return _run("or_gadi_ir", A, b, x0, alpha, omega, tol, eps_inner, max_inner, max_outer, stop,
                prec)


def sylv_norm_inf(a, b):
    m, n = len(a[1]), len(b[1])
    arrs = [_f64(v) for v in (*a, *b)]
    return _load().or_sylv_norm_inf(m, n, *[_p(v, C.c_double) for v in arrs])


def sylv_gadi_ab(a, b, Cm, alpha, omega, prec=PREC_HALF, tol=1e-13, max_outer=10000, x0=None):
    """GADI-AB for A X + X B = C (see or_sylv_gadi_ab); a, b = (lo, dg, up).
    Returns (X, info, eta history)."""
    m, n = len(a[1]), len(b[1])
    arrs = [_f64(v) for v in (*a, *b)]
    Cm = np.ascontiguousarray(Cm, dtype=np.float64)
    X = np.zeros((m, n)) if x0 is None else np.array(x0, dtype=np.float64, order="C")
    info = Info()
    hist = np.zeros(max_outer + 1)
    _load().or_sylv_gadi_ab(m, n, *[_p(v, C.c_double) for v in arrs], _p(Cm, C.c_double), _p(X, C.c_double),
                            float(alpha), float(omega), int(prec), float(tol), int(max_outer), C.byref(info),
                            _p(hist, C.c_double))
    d = info.as_dict()
    return X, d, hist[:d["outer_iters"] + 1]


def lp_apply(A, alpha, which, prec, x, m_user=None):
    """One operator application as GADI-IR does it (see or_lp_apply):
    which 0 A, 1 H', 2 S', 3 S'^T. Returns (y, sM, sN)."""
    lib = _load()
    n, rp, ci, v = _csr(A)
    x = _f64(x)
    y = np.empty(n)
    sM, sN = C.c_int32(), C.c_int32()
    mu = None if m_user is None else _f64(m_user)
    st = lib.or_lp_apply(n, _p(rp, C.c_int32), _p(ci, C.c_int32), _p(v, C.c_double),
                         None if mu is None else _p(mu, C.c_double), float(alpha), int(which),
                         int(prec), _p(x, C.c_double), _p(y, C.c_double), C.byref(sM), C.byref(sN))
    if st != OK:
        raise ValueError("or_lp_apply failed")
    return y, sM.value, sN.value


def to_bf16_bits(x) -> np.ndarray:
    """bfloat16 bit patterns of fl_bf16(x), round-to-nearest-even from FP64."""
    x = _f64(x)
    out = np.empty(x.shape, dtype=np.uint16)
    _load().or_to_bf16_bits(x.size, _p(x, C.c_double), _p(out, C.c_uint16))
    return out


def to_e4m3_bits(x) -> np.ndarray:
    """FP8 E4M3 codes of fl_e4m3(x): round to nearest even from FP64,
    saturating at +-448."""
    x = _f64(x)
    out = np.empty(x.shape, dtype=np.uint8)
    _load().or_to_e4m3_bits(x.size, _p(x, C.c_double), _p(out, C.c_uint8))
    return out


def to_half_bits(x) -> np.ndarray:
    """IEEE binary16 bit patterns of fl16(x), round-to-nearest-even from FP64."""
    x = _f64(x)
    out = np.empty(x.shape, dtype=np.uint16)
    _load().or_to_half_bits(x.size, _p(x, C.c_double), _p(out, C.c_uint16))
    return out


# ---------------------------------------------------------------------------
# Dense helpers for tiny systems (plain numpy)
# ---------------------------------------------------------------------------

def dense_split(Ad: np.ndarray):
    """HSS splitting of a dense matrix: (M, N) = ((A+A^T)/2, (A-A^T)/2)."""
    return 0.5 * (Ad + Ad.T), 0.5 * (Ad - Ad.T)


def iteration_matrix(M: np.ndarray, N: np.ndarray, alpha: float, omega: float) -> np.ndarray:
    """T(alpha, omega) = (aI+N)^-1 (aI+M)^-1 (a^2 I + MN - (1-w) a A)  (Thm 1)."""
    n = M.shape[0]
    I = np.eye(n)
    A = M + N
    inner = alpha * alpha * I + M @ N - (1.0 - omega) * alpha * A
    return np.linalg.solve(alpha * I + N, np.linalg.solve(alpha * I + M, inner))
