"""ctypes binding of libgadi.so (include/gadi.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels. Device buffers are torch CUDA tensors (passed as raw pointers);
host buffers are numpy arrays. Loading fails loudly when the library has not
been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgadi.so")

GADI_OK, GADI_ERR_INVALID_ARG, GADI_ERR_OUT_OF_MEMORY, GADI_ERR_CUDA = 0, 1, 2, 3
GADI_ERR_RANGE, GADI_ERR_NOT_CONVERGED, GADI_ERR_DIVERGED, GADI_ERR_TIMEOUT = 4, 5, 6, 7
GADI_ERR_NO_MODEL, GADI_ERR_UNSUPPORTED = 8, 9
GADI_SPLIT_HSS, GADI_SPLIT_USER = 0, 1
GADI_F64, GADI_F32, GADI_F16, GADI_BF16, GADI_E4M3 = 0, 1, 2, 3, 4
GADI_STOP_ETA, GADI_STOP_RES = 0, 1
GADI_KERNEL_AUTO, GADI_KERNEL_SPARSE, GADI_KERNEL_STENCIL = 0, 1, 2
OP_A, OP_H, OP_S, OP_ST = 0, 1, 2, 3

# every entry point declared in include/gadi.h
EXPORTS = [
    "gadi_create", "gadi_set_params", "gadi_set_inner", "gadi_set_stop", "gadi_set_kernel", "gadi_set_item_rows", "gadi_set_traversal", "gadi_set_scaling",
    "gadi_set_launch", "gadi_set_wait_limit", "gadi_debug_force_timeout", "gadi_solve",
    "gadi_apply", "gadi_get_scales", "gadi_predict_params", "gadi_destroy", "gadi_status_str",
    "gadi_last_error", "gadi_solve_stencil_noalloc", "gadi_sweep", "gadi_model_fit",
    "gadi_model_predict", "gadi_model_loss", "gadi_mlp_gradient", "gadi_mlp_param_count",
    "gadi_model_destroy", "gadi_set_model", "gadi_sylv_create", "gadi_sylv_set_params", "gadi_sylv_solve",
    "gadi_sylv_last_error", "gadi_sylv_destroy",
]
GADI_MODEL_MLP, GADI_MODEL_GPR, GADI_MODEL_GRID = 0, 1, 2


class gadi_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("on_device", C.c_int32)]


class gadi_stencil(C.Structure):
    _fields_ = [("dim", C.c_int32), ("N", C.c_int32), ("beta", C.c_double),
                ("variable_k", C.c_int32)]


class gadi_info(C.Structure):
    _fields_ = [("outer_iters", C.c_int32), ("status", C.c_int32),
                ("inner_iters_H", C.c_int64), ("inner_iters_S", C.c_int64),
                ("spmv_count", C.c_int64), ("eta_inf", C.c_double), ("res_rel", C.c_double),
                ("t_solve_s", C.c_double), ("scale_exp_M", C.c_int32), ("scale_exp_N", C.c_int32),
                ("kernel", C.c_int32), ("grid_blocks", C.c_int32), ("block_threads", C.c_int32),
                ("zmarch_planes", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class gadi_sweep_instance(C.Structure):
    _fields_ = [("dim", C.c_int32), ("N", C.c_int32), ("beta", C.c_double)]


class gadi_sweep_candidate(C.Structure):
    _fields_ = [("alpha", C.c_double), ("omega", C.c_double)]


class gadi_sweep_record(C.Structure):
    _fields_ = [("instance", C.c_int32), ("candidate", C.c_int32), ("status", C.c_int32),
                ("raced_out", C.c_int32), ("outer_iters", C.c_int32), ("team_blocks", C.c_int32),
                ("inner_iters_H", C.c_int64), ("inner_iters_S", C.c_int64),
                ("spmv_count", C.c_int64), ("eta_inf", C.c_double), ("time_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class GadiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_str(status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libgadi.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2501_04229_gb300.build` "
                           "(or __graft_entry__.build()); there is no fallback path")
    lib = C.CDLL(path)
    vp, i32, f64 = C.c_void_p, C.c_int32, C.c_double
    sig = {
        "gadi_create": (i32, [C.POINTER(gadi_csr), i32, C.POINTER(gadi_csr),
                              C.POINTER(gadi_stencil), vp, C.POINTER(vp)]),
        "gadi_set_params": (i32, [vp, f64, f64, i32, i32, i32]),
        "gadi_set_inner": (i32, [vp, f64, i32, i32]),
        "gadi_set_stop": (i32, [vp, i32]),
        "gadi_set_kernel": (i32, [vp, i32]),
        "gadi_set_item_rows": (i32, [vp, i32]),
        "gadi_set_traversal": (i32, [vp, i32]),
        "gadi_set_scaling": (i32, [vp, i32]),
        "gadi_set_launch": (i32, [vp, i32, i32]),
        "gadi_set_wait_limit": (i32, [vp, f64]),
        "gadi_debug_force_timeout": (i32, [vp, i32]),
        "gadi_solve": (i32, [vp, vp, vp, f64, C.POINTER(gadi_info)]),
        "gadi_apply": (i32, [vp, i32, vp, vp]),
        "gadi_get_scales": (i32, [vp, C.POINTER(i32), C.POINTER(i32)]),
        "gadi_predict_params": (i32, [vp, C.POINTER(f64), i32, i32, C.POINTER(f64), C.POINTER(f64)]),
        "gadi_destroy": (None, [vp]),
        "gadi_status_str": (C.c_char_p, [i32]),
        "gadi_solve_stencil_noalloc": (i32, [i32, i32, f64, f64, f64, f64, i32, i32, vp, vp, f64, vp,
                                             C.POINTER(gadi_info)]),
        "gadi_last_error": (C.c_char_p, [vp]),
        "gadi_sweep": (i32, [C.POINTER(gadi_sweep_instance), i32, C.POINTER(gadi_sweep_candidate), i32,
                             f64, f64, i32, i32, i32, i32, i32, vp, C.POINTER(gadi_sweep_record)]),
        "gadi_model_fit": (i32, [i32, vp, vp, i32, vp, i32, vp, C.POINTER(vp)]),
        "gadi_model_predict": (i32, [vp, vp, i32, vp]),
        "gadi_model_loss": (i32, [vp, vp, i32, C.POINTER(i32)]),
        "gadi_mlp_gradient": (i32, [vp, vp, vp, i32, vp, vp]),
        "gadi_mlp_param_count": (i32, []),
        "gadi_model_destroy": (None, [vp]),
        "gadi_set_model": (i32, [vp, i32, vp]),
        "gadi_sylv_create": (i32, [C.c_int64, C.c_int64, vp, vp, vp, vp, vp, vp, vp, C.POINTER(vp)]),
        "gadi_sylv_set_params": (i32, [vp, f64, f64, i32]),
        "gadi_sylv_solve": (i32, [vp, vp, vp, f64, i32, C.POINTER(gadi_info)]),
        "gadi_sylv_last_error": (C.c_char_p, [vp]),
        "gadi_sylv_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_str(st: int) -> str:
    return load().gadi_status_str(int(st)).decode()


def last_error(h) -> str:
    return load().gadi_last_error(h).decode()


def _ptr(a):
    """Raw address of a torch tensor or numpy array (contiguous)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported buffer type {type(a)}")


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _check(h, st):
    if st not in (GADI_OK,):
        raise GadiError(st, last_error(h) if h else "")


def gadi_create(row_ptr, col_idx, val, split=GADI_SPLIT_HSS, m_val=None, stencil=None,
                stream=None):
    """Create a handle from CSR arrays (numpy on the host or torch on the
    device). stencil: None or (dim, N, beta, variable_k). Returns the handle
    (a c_void_p). Keeps no reference to the inputs: the library copies them."""
    lib = load()
    n = len(row_ptr) - 1
    dev = _is_device(val)
    A = gadi_csr(n, len(val), _ptr(row_ptr), _ptr(col_idx), _ptr(val), 1 if dev else 0)
    M = None
    if m_val is not None:
        M = gadi_csr(n, len(val), _ptr(row_ptr), _ptr(col_idx), _ptr(m_val), 1 if dev else 0)
    S = None
    if stencil is not None:
        S = gadi_stencil(int(stencil[0]), int(stencil[1]), float(stencil[2]), int(stencil[3]))
    h = C.c_void_p()
    st = lib.gadi_create(C.byref(A), int(split), C.byref(M) if M is not None else None,
                         C.byref(S) if S is not None else None,
                         C.c_void_p(stream) if stream else None, C.byref(h))
    if st != GADI_OK:
        raise GadiError(st, "gadi_create failed")
    return h


def gadi_destroy(h):
    load().gadi_destroy(h)


def gadi_set_params(h, alpha, omega, u_r=GADI_F16, u=GADI_F64, u_f=GADI_F64):
    st = load().gadi_set_params(h, float(alpha), float(omega), int(u_r), int(u), int(u_f))
    _check(h, st)


def gadi_set_inner(h, eps_inner, max_inner=200, max_outer=100000):
    _check(h, load().gadi_set_inner(h, float(eps_inner), int(max_inner), int(max_outer)))


def gadi_set_stop(h, kind):
    _check(h, load().gadi_set_stop(h, int(kind)))


def gadi_set_kernel(h, kind):
    _check(h, load().gadi_set_kernel(h, int(kind)))


def gadi_set_item_rows(h, rows):
    _check(h, load().gadi_set_item_rows(h, int(rows)))


def gadi_set_traversal(h, mode):
    _check(h, load().gadi_set_traversal(h, int(mode)))


def gadi_set_scaling(h, on):
    _check(h, load().gadi_set_scaling(h, int(on)))


def gadi_set_launch(h, grid_blocks=0, block_threads=0):
    _check(h, load().gadi_set_launch(h, int(grid_blocks), int(block_threads)))


def gadi_set_wait_limit(h, ms):
    _check(h, load().gadi_set_wait_limit(h, float(ms)))


def gadi_debug_force_timeout(h, on):
    _check(h, load().gadi_debug_force_timeout(h, int(bool(on))))


def gadi_solve(h, b, x, tol):
    """Solve in place into x (both torch CUDA tensors or both numpy arrays,
    float64). Returns (status, info dict); does not raise on NOT_CONVERGED,
    DIVERGED or TIMEOUT so callers can inspect the result."""
    info = gadi_info()
    st = load().gadi_solve(h, C.c_void_p(_ptr(b)), C.c_void_p(_ptr(x)), float(tol), C.byref(info))
    if st in (GADI_ERR_INVALID_ARG, GADI_ERR_CUDA, GADI_ERR_OUT_OF_MEMORY, GADI_ERR_UNSUPPORTED,
              GADI_ERR_RANGE):
        raise GadiError(st, last_error(h))
    return st, info.as_dict()


def gadi_apply(h, which, x, y):
    _check(h, load().gadi_apply(h, int(which), C.c_void_p(_ptr(x)), C.c_void_p(_ptr(y))))


def gadi_get_scales(h):
    sM, sN = C.c_int32(), C.c_int32()
    _check(h, load().gadi_get_scales(h, C.byref(sM), C.byref(sN)))
    return sM.value, sN.value


def gadi_predict_params(h, features, kind):
    f = np.ascontiguousarray(features if features is not None else [0.0, 0.0], dtype=np.float64)
    a, w = C.c_double(), C.c_double()
    st = load().gadi_predict_params(h, f.ctypes.data_as(C.POINTER(C.c_double)), len(f), int(kind),
                                    C.byref(a), C.byref(w))
    return st, a.value, w.value


def gadi_solve_stencil_noalloc(dim, N, beta, alpha, omega, b, x, tol, eps_inner=1e-2,
                               max_inner=200, max_outer=100000, stream=None):
    """Allocation-free stencil solve into x (torch CUDA tensors, float64).
    Returns (status, info dict)."""
    info = gadi_info()
    st = load().gadi_solve_stencil_noalloc(int(dim), int(N), float(beta), float(alpha), float(omega),
                                           float(eps_inner), int(max_inner), int(max_outer),
                                           C.c_void_p(_ptr(b)), C.c_void_p(_ptr(x)), float(tol),
                                           C.c_void_p(stream) if stream else None, C.byref(info))
    return st, info.as_dict()


def gadi_sweep(instances, candidates, tol=1e-13, eps_inner=0.1, max_inner=200, max_outer=5000,
               race=True, block_threads=0, team_blocks=0, stream=None):
    """instances: [(dim, N, beta)], candidates: [(alpha, omega)]. Returns a
    list of record dicts, one per (instance, candidate), instance-major.
    block_threads / team_blocks: 0 = the autotuned schedule."""
    ni, nc = len(instances), len(candidates)
    I = (gadi_sweep_instance * ni)(*[gadi_sweep_instance(int(d), int(N), float(b)) for d, N, b in instances])
    Cd = (gadi_sweep_candidate * nc)(*[gadi_sweep_candidate(float(a), float(w)) for a, w in candidates])
    R = (gadi_sweep_record * (ni * nc))()
    st = load().gadi_sweep(I, ni, Cd, nc, float(tol), float(eps_inner), int(max_inner), int(max_outer),
                           int(bool(race)), int(block_threads), int(team_blocks),
                           C.c_void_p(stream) if stream else None, R)
    if st != GADI_OK:
        raise GadiError(st, "gadi_sweep failed")
    return [r.as_dict() for r in R]


def _f64c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def gadi_model_fit(kind, X, Y, hyper=None, stream=None):
    """Fit a predictor (GADI_MODEL_MLP or GADI_MODEL_GPR) on X (m x 2
    features) and Y (m x 2 targets); returns the model handle."""
    X, Y = _f64c(X), _f64c(Y)
    h = None if hyper is None else _f64c(hyper)
    m = C.c_void_p()
    st = load().gadi_model_fit(int(kind), X.ctypes.data, Y.ctypes.data, len(X),
                               None if h is None else h.ctypes.data, 0 if h is None else len(h),
                               C.c_void_p(stream) if stream else None, C.byref(m))
    if st != GADI_OK:
        raise GadiError(st, "gadi_model_fit failed")
    return m


def gadi_model_predict(model, X):
    X = _f64c(X)
    Y = np.empty((len(X), 2))
    st = load().gadi_model_predict(model, X.ctypes.data, len(X), Y.ctypes.data)
    if st != GADI_OK:
        raise GadiError(st, "gadi_model_predict failed")
    return Y


def gadi_model_loss(model):
    cnt = C.c_int32()
    load().gadi_model_loss(model, None, 0, C.byref(cnt))
    out = np.empty(max(cnt.value, 1))
    load().gadi_model_loss(model, out.ctypes.data, cnt.value, C.byref(cnt))
    return out[:cnt.value]


def gadi_mlp_gradient(params, X, T, stream=None):
    params, X, T = _f64c(params), _f64c(X), _f64c(T)
    g = np.empty(load().gadi_mlp_param_count())
    st = load().gadi_mlp_gradient(params.ctypes.data, X.ctypes.data, T.ctypes.data, len(X),
                                  C.c_void_p(stream) if stream else None, g.ctypes.data)
    if st != GADI_OK:
        raise GadiError(st, "gadi_mlp_gradient failed")
    return g


def gadi_mlp_param_count():
    return int(load().gadi_mlp_param_count())


def gadi_model_destroy(model):
    load().gadi_model_destroy(model)


def gadi_set_model(h, kind, model):
    _check(h, load().gadi_set_model(h, int(kind), model))


# ---------------------------------------------------------------------------
# GADI-AB for the Sylvester equation A X + X B = C
# ---------------------------------------------------------------------------

def gadi_sylv_create(a, b, stream=None):
    """a, b = (lo, diag, up) host arrays of the tridiagonal A (m x m) and B (n x n)."""
    arrs = [np.ascontiguousarray(v, dtype=np.float64) for v in (*a, *b)]
    m, n = len(arrs[1]), len(arrs[4])
    if any(len(v) != m for v in arrs[:3]) or any(len(v) != n for v in arrs[3:]):
        raise GadiError(GADI_ERR_INVALID_ARG, "lo, diag, up of one matrix must have equal lengths")
    out = C.c_void_p()
    st = load().gadi_sylv_create(m, n, *[v.ctypes.data for v in arrs], C.c_void_p(stream or 0), C.byref(out))
    if st != GADI_OK:
        raise GadiError(st, "gadi_sylv_create failed")
    return out


def _sylv_check(s, st):
    if st != GADI_OK:
        raise GadiError(st, load().gadi_sylv_last_error(s).decode())


def gadi_sylv_set_params(s, alpha, omega, u_r=GADI_F16):
    _sylv_check(s, load().gadi_sylv_set_params(s, float(alpha), float(omega), int(u_r)))


def gadi_sylv_solve(s, Cm, X, tol=1e-13, max_outer=100000):
    """Cm, X: torch CUDA float64 tensors (m x n, row-major). Returns (status, info)."""
    info = gadi_info()
    st = load().gadi_sylv_solve(s, C.c_void_p(_ptr(Cm)), C.c_void_p(_ptr(X)), float(tol), int(max_outer),
                                C.byref(info))
    if st in (GADI_ERR_INVALID_ARG, GADI_ERR_CUDA, GADI_ERR_OUT_OF_MEMORY):
        raise GadiError(st, load().gadi_sylv_last_error(s).decode())
    return st, info.as_dict()


def gadi_sylv_destroy(s):
    load().gadi_sylv_destroy(s)


class Solver:
    """Convenience owner of a handle for a problems.Problem-like input."""

    def __init__(self, A, stencil=None, stream=None, device=False):
        if device:
            import torch
            rp = torch.from_numpy(np.asarray(A.row_ptr, np.int32)).cuda()
            ci = torch.from_numpy(np.asarray(A.col_idx, np.int32)).cuda()
            va = torch.from_numpy(np.asarray(A.val, np.float64)).cuda()
            self.h = gadi_create(rp, ci, va, stencil=stencil, stream=stream)
        else:
            self.h = gadi_create(np.ascontiguousarray(A.row_ptr, np.int32),
                                 np.ascontiguousarray(A.col_idx, np.int32),
                                 np.ascontiguousarray(A.val, np.float64), stencil=stencil,
                                 stream=stream)
        self.n = A.n

    def close(self):
        if self.h:
            gadi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
