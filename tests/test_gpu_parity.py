"""GPU path (libgadi.so through its C ABI) against the CPU oracle.

Kernel level: one operator application per kernel family and precision is
compared bit for bit with the oracle's application (same splitting, same
power-of-two scales, same FP16 rounding, same row order).
Solver level: GADI-IR / GADI results reach the requested backward error,
agree with the oracle's solution within the stated bound, and the outer
iteration counts agree (exactly up to reduction order in FP64; within 15 %
with FP16 inner solves, where the dot products are summed in another order).
"""
import numpy as np
import pytest

import oracle
from paper_2501_04229_gb300 import gadi as G
from paper_2501_04229_gb300 import problems as P

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


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def _handle(p, stencil=True, device=True, split=G.GADI_SPLIT_HSS, m_user=None):
    A = p.A
    st = None
    if stencil and split == G.GADI_SPLIT_HSS:
        st = (p.dim, p.N, p.beta, 1 if p.faces is not None else 0)
    if device:
        rp = _dev(A.row_ptr, torch.int32)
        ci = _dev(A.col_idx, torch.int32)
        va = _dev(A.val)
        mu = None if m_user is None else _dev(m_user)
    else:
        rp = np.ascontiguousarray(A.row_ptr, np.int32)
        ci = np.ascontiguousarray(A.col_idx, np.int32)
        va = np.ascontiguousarray(A.val, np.float64)
        mu = None if m_user is None else np.ascontiguousarray(m_user, np.float64)
    return G.gadi_create(rp, ci, va, split=split, m_val=mu, stencil=st)


def _half_vector(n, seed):
    x = P.random_vector(n, seed)
    return oracle.to_half_bits(x).view(np.float16).astype(np.float64)


PROBLEMS = {
    "2d_33_b10": lambda: P.make_problem(2, 33, 10.0, rhs="ones"),
    "3d_13_b100": lambda: P.make_problem(3, 13, 100.0),
    "3d_12_b50_grf": lambda: P.make_problem(3, 12, 50.0, grf_seed=3),
    "3d_1_b5": lambda: P.make_problem(3, 1, 5.0),
    "2d_2_b1": lambda: P.make_problem(2, 2, 1.0),
}


# ---------------------------------------------------------------------------
# kernel level: bit-exact operator applications
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("kernel", [G.GADI_KERNEL_SPARSE, G.GADI_KERNEL_STENCIL])
@pytest.mark.parametrize("u_r", [G.GADI_F16, G.GADI_F64])
@pytest.mark.parametrize("alpha", [0.37, 12.0])
def test_apply_bit_exact(name, kernel, u_r, alpha):
    p = PROBLEMS[name]()
    h = _handle(p)
    try:
        G.gadi_set_params(h, alpha, 1.0, u_r=u_r)
        G.gadi_set_kernel(h, kernel)
        prec = oracle.PREC_HALF if u_r == G.GADI_F16 else oracle.PREC_DOUBLE
        tdt = torch.float16 if u_r == G.GADI_F16 else torch.float64
        for which in (G.OP_A, G.OP_H, G.OP_S, G.OP_ST):
            x = _half_vector(p.n, 10 + which) if (which != G.OP_A and u_r == G.GADI_F16) \
                else P.random_vector(p.n, 20 + which)
            want, sM, sN = oracle.lp_apply(p.A, alpha, which, prec, x)
            dt = torch.float64 if which == G.OP_A else tdt
            xd = _dev(x, dt)
            yd = torch.empty_like(xd)
            G.gadi_apply(h, which, xd, yd)
            torch.cuda.synchronize()
            got = yd.double().cpu().numpy()
            if (kernel == G.GADI_KERNEL_STENCIL and p.faces is not None and u_r == G.GADI_F64
                    and which in (G.OP_S, G.OP_ST)):
                # the face-coefficient stencil applies N as the constant convection
                # c = beta h / 2, the split stores (a_ij - a_ji)/2, which differs by ulps
                assert np.allclose(got, want, rtol=1e-14, atol=1e-15 * np.abs(want).max())
            else:
                assert np.array_equal(got, want), (which, np.abs(got - want).max())
        assert G.gadi_get_scales(h) == (sM, sN)
    finally:
        G.gadi_destroy(h)


ROWS_PROBLEMS = {
    "3d_16_b40": lambda: P.make_problem(3, 16, 40.0),
    "3d_16_b30_grf": lambda: P.make_problem(3, 16, 30.0, grf_seed=5),
    "2d_40_b20": lambda: P.make_problem(2, 40, 20.0, rhs="ones"),
    "3d_12_b50_grf": lambda: P.make_problem(3, 12, 50.0, grf_seed=3),
}


@pytest.mark.parametrize("name", list(ROWS_PROBLEMS))
@pytest.mark.parametrize("rows", [1, 4, 8])
@pytest.mark.parametrize("u_r", [G.GADI_F16, G.GADI_F64])
def test_apply_item_rows_bit_exact(name, rows, u_r):
    """Stencil items of 1, 4 and 8 rows of a grid line give the oracle's
    application bit for bit (N = 12 is not a multiple of 8: rows 8 falls back
    to single rows there)."""
    p = ROWS_PROBLEMS[name]()
    h = _handle(p)
    try:
        G.gadi_set_params(h, 0.37, 1.0, u_r=u_r)
        G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL)
        G.gadi_set_item_rows(h, rows)
        prec = oracle.PREC_HALF if u_r == G.GADI_F16 else oracle.PREC_DOUBLE
        tdt = torch.float16 if u_r == G.GADI_F16 else torch.float64
        for which in (G.OP_A, G.OP_H, G.OP_S, G.OP_ST):
            x = _half_vector(p.n, 30 + which) if (which != G.OP_A and u_r == G.GADI_F16) \
                else P.random_vector(p.n, 40 + which)
            want, _, _ = oracle.lp_apply(p.A, 0.37, which, prec, x)
            xd = _dev(x, torch.float64 if which == G.OP_A else tdt)
            yd = torch.empty_like(xd)
            G.gadi_apply(h, which, xd, yd)
            torch.cuda.synchronize()
            got = yd.double().cpu().numpy()
            if p.faces is not None and u_r == G.GADI_F64 and which in (G.OP_S, G.OP_ST):
                assert np.allclose(got, want, rtol=1e-14, atol=1e-15 * np.abs(want).max())
            else:
                assert np.array_equal(got, want), (which, np.abs(got - want).max())
    finally:
        G.gadi_destroy(h)


@pytest.mark.parametrize("N", [24, 48, 96, 176])
def test_apply_staged_bit_exact(N):
    """The shared-memory staged FP16 stencil application (a block owns whole
    y-lines of a z segment; planes stream through a ring of shared-memory
    slots filled by cp.async, with halo lines above and below) gives the
    oracle's application bit for bit, and the same bits as the
    one-item-per-thread kernel that a set launch shape selects. N = 24, 48:
    one block of y-lines per segment, 6 and 12 segments; N = 96: 3 blocks
    of 32 y-lines per plane, 24 segments; N = 176: 8 blocks of 22 y-lines,
    segments of 5 planes with a last one of 1 plane."""
    p = P.make_problem(3, N, 60.0)
    h = _handle(p)
    try:
        G.gadi_set_params(h, 0.37, 1.0, u_r=G.GADI_F16)
        G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL)
        G.gadi_set_item_rows(h, 8)
        for which in (G.OP_H, G.OP_S, G.OP_ST):
            x = _half_vector(p.n, 70 + which)
            want, _, _ = oracle.lp_apply(p.A, 0.37, which, oracle.PREC_HALF, x)
            xd = _dev(x, torch.float16)
            y1 = torch.empty_like(xd)
            y2 = torch.empty_like(xd)
            G.gadi_set_launch(h, 0, 0)
            G.gadi_apply(h, which, xd, y1)
            G.gadi_set_launch(h, 0, 256)
            G.gadi_apply(h, which, xd, y2)
            torch.cuda.synchronize()
            assert np.array_equal(y1.double().cpu().numpy(), want), which
            assert torch.equal(y1, y2), which
    finally:
        G.gadi_destroy(h)


def test_apply_user_split_bit_exact():
    p = P.make_problem(3, 9, 30.0)
    m_hss, _ = oracle.hss_split(p.A)
    d = np.zeros_like(m_hss)
    rows = np.repeat(np.arange(p.n), np.diff(p.A.row_ptr))
    diag = rows == p.A.col_idx
    d[diag] = 0.5 + P.random_vector(p.n, 3, "uniform") ** 2
    m_user = m_hss + d
    h = _handle(p, stencil=False, split=G.GADI_SPLIT_USER, m_user=m_user)
    try:
        G.gadi_set_params(h, 0.8, 1.0, u_r=G.GADI_F16)
        for which in (G.OP_H, G.OP_S, G.OP_ST):
            x = _half_vector(p.n, 30 + which)
            want, sM, sN = oracle.lp_apply(p.A, 0.8, which, oracle.PREC_HALF, x, m_user=m_user)
            xd = _dev(x, torch.float16)
            yd = torch.empty_like(xd)
            G.gadi_apply(h, which, xd, yd)
            torch.cuda.synchronize()
            assert np.array_equal(yd.double().cpu().numpy(), want)
    finally:
        G.gadi_destroy(h)


# ---------------------------------------------------------------------------
# solver level
# ---------------------------------------------------------------------------

def _solve(h, p, tol, x0=None, device=True):
    if device:
        b = _dev(p.b)
        x = _dev(np.zeros(p.n) if x0 is None else x0)
    else:
        b = np.ascontiguousarray(p.b)
        x = np.zeros(p.n) if x0 is None else np.array(x0, dtype=np.float64)
    st, info = G.gadi_solve(h, b, x, tol)
    xh = x.cpu().numpy() if device else x
    return st, info, xh


def test_fp64_gadi_config_2d_matches_oracle():
    """2D 32x32, beta 10, b = A 1, alpha 0.5, omega 1, inner eps 1e-10, RES <= 1e-12:
    plain FP64 GADI (eq. (gadi)) on the oracle, FP64 GADI-IR on the GPU, which
    is the same iteration (x^{k+1/2} = x^k + H^-1 r^k)."""
    p = P.workload("convdiff2d_32_b10")
    want, oinfo, _ = oracle.gadi(p.A, p.b, 0.5, 1.0, tol=1e-12, eps_inner=1e-10,
                                 stop=oracle.STOP_RES)
    for kernel in (G.GADI_KERNEL_SPARSE, G.GADI_KERNEL_STENCIL):
        h = _handle(p)
        try:
            G.gadi_set_params(h, 0.5, 1.0, u_r=G.GADI_F64)
            G.gadi_set_inner(h, 1e-10, 10000, 100000)
            G.gadi_set_stop(h, G.GADI_STOP_RES)
            G.gadi_set_kernel(h, kernel)
            st, info, x = _solve(h, p, 1e-12)
            assert st == G.GADI_OK, G.last_error(h)
            assert info["res_rel"] <= 1e-12
            assert abs(info["outer_iters"] - oinfo["outer_iters"]) <= 1
            assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)
            eta_o = oracle.backward_error(p.A, p.b, want)
            assert oracle.backward_error(p.A, p.b, x) <= 1.1 * eta_o
        finally:
            G.gadi_destroy(h)


@pytest.mark.parametrize("name,alpha,omega", [("3d_13_b100", 3.0, 1.0), ("3d_12_b50_grf", 2.0, 0.5),
                                              ("2d_33_b10", 0.4, 1.2)])
@pytest.mark.parametrize("kernel", [G.GADI_KERNEL_SPARSE, G.GADI_KERNEL_STENCIL])
def test_fp16_gadi_ir_matches_oracle(name, alpha, omega, kernel):
    p = PROBLEMS[name]()
    want, oinfo, _ = oracle.gadi_ir(p.A, p.b, alpha, omega, tol=1e-13, eps_inner=1e-2,
                                    prec=oracle.PREC_HALF, max_outer=5000)
    assert oinfo["status"] == oracle.OK
    h = _handle(p)
    try:
        G.gadi_set_params(h, alpha, omega, u_r=G.GADI_F16)
        G.gadi_set_inner(h, 1e-2, 200, 5000)
        G.gadi_set_kernel(h, kernel)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK, G.last_error(h)
        eta = oracle.backward_error(p.A, p.b, x)
        assert eta <= 1e-13 and info["eta_inf"] <= 1e-13
        assert abs(eta - info["eta_inf"]) <= 1e-3 * eta + 1e-18
        cond = np.linalg.cond(p.A.to_dense(), np.inf) if p.n <= 3000 else 1e4
        bound = max(1e-9, 4 * cond * 1e-13)
        assert np.linalg.norm(x - want) <= bound * np.linalg.norm(want)
        assert abs(info["outer_iters"] - oinfo["outer_iters"]) <= max(2, 0.15 * oinfo["outer_iters"])
        assert (info["scale_exp_M"], info["scale_exp_N"]) == (oinfo["scale_exp_M"], oinfo["scale_exp_N"])
    finally:
        G.gadi_destroy(h)


def test_user_split_solve_matches_oracle():
    p = P.make_problem(3, 9, 30.0)
    m_hss, _ = oracle.hss_split(p.A)
    rows = np.repeat(np.arange(p.n), np.diff(p.A.row_ptr))
    d = np.where(rows == p.A.col_idx, 0.25, 0.0)
    m_user = m_hss + d
    want, oinfo, _ = oracle.gadi_ir(p.A, p.b, 1.5, 1.0, tol=1e-13, prec=oracle.PREC_HALF,
                                    m_user=m_user, max_outer=5000)
    assert oinfo["status"] == oracle.OK
    h = _handle(p, stencil=False, split=G.GADI_SPLIT_USER, m_user=m_user)
    try:
        G.gadi_set_params(h, 1.5, 1.0, u_r=G.GADI_F16)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK
        assert oracle.backward_error(p.A, p.b, x) <= 1e-13
        assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)
        assert abs(info["outer_iters"] - oinfo["outer_iters"]) <= max(2, 0.15 * oinfo["outer_iters"])
    finally:
        G.gadi_destroy(h)


@pytest.mark.parametrize("rows", [1, 4, 8])
@pytest.mark.parametrize("u_r", [G.GADI_F16, G.GADI_F64])
def test_item_rows_solve_matches_oracle(rows, u_r):
    p = ROWS_PROBLEMS["3d_16_b40"]()
    prec = oracle.PREC_HALF if u_r == G.GADI_F16 else oracle.PREC_DOUBLE
    eps = 1e-2 if u_r == G.GADI_F16 else 1e-10
    want, oinfo, _ = oracle.gadi_ir(p.A, p.b, 2.5, 0.5, tol=1e-13, eps_inner=eps, prec=prec, max_outer=5000)
    assert oinfo["status"] == oracle.OK
    h = _handle(p)
    try:
        G.gadi_set_params(h, 2.5, 0.5, u_r=u_r)
        G.gadi_set_inner(h, eps, 200, 5000)
        G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL)
        G.gadi_set_item_rows(h, rows)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK, G.last_error(h)
        assert oracle.backward_error(p.A, p.b, x) <= 1e-13
        assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)
        slack = 0.15 if u_r == G.GADI_F16 else 0.0
        assert abs(info["outer_iters"] - oinfo["outer_iters"]) <= max(1, slack * oinfo["outer_iters"])
    finally:
        G.gadi_destroy(h)


@pytest.mark.parametrize("blocks,threads", [(1, 1024), (3, 128), (16, 256), (0, 0)])
def test_launch_shapes_agree(blocks, threads):
    """Single-block and multi-block (grid-barrier) launches of the persistent
    kernel give the same solution up to reduction order."""
    p = P.make_problem(3, 27, 80.0)          # n = 19683: ragged against every block size
    h = _handle(p)
    try:
        G.gadi_set_params(h, 3.0, 1.0, u_r=G.GADI_F16)
        G.gadi_set_launch(h, blocks, threads)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK, G.last_error(h)
        if blocks:
            assert info["grid_blocks"] == blocks
        assert oracle.backward_error(p.A, p.b, x) <= 1e-13
        assert np.abs(x - p.x_exact).max() <= 1e-9
    finally:
        G.gadi_destroy(h)


def test_host_and_device_buffers_agree():
    p = PROBLEMS["3d_13_b100"]()
    h = _handle(p, device=False)
    try:
        G.gadi_set_params(h, 3.0, 1.0)
        st1, i1, x1 = _solve(h, p, 1e-13, device=False)
        st2, i2, x2 = _solve(h, p, 1e-13, device=True)
        assert st1 == st2 == G.GADI_OK
        assert np.array_equal(x1, x2)
        assert i1["outer_iters"] == i2["outer_iters"]
    finally:
        G.gadi_destroy(h)


def test_edge_cases():
    # already converged start: zero outer steps
    p = PROBLEMS["3d_13_b100"]()
    h = _handle(p)
    try:
        G.gadi_set_params(h, 3.0, 1.0)
        xs = np.linalg.solve(p.A.to_dense(), p.b)
        st, info, x = _solve(h, p, 1e-12, x0=xs)
        assert st == G.GADI_OK and info["outer_iters"] == 0
        assert np.array_equal(x, xs)
        # zero right-hand side: x = 0 is exact
        b0 = P.Problem(p.name, p.dim, p.N, p.beta, p.A, np.zeros(p.n), np.zeros(p.n), None)
        st, info, x = _solve(h, b0, 1e-13)
        assert st == G.GADI_OK and info["outer_iters"] == 0 and not x.any()
        # max_outer reached
        G.gadi_set_inner(h, 1e-2, 200, 2)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_ERR_NOT_CONVERGED and info["outer_iters"] == 2
        assert np.isfinite(x).all()
    finally:
        G.gadi_destroy(h)
    # 1 x 1 system
    p1 = PROBLEMS["3d_1_b5"]()
    for kernel in (G.GADI_KERNEL_SPARSE, G.GADI_KERNEL_STENCIL):
        h = _handle(p1)
        try:
            G.gadi_set_params(h, 1.0, 1.0)
            G.gadi_set_kernel(h, kernel)
            st, info, x = _solve(h, p1, 1e-14)
            assert st == G.GADI_OK
            assert abs(x[0] - p1.b[0] / p1.A.val[0]) <= 1e-14 * abs(x[0])
        finally:
            G.gadi_destroy(h)


def test_invalid_arguments_rejected():
    p = PROBLEMS["2d_2_b1"]()
    h = _handle(p)
    try:
        for a, w in ((0.0, 1.0), (-1.0, 1.0), (1.0, 2.0), (1.0, -0.5), (float("nan"), 1.0)):
            with pytest.raises(G.GadiError) as e:
                G.gadi_set_params(h, a, w)
            assert e.value.status == G.GADI_ERR_INVALID_ARG
        for kw in (dict(u=G.GADI_F32), dict(u_f=G.GADI_F16)):
            with pytest.raises(G.GadiError) as e:
                G.gadi_set_params(h, 1.0, 1.0, **kw)
            assert e.value.status == G.GADI_ERR_UNSUPPORTED
        with pytest.raises(G.GadiError) as e:
            G.gadi_set_params(h, 1.0, 1.0, u_r=7)
        assert e.value.status == G.GADI_ERR_INVALID_ARG
        b = _dev(p.b)
        x = torch.full((p.n,), 7.0, dtype=torch.float64, device="cuda")
        with pytest.raises(G.GadiError):
            G.gadi_solve(h, b, x, 0.0)
        bn = b.clone()
        bn[1] = float("nan")
        with pytest.raises(G.GadiError) as e:
            G.gadi_solve(h, bn, x, 1e-10)
        assert e.value.status == G.GADI_ERR_INVALID_ARG
        assert (x == 7.0).all()
        with pytest.raises(G.GadiError):
            G.gadi_solve(h, b, x.cpu().numpy(), 1e-10)
        for rows in (-1, 2, 3, 16):
            with pytest.raises(G.GadiError) as e:
                G.gadi_set_item_rows(h, rows)
            assert e.value.status == G.GADI_ERR_INVALID_ARG
    finally:
        G.gadi_destroy(h)
    # structurally unsymmetric pattern, unsorted columns, stencil mismatch
    rp = np.array([0, 2, 3], np.int32)
    with pytest.raises(G.GadiError):
        G.gadi_create(rp, np.array([0, 1, 1], np.int32), np.array([2.0, 1.0, 3.0]))
    with pytest.raises(G.GadiError):
        G.gadi_create(np.array([0, 2, 4], np.int32), np.array([1, 0, 0, 1], np.int32),
                      np.array([1.0, 2.0, 1.0, 3.0]))
    q = P.make_problem(3, 5, 10.0)
    with pytest.raises(G.GadiError):
        G.gadi_create(q.A.row_ptr, q.A.col_idx, q.A.val, stencil=(3, 5, 11.0, 0))


def test_bounded_wait_expires_with_timeout_status():
    """A grid-barrier wait whose arrival target nothing reaches expires after
    the wait limit: the solve returns GADI_ERR_TIMEOUT and the handle (and the
    CUDA context) stay usable."""
    p = PROBLEMS["3d_13_b100"]()
    h = _handle(p)
    try:
        G.gadi_set_params(h, 3.0, 1.0)
        G.gadi_set_launch(h, 2, 256)
        G.gadi_set_wait_limit(h, 20.0)
        G.gadi_debug_force_timeout(h, 1)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_ERR_TIMEOUT
        G.gadi_debug_force_timeout(h, 0)
        G.gadi_set_wait_limit(h, 2000.0)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK
        assert oracle.backward_error(p.A, p.b, x) <= 1e-13
    finally:
        G.gadi_destroy(h)


def test_predictor_without_model():
    p = PROBLEMS["2d_2_b1"]()
    h = _handle(p)
    try:
        st, _, _ = G.gadi_predict_params(h, [np.log(4.0), 0.0], 0)
        assert st == G.GADI_ERR_NO_MODEL
    finally:
        G.gadi_destroy(h)


# ---------------------------------------------------------------------------
# full-size workload and degenerate cases
# ---------------------------------------------------------------------------

def test_full_size_64cubed_workload_against_oracle():
    """The bench workload (64^3, beta = 100, manufactured solution) at full
    size, in the bench's launch configuration: eta recomputed by the oracle,
    the solution against the oracle's FP64-inner GADI-IR solution and against
    the manufactured one (forward error <= kappa * eta, kappa(A) < 2e3 here)."""
    p = P.workload("convdiff3d_64_b100")
    h = _handle(p)
    try:
        G.gadi_set_params(h, 3.0, 0.0)
        G.gadi_set_inner(h, 0.1, 500, 100000)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK
    finally:
        G.gadi_destroy(h)
    assert oracle.backward_error(p.A, p.b, x) <= 1e-13
    want, oinfo, _ = oracle.gadi_ir(p.A, p.b, 3.0, 0.0, tol=1e-13, eps_inner=0.1,
                                    prec=oracle.PREC_DOUBLE, max_inner=500, max_outer=5000)
    assert oinfo["status"] == oracle.OK
    assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)
    # A is positive real with symmetric part M: ||x - u_h||_2 <= ||r||_2 / lambda_min(M),
    # lambda_min(M) = 3 (2 - 2 cos(pi h)) for the k = 1 operator (plus the rounding of b)
    lam = 3 * (2 - 2 * np.cos(np.pi / 65))
    rn = np.linalg.norm(oracle.residual(p.A, p.b, x))
    assert np.linalg.norm(x - p.x_exact) <= rn / lam + 1e-11


def test_e4m3_inner_64cubed_reaches_fp64_floor():
    """Cor. 1 at the bench's size: FP8 E4M3 inner storage (4 significant
    bits, scaled like FP16) still drives eta to 1e-13 and the solution to the
    FP64-inner one; the forward error obeys the same bound as FP16."""
    p = P.workload("convdiff3d_64_b100")
    h = _handle(p)
    try:
        G.gadi_set_params(h, 3.0, 0.0, u_r=G.GADI_E4M3)
        G.gadi_set_inner(h, 0.1, 500, 100000)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK, G.last_error(h)
    finally:
        G.gadi_destroy(h)
    assert oracle.backward_error(p.A, p.b, x) <= 1e-13
    lam = 3 * (2 - 2 * np.cos(np.pi / 65))
    rn = np.linalg.norm(oracle.residual(p.A, p.b, x))
    assert np.linalg.norm(x - p.x_exact) <= rn / lam + 1e-11


def test_hbm_workload_192cubed_properties():
    """The bench's HBM-bound system (192^3, n = 7.1e6) at full size, in the
    launch configuration the bench times (automatic: 152 x 512): eta
    recomputed by the oracle, and the forward error against the manufactured
    solution within ||r||_2 / lambda_min(M) (A positive real)."""
    p = P.workload("convdiff3d_192_b100")
    h = _handle(p)
    try:
        G.gadi_set_params(h, 2.0, 0.0)
        G.gadi_set_inner(h, 0.1, 500, 100000)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK and info["grid_blocks"] * info["block_threads"] >= 152 * 256
        # the bench's operator application at this size (staged kernel, 12
        # blocks of 16 y-lines, 8-plane segments) against the
        # one-item-per-thread kernel
        xh = torch.randn(p.n, device="cuda").half()
        for which in (G.OP_H, G.OP_S, G.OP_ST):
            y1 = torch.empty_like(xh)
            y2 = torch.empty_like(xh)
            G.gadi_set_launch(h, 0, 0)
            G.gadi_apply(h, which, xh, y1)
            G.gadi_set_launch(h, 0, 256)
            G.gadi_apply(h, which, xh, y2)
            torch.cuda.synchronize()
            assert torch.equal(y1, y2), which
        G.gadi_set_launch(h, 0, 0)
    finally:
        G.gadi_destroy(h)
    assert oracle.backward_error(p.A, p.b, x) <= 1e-13
    lam = 3 * (2 - 2 * np.cos(np.pi / 193))
    rn = np.linalg.norm(oracle.residual(p.A, p.b, x))
    assert np.linalg.norm(x - p.x_exact) <= rn / lam + 1e-10


def test_grf_128cubed_stencil_and_sparse_kernels():
    """The variable-coefficient 128^3 system at full size with the
    face-coefficient stencil kernel and the general sparse kernel: both reach
    eta <= 1e-13 (recomputed by the oracle) and the manufactured solution."""
    p = P.workload("convdiff3d_128_b50_grf")
    xs = []
    for kernel in (G.GADI_KERNEL_STENCIL, G.GADI_KERNEL_SPARSE):
        h = _handle(p)
        try:
            G.gadi_set_params(h, 1.0, 1.0)
            G.gadi_set_inner(h, 0.1, 500, 100000)
            G.gadi_set_kernel(h, kernel)
            st, info, x = _solve(h, p, 1e-13)
            assert st == G.GADI_OK
        finally:
            G.gadi_destroy(h)
        assert oracle.backward_error(p.A, p.b, x) <= 1e-13
        assert np.abs(x - p.x_exact).max() <= 1e-8
        xs.append(x)
    assert np.abs(xs[0] - xs[1]).max() <= 1e-8


def test_pure_diffusion_beta_zero():
    """beta = 0: N = 0, S = alpha I, so every CGNR solve takes one iteration."""
    p = P.make_problem(3, 16, 0.0)
    h = _handle(p)
    try:
        G.gadi_set_params(h, 0.5, 1.0)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK
        assert info["inner_iters_S"] == info["outer_iters"]
        assert oracle.backward_error(p.A, p.b, x) <= 1e-13
    finally:
        G.gadi_destroy(h)


def test_omega_near_two_still_converges():
    """Thm 1 allows any omega in [0, 2); close to 2 the update (2 - omega) a
    is small and convergence slow, but it converges."""
    p = P.make_problem(2, 16, 5.0)
    h = _handle(p)
    try:
        G.gadi_set_params(h, 1.0, 1.9)
        G.gadi_set_inner(h, 0.1, 200, 100000)
        st, info, x = _solve(h, p, 1e-12)
        assert st == G.GADI_OK
        assert oracle.backward_error(p.A, p.b, x) <= 1e-12
    finally:
        G.gadi_destroy(h)


def test_empty_system_rejected():
    with pytest.raises(G.GadiError) as e:
        G.gadi_create(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    assert e.value.status == G.GADI_ERR_INVALID_ARG


# ---------------------------------------------------------------------------
# unscaled ("naive") FP16 inner precision: the ablation of §4.1's FP16 runs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["2d_33_b10", "3d_13_b100", "3d_12_b50_grf"])
@pytest.mark.parametrize("kernel", [G.GADI_KERNEL_SPARSE, G.GADI_KERNEL_STENCIL])
@pytest.mark.parametrize("alpha", [0.01, 3.0])
def test_naive_apply_bit_exact(name, kernel, alpha):
    p = PROBLEMS[name]()
    h = _handle(p)
    try:
        G.gadi_set_params(h, alpha, 1.0, u_r=G.GADI_F16)
        G.gadi_set_scaling(h, 0)
        G.gadi_set_kernel(h, kernel)
        for which in (G.OP_H, G.OP_S, G.OP_ST):
            x = _half_vector(p.n, 50 + which)
            want, sM, sN = oracle.lp_apply(p.A, alpha, which, oracle.PREC_HALF_NAIVE, x)
            xd = _dev(x, torch.float16)
            yd = torch.empty_like(xd)
            G.gadi_apply(h, which, xd, yd)
            torch.cuda.synchronize()
            got = yd.double().cpu().numpy()
            assert np.array_equal(got, want), (which, np.abs(got - want).max())
        assert G.gadi_get_scales(h) == (0, 0) == (sM, sN)
    finally:
        G.gadi_destroy(h)


def test_naive_apply_item_rows_bit_exact():
    p = ROWS_PROBLEMS["3d_16_b40"]()
    h = _handle(p)
    try:
        G.gadi_set_params(h, 0.37, 1.0, u_r=G.GADI_F16)
        G.gadi_set_scaling(h, 0)
        G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL)
        for rows in (1, 4, 8):
            G.gadi_set_item_rows(h, rows)
            for which in (G.OP_H, G.OP_S, G.OP_ST):
                x = _half_vector(p.n, 60 + which)
                want, _, _ = oracle.lp_apply(p.A, 0.37, which, oracle.PREC_HALF_NAIVE, x)
                xd = _dev(x, torch.float16)
                yd = torch.empty_like(xd)
                G.gadi_apply(h, which, xd, yd)
                torch.cuda.synchronize()
                assert np.array_equal(yd.double().cpu().numpy(), want), (rows, which)
    finally:
        G.gadi_destroy(h)


@pytest.mark.parametrize("kernel", [G.GADI_KERNEL_SPARSE, G.GADI_KERNEL_STENCIL])
def test_naive_fp16_stalls_like_the_oracle(kernel):
    """Table '3d' (§4.1): without scaling the FP16-inner iteration stalls (or
    breaks down) far above double accuracy, on the GPU as in the oracle;
    scaled it reaches RES 1e-13."""
    p = P.make_problem(3, 8, 1.0, rhs="ones")
    _, onaive, _ = oracle.gadi_ir(p.A, p.b, 0.5, 1.0, tol=1e-13, stop=oracle.STOP_RES, eps_inner=1e-2,
                                  max_outer=400, max_inner=300, prec=oracle.PREC_HALF_NAIVE)
    assert onaive["status"] != oracle.OK and onaive["res_rel"] > 1e-9
    h = _handle(p)
    try:
        G.gadi_set_params(h, 0.5, 1.0, u_r=G.GADI_F16)
        G.gadi_set_inner(h, 1e-2, 300, 400)
        G.gadi_set_stop(h, G.GADI_STOP_RES)
        G.gadi_set_kernel(h, kernel)
        G.gadi_set_scaling(h, 0)
        st, info, _ = _solve(h, p, 1e-13)
        assert st != G.GADI_OK and info["res_rel"] > 1e-9
        G.gadi_set_scaling(h, 1)
        st, info, _ = _solve(h, p, 1e-13)
        assert st == G.GADI_OK and info["res_rel"] <= 1e-13
    finally:
        G.gadi_destroy(h)


def test_naive_fp16_loose_tolerance_matches_oracle():
    p = PROBLEMS["3d_13_b100"]()
    want, oinfo, _ = oracle.gadi_ir(p.A, p.b, 3.0, 1.0, tol=1e-6, eps_inner=1e-2, prec=oracle.PREC_HALF_NAIVE,
                                    max_outer=3000)
    assert oinfo["status"] == oracle.OK
    h = _handle(p)
    try:
        G.gadi_set_params(h, 3.0, 1.0, u_r=G.GADI_F16)
        G.gadi_set_inner(h, 1e-2, 200, 3000)
        G.gadi_set_scaling(h, 0)
        st, info, x = _solve(h, p, 1e-6)
        assert st == G.GADI_OK, G.last_error(h)
        assert oracle.backward_error(p.A, p.b, x) <= 1e-6
        assert abs(info["outer_iters"] - oinfo["outer_iters"]) <= max(2, 0.15 * oinfo["outer_iters"])
        with pytest.raises(G.GadiError):
            G.gadi_set_scaling(h, 2)
    finally:
        G.gadi_destroy(h)


# ---------------------------------------------------------------------------
# other inner precisions: FP32, bfloat16 and FP8 E4M3 storage (precision
# variants)
# ---------------------------------------------------------------------------

def _bf16_vector(n, seed):
    bits = oracle.to_bf16_bits(P.random_vector(n, seed))
    return bits, (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _e4m3_table():
    """Value of each 8-bit E4M3 code from the format's layout (sign, 4
    exponent bits with bias 7, 3 fraction bits, subnormals f 2^-9, the two
    all-ones codes NaN)."""
    t = np.empty(256)
    for c in range(256):
        s, e, f = (-1.0 if c & 0x80 else 1.0), (c >> 3) & 0xF, c & 7
        if e == 0xF and f == 7:
            t[c] = np.nan
        elif e == 0:
            t[c] = s * f * 2.0 ** -9
        else:
            t[c] = s * (1 + f / 8) * 2.0 ** (e - 7)
    return t


E4M3 = _e4m3_table()


def _e4m3_vector(n, seed):
    codes = oracle.to_e4m3_bits(P.random_vector(n, seed))
    return codes, E4M3[codes]


def _lp_vector(n, seed, u_r):
    if u_r == G.GADI_BF16:
        return _bf16_vector(n, seed)
    if u_r == G.GADI_E4M3:
        return _e4m3_vector(n, seed)
    return None, P.random_vector(n, seed).astype(np.float32).astype(np.float64)


def _lp_tensor(x, u_r, bits=None):
    if u_r == G.GADI_BF16:
        return torch.from_numpy(bits.view(np.int16).copy()).cuda().view(torch.bfloat16)
    if u_r == G.GADI_E4M3:
        return torch.from_numpy(bits.copy()).cuda()
    return _dev(x, torch.float32)


def _lp_values(yd, u_r):
    if u_r == G.GADI_E4M3:
        return E4M3[yd.cpu().numpy()]
    return yd.double().cpu().numpy()


LP_CASES = [(G.GADI_F32, oracle.PREC_SINGLE), (G.GADI_BF16, oracle.PREC_BF16),
            (G.GADI_E4M3, oracle.PREC_E4M3)]


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("kernel", [G.GADI_KERNEL_SPARSE, G.GADI_KERNEL_STENCIL])
@pytest.mark.parametrize("u_r,prec", LP_CASES)
def test_apply_other_precisions_bit_exact(name, kernel, u_r, prec):
    p = PROBLEMS[name]()
    h = _handle(p)
    try:
        G.gadi_set_params(h, 0.37, 1.0, u_r=u_r)
        G.gadi_set_kernel(h, kernel)
        if u_r == G.GADI_E4M3 and p.faces is not None:
            # GRF face coefficients span more binades than FP8 holds after the
            # scaling: entries below 2^-10 would vanish, and the solver refuses
            bits, x = _lp_vector(p.n, 70, u_r)
            xd = _lp_tensor(x, u_r, bits)
            with pytest.raises(G.GadiError) as e:
                G.gadi_apply(h, G.OP_H, xd, torch.empty_like(xd))
            assert e.value.status == G.GADI_ERR_RANGE
            return
        for which in (G.OP_H, G.OP_S, G.OP_ST):
            bits, x = _lp_vector(p.n, 70 + which, u_r)
            want, sM, sN = oracle.lp_apply(p.A, 0.37, which, prec, x)
            xd = _lp_tensor(x, u_r, bits)
            yd = torch.empty_like(xd)
            G.gadi_apply(h, which, xd, yd)
            torch.cuda.synchronize()
            got = _lp_values(yd, u_r)
            if kernel == G.GADI_KERNEL_STENCIL and p.faces is not None and u_r == G.GADI_F32 \
                    and which in (G.OP_S, G.OP_ST):
                # the face stencil applies N as the constant c = beta h / 2 (see the FP64 case)
                assert np.allclose(got, want, rtol=1e-6, atol=1e-7 * np.abs(want).max())
            else:
                assert np.array_equal(got, want), (which, np.abs(got - want).max())
        assert G.gadi_get_scales(h) == (sM, sN)
    finally:
        G.gadi_destroy(h)


@pytest.mark.parametrize("rows", [1, 4, 8])
@pytest.mark.parametrize("u_r,prec", LP_CASES)
def test_apply_other_precisions_item_rows(rows, u_r, prec):
    p = ROWS_PROBLEMS["3d_16_b40"]()
    h = _handle(p)
    try:
        G.gadi_set_params(h, 2.0, 1.0, u_r=u_r)
        G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL)
        G.gadi_set_item_rows(h, rows)
        for which in (G.OP_H, G.OP_S, G.OP_ST):
            bits, x = _lp_vector(p.n, 80 + which, u_r)
            want, _, _ = oracle.lp_apply(p.A, 2.0, which, prec, x)
            xd = _lp_tensor(x, u_r, bits)
            yd = torch.empty_like(xd)
            G.gadi_apply(h, which, xd, yd)
            torch.cuda.synchronize()
            assert np.array_equal(_lp_values(yd, u_r), want), (rows, which)
    finally:
        G.gadi_destroy(h)


@pytest.mark.parametrize("u_r,prec", LP_CASES)
@pytest.mark.parametrize("kernel", [G.GADI_KERNEL_SPARSE, G.GADI_KERNEL_STENCIL])
def test_other_precision_solves_match_oracle(u_r, prec, kernel):
    p = PROBLEMS["3d_13_b100"]()
    eps = 0.1 if u_r == G.GADI_E4M3 else 1e-2      # FP8 inner solves stop at 0.1 by default
    want, oinfo, _ = oracle.gadi_ir(p.A, p.b, 3.0, 1.0, tol=1e-13, eps_inner=eps, prec=prec, max_outer=5000)
    assert oinfo["status"] == oracle.OK
    h = _handle(p)
    try:
        G.gadi_set_params(h, 3.0, 1.0, u_r=u_r)
        G.gadi_set_inner(h, eps, 200, 5000)
        G.gadi_set_kernel(h, kernel)
        st, info, x = _solve(h, p, 1e-13)
        assert st == G.GADI_OK, G.last_error(h)
        assert oracle.backward_error(p.A, p.b, x) <= 1e-13
        assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)
        assert abs(info["outer_iters"] - oinfo["outer_iters"]) <= max(2, 0.15 * oinfo["outer_iters"])
        assert (info["scale_exp_M"], info["scale_exp_N"]) == (oinfo["scale_exp_M"], oinfo["scale_exp_N"])
    finally:
        G.gadi_destroy(h)
