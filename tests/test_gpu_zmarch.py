"""The z-marching traversal of the solve kernel against grid-stride items and
the oracle.

Solves of the 3D constant-coefficient stencil with FP16 inner vectors walk
each thread along z through a column of 8-row items (gadi_set_traversal 0,
the default); traversal 1 processes the same items grid-stride. Both form
every row with the same terms in the same order; the dot products sum in
another order, so the two solves agree to rounding and reach the same
tolerance in about the same number of steps. Each case checks the z-march
was used (segment length reported in the solve's info), the backward error
recomputed by the oracle, the distance to the oracle's FP64-inner GADI-IR
solution (Algorithm 1 with u_r = u = u_f = double), and the outer-step
count against the grid-stride solve. The launch shapes give segments that
split N evenly, raggedly, and not at all (one segment per column).
"""
import os

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
    oracle.set_threads(os.cpu_count() or 1)
    G.load()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def _solve(p, alpha, omega, traversal, launch=(0, 0)):
    h = G.gadi_create(_dev(p.A.row_ptr, torch.int32), _dev(p.A.col_idx, torch.int32), _dev(p.A.val),
                      stencil=(p.dim, p.N, p.beta, 0))
    try:
        G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL)
        G.gadi_set_params(h, alpha, omega, u_r=G.GADI_F16)
        G.gadi_set_inner(h, 0.1, 500, 100000)
        G.gadi_set_traversal(h, traversal)
        G.gadi_set_launch(h, *launch)
        b = _dev(p.b)
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st, info = G.gadi_solve(h, b, x, 1e-13)
        assert st == G.GADI_OK, G.last_error(h)
        return x.cpu().numpy(), info
    finally:
        G.gadi_destroy(h)


def _planes(N, blocks, threads):
    """The segment length the library picks: about one column segment per
    thread, at least 4 planes (else 0: grid-stride items)."""
    cols = (N // 8) * N
    nseg = max(1, blocks * threads // cols)
    z = -(-N // nseg)
    return z if z >= 4 else 0


@pytest.mark.parametrize("N,beta,alpha,omega,launch", [
    (192, 100.0, 0.8, 0.2, (0, 0)),      # the bench's system and launch
    (128, 50.0, 0.6, 0.3, (0, 0)),
    (48, 100.0, 0.5, 0.5, (8, 128)),     # 3 segments of 16 planes
    (40, 20.0, 0.7, 0.4, (5, 128)),      # segments of 14, 14, 12 planes
    (56, 100.0, 0.5, 0.3, (2, 128)),     # one segment per column
])
def test_zmarch_matches_grid_stride_and_oracle(N, beta, alpha, omega, launch):
    p = P.make_problem(3, N, beta, rhs="manufactured")
    want, oinfo, _ = oracle.gadi_ir(p.A, p.b, alpha, omega, tol=1e-13, eps_inner=0.1,
                                    prec=oracle.PREC_DOUBLE, max_outer=100000, max_inner=500)
    assert oinfo["status"] == oracle.OK
    xz, iz = _solve(p, alpha, omega, 0, launch)
    xg, ig = _solve(p, alpha, omega, 1, launch)
    assert ig["zmarch_planes"] == 0
    assert iz["zmarch_planes"] == _planes(N, iz["grid_blocks"], iz["block_threads"]) > 0
    for x in (xz, xg):
        assert oracle.backward_error(p.A, p.b, x) <= 1e-13
        assert np.linalg.norm(x - want) <= 1e-9 * np.linalg.norm(want)
    assert abs(iz["outer_iters"] - ig["outer_iters"]) <= max(3, 0.1 * ig["outer_iters"])


def test_small_launch_falls_back_to_grid_stride():
    # 24^3 on the full default launch: far more threads than column segments
    # of 4 planes, so the solve runs grid-stride items
    p = P.make_problem(3, 24, 100.0, rhs="manufactured")
    x, info = _solve(p, 0.5, 0.5, 0)
    assert info["zmarch_planes"] == 0
    assert oracle.backward_error(p.A, p.b, x) <= 1e-13


def test_variable_coefficients_do_not_zmarch():
    p = P.workload("convdiff3d_128_b50_grf")
    h = G.gadi_create(_dev(p.A.row_ptr, torch.int32), _dev(p.A.col_idx, torch.int32), _dev(p.A.val),
                      stencil=(p.dim, p.N, p.beta, 1))
    try:
        G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL)
        G.gadi_set_params(h, 1.0, 1.0, u_r=G.GADI_F16)
        G.gadi_set_inner(h, 0.1, 500, 100000)
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st, info = G.gadi_solve(h, _dev(p.b), x, 1e-13)
        assert st == G.GADI_OK, G.last_error(h)
        assert info["zmarch_planes"] == 0
    finally:
        G.gadi_destroy(h)


def test_traversal_rejects_unknown_mode():
    p = P.make_problem(3, 16, 10.0, rhs="ones")
    h = G.gadi_create(_dev(p.A.row_ptr, torch.int32), _dev(p.A.col_idx, torch.int32), _dev(p.A.val),
                      stencil=(p.dim, p.N, p.beta, 0))
    try:
        with pytest.raises(RuntimeError):
            G.gadi_set_traversal(h, 2)
    finally:
        G.gadi_destroy(h)
