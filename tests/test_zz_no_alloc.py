"""The allocation-free stencil solve against the handle-based solve.

gadi_solve_stencil_noalloc exists for callers that cannot allocate device
memory: code under a fixed memory budget or inside a framework that owns all
device memory through its own pool, and latency-critical loops where the
implicit synchronisation of cudaMalloc is not acceptable. It must return the
same solution as gadi_create + gadi_solve on the same system, call after
call, although every call reuses (and leaves behind) the same scratch array.
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


@pytest.mark.parametrize("dim,N,beta,alpha,omega", [(3, 24, 50.0, 3.0, 0.0), (2, 40, 10.0, 0.5, 1.0),
                                                    (3, 13, 100.0, 3.0, 1.0), (3, 64, 100.0, 3.0, 0.0)])
def test_noalloc_matches_handle_solve_on_consecutive_calls(dim, N, beta, alpha, omega):
    p = P.make_problem(dim, N, beta)
    eps, tol = 0.1, 1e-13
    h = G.gadi_create(_dev(p.A.row_ptr, torch.int32), _dev(p.A.col_idx, torch.int32), _dev(p.A.val),
                      stencil=(dim, N, beta, 0))
    try:
        G.gadi_set_params(h, alpha, omega, u_r=G.GADI_F16)
        G.gadi_set_inner(h, eps, 200, 100000)
        b = _dev(p.b)
        x_ref = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st, info_ref = G.gadi_solve(h, b, x_ref, tol)
        assert st == G.GADI_OK
        x_ref = x_ref.cpu().numpy()
    finally:
        G.gadi_destroy(h)
    for _ in range(2):
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st, info = G.gadi_solve_stencil_noalloc(dim, N, beta, alpha, omega, b, x, tol, eps_inner=eps,
                                                max_inner=200)
        assert st == G.GADI_OK, G.status_str(st)
        xh = x.cpu().numpy()
        assert oracle.backward_error(p.A, p.b, xh) <= tol
        assert np.linalg.norm(xh - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
        assert abs(info["outer_iters"] - info_ref["outer_iters"]) <= max(2, 0.05 * info_ref["outer_iters"])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    N = 65                                   # 65^3 = 274625 > GADI_NOALLOC_MAX_N = 262144
    b = torch.ones(N ** 3, dtype=torch.float64, device="cuda")
    x = torch.full((N ** 3,), 3.0, dtype=torch.float64, device="cuda")
    st, _ = G.gadi_solve_stencil_noalloc(3, N, 10.0, 1.0, 1.0, b, x, 1e-10)
    assert st == G.GADI_ERR_INVALID_ARG
    assert bool((x == 3.0).all())
    # host buffers are refused too: the entry point has no device buffer to copy them into
    p = P.make_problem(3, 8, 10.0)
    st, _ = G.gadi_solve_stencil_noalloc(3, 8, 10.0, 1.0, 1.0, np.ascontiguousarray(p.b), np.zeros(p.n),
                                         1e-10)
    assert st == G.GADI_ERR_INVALID_ARG


def test_noalloc_refuses_memory_of_another_gpu():
    # b and x are read and written in place on the current device, so memory
    # of another GPU must be refused before anything is launched
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second visible GPU")
    torch.cuda.set_device(0)
    p = P.make_problem(3, 8, 10.0)
    b = torch.as_tensor(p.b).to(device="cuda:1")
    x = torch.full((p.n,), 3.0, dtype=torch.float64, device="cuda:1")
    st, _ = G.gadi_solve_stencil_noalloc(3, 8, 10.0, 1.0, 1.0, b, x, 1e-10)
    assert st == G.GADI_ERR_INVALID_ARG
    assert bool((x == 3.0).all())
