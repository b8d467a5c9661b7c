"""Batched GADI-IR sweep (teams of one or more blocks per (instance, alpha,
omega) item, one persistent launch per size bin) against single solves
through gadi_solve and against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2501_04229_gb300 import gadi as G
from paper_2501_04229_gb300 import problems as P
from paper_2501_04229_gb300 import sweep as SW

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


INSTANCES = [(2, 16, 5.0), (2, 24, 40.0), (2, 21, 0.7), (3, 8, 20.0), (3, 11, 3.0)]
CANDS = [(0.3, 0.0), (1.0, 1.0), (3.0, 0.5)]


def _single(dim, N, beta, alpha, omega, eps=0.1):
    p = P.make_problem(dim, N, beta, rhs="ones")
    t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt, device="cuda")
    h = G.gadi_create(t(p.A.row_ptr, torch.int32), t(p.A.col_idx, torch.int32), t(p.A.val),
                      stencil=(dim, N, beta, 0))
    try:
        G.gadi_set_params(h, alpha, omega, u_r=G.GADI_F16)
        G.gadi_set_inner(h, eps, 200, 5000)
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        st, info = G.gadi_solve(h, t(p.b), x, 1e-13)
        return p, st, info, x.cpu().numpy()
    finally:
        G.gadi_destroy(h)


@pytest.mark.parametrize("block_threads", [0, 128, 512])
def test_sweep_records_match_single_solves(block_threads):
    recs = G.gadi_sweep(INSTANCES, CANDS, tol=1e-13, eps_inner=0.1, max_outer=5000, race=False,
                        block_threads=block_threads)
    assert len(recs) == len(INSTANCES) * len(CANDS)
    for i, (d, N, b) in enumerate(INSTANCES):
        for j, (a, w) in enumerate(CANDS):
            r = recs[i * len(CANDS) + j]
            assert (r["instance"], r["candidate"]) == (i, j)
            p, st, info, _ = _single(d, N, b, a, w)
            assert r["status"] == st == G.GADI_OK
            assert r["eta_inf"] <= 1e-13
            # FP16 inner solves: counts move with the summation order of the dot
            # products (and the sweep forms b = A 1 on the device), hence 15 %
            assert abs(r["outer_iters"] - info["outer_iters"]) <= max(2, 0.15 * info["outer_iters"])
            assert abs(r["spmv_count"] - info["spmv_count"]) <= max(6, 0.15 * info["spmv_count"])


def test_racing_keeps_the_cheapest_candidate():
    cands = SW.candidates(n_alpha=6, omegas=(0.0, 1.0), lo=-1.5, hi=1.5)
    full = G.gadi_sweep(INSTANCES, cands, race=False, max_outer=3000)
    raced = G.gadi_sweep(INSTANCES, cands, race=True, max_outer=3000)
    nc = len(cands)
    for i in range(len(INSTANCES)):
        b_full = SW.best_candidate(full[i * nc:(i + 1) * nc], cands)
        b_race = SW.best_candidate(raced[i * nc:(i + 1) * nc], cands)
        assert b_full is not None and b_race is not None
        assert b_full["spmv_count"] == b_race["spmv_count"] or \
            abs(b_full["spmv_count"] - b_race["spmv_count"]) <= 0.02 * b_full["spmv_count"]
    assert any(r["raced_out"] for r in raced)
    assert sum(r["time_ms"] for r in raced) < sum(r["time_ms"] for r in full)


def test_sweep_item_matches_oracle_outer_steps():
    d, N, b = 2, 24, 40.0
    recs = G.gadi_sweep([(d, N, b)], [(1.0, 1.0)], tol=1e-13, eps_inner=0.1, race=False)
    p = P.make_problem(d, N, b, rhs="ones")
    _, oinfo, _ = oracle.gadi_ir(p.A, p.b, 1.0, 1.0, tol=1e-13, eps_inner=0.1, prec=oracle.PREC_HALF,
                                 max_outer=5000)
    assert oinfo["status"] == oracle.OK and recs[0]["status"] == G.GADI_OK
    assert abs(recs[0]["outer_iters"] - oinfo["outer_iters"]) <= max(2, 0.15 * oinfo["outer_iters"])


def test_sweep_rejects_bad_arguments():
    with pytest.raises(G.GadiError):
        G.gadi_sweep([(4, 8, 1.0)], [(1.0, 1.0)])
    with pytest.raises(G.GadiError):
        G.gadi_sweep([(2, 8, 1.0)], [(1.0, 2.0)])
    with pytest.raises(G.GadiError):
        G.gadi_sweep([(2, 8, 1.0)], [(1.0, 1.0)], block_threads=100)


def test_sweep_jsonl_resume(tmp_path):
    path = str(tmp_path / "records.jsonl")
    inst = [(2, 16, 2.0), (2, 24, 30.0)]
    cands = [(0.5, 0.0), (2.0, 0.0)]
    first = SW.run(inst[:1], path, cands=cands, max_outer=3000)
    both = SW.run(inst, path, cands=cands, max_outer=3000)
    lines = open(path).read().splitlines()
    assert len(lines) == 2
    assert both[0] == first[0]
    assert both[1]["best"] is not None


@pytest.mark.parametrize("team", [2, 4])
def test_multi_block_teams_match_single_solves(team):
    """Items solved by teams of several blocks (rows shared over the team's
    blocks, team-scoped exchanges) agree with gadi_solve like one-block
    teams do, and with the one-block sweep."""
    inst = [(2, 64, 30.0), (3, 16, 10.0), (2, 40, 3.0)]
    cands = [(1.0, 0.0), (3.0, 0.5)]
    one = G.gadi_sweep(inst, cands, race=False, max_outer=5000, team_blocks=1)
    many = G.gadi_sweep(inst, cands, race=False, max_outer=5000, team_blocks=team)
    for i, (d, N, b) in enumerate(inst):
        for j, (a, w) in enumerate(cands):
            r1, rk = one[i * len(cands) + j], many[i * len(cands) + j]
            assert rk["team_blocks"] == team and r1["team_blocks"] == 1
            assert rk["status"] == r1["status"] == G.GADI_OK and rk["eta_inf"] <= 1e-13
            _, st, info, _ = _single(d, N, b, a, w)
            assert abs(rk["outer_iters"] - info["outer_iters"]) <= max(2, 0.15 * info["outer_iters"])
            assert abs(rk["outer_iters"] - r1["outer_iters"]) <= max(2, 0.15 * r1["outer_iters"])


def test_autotuned_schedule_gives_large_instances_multi_block_teams():
    """The row-bin schedule: an instance of 2^18 or more rows runs on a team
    of 2 or more blocks, a small one on a single block; racing still keeps
    the cheapest candidate."""
    inst = [(3, 64, 100.0), (2, 24, 10.0)]
    cands = [(0.8, 0.2), (2.0, 0.0), (6.0, 0.0)]
    recs = G.gadi_sweep(inst, cands, race=True, max_outer=5000)
    big = recs[:3]
    small = recs[3:]
    assert all(r["team_blocks"] >= 2 for r in big)
    assert all(r["team_blocks"] == 1 for r in small)
    best = SW.best_candidate(big, cands)
    full = G.gadi_sweep(inst[:1], cands, race=False, max_outer=5000)
    assert best["spmv_count"] == SW.best_candidate(full, cands)["spmv_count"]


def test_team_larger_than_the_gpu_is_rejected():
    with pytest.raises(G.GadiError):
        G.gadi_sweep([(2, 8, 1.0)], [(1.0, 1.0)], team_blocks=65)
