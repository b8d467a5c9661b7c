"""Host logic of the sweep driver (no GPU): the candidate grid, the choice
of an instance's best candidate, the seeded instance sets, and the JSONL
checkpoint/resume of records, with the device sweep replaced by a fake."""
import json
import math

from paper_2501_04229_gb300 import gadi as G
from paper_2501_04229_gb300 import sweep as SW


def test_alpha_grid_and_candidates():
    a = SW.alpha_grid(16, -3.0, 2.0)
    assert len(a) == 16 and math.isclose(a[0], 1e-3) and math.isclose(a[-1], 100.0)
    assert all(math.isclose(a[j + 1] / a[j], 10 ** (5 / 15)) for j in range(15))
    c = SW.candidates()
    assert len(c) == 64 and c[0] == (a[0], 0.0) and c[-1] == (a[-1], 1.5)


def _r(cand, spmv, outer, status=G.GADI_OK):
    return {"candidate": cand, "spmv_count": spmv, "outer_iters": outer, "status": status, "eta_inf": 1e-14}


def test_best_candidate_order():
    cands = [(0.1, 0.0), (1.0, 0.0), (10.0, 0.5)]
    # fewest operator applications; ties to fewer outer steps, then larger alpha
    recs = [_r(0, 50, 9), _r(1, 50, 9), _r(2, 40, 20, G.GADI_ERR_NOT_CONVERGED)]
    b = SW.best_candidate(recs, cands)
    assert (b["alpha"], b["omega"]) == (1.0, 0.0)
    recs = [_r(0, 50, 8), _r(1, 50, 9), _r(2, 60, 1)]
    assert SW.best_candidate(recs, cands)["alpha"] == 0.1
    assert SW.best_candidate([_r(0, 1, 1, G.GADI_ERR_DIVERGED)], cands) is None


def test_random_instances_are_seeded_and_in_range():
    a = SW.random_instances(50, seed=4, dim=2, side=(64, 1024), beta=(0.1, 1000.0))
    assert a == SW.random_instances(50, seed=4, dim=2, side=(64, 1024), beta=(0.1, 1000.0))
    assert a != SW.random_instances(50, seed=5, dim=2, side=(64, 1024), beta=(0.1, 1000.0))
    for d, N, b in a:
        assert d == 2 and N % 8 == 0 and 64 <= N <= 1024 and 0.1 <= b <= 1000.0


def test_run_resumes_from_its_records(tmp_path, monkeypatch):
    cands = [(0.5, 0.0), (2.0, 0.5)]
    calls = []

    def fake_sweep(instances, candidates, **kw):
        calls.append(list(instances))
        out = []
        for d, N, b in instances:
            for j in range(len(candidates)):
                out.append(dict(_r(j, N + 10 * j, 3), time_ms=1.0))
        return out

    monkeypatch.setattr(G, "gadi_sweep", fake_sweep)
    path = tmp_path / "rec.jsonl"
    inst = [(2, 16, 1.0), (2, 24, 2.0), (2, 32, 3.0)]
    recs = SW.run(inst[:2], str(path), cands=cands, chunk=1)
    assert [r["N"] for r in recs] == [16, 24] and len(calls) == 2
    assert all(r["best"]["alpha"] == 0.5 for r in recs)
    # a rerun over a larger set sweeps only the new instance and keeps the old records
    recs = SW.run(inst, str(path), cands=cands, chunk=16)
    assert calls[-1] == [inst[2]] and len(calls) == 3
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert [x["N"] for x in lines] == [16, 24, 32]
    assert [r["N"] for r in recs] == [16, 24, 32]
    assert recs[2]["log_n"] == math.log(32 ** 2) and recs[2]["n"] == 1024
