"""Evaluation of the parameter predictors on large 3D systems (§3.3).

    python -m paper_2501_04229_gb300.evaluate [--cases 32] [--N 192] [--out results.json]

Training records come from batched sweeps of smaller systems of the same
structure (§3.3 trains on small systems): a 3D set (sides 8..160, five
convection strengths from 2 to 300) -- the set the bench trains on -- and a
2D set (sides 16..128, beta log-uniform in [0.1, 1000]), each swept over 24
alpha in [0.1, 31.6] x 3 omega to eta_inf <= 1e-13. From each set an MLP
(trained on the GPU by the library's kernels) and a GPR are fitted. The test
systems are the 3D convection-diffusion operator on an N^3 grid with beta
log-uniform in [1, 500] (case c uses seed 5000 + c) and the manufactured
right-hand side. For every case and predictor: the predicted (alpha, omega),
the outer and inner iteration counts, operator applications and the time to
eta_inf <= 1e-13 of FP16-inner GADI-IR, next to the best candidate of a
raced grid search on the case itself, 16 alpha = 10^(-3 + 5 j / 15) x 4
omega in {0, 0.5, 1, 1.5} (the reference for the predictors' error).

Prints one JSON line per case and a summary line. --out receives the same
as JSON lines (every case's full records as soon as the case ends, the
summary last), so an interrupted run keeps the cases it finished.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import gadi as G
from . import problems as P
from . import sweep as SW

TOL = 1e-13
EPS = 0.1


THREE_D_TRAIN = [(3, N, b) for N in (8, 16, 24, 32, 48, 64, 96, 128, 160) for b in (2.0, 10.0, 40.0, 100.0, 300.0)]


def train_sets(seed=11, records=None):
    """The 3D training set (the bench's), and the 2D set: swept here (sides
    16..128), or read from a record file written by `python -m
    paper_2501_04229_gb300.sweep` (e.g. 256 instances with sides 64..1024)."""
    cands = SW.candidates(n_alpha=24, omegas=(0.0, 0.25, 0.5), lo=-1.0, hi=1.5)
    sets = {}
    t0 = time.perf_counter()
    sets["3d"] = SW.run(THREE_D_TRAIN, cands=cands, eps_inner=EPS, max_outer=4000)
    if records:
        with open(records) as f:
            sets["2d"] = [json.loads(line) for line in f]
    else:
        two = SW.random_instances(48, seed=seed, dim=2, side=(16, 128), beta=(0.1, 1000.0))
        sets["2d"] = SW.run(two, cands=cands, eps_inner=EPS, max_outer=4000)
    return sets, time.perf_counter() - t0


def fit(records):
    rows = [r for r in records if r["best"]]
    X = np.array([[r["log_n"], r["log_beta"]] for r in rows])
    Y = np.array([[math.log(r["best"]["alpha"]), r["best"]["omega"]] for r in rows])
    return {"mlp": G.gadi_model_fit(G.GADI_MODEL_MLP, X, Y, hyper=[3000, 1e-2, 1]),
            "gpr": G.gadi_model_fit(G.GADI_MODEL_GPR, X, Y)}, len(rows)


def solve(h, b, x, alpha, omega, max_outer=100000):
    import torch
    G.gadi_set_params(h, alpha, omega, u_r=G.GADI_F16)
    G.gadi_set_inner(h, EPS, 500, max_outer)
    x.zero_()
    torch.cuda.synchronize()
    st, info = G.gadi_solve(h, b, x, TOL)
    return {"alpha": alpha, "omega": omega, "status": G.status_str(st), "outer_iters": info["outer_iters"],
            "inner_iters_H": info["inner_iters_H"], "inner_iters_S": info["inner_iters_S"],
            "spmv_count": info["spmv_count"], "eta_inf": info["eta_inf"], "time_s": info["t_solve_s"]}


def grid_optimum(h, b, x, n_alpha=16, omegas=SW.OMEGAS, start=0.3):
    """Best (fewest operator applications) of the 16 alpha (10^-3 .. 10^2) x
    4 omega grid on the case itself; each candidate is capped at 1.5x the
    outer steps of the best one so far (a candidate that needs more cannot
    be the cheapest unless its inner solves are much cheaper), and the grid
    is walked from alpha = start outwards so that a cap exists early."""
    best, cap, tried = None, 100000, []
    for a in sorted(SW.alpha_grid(n_alpha, -3.0, 2.0), key=lambda v: abs(math.log(v / start))):
        for w in omegas:
            r = solve(h, b, x, a, w, max_outer=cap)
            tried.append(r)
            if r["status"] == "GADI_OK" and (best is None or r["spmv_count"] < best["spmv_count"]):
                best = r
                cap = max(1, int(r["outer_iters"] * 1.5))
    return best, tried


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--cases", type=int, default=32)
    ap.add_argument("--N", type=int, default=192)
    ap.add_argument("--out", default=None)
    ap.add_argument("--records", default=None, help="2D training records (JSONL) instead of a small sweep")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    G.load()
    sets, t_sweep = train_sets(records=args.records)
    models = {}
    counts = {}
    for name, recs in sets.items():
        ms, counts[name] = fit(recs)
        for kind, m in ms.items():
            models[f"{kind}_{name}"] = m
    results = []
    out = open(args.out, "w") if args.out else None
    try:
        for c in range(args.cases):
            rng = np.random.default_rng(5000 + c)
            beta = float(math.exp(rng.uniform(math.log(1.0), math.log(500.0))))
            p = P.make_problem(3, args.N, beta)
            t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt, device="cuda")
            h = G.gadi_create(t(p.A.row_ptr, torch.int32), t(p.A.col_idx, torch.int32), t(p.A.val),
                              stencil=(3, args.N, beta, 0))
            b = t(p.b)
            x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
            try:
                G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL)
                solve(h, b, x, 2.0, 0.0)                       # warm-up
                row = {"case": c, "seed": 5000 + c, "N": args.N, "beta": beta}
                q = [[math.log(p.n), math.log(beta)]]
                for name, m in models.items():
                    y = G.gadi_model_predict(m, q)[0]
                    a, w = float(math.exp(y[0])), float(min(1.999, max(0.0, y[1])))
                    row[name] = solve(h, b, x, a, w)
                row["grid"], _ = grid_optimum(h, b, x, start=row["mlp_3d"]["alpha"] if "mlp_3d" in row else 0.3)
                results.append(row)
                if out:
                    out.write(json.dumps(row) + "\n")
                    out.flush()
                print(json.dumps({k: (v if not isinstance(v, dict) else
                                      {kk: v[kk] for kk in ("alpha", "omega", "spmv_count", "time_s", "status")})
                                  for k, v in row.items()}), flush=True)
            finally:
                G.gadi_destroy(h)
    finally:
        for m in models.values():
            G.gadi_model_destroy(m)
    summary = summarize(results, list(models))
    summary.update({"N": args.N, "train_records": counts, "sweep_s": round(t_sweep, 2)})
    if out:
        out.write(json.dumps({"summary": summary}) + "\n")
        out.close()
    print(json.dumps(summary))


def summarize(results, names):
    """Per predictor: cases converged, and the means over them of operator
    applications, outer steps and time relative to the grid's best, and of
    the time itself."""
    summary = {"cases": len(results)}
    for name in names:
        ok = [r for r in results if r[name]["status"] == "GADI_OK" and r["grid"]]
        if ok:
            rel = lambda key: float(np.mean([r[name][key] / r["grid"][key] for r in ok]))
            summary[name] = {"converged": len(ok), "spmv_vs_grid_mean": rel("spmv_count"),
                             "outer_vs_grid_mean": rel("outer_iters"), "time_vs_grid_mean": rel("time_s"),
                             "time_s_mean": float(np.mean([r[name]["time_s"] for r in ok]))}
        else:
            summary[name] = {"converged": 0}
    summary["grid_time_s_mean"] = float(np.mean([r["grid"]["time_s"] for r in results if r["grid"]]))
    return summary


if __name__ == "__main__":
    main()
