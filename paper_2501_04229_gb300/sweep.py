"""Training records for the parameter predictors from batched GADI-IR sweeps.

A record is one instance (dim, N, beta) with the cheapest converged candidate
(alpha*, omega*) of a candidate grid: cheapest = fewest operator
applications to eta_inf <= tol; ties go to fewer outer steps, then to the
larger alpha. Records are appended to a JSONL file as instances finish, and
a rerun skips the instances already in the file (checkpoint and resume).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import gadi as G


def alpha_grid(n_alpha=16, lo=-3.0, hi=2.0):
    """alpha = 10^(lo + (hi - lo) j / (n_alpha - 1)), j = 0..n_alpha-1."""
    return [10.0 ** (lo + (hi - lo) * j / (n_alpha - 1)) for j in range(n_alpha)]


OMEGAS = (0.0, 0.5, 1.0, 1.5)


def candidates(n_alpha=16, omegas=OMEGAS, lo=-3.0, hi=2.0):
    return [(a, w) for a in alpha_grid(n_alpha, lo, hi) for w in omegas]


def best_candidate(recs, cands):
    """The cheapest converged candidate among one instance's records."""
    ok = [r for r in recs if r["status"] == G.GADI_OK]
    if not ok:
        return None
    r = min(ok, key=lambda r: (r["spmv_count"], r["outer_iters"], -cands[r["candidate"]][0]))
    a, w = cands[r["candidate"]]
    return {"alpha": a, "omega": w, "spmv_count": r["spmv_count"], "outer_iters": r["outer_iters"],
            "eta_inf": r["eta_inf"]}


def random_instances(count, seed, dim=2, side=(16, 128), beta=(0.1, 1000.0), multiple=8):
    """Sides log-uniform in side (rounded to a multiple of `multiple`), beta
    log-uniform in beta."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(round(math.exp(rng.uniform(math.log(side[0]), math.log(side[1]))) / multiple)) * multiple
        N = max(multiple, N)
        b = math.exp(rng.uniform(math.log(beta[0]), math.log(beta[1])))
        out.append((dim, N, b))
    return out


def run(instances, path=None, cands=None, chunk=16, **kw):
    """Sweep instances over cands (default 16 alpha x 4 omega); append one
    record per instance to the JSONL file at path, skipping instances that
    are already there. Returns all records of the requested instances."""
    cands = cands or candidates()
    done = {}
    if path and os.path.exists(path):
        for line in open(path):
            r = json.loads(line)
            done[(r["dim"], r["N"], r["beta"])] = r
    todo = [t for t in instances if (t[0], t[1], t[2]) not in done]
    for k in range(0, len(todo), chunk):
        part = todo[k:k + chunk]
        recs = G.gadi_sweep(part, cands, **kw)
        for i, (d, N, b) in enumerate(part):
            best = best_candidate(recs[i * len(cands):(i + 1) * len(cands)], cands)
            row = {"dim": d, "N": N, "beta": b, "n": N ** d, "log_n": math.log(N ** d),
                   "log_beta": math.log(b), "best": best,
                   "time_ms": sum(r["time_ms"] for r in recs[i * len(cands):(i + 1) * len(cands)])}
            done[(d, N, b)] = row
            if path:
                with open(path, "a") as f:
                    f.write(json.dumps(row) + "\n")
    return [done[(t[0], t[1], t[2])] for t in instances]


def main(argv=None):
    """Command line: sweep a seeded random instance set and append records.

        python -m paper_2501_04229_gb300.sweep --count 256 --seed 4 --dim 2 \\
            --side 64 1024 --beta 0.1 1000 --out records.jsonl

    (the defaults: 256 2D instances, sides log-uniform in [64, 1024], beta
    log-uniform in [0.1, 1000], 16 alpha x 4 omega, max_outer 5000)."""
    import argparse
    import time
    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=256)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--side", type=int, nargs=2, default=(64, 1024))
    ap.add_argument("--beta", type=float, nargs=2, default=(0.1, 1000.0))
    ap.add_argument("--max-outer", type=int, default=5000)
    ap.add_argument("--chunk", type=int, default=16)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    build.build()
    G.load()
    inst = random_instances(args.count, args.seed, dim=args.dim, side=tuple(args.side), beta=tuple(args.beta))
    t0 = time.perf_counter()
    recs = run(inst, args.out, chunk=args.chunk, max_outer=args.max_outer)
    dt = time.perf_counter() - t0
    found = [r for r in recs if r["best"]]
    print(json.dumps({"instances": len(recs), "with_best": len(found), "seconds": round(dt, 2),
                      "n_max": max(r["n"] for r in recs), "sum_item_ms": round(sum(r["time_ms"] for r in recs), 1)}))


if __name__ == "__main__":
    main()
