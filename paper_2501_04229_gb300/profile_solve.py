"""Repeated solves of one workload, for counter captures of the solve kernel.

    python -m paper_2501_04229_gb300.profile_solve --workload convdiff3d_160_b100 \\
        [--alpha 0.8] [--omega 0.2] [--eps 0.1] [--max-outer M] [--solves 3] [--kernel stencil] [--traversal 0]

Each solve runs from x0 = 0 with FP16 inner solves (one persistent launch
of gadi_solve_kernel). --max-outer caps the outer steps (0: the launch does
one FP64 residual pass and stops), so that a capture can isolate the
residual pass or a bounded number of outer steps. Prints one JSON line per
solve (status, counters, device time).
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import gadi as G
from . import problems as P


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="convdiff3d_160_b100")
    ap.add_argument("--alpha", type=float, default=0.8)
    ap.add_argument("--omega", type=float, default=0.2)
    ap.add_argument("--eps", type=float, default=0.1)
    ap.add_argument("--max-outer", type=int, default=100000)
    ap.add_argument("--solves", type=int, default=3)
    ap.add_argument("--kernel", default="stencil", choices=["stencil", "sparse"])
    ap.add_argument("--traversal", type=int, default=0, choices=[0, 1],
                    help="0: z-marching where available, 1: grid-stride items")
    args = ap.parse_args(argv)
    from . import build
    build.build()
    G.load()
    p = P.workload(args.workload)
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt, device="cuda")
    h = G.gadi_create(dev(p.A.row_ptr, torch.int32), dev(p.A.col_idx, torch.int32), dev(p.A.val),
                      stencil=(p.dim, p.N, p.beta, 1 if p.faces is not None else 0))
    try:
        G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL if args.kernel == "stencil" else G.GADI_KERNEL_SPARSE)
        G.gadi_set_params(h, args.alpha, args.omega, u_r=G.GADI_F16)
        G.gadi_set_inner(h, args.eps, 500, args.max_outer)
        G.gadi_set_traversal(h, args.traversal)
        b = dev(p.b)
        x = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        for i in range(args.solves):
            x.zero_()
            st, info = G.gadi_solve(h, b, x, 1e-13)
            if st not in (G.GADI_OK, G.GADI_ERR_NOT_CONVERGED):
                raise RuntimeError(G.last_error(h))
            print(json.dumps({"solve": i, "workload": args.workload, "n": p.n, "status": G.status_str(st),
                              **{k: info[k] for k in ("outer_iters", "inner_iters_H", "inner_iters_S",
                                                      "spmv_count", "eta_inf", "t_solve_s", "grid_blocks",
                                                      "block_threads", "zmarch_planes")}}), flush=True)
    finally:
        G.gadi_destroy(h)


if __name__ == "__main__":
    main()
