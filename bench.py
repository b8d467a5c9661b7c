"""Time-to-tolerance benchmark of FP16-inner GADI-IR on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Workload (the largest single-GPU system of the measurement plan): the 3D
convection-diffusion operator of §4.1 on a 192^3 grid (n = 7,077,888,
7-point, h^2-scaled, beta = 100, manufactured solution sin(pi x) sin(pi y)
sin(pi z)), solved from x0 = 0 to normwise backward error eta_inf <= 1e-13
by Algorithm 1 with FP16 inner solves (FP16 storage, FP32 arithmetic) and
FP64 residual and update, (alpha, omega) predicted by the MLP trained on the
GPU on batched sweeps of smaller 3D systems (untimed set-up; the fixed pair
is the fallback). One step = one complete solve. Inputs are resident on the
device when a step's timing starts; the working set (about 3 GB) is many
times the 129 MB L2, and L2 is flushed before every timed step as well.

`value` is the median solve time over the K timed steps (CUDA events on the
solver's stream); `e2e` is the same solve through the C ABI with pinned host
buffers (copies of b, x0 and x inside the timed call); `roofline` is the
persistent solve kernel's algorithmic bytes over its mean launch time;
`cpu_baseline` is the FP64-inner oracle on the host cores. Secondary numbers
in the same line: plain FP64 GADI on the same GPU, the 64^3 system, the
inner-precision ablation, the 128^3 variable-coefficient system with both
kernels, operator-application bandwidths, the Sylvester case, and the
predictor's choice against the fixed pair.

`--impl reference` times the oracle (the only other implementation of the
method) on the host cores with the same (alpha, omega), obtained the same way.

Under torchrun (N > 1) every rank solves its own copy of the system
(replicas: a single solve is not sharded), the step time is the maximum
over ranks and rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-13 backward error (s) and SpMV GB/s: FP16-inner GADI-IR vs FP64 GADI"
WORKLOAD = "convdiff3d_192_b100"
SECONDARY = "convdiff3d_64_b100"
TOL = 1e-13
# inner relative tolerance of the timed FP16-inner solves: the best of
# 0.3, 0.2, 0.1, 0.05, 0.03, 0.01 on the 192^3 system at the predicted
# (alpha, omega) (0.05: 279 outer steps, 0.145 s; 0.1: 311, 0.154 s)
EPS16 = 5e-2
# inner tolerance of the training sweeps (the records of the evaluation and
# of the sweep workload use the same) and of FP8 E4M3 inner solves (4
# significant bits do not resolve a smaller reduction reliably)
EPS_TRAIN = 1e-1
EPS_FP8 = 1e-1
EPS64 = 1e-10
# fallback (alpha, omega) per system: the best of small alpha sweeps with omega = 0
FIXED = {"convdiff3d_192_b100": (2.0, 0.0), "convdiff3d_64_b100": (3.0, 0.0),
         "convdiff3d_128_b50_grf": (1.0, 1.0)}
L2_BYTES = 129e6
# the predictors' training instances: 3D systems of the targets' structure,
# up to 160^3 (the large ones solved by multi-block teams in the sweep)
TRAIN_SIDES = (8, 16, 24, 32, 48, 64, 96, 128, 160)
TRAIN_BETAS = (2.0, 10.0, 40.0, 100.0, 300.0)


def fixed_pair(name):
    return FIXED.get(name, (2.0, 0.0))


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, help="system of problems.WORKLOADS to time")
    ap.add_argument("--params", default="mlp", choices=["mlp", "gpr", "fixed"],
                    help="(alpha, omega): predicted by the MLP or GPR trained on sweeps of smaller "
                         "3D systems (untimed set-up), or the fixed pair (--alpha/--omega)")
    ap.add_argument("--alpha", type=float, default=None)
    ap.add_argument("--omega", type=float, default=None)
    ap.add_argument("--eps", type=float, default=EPS16, help="inner relative tolerance (FP16 inner)")
    ap.add_argument("--kernel", default="stencil", choices=["stencil", "sparse"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GADI comparison")
    ap.add_argument("--no-spmv", action="store_true", help="skip the operator bandwidth runs")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 64^3 system")
    ap.add_argument("--no-ablation", action="store_true", help="skip the inner-precision ablation")
    ap.add_argument("--no-sylvester", action="store_true", help="skip the Sylvester GADI-AB case")
    ap.add_argument("--no-grf", action="store_true", help="skip the 128^3 variable-coefficient case")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end timing")
    ap.add_argument("--cpu-sample-s", type=float, default=30.0,
                    help="bound on the CPU oracle's time for cpu_baseline")
    return ap.parse_args(argv)


def dist_init(args):
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "gb300" else "gloo"
        dist.init_process_group(backend)
    return rank, world


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Algorithmic bytes (the per-row counts of the measurement plan)
# ---------------------------------------------------------------------------
def spmv_bytes(kind, fp16, nnz_per_row=7.0, faces=False, op="H"):
    """Bytes per row of one inner operator application: x read and y written
    in the inner precision, plus the matrix bytes as stored.
      stencil, constant k: x, y only            4 B (FP16) / 16 B (FP64)
      stencil, face k (H only; S is constant):  3 FP16 faces + x, y = 10 B / 40 B
      CSR (7-point):  values 7 x 2, columns 7 x 4, row pointer 4, x, y = 50 B / 104 B"""
    vs = 2 if fp16 else 8
    if kind == "stencil":
        return 2 * vs + (3 * vs if (faces and op == "H") else 0)
    return nnz_per_row * (vs + 4) + 4 + 2 * vs


def residual_matrix_bytes(kind, nnz_per_row=7.0, faces=False):
    """Matrix bytes per row of the FP64 residual's product with A: none for
    the constant-coefficient stencil, the three FP64 face coefficients for
    the face form, values + columns + row pointer for CSR."""
    if kind == "stencil":
        return 3 * 8 if faces else 0
    return nnz_per_row * 12 + 4


def algorithmic_bytes(n, nnz, info, kind, fp16=True, faces=False):
    """Minimum bytes one solve moves, from its counters, per row:
      outer step   34 B (FP64 residual, norms, demotion) + the residual's
                   matrix bytes, for every residual evaluated (outer + 1,
                   the last one is the stopping test), + 18 B FP64 update
                   per completed step;
      CG iteration 20 B of vectors (80 B with FP64 inner vectors) + one H
                   application;
      CGNR iteration 26 B of vectors (104 B) + two S applications."""
    npr = nnz / n
    outer, itH, itS = info["outer_iters"], info["inner_iters_H"], info["inner_iters_S"]
    cg_v, cgnr_v = (20, 26) if fp16 else (80, 104)
    per_row = ((outer + 1) * (34 + residual_matrix_bytes(kind, npr, faces)) + outer * 18
               + itH * (cg_v + spmv_bytes(kind, fp16, npr, faces, "H"))
               + itS * (cgnr_v + 2 * spmv_bytes(kind, fp16, npr, faces, "S")))
    return float(n * per_row)


def reduce_max(value, world, device="cpu"):
    """Maximum of a per-rank value over all ranks (identity for one rank)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# the sources the solve kernel and its launch are built from
SOLVE_SOURCES = ("gadi_api.cu", "gadi_solve.cuh", "gadi_ops.cuh", "gadi_device.cuh", "gadi_bits.cuh")


def kernel_source_digest():
    """Hash of the solve kernel's sources with comments and blank space
    removed, so that a change of wording alone keeps a capture current."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in SOLVE_SOURCES:
        text = open(os.path.join(ROOT, "paper_2501_04229_gb300", "csrc", name)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(name.encode())
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(name, algorithmic):
    """DRAM bytes per launch from a committed ncu summary, scaled from the
    profiled launch to this one by their algorithmic bytes (the same kernel on
    the same system: traffic grows with the outer and inner steps), or None
    when the kernel sources changed since that capture."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    keys = ("kernel-source-sha256:", "dram-bytes-per-launch:", "algorithmic-bytes-per-launch:")
    fields = dict(line.split(":", 1) for line in txt.splitlines() if line.startswith(keys))
    if fields.get("kernel-source-sha256", "").strip() != kernel_source_digest():
        return None
    return round(float(fields["dram-bytes-per-launch"]) * algorithmic / float(fields["algorithmic-bytes-per-launch"]))


def solve_kernel_name(kind, info):
    """The solve kernel a solve ran, from its info (stencil item rows are 8
    for every bench workload)."""
    if kind != "stencil":
        return "gadi_solve_kernel<EllOp<half>>"
    if info.get("zmarch_planes", 0) > 0:
        return "gadi_solve_kernel<ZMarchOp<StencilOp<half,3,8>>>"
    return "gadi_solve_kernel<StencilOp<half,3,8>>"


def peaks():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(pk["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "fallback 6800 GB/s (of fallback)"


def backward_error(A, b, x):
    """eta_inf = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf), FP64 on
    the host (a check of the returned x)."""
    S = A.to_scipy()
    r = b - S @ x
    anorm = float(np.abs(S).sum(axis=1).max())
    return float(np.abs(r).max() / (anorm * np.abs(x).max() + np.abs(b).max()))


# ---------------------------------------------------------------------------
# GPU pieces
# ---------------------------------------------------------------------------
class Ctx:
    """Device, stream and L2 flush shared by the GPU measurements."""

    def __init__(self, torch, G, P, dev):
        self.torch, self.G, self.P = torch, G, P
        torch.cuda.set_device(dev)
        self.dev = dev
        self.stream = torch.cuda.current_stream()
        self._flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush_l2(self):
        # write 256 MB (evicts everything), then read it back so that L2 holds
        # clean lines: no write-back of flush data inside a timed region
        self._flush.fill_(1.0)
        self._flush.sum()

    def dev_tensor(self, a, dt=None):
        torch = self.torch
        return torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt or torch.float64, device="cuda")

    def create(self, p, kernel="stencil"):
        torch, G = self.torch, self.G
        st = (p.dim, p.N, p.beta, 1 if p.faces is not None else 0)
        h = G.gadi_create(self.dev_tensor(p.A.row_ptr, torch.int32), self.dev_tensor(p.A.col_idx, torch.int32),
                          self.dev_tensor(p.A.val), stencil=st, stream=self.stream.cuda_stream)
        G.gadi_set_kernel(h, G.GADI_KERNEL_STENCIL if kernel == "stencil" else G.GADI_KERNEL_SPARSE)
        return h

    def timed_solve(self, h, b, x, u_r, alpha, omega, eps, max_inner=500, max_outer=100000):
        """One solve from x0 = 0, L2 flushed before it, CUDA-event time on the
        solver's stream."""
        torch, G = self.torch, self.G
        G.gadi_set_params(h, alpha, omega, u_r=u_r)
        G.gadi_set_inner(h, eps, max_inner, max_outer)
        x.zero_()
        self.flush_l2()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        st, info = G.gadi_solve(h, b, x, TOL)
        e1.record(self.stream)
        torch.cuda.synchronize()
        return st, info, e0.elapsed_time(e1) * 1e-3


def summary(info, keys=("outer_iters", "inner_iters_H", "inner_iters_S", "spmv_count", "eta_inf")):
    return {k: info[k] for k in keys}


def spread(ts):
    return {"median": statistics.median(ts), "min": min(ts), "max": max(ts),
            "stdev": statistics.stdev(ts) if len(ts) > 1 else 0.0, "n": len(ts)}


def learned_params(G, queries):
    """Training records from batched sweeps of 3D systems of the same
    structure as the targets (sides 8..160, five convection strengths, 24
    alpha in [0.1, 31.6] x 3 omega: a fine alpha grid keeps the targets from
    being quantised), then the MLP (trained on the GPU) and the GPR; their
    (alpha, omega) for each (n, beta) of queries."""
    from paper_2501_04229_gb300 import sweep as SW
    inst = [(3, N, b) for N in TRAIN_SIDES for b in TRAIN_BETAS]
    cands = SW.candidates(n_alpha=24, omegas=(0.0, 0.25, 0.5), lo=-1.0, hi=1.5)
    t0 = time.perf_counter()
    recs = SW.run(inst, cands=cands, eps_inner=EPS_TRAIN, max_outer=4000)
    t_sweep = time.perf_counter() - t0
    rows = [r for r in recs if r["best"]]
    X = np.array([[r["log_n"], r["log_beta"]] for r in rows])
    Y = np.array([[math.log(r["best"]["alpha"]), r["best"]["omega"]] for r in rows])
    q = np.array([[math.log(qn), math.log(qb)] for qn, qb in queries])
    out = {"train_instances": len(rows), "train_sides": sorted({r["N"] for r in rows}),
           "candidates": len(cands), "sweep_s": round(t_sweep, 3)}
    t0 = time.perf_counter()
    mlp = G.gadi_model_fit(G.GADI_MODEL_MLP, X, Y, hyper=[3000, 1e-2, 1])
    out["mlp_train_s"] = round(time.perf_counter() - t0, 3)
    gpr = G.gadi_model_fit(G.GADI_MODEL_GPR, X, Y)
    try:
        for name, m in (("mlp", mlp), ("gpr", gpr)):
            ys = G.gadi_model_predict(m, q)
            out[name] = [{"alpha": float(math.exp(y[0])), "omega": float(min(1.999, max(0.0, y[1])))} for y in ys]
    finally:
        G.gadi_model_destroy(mlp)
        G.gadi_model_destroy(gpr)
    return out


def resolve_params(args, names):
    """(alpha, omega) for each workload name: the fixed pair (or --alpha /
    --omega), or the predictor's (MLP / GPR) trained on the GPU; returns
    ({name: (alpha, omega, source)}, predictor record or None)."""
    from paper_2501_04229_gb300 import problems as P
    out = {nm: (*fixed_pair(nm), "fixed") for nm in names}
    if args.alpha is not None or args.omega is not None:
        nm = names[0]
        out[nm] = (args.alpha if args.alpha is not None else fixed_pair(nm)[0],
                   args.omega if args.omega is not None else fixed_pair(nm)[1], "given")
        return out, None
    if args.params == "fixed":
        return out, None
    from paper_2501_04229_gb300 import gadi as G
    wls = [P.WORKLOADS[nm] for nm in names]
    pred = learned_params(G, [(w["N"] ** w["dim"], w["beta"]) for w in wls])
    for nm, q in zip(names, pred[args.params]):
        out[nm] = (q["alpha"], q["omega"], args.params)
    return out, pred


def apply_bandwidth(ctx, p, kernels, reps=10, precs=("fp16", "fp64")):
    """GB/s of H' applications per kernel variant and inner precision, on
    algorithmic bytes (x read once, y written once, matrix bytes as stored):
      GBps           one launch, L2 flushed before it (median CUDA-event time);
      GBps_streamed  back-to-back launches over rotating (x, y) pairs whose
                     footprint exceeds twice the L2, per-launch time from one
                     event pair (None where the matrix arrays, read by every
                     launch, fit in L2)."""
    torch, G = ctx.torch, ctx.G
    h = ctx.create(p)
    n, nnz = p.n, p.A.nnz
    kinds = {"fp16": (G.GADI_F16, torch.float16, 2), "fp64": (G.GADI_F64, torch.float64, 8),
             "fp8_e4m3": (G.GADI_E4M3, torch.uint8, 1)}
    out = {}

    def vec(dt):
        if dt == torch.uint8:
            # E4M3 codes of moderate magnitude with random signs (no NaN codes)
            return (torch.randint(0x20, 0x60, (n,), dtype=torch.uint8, device="cuda")
                    | (torch.randint(0, 2, (n,), dtype=torch.uint8, device="cuda") << 7))
        return torch.randn(n, device="cuda").to(dt)

    try:
        for kname, kk in kernels:
            G.gadi_set_kernel(h, kk)
            for prec in precs:
                u_r, dt, vs = kinds[prec]
                G.gadi_set_params(h, 3.0, 0.0, u_r=u_r)
                xi = vec(dt)
                yo = torch.empty_like(xi)
                for _ in range(3):
                    G.gadi_apply(h, G.OP_H, xi, yo)
                ts = []
                for _ in range(reps):
                    ctx.flush_l2()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(ctx.stream)
                    G.gadi_apply(h, G.OP_H, xi, yo)
                    e1.record(ctx.stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1) * 1e-3)
                if kname == "sparse":
                    mat = nnz * (vs + 4)
                elif p.faces is not None:
                    mat = 4 * n * vs            # diagonal + 3 face couplings per node, as stored
                else:
                    mat = 0
                byts = 2 * n * vs + mat
                med = statistics.median(ts)
                key = f"{p.name}_{kname}_{prec}_H"
                out[key] = {"GBps": round(byts / med / 1e9, 1), "bytes": byts, "us": round(med * 1e6, 2)}
                if 0 < mat < 1.5 * L2_BYTES:
                    out[key]["GBps_streamed"] = None
                    continue
                npairs = int(min(32, max(2, np.ceil(2 * L2_BYTES / (2 * n * vs)))))
                xs = [vec(dt) for _ in range(npairs)]
                ys = [torch.empty_like(xi) for _ in range(npairs)]
                launches = max(20, 2 * npairs)
                ctx.flush_l2()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(ctx.stream)
                for k in range(launches):
                    G.gadi_apply(h, G.OP_H, xs[k % npairs], ys[k % npairs])
                e1.record(ctx.stream)
                torch.cuda.synchronize()
                per = e0.elapsed_time(e1) * 1e-3 / launches
                del xs, ys
                out[key].update({"GBps_streamed": round(byts / per / 1e9, 1), "us_streamed": round(per * 1e6, 2),
                                 "streamed_pairs": npairs, "streamed_launches": launches})
    finally:
        G.gadi_destroy(h)
    return out


def precision_ablation(ctx, h, b, x, alpha, omega, eps, larger_alpha=None):
    """The inner precision u_r varied on the same system and parameters (§4.1's
    precision study): FP16 (scaled, the method), bfloat16 (scaled), FP8 E4M3
    (scaled), FP32, FP64, and the unscaled FP16 mode. Per variant one
    untimed solve (operator demotion, first launch), then one timed solve to
    eta_inf <= 1e-13 (the unscaled mode, which stalls, is capped at 500
    outer steps and 50 inner iterations per solve). FP8's 4 significant
    bits resolve the inner systems only while u_r kappa(H) stays below about
    1, i.e. for alpha large enough; when FP8 fails at (alpha, omega) it is
    also run at larger_alpha = (alpha', omega')."""
    G = ctx.G
    out = {}
    for name, u_r, scaling in (("fp16", G.GADI_F16, 1), ("bf16", G.GADI_BF16, 1), ("fp8_e4m3", G.GADI_E4M3, 1),
                               ("fp32", G.GADI_F32, 1), ("fp64", G.GADI_F64, 1), ("fp16_unscaled", G.GADI_F16, 0)):
        G.gadi_set_scaling(h, scaling)
        mo, mi = (500, 50) if scaling == 0 else (100000, 500)
        ev = max(eps, EPS_FP8) if u_r == G.GADI_E4M3 else eps
        for _ in range(2):
            st, info, dt = ctx.timed_solve(h, b, x, u_r, alpha, omega, ev, max_inner=mi, max_outer=mo)
        out[name] = dict(status=G.status_str(st), time_s=dt, eps_inner=ev, **summary(info))
    G.gadi_set_scaling(h, 1)
    if larger_alpha and out["fp8_e4m3"]["status"] != "GADI_OK":
        a8, w8 = larger_alpha
        for _ in range(2):
            st, info, dt = ctx.timed_solve(h, b, x, G.GADI_E4M3, a8, w8, max(eps, EPS_FP8))
        out["fp8_e4m3_larger_alpha"] = dict(alpha=a8, omega=w8, status=G.status_str(st), time_s=dt,
                                            eps_inner=max(eps, EPS_FP8), **summary(info))
    return out


def grf_case(ctx):
    """The 128^3 system with GRF face coefficients (beta = 50): time to
    eta_inf <= 1e-13 of FP16-inner GADI-IR with the face-coefficient stencil
    kernel and with the general sparse (ELL) kernel, and plain FP64 GADI with
    the stencil kernel, on the same GPU (one warm-up solve per kernel first)."""
    G, P = ctx.G, ctx.P
    p = P.workload("convdiff3d_128_b50_grf")
    alpha, omega = FIXED["convdiff3d_128_b50_grf"]
    h = ctx.create(p)
    b = ctx.dev_tensor(p.b)
    x = ctx.torch.zeros(p.n, dtype=ctx.torch.float64, device="cuda")
    out = {"workload": p.name, "n": p.n, "alpha": alpha, "omega": omega}
    try:
        for name, kern, u_r, eps, reps in (("fp16_stencil", G.GADI_KERNEL_STENCIL, G.GADI_F16, EPS16, 2),
                                           ("fp16_sparse", G.GADI_KERNEL_SPARSE, G.GADI_F16, EPS16, 2),
                                           ("fp64_gadi_stencil", G.GADI_KERNEL_STENCIL, G.GADI_F64, EPS64, 1)):
            G.gadi_set_kernel(h, kern)
            for _ in range(reps):
                st, info, dt = ctx.timed_solve(h, b, x, u_r, alpha, omega, eps,
                                               max_inner=500 if u_r == G.GADI_F16 else 10000)
            kind = "stencil" if kern == G.GADI_KERNEL_STENCIL else "sparse"
            alg = algorithmic_bytes(p.n, p.A.nnz, info, kind, u_r == G.GADI_F16, faces=True)
            out[name] = dict(status=G.status_str(st), time_s=dt, **summary(info),
                             effective_GBps=round(alg / info["t_solve_s"] / 1e9, 1),
                             max_abs_err_vs_exact=float(np.abs(x.cpu().numpy() - p.x_exact).max()))
        if out["fp16_stencil"]["status"] == "GADI_OK" and out["fp64_gadi_stencil"]["status"] == "GADI_OK":
            out["speedup_fp16_vs_fp64_gadi"] = out["fp64_gadi_stencil"]["time_s"] / out["fp16_stencil"]["time_s"]
    finally:
        G.gadi_destroy(h)
    return out


def sylvester_case(ctx, m=1024, n=1024, r=0.1, alpha=0.05, omega=1.0):
    """GADI-AB for the Sylvester equation of §4.3 (A = B = M + 2 r N + 100/(n+1)^2 I,
    m = n = 1024, X* random, C = A X* + X* B): time to eta <= 1e-13 with FP16
    and FP64 inner solves on the GPU (one warm-up solve each first)."""
    torch, G, P = ctx.torch, ctx.G, ctx.P
    a, b, Xs, Cm = P.sylvester_problem(m, n, r, seed=0)
    Cm = torch.from_numpy(Cm).cuda()
    out = {"m": m, "n": n, "r": r, "alpha": alpha, "omega": omega}
    s = G.gadi_sylv_create(a, b)
    try:
        for name, u_r in (("fp16", G.GADI_F16), ("fp64", G.GADI_F64)):
            G.gadi_sylv_set_params(s, alpha, omega, u_r)
            X = torch.zeros_like(Cm)
            G.gadi_sylv_solve(s, Cm, X, TOL)
            X.zero_()
            torch.cuda.synchronize()
            st, info = G.gadi_sylv_solve(s, Cm, X, TOL)
            err = float((X.cpu() - torch.from_numpy(Xs)).abs().max())
            out[name] = {"status": G.status_str(st), "time_s": info["t_solve_s"], "outer_iters": info["outer_iters"],
                         "eta_inf": info["eta_inf"], "max_abs_err_vs_exact": err}
    finally:
        G.gadi_sylv_destroy(s)
    return out


def run_gpu(args, rank, world):
    import torch
    from paper_2501_04229_gb300 import build as B
    from paper_2501_04229_gb300 import gadi as G
    from paper_2501_04229_gb300 import problems as P

    B.build()
    dev = int(os.environ.get("LOCAL_RANK", 0))
    ctx = Ctx(torch, G, P, dev)
    names = [args.workload] + ([SECONDARY] if not args.no_secondary and args.workload != SECONDARY else [])
    params, predictor = resolve_params(args, names)
    p = P.workload(args.workload)
    n, nnz = p.n, p.A.nnz
    h = ctx.create(p, args.kernel)
    b = ctx.dev_tensor(p.b)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    alpha, omega, source = params[args.workload]
    res = {"p": p, "params": {"source": source, "alpha": alpha, "omega": omega}, "predictor": predictor}

    # warm-up (operator demotion, first launch); a predicted pair that fails
    # to converge falls back to the fixed pair
    for i in range(args.warmup):
        st, info, _ = ctx.timed_solve(h, b, x, G.GADI_F16, alpha, omega, args.eps)
        if st != G.GADI_OK and source != "fixed":
            res["params"]["fallback_from"] = {"source": source, "alpha": alpha, "omega": omega,
                                              "status": G.status_str(st)}
            alpha, omega = fixed_pair(args.workload)
            source = "fixed"
            res["params"].update(source=source, alpha=alpha, omega=omega)
            st, info, _ = ctx.timed_solve(h, b, x, G.GADI_F16, alpha, omega, args.eps)
        assert st == G.GADI_OK, G.last_error(h)

    # the K timed steps, clocks sampled meanwhile
    times, kern_t, infos = [], [], []
    clocks = ClockSampler(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with clocks:
        for _ in range(args.steps):
            st, info, dt = ctx.timed_solve(h, b, x, G.GADI_F16, alpha, omega, args.eps)
            assert st == G.GADI_OK, G.last_error(h)
            times.append(dt)
            kern_t.append(info["t_solve_s"])
            infos.append(info)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    info = infos[-1]
    xh = x.cpu().numpy()
    res.update(times=times, kern_t=kern_t, info=info, x=xh,
               total=reduce_max(sum(times), world, "cuda"),
               median=reduce_max(statistics.median(times), world, "cuda"), clocks=clocks.summary())
    kind = args.kernel
    faces = p.faces is not None
    alg = algorithmic_bytes(n, nnz, info, kind, True, faces)
    hbm, peak_src = peaks()
    achieved = alg / statistics.mean(kern_t) / 1e9
    res["roofline"] = {
        "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
        "frac": round(achieved / hbm, 4),
        "traffic": profiled_traffic(f"gadi_solve_kernel_{args.workload}.md", alg),
        "algorithmic_bytes": alg,
        "algorithmic_bytes_rule": "per row: (outer+1) x (34 B + residual matrix bytes) + outer x 18 B "
                                  "+ CG x (20 B + H application) + CGNR x (26 B + 2 S applications); "
                                  "constant-coefficient stencil application 4 B (FP16 x, y)",
        "traffic_note": "ncu dram bytes of the profiled launch, scaled to this launch by algorithmic bytes; "
                        "null when the kernel changed since the capture",
        "kernel": solve_kernel_name(kind, info),
        "kernel_time_s_mean": statistics.mean(kern_t),
        "peak_source": peak_src}

    # FP64 GADI on the same GPU (the baseline of the comparison)
    if not args.no_fp64:
        a64, w64 = fixed_pair(args.workload)
        t64 = []
        for _ in range(2):
            st, i64, dt = ctx.timed_solve(h, b, x, G.GADI_F64, a64, w64, EPS64, max_inner=10000)
            t64.append(dt)
        res["fp64"] = dict(time_s=statistics.median(t64), status=G.status_str(st), alpha=a64, omega=w64,
                           eps_inner=EPS64, spread=spread(t64), **summary(i64))

    # the predictor's choice against the fixed pair on the same system
    if source != "fixed":
        fa, fw = fixed_pair(args.workload)
        st, ifx, dt = ctx.timed_solve(h, b, x, G.GADI_F16, fa, fw, args.eps)
        res["fixed_pair"] = dict(alpha=fa, omega=fw, status=G.status_str(st), time_s=dt, **summary(ifx))
        if predictor is not None:
            ga, gw = predictor["gpr"][0]["alpha"], predictor["gpr"][0]["omega"]
            st, igp, dt = ctx.timed_solve(h, b, x, G.GADI_F16, ga, gw, args.eps)
            res["gpr_pair"] = dict(alpha=ga, omega=gw, status=G.status_str(st), time_s=dt, **summary(igp))

    if not args.no_ablation:
        res["ablation"] = precision_ablation(ctx, h, b, x, alpha, omega, args.eps,
                                             larger_alpha=fixed_pair(args.workload))

    # end to end through the C ABI with pinned host buffers (copies inside)
    if not args.no_e2e:
        G.gadi_set_params(h, alpha, omega, u_r=G.GADI_F16)
        G.gadi_set_inner(h, args.eps, 500, 100000)
        bh = torch.from_numpy(p.b.copy()).pin_memory()
        xh_pin = torch.zeros(n, dtype=torch.float64).pin_memory()
        e2e = []
        for i in range(args.warmup + args.steps):
            xh_pin.zero_()
            ctx.flush_l2()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, _ = G.gadi_solve(h, bh, xh_pin, TOL)
            t1 = time.perf_counter()
            assert st == G.GADI_OK, G.last_error(h)
            if i >= args.warmup:
                e2e.append(t1 - t0)
        res["e2e"] = {"value": statistics.median(e2e), "unit": "s", "h2d_bytes_per_step": 2 * n * 8,
                      "d2h_bytes_per_step": n * 8, "spread": spread(e2e),
                      "path": "gadi_solve with pinned host b and x (H2D b, x0; solve; D2H x)"}
    G.gadi_destroy(h)

    # the 64^3 system (L2-resident: an effective rate, no HBM claim)
    if SECONDARY in params and args.workload != SECONDARY:
        ps = P.workload(SECONDARY)
        a2, w2, src2 = params[SECONDARY]
        hs = ctx.create(ps)
        bs = ctx.dev_tensor(ps.b)
        xs = torch.zeros(ps.n, dtype=torch.float64, device="cuda")
        ts, ks = [], []
        for i in range(3 + max(5, args.steps)):
            st, i2, dt = ctx.timed_solve(hs, bs, xs, G.GADI_F16, a2, w2, args.eps)
            if st != G.GADI_OK and src2 != "fixed":
                a2, w2 = FIXED[SECONDARY]
                src2 = "fixed (predicted pair did not converge)"
                continue
            if i >= 3:
                ts.append(dt)
                ks.append(i2["t_solve_s"])
        alg2 = algorithmic_bytes(ps.n, ps.A.nnz, i2, "stencil", True)
        st64, i64s, t64s = ctx.timed_solve(hs, bs, xs, G.GADI_F64, a2, w2, EPS64, max_inner=10000)
        res["secondary"] = dict(workload=SECONDARY, n=ps.n, params={"source": src2, "alpha": a2, "omega": w2},
                                time_s=statistics.median(ts), spread=spread(ts), **summary(i2),
                                effective_GBps=round(alg2 / statistics.mean(ks) / 1e9, 1),
                                note="working set L2-resident: effective rate, no HBM claim",
                                fp64_gadi_same_gpu=dict(time_s=t64s, status=G.status_str(st64), **summary(i64s)))
        G.gadi_destroy(hs)

    if not args.no_spmv:
        spmv = {}
        p128 = P.make_problem(3, 128, 50.0, grf_seed=3, name="convdiff3d_128_b50_grf")
        spmv.update(apply_bandwidth(ctx, p128, (("stencil", G.GADI_KERNEL_STENCIL), ("sparse", G.GADI_KERNEL_SPARSE))))
        del p128
        spmv.update(apply_bandwidth(ctx, P.workload("convdiff3d_192_b100"),
                                    (("stencil", G.GADI_KERNEL_STENCIL), ("sparse", G.GADI_KERNEL_SPARSE)),
                                    precs=("fp16", "fp8_e4m3", "fp64")))
        res["spmv"] = spmv
    if not args.no_sylvester:
        res["sylvester"] = sylvester_case(ctx)
    if not args.no_grf:
        res["grf"] = grf_case(ctx)
    return res


# ---------------------------------------------------------------------------
# CPU pieces: the oracle on the host cores
# ---------------------------------------------------------------------------
def host_info(n_doubles=1 << 26, reps=5):
    """The host's CPU model and its memory copy rate (STREAM-style copy of a
    512 MB FP64 array over all cores, bytes read + written per second, best
    of reps), so that the oracle's time can be set against the host's own
    bandwidth."""
    import platform
    from concurrent.futures import ThreadPoolExecutor
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    cores = os.cpu_count() or 1
    src = np.ones(n_doubles)
    dst = np.zeros(n_doubles)
    bounds = np.linspace(0, n_doubles, cores + 1).astype(np.int64)
    chunks = [(int(bounds[i]), int(bounds[i + 1])) for i in range(cores)]

    def part(c):
        np.copyto(dst[c[0]:c[1]], src[c[0]:c[1]])

    best = float("inf")
    with ThreadPoolExecutor(cores) as pool:
        list(pool.map(part, chunks))
        for _ in range(reps):
            t0 = time.perf_counter()
            list(pool.map(part, chunks))
            best = min(best, time.perf_counter() - t0)
    return {"cpu_model": model, "host_copy_gbs": round(2 * 8 * n_doubles / best / 1e9, 1),
            "host_copy_threads": cores}


def oracle_steps(p, alpha, omega, eps, max_outer):
    """The oracle's FP64-inner GADI-IR from x0 = 0 with at most max_outer
    outer steps, on all host cores: (seconds, info)."""
    import oracle
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    _, info, _ = oracle.gadi_ir(p.A, p.b, alpha, omega, tol=TOL, eps_inner=eps, prec=oracle.PREC_DOUBLE,
                                max_outer=max_outer, max_inner=500)
    return time.perf_counter() - t0, info


def oracle_setup_s(p, alpha, omega, eps):
    """Seconds of an oracle call that stops at its first residual (the
    splitting, the allocations and one residual): the part of a call that
    does not grow with its outer steps, so that a sample of k steps scales
    to n steps as setup + (t - setup) n / k. The faster of two calls."""
    return min(oracle_steps(p, alpha, omega, eps, 0)[0] for _ in range(2))


def cpu_baseline(p, alpha, omega, eps, budget_s, gpu_outer=None):
    """The oracle (FP64-inner GADI-IR, all host cores) on the same system and
    parameters: a full solve when it fits the budget (estimated from two outer
    steps), else as many outer steps as fit, scaled per outer step (set-up
    apart) to the outer-step count of the GPU solve."""
    import oracle
    cores = os.cpu_count() or 1
    t_set = oracle_setup_s(p, alpha, omega, eps)
    t2, i2 = oracle_steps(p, alpha, omega, eps, 2)
    per = max(t2 - t_set, 1e-9) / max(1, i2["outer_iters"])
    want = gpu_outer or 1000
    if per * want <= budget_s:
        dt, info = oracle_steps(p, alpha, omega, eps, 100000)
        if info["status"] == oracle.OK:
            return {"value": dt, "unit": "s", "cores": cores, "kind": "oracle",
                    "sample": f"one full FP64-inner GADI-IR solve of {p.name} to eta 1e-13 "
                              f"({info['outer_iters']} outer steps), alpha {alpha:.4g}, omega {omega:.4g}"}
    m = max(2, int(budget_s / max(per, 1e-9)))
    dt, info = oracle_steps(p, alpha, omega, eps, m)
    k = max(1, info["outer_iters"])
    scale = gpu_outer or k
    return {"value": t_set + (dt - t_set) / k * scale, "unit": "s", "cores": cores, "kind": "oracle",
            "sample": f"{k} outer steps of FP64-inner GADI-IR on {p.name} in {dt:.2f} s (set-up and first "
                      f"residual {t_set:.2f} s), alpha {alpha:.4g}, omega {omega:.4g}, scaled per outer step "
                      f"to the GPU solve's {scale} outer steps"}


def run_reference(args, base, cfg):
    """The oracle as the reference arm: one full solve first (untimed: its
    outer-step count and time), the set-up time of a call, and one untimed
    sample of the first outer steps (about 3 s); then K timed steps, each
    the same bounded sample, scaled to a full solve by the ratio of the full
    solve's steps to the calibration sample's (set-up apart), so that the
    early steps' different cost does not bias the estimate. (alpha, omega)
    come from the same predictor as the GPU arm's (trained on the GPU in the
    set-up; the fixed pair without a GPU)."""
    from paper_2501_04229_gb300 import problems as P
    names = [args.workload]
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except ImportError:
        have_gpu = False
    if args.params != "fixed" and args.alpha is None and args.omega is None and not have_gpu:
        params, pred = {nm: (*fixed_pair(nm), "fixed (no GPU for the predictor)") for nm in names}, None
    else:
        if have_gpu and args.params != "fixed":
            from paper_2501_04229_gb300 import build as B
            B.build()
        params, pred = resolve_params(args, names)
    alpha, omega, source = params[args.workload]
    p = P.workload(args.workload)
    t_full, i_full = oracle_steps(p, alpha, omega, args.eps, 100000)
    t_set = oracle_setup_s(p, alpha, omega, args.eps)
    full_outer = max(1, i_full["outer_iters"])
    per_full = max(t_full - t_set, 1e-6) / full_outer
    sample_outer = max(2, min(full_outer, int(math.ceil(3.0 / per_full))))
    t_cal, _ = oracle_steps(p, alpha, omega, args.eps, sample_outer)
    scale = (t_full - t_set) / max(t_cal - t_set, 1e-9)
    times = []
    for i in range(args.warmup + args.steps):
        dt, info = oracle_steps(p, alpha, omega, args.eps, sample_outer)
        if i >= args.warmup:
            times.append(t_set + (dt - t_set) * scale)
    v = statistics.median(times)
    cb = {"value": v, "unit": "s", "cores": os.cpu_count() or 1, "kind": "oracle",
          "sample": f"each step: the first {sample_outer} outer steps of FP64-inner GADI-IR on {p.name}, "
                    f"scaled (set-up and first residual, {t_set:.2f} s, apart) by {scale:.2f}, the ratio of "
                    f"one full oracle solve ({full_outer} outer steps, {t_full:.2f} s, status "
                    f"{i_full['status']}, eta {i_full['eta_inf']:.3g}) to an untimed sample ({t_cal:.2f} s)",
          "full_solve_s": t_full}
    cb.update(host_info())
    line = dict(base, impl="reference", value=v, ms_per_step=v * 1e3, dtype="f64", config=cfg,
                cpu_baseline=cb, params_used={"source": source, "alpha": alpha, "omega": omega},
                spread=spread(times),
                e2e={"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})
    if pred is not None:
        line["predictor"] = {k: pred[k] for k in ("train_instances", "train_sides", "candidates")}
    print(json.dumps(line))


def main():
    args = parse()
    rank, world = dist_init(args)
    from paper_2501_04229_gb300 import problems as P
    wl = P.WORKLOADS[args.workload]
    n_wl = wl["N"] ** wl["dim"]
    nnz_wl = (7 * wl["N"] ** 3 - 6 * wl["N"] ** 2) if wl["dim"] == 3 else (5 * wl["N"] ** 2 - 4 * wl["N"])
    base = {"metric": METRIC, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic (3D convection-diffusion of §4.1, manufactured solution)"}
    cfg = {"workload": args.workload, "n": n_wl, "nnz": nnz_wl, "beta": wl["beta"], "tol_eta_inf": TOL,
           "params": args.params, "eps_inner": args.eps,
           "precisions": "u_r=fp16 (fp32 arithmetic), u=u_f=fp64", "kernel": args.kernel,
           "l2": "working set (about 3 GB) larger than L2; L2 also flushed before every timed step "
                 "(256 MB write, then read back)",
           "parallelism": "replicas" if world > 1 else "single GPU"}
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, base, cfg)
        return

    r = run_gpu(args, rank, world)
    if rank != 0:
        return
    p = r["p"]
    info = r["info"]
    eta_host = backward_error(p.A, p.b, r["x"])
    fwd = float(np.abs(r["x"] - p.x_exact).max()) if p.x_exact is not None else None
    cb = cpu_baseline(p, r["params"]["alpha"], r["params"]["omega"], args.eps, args.cpu_sample_s,
                      gpu_outer=info["outer_iters"])
    cb.update(host_info())
    line = dict(base)
    line.update({
        "value": r["median"], "ms_per_step": r["total"] / args.steps * 1e3, "dtype": "fp16-inner/fp64-outer",
        "config": cfg,
        "spread": spread(r["times"]),
        "roofline": r["roofline"],
        "cpu_baseline": cb,
        "e2e": r.get("e2e"),
        "gpu_launches": 3 * args.steps,
        "clocks": r["clocks"],
        "solve": {k: info[k] for k in ("outer_iters", "inner_iters_H", "inner_iters_S", "spmv_count",
                                       "grid_blocks", "block_threads")},
        "eta_inf_gpu": info["eta_inf"], "eta_inf_host_check": eta_host, "max_abs_err_vs_exact": fwd,
        "params_used": r["params"],
        "predictor": r["predictor"],
        "fixed_pair_same_gpu": r.get("fixed_pair"),
        "gpr_pair_same_gpu": r.get("gpr_pair"),
        "fp64_gadi_same_gpu": r.get("fp64"),
        "speedup_vs_fp64_gadi": (r["fp64"]["time_s"] / r["median"]) if r.get("fp64") else None,
        "secondary": r.get("secondary"),
        "precision_ablation": r.get("ablation"),
        "spmv": r.get("spmv"),
        "sylvester_gadi_ab": r.get("sylvester"),
        "grf_case": r.get("grf"),
    })
    print(json.dumps(line))


if __name__ == "__main__":
    main()
