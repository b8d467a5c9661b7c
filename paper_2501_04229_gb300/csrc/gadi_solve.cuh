// gadi_solve.cuh -- the persistent GADI-IR solve kernel (Algorithm 1).
//
// One cooperative launch runs the whole solve: the outer refinement loop
// and both inner Krylov solves. Phases over the rows are separated by the
// bounded grid barrier of gadi_device.cuh; every reduction is combined by
// all blocks identically, so all blocks take the same branches and the
// scalars of CG and CGNR never leave the device.
//
// Outer step k (Algorithm 1, with the readings of the library header):
//   R  r = b - A x in FP64, ||r||_inf, ||r||_2^2, ||x||_inf; stopping test
//   D  e = floor(log2 ||r||_inf); r^ = fl_r(2^-e r)       (§2.2: r^ = fl_r(s^))
//   CG on H' = 2^-sM (aI + M):  z ~ H'^-1 r^              (Alg. 1 step 2)
//   C0 ez = floor(log2 ||z||_inf); z^ = 2^-ez z; s = S'^T z^
//   CGNR on S' = 2^-sN (aI + N): y ~ S'^-1 z^             (Alg. 1 step 3)
//   U  x += (2-w) a 2^(e - sM + ez - sN) y  in FP64       (Alg. 1 step 4)
// With FP64 inner precision the scales are all 2^0.
//
// Barrier count per CG iteration: 2 (the search-direction update
// p = r + beta p is recomputed at the neighbours inside the next operator
// application instead of in a phase of its own); per CGNR iteration: 2
// (likewise, and the residual update is fused with the S^T product).
#pragma once

#include "gadi_ops.cuh"

namespace gadi {

template <class Op, class T>
struct SolveArgs {
    Op op;
    int64_t n;
    const double *b;
    double *x;
    double *r64;
    T *rc, *pA, *pB, *q, *z, *rsA, *rsB, *s, *y;
    double anorm, bnorm, tol, eps, pfac;
    int sM, sN, half, stop_kind;
    int max_inner, max_outer;
    Ctl *ctl;
    unsigned long long *slots;   // [2][kMaxWords][gridDim] exchange words, zeroed before launch
    double *eta_hist;            // optional, max_outer + 1 entries
    unsigned long long wait_ns;
    unsigned extra;
};

template <class Op, class T>
__global__ void __launch_bounds__(1024, 1) gadi_solve_kernel(const SolveArgs<Op, T> a)
{
    using P = Prec<T>;
    using Acc = typename P::Acc;
    const int64_t n = a.n;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    const Op &op = a.op;
    GridExchange ex{a.ctl, a.slots, 0u, a.wait_ns, a.extra};
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const Acc eps2 = (Acc)(a.eps * a.eps);

    double r0 = 0.0, best = INFINITY, eta = 0.0, res = 0.0;
    long long itH = 0, itS = 0, spmv = 0;
    int k = 0, status = kErrNotConverged;

    for (;;) {
        // ---- R: outer residual in FP64 -------------------------------------
        {
            double v[3] = {0.0, 0.0, 0.0};
            const int ops[3] = {kMax, kSum, kMax};
            const double *x = a.x;
            for (int64_t i = t0; i < n; i += nt) {
                double ax = op.rowA(i, [&](int64_t j) { return x[j]; });
                double r = __dsub_rn(a.b[i], ax);
                a.r64[i] = r;
                v[0] = fmax(v[0], fabs(r));
                v[1] = d_madd(v[1], r, r);
                v[2] = fmax(v[2], fabs(x[i]));
            }
            if (!ex.allreduce(v, ops)) return;
            ++spmv;
            const double rinf = v[0], rn2 = sqrt(v[1]), xinf = v[2];
            const double den = a.anorm * xinf + a.bnorm;
            eta = den > 0.0 ? rinf / den : (rinf == 0.0 ? 0.0 : INFINITY);
            if (k == 0) r0 = rn2;
            res = r0 > 0.0 ? rn2 / r0 : 0.0;
            if (lead && a.eta_hist) a.eta_hist[k] = eta;
            bool done = true;
            if (!isfinite(rn2) || !isfinite(eta)) status = kErrDiverged;
            else {
                if (rn2 < best) best = rn2;
                const double crit = a.stop_kind == 1 ? res : eta;
                if (crit <= a.tol) status = kOk;
                else if (rn2 > 1e3 * best) status = kErrDiverged;
                else if (k >= a.max_outer) status = kErrNotConverged;
                else done = false;
            }
            if (done) break;

            // ---- D: scale and round the residual; CG start -----------------
            const int e = (a.half && rinf > 0.0) ? ilogb(rinf) : 0;
            const double sc = ldexp(1.0, -e);
            Acc w[1] = {0};
            const int ops1[1] = {kSum};
            {
                Acc acc = 0;
                for (int64_t i = t0; i < n; i += nt) {
                    T vr = P::from64(__dmul_rn(a.r64[i], sc));
                    a.rc[i] = vr;
                    a.pA[i] = vr;
                    a.z[i] = P::st(Acc(0));
                    Acc f = P::ld(vr);
                    acc = P::add(acc, P::mul(f, f));
                }
                w[0] = acc;
            }
            if (!ex.allreduce(w, ops1)) return;
            const Acc rr0 = (Acc)w[0];

            // ---- CG on H' ----------------------------------------------------
            Acc zinf = 0;
            int it = 0;
            if (rr0 > Acc(0)) {
                T *pc = a.pA, *pn = a.pB;
                Acc rho = rr0, beta = 0;
                bool first = true;
                for (;;) {
                    // A: p <- r + beta p (fused), q = H' p, <p, q>
                    Acc u[1] = {0};
                    {
                        Acc acc = 0;
                        if (first) {
                            auto fp = [&](int64_t j) -> Acc { return P::ld(pc[j]); };
                            for (int64_t i = t0; i < n; i += nt) {
                                T qs = P::st(op.row(kOpH, i, fp));
                                a.q[i] = qs;
                                acc = P::add(acc, P::mul(fp(i), P::ld(qs)));
                            }
                        } else {
                            const T *rc = a.rc;
                            auto fp = [&](int64_t j) -> Acc {
                                return P::rnd(P::add(P::ld(rc[j]), P::mul(beta, P::ld(pc[j]))));
                            };
                            for (int64_t i = t0; i < n; i += nt) {
                                Acc pi = fp(i);
                                pn[i] = P::st(pi);
                                T qs = P::st(op.row(kOpH, i, fp));
                                a.q[i] = qs;
                                acc = P::add(acc, P::mul(pi, P::ld(qs)));
                            }
                        }
                        u[0] = acc;
                    }
                    if (!ex.allreduce(u, ops1)) return;
                    if (!first) { T *t = pc; pc = pn; pn = t; }
                    ++it;
                    ++spmv;
                    const Acc pq = u[0];
                    if (!(pq > Acc(0)) || !isfinite((double)pq)) { status = kErrDiverged; break; }
                    const Acc al = rho / pq;
                    // B: z += al p, r -= al q, <r, r>, ||z||_inf
                    Acc vb[2] = {0, 0};
                    const int opsb[2] = {kSum, kMax};
                    {
                        Acc acc = 0, zm = 0;
                        for (int64_t i = t0; i < n; i += nt) {
                            Acc zn = P::rnd(P::add(P::ld(a.z[i]), P::mul(al, P::ld(pc[i]))));
                            a.z[i] = P::st(zn);
                            Acc rn = P::rnd(P::sub(P::ld(a.rc[i]), P::mul(al, P::ld(a.q[i]))));
                            a.rc[i] = P::st(rn);
                            acc = P::add(acc, P::mul(rn, rn));
                            zm = fmax(zm, fabs(zn));
                        }
                        vb[0] = acc;
                        vb[1] = zm;
                    }
                    if (!ex.allreduce(vb, opsb)) return;
                    const Acc rrn = vb[0];
                    zinf = vb[1];
                    if (!isfinite((double)rrn)) { status = kErrDiverged; break; }
                    if (rrn <= eps2 * rr0 || it >= a.max_inner) break;
                    beta = rrn / rho;
                    rho = rrn;
                    first = false;
                }
                if (status == kErrDiverged) break;
            }
            itH += it;

            // ---- C0: rescale z, CGNR start (s = S'^T z^, p = s, y = 0) --------
            const int ez = (a.half && zinf > Acc(0) && isfinite((double)zinf)) ? ilogb((double)zinf) : 0;
            const Acc scz = (Acc)ldexp(1.0, -ez);
            Acc c0[2] = {0, 0};
            const int opsc[2] = {kSum, kSum};
            {
                const T *z = a.z;
                auto fz = [&](int64_t j) -> Acc { return P::rnd(P::mul(P::ld(z[j]), scz)); };
                Acc acc0 = 0, acc1 = 0;
                for (int64_t i = t0; i < n; i += nt) {
                    Acc rs = fz(i);
                    a.rsA[i] = P::st(rs);
                    Acc si = P::rnd(op.row(kOpST, i, fz));
                    a.s[i] = P::st(si);
                    a.pA[i] = P::st(si);
                    a.y[i] = P::st(Acc(0));
                    acc0 = P::add(acc0, P::mul(rs, rs));
                    acc1 = P::add(acc1, P::mul(si, si));
                }
                c0[0] = acc0;
                c0[1] = acc1;
            }
            if (!ex.allreduce(c0, opsc)) return;
            const Acc rr0s = c0[0];

            // ---- CGNR on S' ------------------------------------------------------
            it = 0;
            if (rr0s > Acc(0)) {
                ++spmv;
                T *pc = a.pA, *pn = a.pB, *rsc = a.rsA, *rsn = a.rsB;
                Acc gam = c0[1], beta = 0;
                bool first = true;
                for (;;) {
                    // A: p <- s + beta p (fused), q = S' p, <q, q>
                    Acc u[1] = {0};
                    {
                        Acc acc = 0;
                        if (first) {
                            auto fp = [&](int64_t j) -> Acc { return P::ld(pc[j]); };
                            for (int64_t i = t0; i < n; i += nt) {
                                Acc qi = P::rnd(op.row(kOpS, i, fp));
                                a.q[i] = P::st(qi);
                                acc = P::add(acc, P::mul(qi, qi));
                            }
                        } else {
                            const T *s = a.s;
                            auto fp = [&](int64_t j) -> Acc {
                                return P::rnd(P::add(P::ld(s[j]), P::mul(beta, P::ld(pc[j]))));
                            };
                            for (int64_t i = t0; i < n; i += nt) {
                                pn[i] = P::st(fp(i));
                                Acc qi = P::rnd(op.row(kOpS, i, fp));
                                a.q[i] = P::st(qi);
                                acc = P::add(acc, P::mul(qi, qi));
                            }
                        }
                        u[0] = acc;
                    }
                    if (!ex.allreduce(u, ops1)) return;
                    if (!first) { T *t = pc; pc = pn; pn = t; }
                    ++it;
                    ++spmv;
                    const Acc qq = u[0];
                    if (!(qq > Acc(0)) || !isfinite((double)qq)) { status = kErrDiverged; break; }
                    const Acc ac = gam / qq;
                    // B: y += ac p; rs' = rs - ac q (fused into s = S'^T rs')
                    Acc vb[2] = {0, 0};
                    {
                        const T *q = a.q;
                        const T *rcur = rsc;
                        auto frs = [&](int64_t j) -> Acc {
                            return P::rnd(P::sub(P::ld(rcur[j]), P::mul(ac, P::ld(q[j]))));
                        };
                        Acc acc0 = 0, acc1 = 0;
                        for (int64_t i = t0; i < n; i += nt) {
                            Acc yn = P::rnd(P::add(P::ld(a.y[i]), P::mul(ac, P::ld(pc[i]))));
                            a.y[i] = P::st(yn);
                            Acc rn = frs(i);
                            rsn[i] = P::st(rn);
                            Acc si = P::rnd(op.row(kOpST, i, frs));
                            a.s[i] = P::st(si);
                            acc0 = P::add(acc0, P::mul(rn, rn));
                            acc1 = P::add(acc1, P::mul(si, si));
                        }
                        vb[0] = acc0;
                        vb[1] = acc1;
                    }
                    if (!ex.allreduce(vb, opsc)) return;
                    { T *t = rsc; rsc = rsn; rsn = t; }
                    ++spmv;
                    const Acc rr = vb[0];
                    if (!isfinite((double)rr)) { status = kErrDiverged; break; }
                    if (rr <= eps2 * rr0s || it >= a.max_inner) break;
                    const Acc gn = vb[1];
                    beta = gn / gam;
                    gam = gn;
                    first = false;
                }
                if (status == kErrDiverged) break;
            }
            itS += it;

            // ---- U: x += (2-w) a 2^(e - sM + ez - sN) y (FP64) ---------------------
            const double upd = ldexp(a.pfac, e - a.sM + ez - a.sN);
            for (int64_t i = t0; i < n; i += nt)
                a.x[i] = __dadd_rn(a.x[i], __dmul_rn(upd, (double)P::ld(a.y[i])));
            if (!ex.sync()) return;
            ++k;
        }
    }
    if (lead) {
        Ctl *c = a.ctl;
        c->status = status;
        c->outer_iters = k;
        c->itH = itH;
        c->itS = itS;
        c->spmv = spmv;
        c->eta = eta;
        c->res = res;
        c->r0 = r0;
    }
}

// One operator application y = K x (kernel-level tests, bandwidth runs).
template <class Op, class T>
__global__ void gadi_apply_kernel(const Op op, int which, const void *xv, void *yv)
{
    using P = Prec<T>;
    const int64_t n = op.n;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    if (which == kOpA) {
        const double *x = (const double *)xv;
        double *y = (double *)yv;
        for (int64_t i = t0; i < n; i += nt) y[i] = op.rowA(i, [&](int64_t j) { return x[j]; });
        return;
    }
    const T *x = (const T *)xv;
    T *y = (T *)yv;
    auto f = [&](int64_t j) { return P::ld(x[j]); };
    for (int64_t i = t0; i < n; i += nt) y[i] = P::st(op.row(which, i, f));
}

}  // namespace gadi
