// gadi_solve.cuh -- the persistent GADI-IR solve kernel (Algorithm 1).
//
// One cooperative launch runs the whole solve: the outer refinement loop
// and both inner Krylov solves. Phases over the rows are separated by the
// grid all-reduce of gadi_device.cuh (bounded waits); all blocks hold
// identical scalars, so they take identical branches and the Krylov scalars
// never leave the device.
//
// Outer step k:
//   R   r = b - A x in FP64; ||r||_inf, ||r||_2^2, ||x||_inf; stopping test;
//       the round-to-odd FP32 copy of r (FP16 and FP8 inner paths)
//   D   e = floor(log2 ||r||_inf), r^ = fl_r(2^-e r) (§2.2: r^ = fl_r(s^));
//       CG start u = H' r^
//   CG  on H' = 2^-sM (aI + M): z ~ H'^-1 r^              (Alg. 1 step 2)
//   C0  ez = floor(log2 ||z||_inf), z^ = 2^-ez z, s = S'^T z^
//   CGNR on S' = 2^-sN (aI + N): y ~ S'^-1 z^            (Alg. 1 step 3)
//       each second pass also forms x + (2-w) a 2^(e - sM + ez - sN) y in
//       FP64 into the other iterate buffer (Alg. 1 step 4); after the last
//       pass that buffer holds the new iterate
// With FP64 inner precision the scales are all 2^0.
//
// CG is the single-reduction (Chronopoulos-Gear) form: one exchange per
// iteration; the residual update is recomputed at the neighbours inside the
// operator application, so r_{i+1} and u_{i+1} = H' r_{i+1} come out of one
// pass. CGNR (CG on S'^T S') needs two exchanges per iteration; its
// search-direction and residual updates are fused into the products the
// same way.
//
// A pass visits its rows in items of R consecutive rows of an x-line, taken
// grid-stride; with the ZMarchOp family (3D constant-coefficient stencil,
// 8-row items) the R, D, C0 and CGNR-A passes instead walk z-columns of
// items (zmarch_items below), which forms the same rows from the same
// terms in the same order.
#pragma once

#include <type_traits>

#include "gadi_ops.cuh"

namespace gadi {

template <class Op, class T>
struct SolveArgs {
    Op op;
    int64_t n, nitems;
    const double *b;
    double *x;                   // in: x0, out: the result
    double *x2;                  // n doubles: the iterates alternate between x and x2
    double *r64;
    float *r32;                  // n floats: round-to-odd copy of r (FP16 / FP8 inner paths)
    T *v[9];                     // inner work vectors, n elements each
    double anorm, bnorm, tol, eps, pfac;
    int sM, sN, stop_kind;
    int half;                    // inner precision below FP64: r and z scaled by powers of two
    int naive;                   // unscaled FP16 mode: no 2^-e, 2^-ez; (2-w) a applied to z in FP16
    int max_inner, max_outer;
    Ctl *ctl;
    double *part;                // [2][kMaxSlots][gridDim] partial sums
    double *eta_hist;            // optional, max_outer + 1 entries
    const long long *race_bound; // optional (batched sweeps): stop once spmv exceeds it
    unsigned long long wait_ns;
    unsigned extra;
    int zlen;                    // z-marching operator family: planes per column segment
};

// ---------------------------------------------------------------------------
// z-marching traversal of the 8-row items (3D constant-coefficient FP16
// stencil, operator family ZMarchOp). A unit of work is one column of items
// (the 8-row chunk of an x-line at fixed y) over zlen consecutive planes;
// thread t takes units t, t + nt, ... The values of the expression f at
// planes z-1, z, z+1 come from the march (the raw chunk of plane z+2 is
// requested while plane z is worked on), so only the y neighbours and the x
// ends are loaded per plane; the pass's own vectors (loader O) are requested
// one plane ahead. work(it, zc, z, c, zl, zu, own) forms the rows of item
// it; the passes' work objects below keep their partial sums as members.
// The residual, demotion, CGNR-start and CGNR pass A march; the CG pass and
// CGNR pass B, which read five and three vectors of their own per row and
// write five and four, measured faster as grid-stride items (192^3: CG pass
// 29.2 against 31.2 us, pass B 40.6 against 44.7 us), and stay so.
// ---------------------------------------------------------------------------
struct OwnNone {
    struct Raw {};
    __device__ __forceinline__ void load8(int64_t, Raw &) const {}
};

template <class Op, class F, class O, class Work>
__device__ __forceinline__ void zmarch_items(const Op &op, int zlen, int64_t t0, int64_t nt, const F &f,
                                             const O &own, Work &work)
{
    using V = typename F::Val;
    const int N = op.N, last = N - 1;
    const int64_t cols = (int64_t)(N / 8) * N;
    const int nseg = (N + zlen - 1) / zlen;
    const int64_t units = cols * nseg;
    for (int64_t u = t0; u < units; u += nt) {
        const int64_t col = u % cols;
        const int z0 = (int)(u / cols) * zlen, z1 = min(N, z0 + zlen);
        const auto zc = op.zcol(col);
        typename F::Raw fr{};
        typename O::Raw ocur{}, onext{};
        V zl[8], c[8], zu[8];
        if (z0 > 0) {
            f.load8((col + (int64_t)(z0 - 1) * cols) * 8, fr);
            f.eval8(fr, zl);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) zl[k] = V(0);
        }
        f.load8((col + (int64_t)z0 * cols) * 8, fr);
        f.eval8(fr, c);
        if (z0 < last) f.load8((col + (int64_t)(z0 + 1) * cols) * 8, fr);
        own.load8((col + (int64_t)z0 * cols) * 8, ocur);
        for (int z = z0; z < z1; ++z) {
            if (z < last) {
                f.eval8(fr, zu);
            } else {
#pragma unroll
                for (int k = 0; k < 8; ++k) zu[k] = V(0);
            }
            if (z + 2 <= last && z + 1 < z1) f.load8((col + (int64_t)(z + 2) * cols) * 8, fr);
            if (z + 1 < z1) own.load8((col + (int64_t)(z + 1) * cols) * 8, onext);
            work(col + (int64_t)z * cols, zc, z, c, zl, zu, ocur);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                zl[k] = c[k];
                c[k] = zu[k];
            }
            ocur = onext;
        }
    }
}

// The passes of one outer step along the march (same arithmetic as the
// grid-stride passes of solve_body, which describes them).
template <class Op, class T>
struct ZmResid {                     // R: r = b - A x, maxima, round-to-odd copy, ||r||_2^2
    const Op *op;
    const XLoad64 *f;
    double *r64;
    float *r32;
    int last;
    bool sq32;
    float sc32;
    double lsum = 0.0;
    float lsum32 = 0.0f;
    uint64_t lmax = 0, xmax = 0;
    __device__ __forceinline__ void operator()(int64_t it, const typename Op::ZCol &zc, int zi, const double (&c)[8],
                                               const double (&zl)[8], const double (&zu)[8],
                                               const XLoad64::Raw &ob)
    {
        constexpr uint64_t kMag = 0x7FFFFFFFFFFFFFFFull;
        double bb[8], rr[8];
        cvt8(ob.v, bb);
        op->resid_zm(it, *f, zc, zi > 0, zi < last, c, zl, zu, bb, rr);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            lmax = umax64(lmax, bits_of(rr[q]) & kMag);
            xmax = umax64(xmax, bits_of(c[q]) & kMag);
        }
        ItemIO64<8>::st(r64, it, rr);
        if constexpr (kDemoteFromOdd<T>) {
            float ro[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) ro[q] = __uint_as_float(float_bits_round_odd(rr[q]));
            stv<8>(r32, it * 8, ro);
            if (sq32) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float t = __fmul_rn(ro[q], sc32);
                    lsum32 = __fmaf_rn(t, t, lsum32);
                }
            }
        }
        if (!sq32) {
#pragma unroll
            for (int q = 0; q < 8; ++q) lsum = __fma_rn(rr[q], rr[q], lsum);
        }
    }
};

template <class Op, class T, class F>
struct ZmDemote {                    // D: r^ = fl(2^-e r), u = H' r^, z = 0
    using Acc = typename Prec<T>::Acc;
    using P = Prec<T>;
    const Op *op;
    const F *f;
    T *rc, *uc, *z;
    int last;
    Acc l0 = 0, l1 = 0;
    __device__ __forceinline__ void operator()(int64_t it, const typename Op::ZCol &zc, int zi, const Acc (&c)[8],
                                               const Acc (&zl)[8], const Acc (&zu)[8], const OwnNone::Raw &)
    {
        Acc uu[8], zz[8];
        op->rows_zm(kOpH, it, *f, zc, zi > 0, zi < last, c, zl, zu, uu);
        P::rndv(uu);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            zz[q] = Acc(0);
            l0 = P::madd(l0, c[q], c[q]);
            l1 = P::madd(l1, uu[q], c[q]);
        }
        ItemIO<T, 8>::st(rc, it, c);
        ItemIO<T, 8>::st(uc, it, uu);
        ItemIO<T, 8>::st(z, it, zz);
    }
};

template <class Op, class T, class F>
struct ZmC0 {                        // C0: z^ = 2^-ez z, s = S'^T z^, p = s, y = 0
    using Acc = typename Prec<T>::Acc;
    using P = Prec<T>;
    const Op *op;
    const F *f;
    T *rsc, *s, *pc, *y;
    int last;
    Acc l0 = 0, l1 = 0;
    __device__ __forceinline__ void operator()(int64_t it, const typename Op::ZCol &zc, int zi, const Acc (&c)[8],
                                               const Acc (&zl)[8], const Acc (&zu)[8], const OwnNone::Raw &)
    {
        Acc ss[8], yy[8];
        op->rows_zm(kOpST, it, *f, zc, zi > 0, zi < last, c, zl, zu, ss);
        P::rndv(ss);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            yy[j] = Acc(0);
            l0 = P::madd(l0, c[j], c[j]);
            l1 = P::madd(l1, ss[j], ss[j]);
        }
        ItemIO<T, 8>::st(rsc, it, c);
        ItemIO<T, 8>::st(s, it, ss);
        ItemIO<T, 8>::st(pc, it, ss);
        ItemIO<T, 8>::st(y, it, yy);
    }
};

template <class Op, class T, class F>
struct ZmCgnrA {                     // CGNR pass A: p = s + be p (stored unless first), q = S' p
    using Acc = typename Prec<T>::Acc;
    using P = Prec<T>;
    const Op *op;
    const F *f;
    T *pn, *q;
    bool store_p;
    int last;
    Acc l0 = 0;
    __device__ __forceinline__ void operator()(int64_t it, const typename Op::ZCol &zc, int zi, const Acc (&c)[8],
                                               const Acc (&zl)[8], const Acc (&zu)[8], const OwnNone::Raw &)
    {
        Acc qq[8];
        if (store_p) ItemIO<T, 8>::st(pn, it, c);
        op->rows_zm(kOpS, it, *f, zc, zi > 0, zi < last, c, zl, zu, qq);
        P::rndv(qq);
#pragma unroll
        for (int j = 0; j < 8; ++j) l0 = P::madd(l0, qq[j], qq[j]);
        ItemIO<T, 8>::st(q, it, qq);
    }
};

// status of a solve stopped by race_bound (reported as not converged)
constexpr int kRacedOut = 100;

// launch bound: 1024 threads for one-row items, 512 for 4- and 8-row items
// (whose per-thread state is larger: an item holds all its neighbour chunks
// at once). For 8-row items 512 threads cap the registers at 128 and the
// compiler keeps some values in local memory, yet the extra warps hide more
// memory latency: measured at 192^3, 0.178 s with 384 threads (168
// registers) against 0.167 s with 512.
template <class Op>
__host__ __device__ constexpr int max_threads() { return Op::R > 1 ? 512 : 1024; }

// The solve, run by a team of threads: the whole grid (ex.block_only false,
// t0/nt the global thread index and count) or one block (ex.block_only true,
// t0/nt the block's). lead is the one thread that writes the results.
template <class Op, class T, class Ex>
__device__ __forceinline__ void solve_body(const SolveArgs<Op, T> &a, Ex &ex, const int64_t t0,
                                           const int64_t nt, const bool lead)
{
    using P = Prec<T>;
    using Acc = typename P::Acc;
    constexpr int R = Op::R;
    using IO = ItemIO<T, R>;
    using IO64 = ItemIO64<R>;
    const int64_t items = a.nitems;
    const Op &op = a.op;
    const Acc eps2 = (Acc)(a.eps * a.eps);
    const int ops1[1] = {kSum};
    const int ops2[2] = {kSum, kSum};
    const int ops3[3] = {kSum, kSum, kMax};

    // work vectors: CG uses r (2), u (2), s (2), p, z; CGNR reuses them
    T *const z = a.v[8];

    double r0 = 0.0, best = INFINITY, eta = 0.0, res = 0.0, rinf_prev = 0.0;
    long long itH = 0, itS = 0, spmv = 0;
    int k = 0, status = kErrNotConverged;
    double *xcur = a.x;              // the buffer holding the current iterate

    for (;;) {
        // ---- R: outer residual in FP64 -----------------------------------------
        double vR[3] = {0.0, 0.0, 0.0};
        // ||r||_2^2 in FP64, or (FP16 / FP8 inner paths stopping on eta_inf,
        // where ||r||_2 only watches for growth and gives RES for the
        // record; from the second step on) in FP32 from the round-to-odd
        // copy scaled by 2^-esq, esq the exponent of the previous ||r||_inf,
        // so that the squares stay far inside FP32's range
        const bool sq32 = kDemoteFromOdd<T> && a.stop_kind != 1 && k > 0;
        const int esq = rinf_prev > 0.0 ? ilogb(rinf_prev) : 0;
        {
            // r = b - A x with each product subtracted by a fused
            // multiply-add (7 FP64 operations per 7-point row: GB300 issues
            // FP64 at 2 lanes per clock per SM, so this pass is bound by the
            // FP64 rate); the maxima of |r| and |x| as integer maxima of the
            // magnitudes' bit patterns (same value for finite inputs; FP64
            // compares issue at the FP64 rate, integer ones at the integer
            // rate)
            double lsum = 0.0;
            float lsum32 = 0.0f;
            const float sc32 = ldexpf(1.0f, -max(-126, min(126, esq)));
            uint64_t lmax = 0, xmax = 0;
            constexpr uint64_t kMag = 0x7FFFFFFFFFFFFFFFull;
            const XLoad64 fx{xcur};
            if constexpr (Op::kZMarch) {
                ZmResid<Op, T> w{&op, &fx, a.r64, a.r32, op.N - 1, sq32, sc32};
                zmarch_items(op, a.zlen, t0, nt, fx, XLoad64{a.b}, w);
                lsum = w.lsum;
                lsum32 = w.lsum32;
                lmax = w.lmax;
                xmax = w.xmax;
            } else
            for (int64_t it = t0; it < items; it += nt) {
                double bb[R], xx[R], rr[R];
                IO64::ld(a.b, it, bb);
                IO64::ld(xcur, it, xx);
                op.resid(it, fx, bb, rr);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    lmax = umax64(lmax, bits_of(rr[q]) & kMag);
                    xmax = umax64(xmax, bits_of(xx[q]) & kMag);
                }
                IO64::st(a.r64, it, rr);
                if constexpr (kDemoteFromOdd<T>) {
                    float ro[R];
#pragma unroll
                    for (int q = 0; q < R; ++q) ro[q] = __uint_as_float(float_bits_round_odd(rr[q]));
                    if constexpr (R > 1) stv<R>(a.r32, it * R, ro);
                    else a.r32[it] = ro[0];
                    if (sq32) {
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            const float t = __fmul_rn(ro[q], sc32);
                            lsum32 = __fmaf_rn(t, t, lsum32);
                        }
                    }
                }
                if (!sq32) {
#pragma unroll
                    for (int q = 0; q < R; ++q) lsum = __fma_rn(rr[q], rr[q], lsum);
                }
            }
            vR[0] = sq32 ? (double)lsum32 : lsum;
            vR[1] = double_of(lmax);
            vR[2] = double_of(xmax);
        }
        {
            const int opsR[3] = {kSum, kMax, kMax};
            if (!ex.allreduce(vR, opsR)) return;
        }
        ++spmv;
        const double rinf = vR[1], xinf = vR[2];
        const double rn2 = sq32 ? ldexp(sqrt(vR[0]), max(-126, min(126, esq))) : sqrt(vR[0]);
        rinf_prev = rinf;
        const double den = __dadd_rn(__dmul_rn(a.anorm, xinf), a.bnorm);   // as written, not fused
        eta = den > 0.0 ? rinf / den : (rinf == 0.0 ? 0.0 : INFINITY);
        if (k == 0) r0 = rn2;
        res = r0 > 0.0 ? rn2 / r0 : 0.0;
        if (lead && a.eta_hist) a.eta_hist[k] = eta;
        {
            bool done = true;
            if (!isfinite(rn2) || !isfinite(eta) || !isfinite(xinf)) status = kErrDiverged;
            else {
                if (rn2 < best) best = rn2;
                const double crit = a.stop_kind == 1 ? res : eta;
                if (crit <= a.tol) status = kOk;
                else if (rn2 > 1e3 * best) status = kErrDiverged;
                else if (k >= a.max_outer) status = kErrNotConverged;
                else done = false;
            }
            if (done) break;
        }

        // ---- D: r^ = fl_r(2^-e r), u = H' r^, z = 0 (CG start) ----------------
        const int e = (a.half && !a.naive && rinf > 0.0) ? ilogb(rinf) : 0;
        T *rc = a.v[0], *rn = a.v[1], *uc = a.v[2], *un = a.v[3];
        T *sc = a.v[4], *sn = a.v[5], *p = a.v[6];
        // g[2]: a raced-out flag (batched sweeps): thread 0 of every block
        // reads the bound, and the maximum over the team makes the decision
        // the same in every block
        Acc g[3] = {0, 0, 0};
        if (a.race_bound && threadIdx.x == 0 && spmv > *(const volatile long long *)a.race_bound) g[2] = Acc(1);
        auto d_pass = [&](const auto &fr) {
            Acc l0 = 0, l1 = 0;
            for (int64_t it = t0; it < items; it += nt) {
                Acc rr[R], uu[R], zz[R];
                op.rows(kOpH, it, fr, uu);
                if constexpr (R > 1) fr.template many<R>(it * R, rr);
                else rr[0] = fr.one(it);
                P::rndv(uu);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    zz[q] = Acc(0);
                    l0 = P::madd(l0, rr[q], rr[q]);
                    l1 = P::madd(l1, uu[q], rr[q]);
                }
                IO::st(rc, it, rr);
                IO::st(uc, it, uu);
                IO::st(z, it, zz);
            }
            g[0] = l0;
            g[1] = l1;
        };
        if constexpr (Op::kZMarch) {
            if (e >= -100 && e <= 126) {
                const XDemoteOdd<T> fr{a.r32, ldexpf(1.0f, -e)};
                ZmDemote<Op, T, XDemoteOdd<T>> w{&op, &fr, rc, uc, z, op.N - 1};
                zmarch_items(op, a.zlen, t0, nt, fr, OwnNone{}, w);
                g[0] = w.l0;
                g[1] = w.l1;
            } else {
                const XDemote<T> fr{a.r64, ldexp(1.0, -e)};
                ZmDemote<Op, T, XDemote<T>> w{&op, &fr, rc, uc, z, op.N - 1};
                zmarch_items(op, a.zlen, t0, nt, fr, OwnNone{}, w);
                g[0] = w.l0;
                g[1] = w.l1;
            }
        } else if constexpr (kDemoteFromOdd<T>) {
            // from the round-to-odd FP32 copy where that is exact, else from FP64
            if (e >= -100 && e <= 126) d_pass(XDemoteOdd<T>{a.r32, ldexpf(1.0f, -e)});
            else d_pass(XDemote<T>{a.r64, ldexp(1.0, -e)});
        } else {
            d_pass(XDemote<T>{a.r64, ldexp(1.0, -e)});
        }
        {
            const int opsD[3] = {kSum, kSum, kMax};
            if (!ex.allreduce(g, opsD)) return;
        }
        if (g[2] > Acc(0)) { status = kRacedOut; break; }
        ++spmv;
        const Acc gam0 = g[0];

        // ---- CG on H' (single reduction per iteration) -----------------------------
        Acc zinf = 0;
        int it_cg = 0;
        if (gam0 > Acc(0)) {
            Acc gam = gam0, del = g[1];
            if (!(del > Acc(0)) || !isfinite((double)del)) { status = kErrDiverged; break; }
            Acc al = gam / del, be = 0;
            bool first = true;
            for (;;) {
                // p = r + be p; s = u + be s; z += al p; r' = r - al s; u' = H' r'
                // (on the first iteration p = r, s = u, and the previous s is not read)
                Acc w3[3] = {0, 0, 0};
                auto cg_pass = [&](const auto &frn) {
                    Acc l0 = 0, l1 = 0, zm = 0;
                    for (int64_t it = t0; it < items; it += nt) {
                        Acc r_[R], u_[R], p_[R], s_[R], z_[R], rnew[R], unew[R];
                        IO::ld(rc, it, r_);
                        IO::ld(uc, it, u_);
                        IO::ld(z, it, z_);
                        if (first) {
#pragma unroll
                            for (int q = 0; q < R; ++q) { p_[q] = r_[q]; s_[q] = u_[q]; }
                        } else {
                            IO::ld(p, it, p_);
                            IO::ld(sc, it, s_);
                            P::madd_s(p_, r_, be, p_);
                            P::madd_s(s_, u_, be, s_);
                            P::rndv(p_);
                            P::rndv(s_);
                        }
                        op.rows(kOpH, it, frn, unew);
                        P::madd_s(z_, z_, al, p_);
                        P::madd_s(rnew, r_, -al, s_);
                        P::rndv(z_);
                        P::rndv(rnew);
                        P::rndv(unew);
#pragma unroll
                        for (int q = 0; q < R; ++q) {
                            l0 = P::madd(l0, rnew[q], rnew[q]);
                            l1 = P::madd(l1, unew[q], rnew[q]);
                            zm = fmax(zm, fabs(z_[q]));
                        }
                        IO::st(p, it, p_);
                        IO::st(sn, it, s_);
                        IO::st(z, it, z_);
                        IO::st(rn, it, rnew);
                        IO::st(un, it, unew);
                    }
                    w3[0] = l0;
                    w3[1] = l1;
                    w3[2] = zm;
                };
                if (first) {
                    cg_pass(XAxpy<T>{rc, uc, -al});
                } else {
                    cg_pass(XAxpy2<T>{rc, uc, sc, al, be});
                }
                if (!ex.allreduce(w3, ops3)) return;
                ++it_cg;
                ++spmv;
                { T *t = rc; rc = rn; rn = t; }
                { T *t = uc; uc = un; un = t; }
                { T *t = sc; sc = sn; sn = t; }
                const Acc gn = w3[0], dn = w3[1];
                zinf = w3[2];
                if (!isfinite((double)gn) || !isfinite((double)dn)) { status = kErrDiverged; break; }
                if (gn <= eps2 * gam0 || it_cg >= a.max_inner) break;
                const Acc bn = gn / gam;
                const Acc den2 = dn - bn * gn / al;
                if (!(den2 > Acc(0))) { status = kErrDiverged; break; }
                al = gn / den2;
                be = bn;
                gam = gn;
                first = false;
            }
            if (status == kErrDiverged) break;
        }
        itH += it_cg;

        // ---- C0: ez, z^ = 2^-ez z, s = S'^T z^, p = s, y = 0 (CGNR start) -------
        const int ez = (a.half && !a.naive && zinf > Acc(0) && isfinite((double)zinf)) ? ilogb((double)zinf) : 0;
        T *rsc = a.v[0], *rsn = a.v[1], *s = a.v[2], *pc = a.v[3], *pn = a.v[4], *q = a.v[5], *y = a.v[6];
        Acc c0[2] = {0, 0};
        {
            // z^ = 2^-ez z; unscaled mode: (2-w) a z formed in the inner precision
            const XScale<T> fz{z, a.naive ? (Acc)a.pfac : (Acc)ldexp(1.0, -ez)};
            Acc l0 = 0, l1 = 0;
            if constexpr (Op::kZMarch) {
                ZmC0<Op, T, XScale<T>> w{&op, &fz, rsc, s, pc, y, op.N - 1};
                zmarch_items(op, a.zlen, t0, nt, fz, OwnNone{}, w);
                l0 = w.l0;
                l1 = w.l1;
            } else
            for (int64_t it = t0; it < items; it += nt) {
                Acc rs[R], ss[R], yy[R];
                if constexpr (R > 1) fz.template many<R>(it * R, rs);
                else rs[0] = fz.one(it);
                op.rows(kOpST, it, fz, ss);
                P::rndv(ss);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    yy[j] = Acc(0);
                    l0 = P::madd(l0, rs[j], rs[j]);
                    l1 = P::madd(l1, ss[j], ss[j]);
                }
                IO::st(rsc, it, rs);
                IO::st(s, it, ss);
                IO::st(pc, it, ss);
                IO::st(y, it, yy);
            }
            c0[0] = l0;
            c0[1] = l1;
        }
        if (!ex.allreduce(c0, ops2)) return;
        const Acc rr0s = c0[0];

        // ---- CGNR on S' ----------------------------------------------------------
        // Every B pass also forms the candidate update (Alg. 1 step 4, FP64)
        //   x_next = x + (2-w) a 2^(e - sM + ez - sN) y
        // for its own rows; after the last pass x_next is the new iterate, so
        // no separate update pass and grid synchronisation are needed.
        const double upd = a.naive ? 1.0 : ldexp(a.pfac, e - a.sM + ez - a.sN);
        double *const xnext = xcur == a.x ? a.x2 : a.x;
        int it_s = 0;
        if (rr0s > Acc(0)) {
            ++spmv;
            Acc gam = c0[1], be = 0;
            bool first = true;
            for (;;) {
                // A: p = s + be p (fused), q = S' p, <q, q>
                Acc u1[1] = {0};
                {
                    Acc l0 = 0;
                    if constexpr (Op::kZMarch) {
                        if (first) {
                            const XLoad<T> fp{pc};
                            ZmCgnrA<Op, T, XLoad<T>> w{&op, &fp, pn, q, false, op.N - 1};
                            zmarch_items(op, a.zlen, t0, nt, fp, OwnNone{}, w);
                            l0 = w.l0;
                        } else {
                            const XAxpy<T> fp{s, pc, be};
                            ZmCgnrA<Op, T, XAxpy<T>> w{&op, &fp, pn, q, true, op.N - 1};
                            zmarch_items(op, a.zlen, t0, nt, fp, OwnNone{}, w);
                            l0 = w.l0;
                        }
                    } else if (first) {
                        const XLoad<T> fp{pc};
                        for (int64_t it = t0; it < items; it += nt) {
                            Acc qq[R];
                            op.rows(kOpS, it, fp, qq);
                            P::rndv(qq);
#pragma unroll
                            for (int j = 0; j < R; ++j) l0 = P::madd(l0, qq[j], qq[j]);
                            IO::st(q, it, qq);
                        }
                    } else {
                        const XAxpy<T> fp{s, pc, be};
                        for (int64_t it = t0; it < items; it += nt) {
                            Acc pp[R], qq[R];
                            if constexpr (R > 1) fp.template many<R>(it * R, pp);
                            else pp[0] = fp.one(it);
                            IO::st(pn, it, pp);
                            op.rows(kOpS, it, fp, qq);
                            P::rndv(qq);
#pragma unroll
                            for (int j = 0; j < R; ++j) l0 = P::madd(l0, qq[j], qq[j]);
                            IO::st(q, it, qq);
                        }
                    }
                    u1[0] = l0;
                }
                if (!ex.allreduce(u1, ops1)) return;
                if (!first) { T *t = pc; pc = pn; pn = t; }
                ++it_s;
                ++spmv;
                const Acc qq = u1[0];
                if (!(qq > Acc(0)) || !isfinite((double)qq)) { status = kErrDiverged; break; }
                const Acc ac = gam / qq;
                // B: y += ac p; rs' = rs - ac q; s = S'^T rs' (rs' recomputed at the neighbours)
                Acc vb[2] = {0, 0};
                {
                    const XAxpy<T> frs{rsc, q, -ac};
                    Acc l0 = 0, l1 = 0;
                    for (int64_t it = t0; it < items; it += nt) {
                        Acc yy[R], pp[R], rn_[R], ss[R];
                        double xx[R];
                        IO::ld(y, it, yy);
                        IO::ld(pc, it, pp);
                        IO64::ld(xcur, it, xx);
                        if constexpr (R > 1) frs.template many<R>(it * R, rn_);
                        else rn_[0] = frs.one(it);
                        op.rows(kOpST, it, frs, ss);
                        P::madd_s(yy, yy, ac, pp);
                        P::rndv(yy);
                        P::rndv(ss);
#pragma unroll
                        for (int j = 0; j < R; ++j) xx[j] = __fma_rn(upd, P::to64(yy[j]), xx[j]);
                        IO64::st(xnext, it, xx);
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            l0 = P::madd(l0, rn_[j], rn_[j]);
                            l1 = P::madd(l1, ss[j], ss[j]);
                        }
                        IO::st(y, it, yy);
                        IO::st(rsn, it, rn_);
                        IO::st(s, it, ss);
                    }
                    vb[0] = l0;
                    vb[1] = l1;
                }
                if (!ex.allreduce(vb, ops2)) return;
                { T *t = rsc; rsc = rsn; rsn = t; }
                ++spmv;
                const Acc rr = vb[0];
                if (!isfinite((double)rr)) { status = kErrDiverged; break; }
                if (rr <= eps2 * rr0s || it_s >= a.max_inner) break;
                const Acc gn = vb[1];
                be = gn / gam;
                gam = gn;
                first = false;
            }
            if (status == kErrDiverged) break;
            xcur = xnext;            // (no CGNR step: y = 0 and x stays)
        }
        itS += it_s;

        ++k;
    }
    // the result belongs in x: copy the own items when the last iterate is in x2
    if (xcur != a.x)
        for (int64_t it = t0; it < items; it += nt) {
            double xx[R];
            IO64::ld(xcur, it, xx);
            IO64::st(a.x, it, xx);
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

template <class Op, class T>
__global__ void __launch_bounds__(max_threads<Op>(), 1) gadi_solve_kernel(const SolveArgs<Op, T> a)
{
    // one batch of partial loads covers 160 blocks (152 SMs) where registers allow
    GridExchangeT<(max_threads<Op>() >= 1024 ? 4 : 5)> ex{a.ctl, a.part, 0u, a.wait_ns, a.extra, false};
    solve_body(a, ex, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
               blockIdx.x == 0 && threadIdx.x == 0);
}

// One operator application y = K x (kernel-level tests, bandwidth runs).
template <class Op, class T>
__device__ __forceinline__ void apply_body(const Op &op, int64_t nitems, int which, const void *xv, void *yv)
{
    using P = Prec<T>;
    using Acc = typename P::Acc;
    constexpr int R = Op::R;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (int64_t)gridDim.x * blockDim.x;
    if (which == kOpA) {
        const XLoad64 f{(const double *)xv};
        for (int64_t it = t0; it < nitems; it += nt) {
            double o[R];
            op.rowsA(it, f, o);
            ItemIO64<R>::st((double *)yv, it, o);
        }
        return;
    }
    const XLoad<T> f{(const T *)xv};
    for (int64_t it = t0; it < nitems; it += nt) {
        Acc o[R];
        op.rows(which, it, f, o);
        ItemIO<T, R>::st((T *)yv, it, o);
    }
}

template <class Op, class T>
__global__ void gadi_apply_kernel(const Op op, int64_t nitems, int which, const void *xv, void *yv)
{
    apply_body<Op, T>(op, nitems, which, xv, yv);
}

// The same for 8-row stencil items, which hold all their neighbour chunks
// at once: at most 128 registers, so that two 256-thread blocks share an SM.
template <class Op, class T>
__global__ void __maxnreg__(128) gadi_apply_kernel_wide(const Op op, int64_t nitems, int which, const void *xv,
                                                        void *yv)
{
    apply_body<Op, T>(op, nitems, which, xv, yv);
}

__device__ __forceinline__ void half8_to_float(const uint4 &u, float (&o)[8])
{
    const __half2 *h = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __half22float2(h[k]);
        o[2 * k] = f.x;
        o[2 * k + 1] = f.y;
    }
}

// 16-byte asynchronous copy global -> shared (cp.async, bypassing L1) and
// its group bookkeeping
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Operator application for the constant-coefficient 3D stencil with FP16
// vectors and 8-row items, staged through shared memory. A block owns ty
// consecutive y-lines (all nx8 = N/8 chunks of each, one thread per chunk)
// for a segment of zlen planes and streams the planes through a ring of S
// shared-memory slots: each slot holds the block's ty lines of one plane
// plus the y-lines just below and above them (halo), copied with 16-byte
// cp.async by the threads that own them (threads of rows 0 and 1 copy the
// two halo lines). Planes z-1, z, z+1 are read from the ring while S-4
// later planes are in flight, so the block keeps (S-3) x (ty+2) x nx8 x 16
// bytes requested without holding them in registers; a thread's own chunk
// of planes z-1 and z stays converted in registers from the previous plane,
// so a plane costs three chunk conversions (z+1 and the two y neighbours). Each row is formed
// with the terms of StencilOp::rows in the same order, so the result is
// bit for bit that of gadi_apply_kernel. Shared memory: S (ty+2) nx8 16 B.
template <class Op, int S>
__global__ void __launch_bounds__(512, 2) gadi_apply_staged_kernel(const Op op, int which, int ty, int zlen,
                                                                   const __half *x, __half *y)
{
    static_assert(Op::kDim == 3 && Op::R == 8 && S >= 4, "3D stencil with 8-row items");
    using P = Prec<__half>;
    constexpr int R = 8;
    extern __shared__ uint4 ring[];
    const int N = op.N, nx8 = N / R, last = N - 1;
    const int64_t NN = (int64_t)N * N;
    const int ytiles = N / ty;
    const int y0 = (int)(blockIdx.x % ytiles) * ty;
    const int z0 = (int)(blockIdx.x / ytiles) * zlen;
    const int z1 = min(N, z0 + zlen);
    const int cx = (int)threadIdx.x % nx8, r = (int)threadIdx.x / nx8;   // blockDim.x = nx8 * ty
    const int yy = y0 + r;
    const int lines = ty + 2;
    // copies of plane zp (planes z0-1 .. z1 inside the grid are needed)
    auto load_plane = [&](int zp) {
        if (zp < 0 || zp > last || zp > z1) return;
        uint4 *slot = ring + (size_t)((zp + 1 - z0) % S) * lines * nx8;
        const __half *row = x + (int64_t)zp * NN + (int64_t)yy * N + cx * R;
        cp_async16(slot + (r + 1) * nx8 + cx, row);
        if (r == 0 && y0 > 0) cp_async16(slot + cx, row - N);                                    // y0 - 1
        if (r == 1 && y0 + ty <= last) cp_async16(slot + (ty + 1) * nx8 + cx, row + (int64_t)(ty - 1) * N);  // y0 + ty
    };
    for (int k = 0; k < S - 1; ++k) {
        load_plane(z0 - 1 + k);
        cp_async_commit();
    }
    const bool hly = yy > 0, huy = yy < last, hxm = cx > 0, hxp = cx < nx8 - 1;
    const int plane = lines * nx8, own_off = (r + 1) * nx8 + cx;
    float zl[R], c[R];               // this thread's chunk of planes z - 1 and z, carried
    for (int z = z0; z < z1; ++z) {
        // the groups of planes up to z + 1 are complete when at most S - 4
        // of the (S - 1) + (z - z0) committed ones are pending
        cp_async_wait<S - 4>();
        __syncthreads();
        const unsigned q = (unsigned)(z - z0);
        const uint4 *pc = ring + (size_t)((q + 1u) % S) * plane;   // plane z
        const uint4 *pu = ring + (size_t)((q + 2u) % S) * plane;   // plane z + 1
        if (z == z0) {
            half8_to_float(ring[(size_t)(q % S) * plane + own_off], zl);   // plane z - 1
            half8_to_float(pc[own_off], c);
        }
        float zu[R], yl[R], yu[R], acc[R], sh[R];
        half8_to_float(pu[own_off], zu);
        half8_to_float(pc[r * nx8 + cx], yl);
        half8_to_float(pc[(r + 2) * nx8 + cx], yu);
        const __half *own = reinterpret_cast<const __half *>(pc + (own_off - cx));
        const float xm = hxm ? P::ld(own[cx * R - 1]) : 0.0f, xp = hxp ? P::ld(own[cx * R + R]) : 0.0f;
        const bool hlz = z > 0, huz = z < last;
        if (which == kOpH) {
            P::mul_s(acc, op.sigH, c);
            if (hlz) P::madd_s(acc, acc, op.h_off, zl);
            if (hly) P::madd_s(acc, acc, op.h_off, yl);
#pragma unroll
            for (int k = 0; k < R; ++k) sh[k] = k ? c[k - 1] : xm;
            P::madd_s(acc, acc, op.h_off, sh);
            P::madd_s(acc, acc, op.h_diag, c);
#pragma unroll
            for (int k = 0; k < R; ++k) sh[k] = k < R - 1 ? c[k + 1] : xp;
            P::madd_s(acc, acc, op.h_off, sh);
            if (huy) P::madd_s(acc, acc, op.h_off, yu);
            if (huz) P::madd_s(acc, acc, op.h_off, zu);
        } else {
            const float lo = which == kOpS ? -op.s_c : op.s_c;
            P::mul_s(acc, op.sigS, c);
            if (hlz) P::madd_s(acc, acc, lo, zl);
            if (hly) P::madd_s(acc, acc, lo, yl);
#pragma unroll
            for (int k = 0; k < R; ++k) sh[k] = k ? c[k - 1] : xm;
            P::madd_s(acc, acc, lo, sh);
            if (op.s_diag != 0.0f) P::madd_s(acc, acc, op.s_diag, c);
#pragma unroll
            for (int k = 0; k < R; ++k) sh[k] = k < R - 1 ? c[k + 1] : xp;
            P::madd_s(acc, acc, -lo, sh);
            if (huy) P::madd_s(acc, acc, -lo, yu);
            if (huz) P::madd_s(acc, acc, -lo, zu);
        }
        ItemIO<__half, R>::st(y, ((int64_t)z * NN + (int64_t)yy * N + cx * R) / R, acc);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            zl[k] = c[k];
            c[k] = zu[k];
        }
        __syncthreads();             // every thread is done with plane z - 1's slot
        load_plane(z + S - 2);       // into that slot
        cp_async_commit();
    }
    cp_async_wait<0>();
}

}  // namespace gadi
