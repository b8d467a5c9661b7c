/*
 * gadi_oracle.c -- plain, slow, obviously correct CPU implementation of GADI
 * and GADI-IR (arXiv 2501.04229).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library path may call, link or
 * load this file; only the tests, the smoke check and the bench's CPU
 * baseline do. It shares no code with the CUDA path.
 *
 * What it implements, and where the paper defines it:
 *   or_hss_split      M = (A+A^T)/2, N = (A-A^T)/2                 (§4.1, HSS splitting)
 *   or_spmv_shift     y = (sigma I + V) x                          (H = aI+M, S = aI+N, §1.4)
 *   or_cg             CG on the SPD system (sigma I + M) v = rhs    (inner solver, §2.2: "backward stable")
 *   or_cgnr           CG on the normal equations of (sigma I + N)   (inner solver, §2.2)
 *   or_gadi           the two-half-step GADI iteration             (eq. (gadi), §2.1)
 *   or_gadi_ir        three-precision GADI-IR                      (Algorithm 1, §2.1)
 *   or_backward_error eta_inf = ||b-Ax||_inf/(||A||_inf ||x||_inf + ||b||_inf)  (Thm 3 measure)
 *
 * Readings of the paper that this file takes (the paper is silent there):
 *   - inner solvers: CG for H = aI+M (SPD), CGNR for S = aI+N (N skew);
 *   - inner stopping: ||rhs - K v||_2 <= eps * ||rhs - K v0||_2 (relative to the
 *     inner initial residual), with an iteration cap;
 *   - residual sign r = b - Ax; start x0 given by the caller (zero in the
 *     paper's experiments);
 *   - bfloat16 inner precision: as FP16 (scaled the same way), with 8
 *     significant bits and FP32's exponent range;
 *   - FP8 E4M3 inner precision (below the paper's FP16; its future-work
 *     direction): as FP16, with 4 significant bits, largest finite value
 *     448 and saturating rounding;
 *   - FP16 inner precision ("half"): FP16 storage of matrix values and inner
 *     vectors, FP32 arithmetic; the matrix, the residual and the first
 *     correction are scaled by powers of two so that FP16 stays in range; the
 *     shift alpha is applied in FP32 and (2-omega)*alpha is folded into the
 *     FP64 update scalar. The "naive" half mode instead rounds alpha into the
 *     FP16 diagonal and scales nothing, for the paper's unscaled behaviour.
 *
 * Rounding: products are fused with their sum (C99 fma / fmaf, one rounding
 * per term) in FP64 and in the FP32 arithmetic of the low-precision modes,
 * the paper fixing only the precisions (u_f = u = double, FP32 arithmetic
 * for u_r = half); a product that starts a sum (sigma x_i) is rounded on its
 * own. Compile with -ffp-contract=off so that nothing else is fused.
 * Determinism: dot products are summed in fixed blocks of OR_BLK elements and
 * the block sums are added in order, so results do not depend on the number
 * of OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_INVALID 1
#define OR_OOM 2
#define OR_NOT_CONVERGED 5
#define OR_DIVERGED 6

#define OR_BLK 4096
/* loops over fewer elements than this run on one thread */
#define OR_PAR_MIN 32768

enum { OR_PREC_DOUBLE = 0, OR_PREC_SINGLE = 1, OR_PREC_HALF = 2, OR_PREC_HALF_NAIVE = 3, OR_PREC_BF16 = 4,
       OR_PREC_E4M3 = 5 };
enum { OR_STOP_ETA = 0, OR_STOP_RES = 1 };

typedef struct {
    double alpha, omega;     /* GADI parameters, alpha > 0, omega in [0, 2) (Thm 1) */
    double tol;              /* outer stopping tolerance on eta_inf or RES */
    double eps_inner;        /* inner relative tolerance */
    int32_t max_inner, max_outer;
    int32_t stop_kind;       /* OR_STOP_ETA or OR_STOP_RES */
    int32_t inner_prec;      /* OR_PREC_* (GADI-IR only) */
} or_params;

typedef struct {
    int32_t status, outer_iters;
    int64_t inner_iters_H, inner_iters_S, spmv_count;
    double eta_inf, res_rel, res0;
    int32_t scale_exp_M, scale_exp_N;   /* FP16 matrix scale exponents (half mode) */
} or_info;

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* FP64 vector helpers                                                 */
/* ------------------------------------------------------------------ */

static double dot64(int64_t n, const double *a, const double *b)
{
    int64_t nb = (n + OR_BLK - 1) / OR_BLK;
    double *part = (double *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(double));
    #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t k = 0; k < nb; ++k) {
        int64_t lo = k * OR_BLK, hi = lo + OR_BLK < n ? lo + OR_BLK : n;
        double s = 0.0;
        for (int64_t i = lo; i < hi; ++i) s = fma(a[i], b[i], s);
        part[k] = s;
    }
    double s = 0.0;
    for (int64_t k = 0; k < nb; ++k) s += part[k];
    free(part);
    return s;
}

static double norm_inf64(int64_t n, const double *a)
{
    double m = 0.0;
    #pragma omp parallel for reduction(max : m) schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double v = fabs(a[i]);
        if (v > m || v != v) m = (v != v) ? INFINITY : v;
    }
    return m;
}

/* y = (sigma I + V) x, V in CSR */
void or_spmv_shift(int64_t n, const int32_t *rp, const int32_t *ci, const double *v,
                   double sigma, const double *x, double *y)
{
    #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double s = sigma * x[i];
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s = fma(v[k], x[ci[k]], s);
        y[i] = s;
    }
}

/* r = b - A x */
void or_residual(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
                 const double *b, const double *x, double *r)
{
    #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s = fma(a[k], x[ci[k]], s);
        r[i] = b[i] - s;
    }
}

double or_matrix_norm_inf(int64_t n, const int32_t *rp, const double *a)
{
    double m = 0.0;
    #pragma omp parallel for reduction(max : m) schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s += fabs(a[k]);
        if (s > m) m = s;
    }
    return m;
}

/* Normwise backward error in the infinity norm (the measure of Thm 3 with the
 * b term added): ||b - Ax||_inf / (||A||_inf ||x||_inf + ||b||_inf). */
double or_backward_error(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
                         const double *b, const double *x)
{
    double *r = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    or_residual(n, rp, ci, a, b, x, r);
    double num = norm_inf64(n, r);
    double den = or_matrix_norm_inf(n, rp, a) * norm_inf64(n, x) + norm_inf64(n, b);
    free(r);
    if (den == 0.0) return num == 0.0 ? 0.0 : INFINITY;
    return num / den;
}

/* ------------------------------------------------------------------ */
/* HSS splitting (§4.1): M = (A + A^T)/2, N = (A - A^T)/2 on A's pattern */
/* ------------------------------------------------------------------ */

static int32_t find_in_row(const int32_t *rp, const int32_t *ci, int64_t row, int64_t col)
{
    int32_t lo = rp[row], hi = rp[row + 1] - 1;
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (ci[mid] == col) return mid;
        if (ci[mid] < col) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Returns OR_OK, or OR_INVALID when A's pattern is not symmetric or a row's
 * columns are not sorted ascending (then M and N are left undefined). */
int or_hss_split(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
                 double *m, double *nv)
{
    int bad = 0;
    #pragma omp parallel for schedule(static) reduction(| : bad) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            if (k > rp[i] && ci[k] <= ci[k - 1]) { bad = 1; continue; }
            int64_t j = ci[k];
            if (j < 0 || j >= n) { bad = 1; continue; }
            int32_t kt = find_in_row(rp, ci, j, i);
            if (kt < 0) { bad = 1; continue; }
            m[k] = 0.5 * (a[k] + a[kt]);
            nv[k] = 0.5 * (a[k] - a[kt]);
        }
    }
    return bad ? OR_INVALID : OR_OK;
}

/* Explicit transpose of a CSR matrix (counting sort by column). */
static int transpose_csr(int64_t n, const int32_t *rp, const int32_t *ci, const double *v,
                         int32_t **rpt, int32_t **cit, double **vt)
{
    int64_t nnz = rp[n];
    *rpt = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    *cit = (int32_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    *vt = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    int32_t *fill = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!*rpt || !*cit || !*vt || !fill) { free(fill); return OR_OOM; }
    for (int64_t k = 0; k < nnz; ++k) (*rpt)[ci[k] + 1]++;
    for (int64_t i = 0; i < n; ++i) (*rpt)[i + 1] += (*rpt)[i];
    for (int64_t i = 0; i < n; ++i) fill[i] = (*rpt)[i];
    for (int64_t i = 0; i < n; ++i)
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            int32_t pos = fill[ci[k]]++;
            (*cit)[pos] = (int32_t)i;
            (*vt)[pos] = v[k];
        }
    free(fill);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* FP64 inner solvers                                                  */
/* ------------------------------------------------------------------ */

/* CG for (sigma I + M) v = rhs, M symmetric, starting from v (in/out).
 * Stops when ||rhs - K v||_2 <= eps ||rhs - K v0||_2 or after maxit SpMVs.
 * Returns the number of SpMVs inside the loop; -1 on breakdown (p.q <= 0 or
 * non-finite). */
int64_t or_cg(int64_t n, const int32_t *rp, const int32_t *ci, const double *m, double sigma,
              const double *rhs, double *v, double eps, int32_t maxit)
{
    size_t sz = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *r = (double *)malloc(sz), *p = (double *)malloc(sz), *q = (double *)malloc(sz);
    or_spmv_shift(n, rp, ci, m, sigma, v, q);
    #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) { r[i] = rhs[i] - q[i]; p[i] = r[i]; }
    double rr = dot64(n, r, r), rr0 = rr;
    int64_t it = 0;
    if (rr0 > 0.0) {
        while (it < maxit) {
            or_spmv_shift(n, rp, ci, m, sigma, p, q);
            ++it;
            double pq = dot64(n, p, q);
            if (!(pq > 0.0) || !isfinite(pq)) { it = -1; break; }
            double a = rr / pq;
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) { v[i] = fma(a, p[i], v[i]); r[i] = fma(-a, q[i], r[i]); }
            double rrn = dot64(n, r, r);
            if (!isfinite(rrn)) { it = -1; break; }
            if (rrn <= eps * eps * rr0) break;
            double beta = rrn / rr;
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) p[i] = fma(beta, p[i], r[i]);
            rr = rrn;
        }
    }
    free(r); free(p); free(q);
    return it;
}

/* CGNR for S v = rhs with S = sigma I + V: CG on S^T S v = S^T rhs, where
 * S^T = sigma I + V^T (Vt is V's explicit transpose). Same stopping rule as
 * or_cg, on the residual of S v = rhs. Returns the number of iterations
 * (each one product with S and, unless it is the last, one with S^T). */
int64_t or_cgnr(int64_t n, const int32_t *rp, const int32_t *ci, const double *vv,
                const int32_t *rpt, const int32_t *cit, const double *vt, double sigma,
                const double *rhs, double *v, double eps, int32_t maxit)
{
    size_t sz = (size_t)(n > 0 ? n : 1) * sizeof(double);
    double *r = (double *)malloc(sz), *s = (double *)malloc(sz);
    double *p = (double *)malloc(sz), *q = (double *)malloc(sz);
    or_spmv_shift(n, rp, ci, vv, sigma, v, q);
    #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) r[i] = rhs[i] - q[i];
    double rr0 = dot64(n, r, r);
    int64_t it = 0;
    if (rr0 > 0.0) {
        or_spmv_shift(n, rpt, cit, vt, sigma, r, s);
        memcpy(p, s, sz);
        double g = dot64(n, s, s);
        while (it < maxit) {
            or_spmv_shift(n, rp, ci, vv, sigma, p, q);
            ++it;
            double qq = dot64(n, q, q);
            if (!(qq > 0.0) || !isfinite(qq)) { it = -1; break; }
            double a = g / qq;
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) { v[i] = fma(a, p[i], v[i]); r[i] = fma(-a, q[i], r[i]); }
            double rr = dot64(n, r, r);
            if (!isfinite(rr)) { it = -1; break; }
            if (rr <= eps * eps * rr0) break;
            or_spmv_shift(n, rpt, cit, vt, sigma, r, s);
            double gn = dot64(n, s, s);
            double beta = gn / g;
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) p[i] = fma(beta, p[i], s[i]);
            g = gn;
        }
    }
    free(r); free(s); free(p); free(q);
    return it;
}

/* ------------------------------------------------------------------ */
/* Low-precision inner solvers: FP32 arithmetic, storage rounded to the */
/* inner precision (FP32 itself, FP16 emulated with _Float16, or        */
/* bfloat16 emulated by rounding FP32 bit patterns).                     */
/* Every stored value is the result of rnd(); every sum runs in float,  */
/* each product-sum as one fused multiply-add (fmaf).                   */
/* ------------------------------------------------------------------ */

/* Storage rounding of the low-precision modes: rt = 0 FP32 (none), 1 FP16,
 * 2 bfloat16 (8 significant bits, FP32's exponent range), 3 FP8 E4M3, all
 * round to nearest even. */
enum { RT_F32 = 0, RT_F16 = 1, RT_BF16 = 2, RT_E4M3 = 3 };

/* FP8 E4M3 (the OCP 8-bit floating-point format): a sign bit, 4 exponent
 * bits with bias 7 and 3 fraction bits. Exponent field 0 holds the
 * subnormals m 2^-9 (m = 0..7); there is no infinity and only the all-ones
 * pattern is NaN, so the largest finite magnitude is 1.75 2^8 = 448.
 * v is rounded to the nearest representable value, ties to the even
 * fraction; magnitudes beyond 448 saturate to 448 (the saturating
 * conversion an inner storage needs: no value becomes NaN). */
static double e4m3_of_double(double v)
{
    if (v != v) return v;
    const double a = fabs(v);
    if (a >= 448.0) return copysign(448.0, v);
    /* spacing of the representable values near a: 2^-9 below 2^-5, then
     * 2^(e-3) on [2^e, 2^(e+1)) */
    double ulp = ldexp(1.0, -9);
    while (ulp * 16.0 <= a) ulp *= 2.0;
    const double k = a / ulp;                    /* exact: ulp is a power of two */
    double f = floor(k);
    const double rem = k - f;
    if (rem > 0.5 || (rem == 0.5 && fmod(f, 2.0) != 0.0)) f += 1.0;
    return copysign(f * ulp, v);
}

static inline float bf16_of_float(float x)
{
    uint32_t u;
    memcpy(&u, &x, sizeof u);
    if ((u & 0x7f800000u) == 0x7f800000u) {
        if (u & 0x7fffffu) u |= 0x400000u;            /* NaN stays (quiet) NaN */
        u &= 0xffff0000u;
    } else {
        u += 0x7fffu + ((u >> 16) & 1u);              /* nearest, ties to even; overflow -> inf */
        u &= 0xffff0000u;
    }
    memcpy(&x, &u, sizeof x);
    return x;
}

/* x rounded to FP32 with round-to-odd: truncated toward zero, last bit set
 * when inexact. Rounding that to bfloat16 (round to nearest even) equals
 * rounding x directly, since 24 >= 8 + 2 significant bits. */
static inline float float_round_odd(double x)
{
    float t = (float)x;
    if (!(x == x) || (double)t == x) return t;
    if (fabs((double)t) > fabs(x)) t = nextafterf(t, 0.0f);
    uint32_t u;
    memcpy(&u, &t, sizeof u);
    u |= 1u;
    memcpy(&t, &u, sizeof t);
    return t;
}

static inline float rnd_store(float x, int rt)
{
    if (rt == RT_E4M3) return (float)e4m3_of_double((double)x);
    return rt == RT_F16 ? (float)(_Float16)x : (rt == RT_BF16 ? bf16_of_float(x) : x);
}

/* an FP64 value rounded once to the storage precision */
static inline float rnd_from64(double v, int rt)
{
    if (rt == RT_E4M3) return (float)e4m3_of_double(v);
    return rt == RT_F16 ? (float)(_Float16)v : (rt == RT_BF16 ? bf16_of_float(float_round_odd(v)) : (float)v);
}

static float dot32(int64_t n, const float *a, const float *b)
{
    int64_t nb = (n + OR_BLK - 1) / OR_BLK;
    float *part = (float *)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(float));
    #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t k = 0; k < nb; ++k) {
        int64_t lo = k * OR_BLK, hi = lo + OR_BLK < n ? lo + OR_BLK : n;
        float s = 0.0f;
        for (int64_t i = lo; i < hi; ++i) s = fmaf(a[i], b[i], s);
        part[k] = s;
    }
    float s = 0.0f;
    for (int64_t k = 0; k < nb; ++k) s += part[k];
    free(part);
    return s;
}

static float norm_inf32(int64_t n, const float *a)
{
    float m = 0.0f;
    #pragma omp parallel for reduction(max : m) schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        float v = fabsf(a[i]);
        if (v > m || v != v) m = (v != v) ? INFINITY : v;
    }
    return m;
}

/* y = rnd(sigma x + V x), V values already rounded to storage precision */
static void spmv32(int64_t n, const int32_t *rp, const int32_t *ci, const float *v,
                   float sigma, const float *x, float *y, int rt)
{
    #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
    for (int64_t i = 0; i < n; ++i) {
        float s = sigma * x[i];
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s = fmaf(v[k], x[ci[k]], s);
        y[i] = rnd_store(s, rt);
    }
}

/* CG on (sigma I + M) z = rhs from z = 0, low precision. */
static int64_t lp_cg(int64_t n, const int32_t *rp, const int32_t *ci, const float *m, float sigma,
                     const float *rhs, float *z, double eps, int32_t maxit, int rt)
{
    size_t sz = (size_t)(n > 0 ? n : 1) * sizeof(float);
    float *r = (float *)malloc(sz), *p = (float *)malloc(sz), *q = (float *)malloc(sz);
    memcpy(r, rhs, sz); memcpy(p, rhs, sz);
    memset(z, 0, sz);
    float rr = dot32(n, r, r), rr0 = rr;
    float eps2 = (float)(eps * eps);
    int64_t it = 0;
    if (rr0 > 0.0f) {
        while (it < maxit) {
            spmv32(n, rp, ci, m, sigma, p, q, rt);
            ++it;
            float pq = dot32(n, p, q);
            if (!(pq > 0.0f) || !isfinite(pq)) { it = -1; break; }
            float a = rr / pq;
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) {
                z[i] = rnd_store(fmaf(a, p[i], z[i]), rt);
                r[i] = rnd_store(fmaf(-a, q[i], r[i]), rt);
            }
            float rrn = dot32(n, r, r);
            if (!isfinite(rrn)) { it = -1; break; }
            if (rrn <= eps2 * rr0) break;
            float beta = rrn / rr;
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) p[i] = rnd_store(fmaf(beta, p[i], r[i]), rt);
            rr = rrn;
        }
    }
    free(r); free(p); free(q);
    return it;
}

/* CGNR on (sigma I + N) y = rhs from y = 0, low precision. */
static int64_t lp_cgnr(int64_t n, const int32_t *rp, const int32_t *ci, const float *nv,
                       const int32_t *rpt, const int32_t *cit, const float *nvt, float sigma,
                       const float *rhs, float *y, double eps, int32_t maxit, int rt)
{
    size_t sz = (size_t)(n > 0 ? n : 1) * sizeof(float);
    float *r = (float *)malloc(sz), *s = (float *)malloc(sz);
    float *p = (float *)malloc(sz), *q = (float *)malloc(sz);
    memcpy(r, rhs, sz);
    memset(y, 0, sz);
    float rr0 = dot32(n, r, r);
    float eps2 = (float)(eps * eps);
    int64_t it = 0;
    if (rr0 > 0.0f) {
        spmv32(n, rpt, cit, nvt, sigma, r, s, rt);
        memcpy(p, s, sz);
        float g = dot32(n, s, s);
        while (it < maxit) {
            spmv32(n, rp, ci, nv, sigma, p, q, rt);
            ++it;
            float qq = dot32(n, q, q);
            if (!(qq > 0.0f) || !isfinite(qq)) { it = -1; break; }
            float a = g / qq;
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) {
                y[i] = rnd_store(fmaf(a, p[i], y[i]), rt);
                r[i] = rnd_store(fmaf(-a, q[i], r[i]), rt);
            }
            float rr = dot32(n, r, r);
            if (!isfinite(rr)) { it = -1; break; }
            if (rr <= eps2 * rr0) break;
            spmv32(n, rpt, cit, nvt, sigma, r, s, rt);
            float gn = dot32(n, s, s);
            float beta = gn / g;
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) p[i] = rnd_store(fmaf(beta, p[i], s[i]), rt);
            g = gn;
        }
    }
    free(r); free(s); free(p); free(q);
    return it;
}

/* floor(log2 |v|) for finite v > 0 */
static int ilog2_floor(double v)
{
    int e;
    frexp(v, &e);
    return e - 1;
}

/* FP16 range scale of an operator sigma I + V: the exponent s for which
 * (|sigma| + max row sum |V|) * 2^-s lies in (1, 2]. Scaling by a power of
 * two is exact, so this only keeps FP16 values in range: with the inner
 * right-hand side scaled to infinity-norm [1, 2), a product K p (and, in
 * CGNR, K K^T r) stays within a small multiple of the vector's own size. */
static int half_scale_exponent(int64_t n, const int32_t *rp, const double *v, double sigma)
{
    double nrm = or_matrix_norm_inf(n, rp, v) + fabs(sigma);
    if (!(nrm > 0.0) || !isfinite(nrm)) return 0;
    int e;
    double m = frexp(nrm, &e);       /* nrm = m 2^e, m in [0.5, 1) */
    int c = (m == 0.5) ? e - 1 : e;  /* ceil(log2 nrm) */
    return c - 1;
}

/* ------------------------------------------------------------------ */
/* Outer iterations                                                    */
/* ------------------------------------------------------------------ */

static int check_params(const or_params *P)
{
    if (!(P->alpha > 0.0) || !isfinite(P->alpha)) return OR_INVALID;
    if (!(P->omega >= 0.0 && P->omega < 2.0)) return OR_INVALID;
    if (!(P->tol >= 0.0) || !(P->eps_inner > 0.0)) return OR_INVALID;
    if (P->max_inner < 1 || P->max_outer < 0) return OR_INVALID;
    return OR_OK;
}

typedef struct {
    double anorm, bnorm, r0;
    double best;
} stop_state;

/* Evaluate the stopping test on r = b - Ax (Alg. 1 loop condition, read as
 * RES or eta_inf). Returns 1 to stop (converged), 0 to continue, -1 diverged. */
static int outer_test(int64_t n, const double *r, const double *x, const or_params *P,
                      stop_state *st, or_info *info, double *eta_hist, int k)
{
    double rn2 = sqrt(dot64(n, r, r));
    double rinf = norm_inf64(n, r);
    double den = st->anorm * norm_inf64(n, x) + st->bnorm;
    double eta = den > 0.0 ? rinf / den : (rinf == 0.0 ? 0.0 : INFINITY);
    if (k == 0) st->r0 = rn2;
    double res = st->r0 > 0.0 ? rn2 / st->r0 : 0.0;
    info->eta_inf = eta;
    info->res_rel = res;
    info->res0 = st->r0;
    if (eta_hist) eta_hist[k] = eta;
    if (!isfinite(rn2) || !isfinite(eta)) return -1;
    if (k == 0 || rn2 < st->best) st->best = rn2;
    double crit = P->stop_kind == OR_STOP_RES ? res : eta;
    if (crit <= P->tol) return 1;
    if (rn2 > 1e3 * st->best) return -1;
    return 0;
}

/* Plain GADI, the two-half-step form of eq. (gadi), all in FP64:
 *   (aI + M) x^{k+1/2} = (aI - N) x^k + b
 *   (aI + N) x^{k+1}   = (N - (1-w) aI) x^k + (2-w) a x^{k+1/2}
 * Each half step is solved by CG / CGNR started from x^k.
 * x: in = x0, out = last iterate. eta_hist, itH, itS: optional per-iteration
 * records of length max_outer + 1 (eta) and max_outer (inner counts). */
int or_gadi(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
            const double *b, double *x, const or_params *P, or_info *info,
            double *eta_hist, int32_t *itH, int32_t *itS)
{
    memset(info, 0, sizeof(*info));
    if (check_params(P) != OR_OK) { info->status = OR_INVALID; return OR_INVALID; }
    int64_t nnz = rp[n];
    size_t szv = (size_t)(n > 0 ? n : 1) * sizeof(double);
    size_t szm = (size_t)(nnz > 0 ? nnz : 1) * sizeof(double);
    double *m = (double *)malloc(szm), *nv = (double *)malloc(szm);
    if (or_hss_split(n, rp, ci, a, m, nv) != OR_OK) {
        free(m); free(nv); info->status = OR_INVALID; return OR_INVALID;
    }
    int32_t *rpt, *cit; double *nvt;
    transpose_csr(n, rp, ci, nv, &rpt, &cit, &nvt);
    double *r = (double *)malloc(szv), *t = (double *)malloc(szv);
    double *rhs = (double *)malloc(szv), *xh = (double *)malloc(szv), *xn = (double *)malloc(szv);
    const double al = P->alpha, om = P->omega;
    stop_state st = { or_matrix_norm_inf(n, rp, a), norm_inf64(n, b), 0.0, 0.0 };
    int status = OR_NOT_CONVERGED;
    int k = 0;
    for (;;) {
        or_residual(n, rp, ci, a, b, x, r);
        info->spmv_count++;
        int s = outer_test(n, r, x, P, &st, info, eta_hist, k);
        if (s == 1) { status = OR_OK; break; }
        if (s == -1) { status = OR_DIVERGED; break; }
        if (k >= P->max_outer) break;
        /* first half step: rhs = (aI - N) x + b, solve (aI + M) xh = rhs from x */
        or_spmv_shift(n, rp, ci, nv, -al, x, t);     /* t = -a x + N x */
        #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t i = 0; i < n; ++i) { rhs[i] = b[i] - t[i]; xh[i] = x[i]; }
        int64_t ih = or_cg(n, rp, ci, m, al, rhs, xh, P->eps_inner, P->max_inner);
        if (ih < 0) { status = OR_DIVERGED; break; }
        /* second half step: rhs = (N - (1-w) a I) x + (2-w) a xh, solve (aI + N) xn = rhs from x */
        or_spmv_shift(n, rp, ci, nv, -(1.0 - om) * al, x, t);
        #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
        for (int64_t i = 0; i < n; ++i) { rhs[i] = fma((2.0 - om) * al, xh[i], t[i]); xn[i] = x[i]; }
        int64_t is = or_cgnr(n, rp, ci, nv, rpt, cit, nvt, al, rhs, xn, P->eps_inner, P->max_inner);
        if (is < 0) { status = OR_DIVERGED; break; }
        memcpy(x, xn, szv);
        info->inner_iters_H += ih;
        info->inner_iters_S += is;
        info->spmv_count += ih + 2 * is + 4;  /* + 2 rhs products + 2 initial inner residuals */
        if (itH) itH[k] = (int32_t)ih;
        if (itS) itS[k] = (int32_t)is;
        ++k;
    }
    info->outer_iters = k;
    info->status = status;
    free(m); free(nv); free(rpt); free(cit); free(nvt);
    free(r); free(t); free(rhs); free(xh); free(xn);
    return status;
}

/* Three-precision GADI-IR, Algorithm 1:
 *   step 1  r = b - A x                              (u_f = FP64)
 *   step 2  solve H z = r,            H = aI + M     (u_r = inner_prec)
 *   step 3  solve S y = (2-w) a z,    S = aI + N     (u_r)
 *   step 4  x = x + y                                (u = FP64)
 * until the stopping test holds. In the low-precision modes the residual is
 * rounded to the inner precision (r^ = fl_r(s^), §2.2) after scaling by
 * 2^-e, e = floor(log2 ||r||_inf); z is rescaled by 2^-ez before step 3; the
 * scales and (2-w) a are applied to y in FP64 in step 4. */
int or_gadi_ir_split(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
                     const double *m_user, const double *b, double *x, const or_params *P,
                     or_info *info, double *eta_hist, int32_t *itH, int32_t *itS)
{
    memset(info, 0, sizeof(*info));
    if (check_params(P) != OR_OK || P->inner_prec < 0 || P->inner_prec > OR_PREC_E4M3) {
        info->status = OR_INVALID; return OR_INVALID;
    }
    int64_t nnz = rp[n];
    size_t szv = (size_t)(n > 0 ? n : 1) * sizeof(double);
    size_t szm = (size_t)(nnz > 0 ? nnz : 1) * sizeof(double);
    double *m = (double *)malloc(szm), *nv = (double *)malloc(szm);
    if (m_user) {
        /* user splitting A = M + N: N = A - M on A's pattern */
        for (int64_t k = 0; k < nnz; ++k) { m[k] = m_user[k]; nv[k] = a[k] - m_user[k]; }
    } else if (or_hss_split(n, rp, ci, a, m, nv) != OR_OK) {
        free(m); free(nv); info->status = OR_INVALID; return OR_INVALID;
    }
    int32_t *rpt, *cit; double *nvt;
    transpose_csr(n, rp, ci, nv, &rpt, &cit, &nvt);
    const double al = P->alpha, om = P->omega, pfac = (2.0 - om) * al;
    const int prec = P->inner_prec;
    const int naive = (prec == OR_PREC_HALF_NAIVE);
    /* storage rounding; the FP16, bfloat16 and FP8 modes scale the operators */
    const int rt = (prec == OR_PREC_HALF || naive) ? RT_F16
                   : (prec == OR_PREC_BF16 ? RT_BF16 : (prec == OR_PREC_E4M3 ? RT_E4M3 : RT_F32));
    const int half = (rt != RT_F32);

    double *r = (double *)malloc(szv), *z = (double *)malloc(szv), *y = (double *)malloc(szv);
    /* low-precision copies */
    size_t szvf = (size_t)(n > 0 ? n : 1) * sizeof(float);
    size_t szmf = (size_t)(nnz > 0 ? nnz : 1) * sizeof(float);
    float *mf = NULL, *nf = NULL, *nft = NULL, *rf = NULL, *zf = NULL, *yf = NULL;
    float sigH = 0.0f, sigS = 0.0f;
    int sM = 0, sN = 0;
    if (prec != OR_PREC_DOUBLE) {
        mf = (float *)malloc(szmf); nf = (float *)malloc(szmf); nft = (float *)malloc(szmf);
        rf = (float *)malloc(szvf); zf = (float *)malloc(szvf); yf = (float *)malloc(szvf);
        if (naive) {
            /* alpha rounded into the stored diagonal, no scaling */
            for (int64_t i = 0; i < n; ++i)
                for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
                    double dm = m[k] + (ci[k] == i ? al : 0.0);
                    double dn = nv[k] + (ci[k] == i ? al : 0.0);
                    mf[k] = (float)(_Float16)dm;
                    nf[k] = (float)(_Float16)dn;
                }
            for (int64_t i = 0; i < n; ++i)
                for (int32_t k = rpt[i]; k < rpt[i + 1]; ++k) {
                    double dn = nvt[k] + (cit[k] == i ? al : 0.0);
                    nft[k] = (float)(_Float16)dn;
                }
            sigH = 0.0f; sigS = 0.0f;
        } else {
            if (half) {
                sM = half_scale_exponent(n, rp, m, al);
                sN = half_scale_exponent(n, rp, nv, al);
                int sNt = half_scale_exponent(n, rpt, nvt, al);
                if (sNt > sN) sN = sNt;     /* one scale for S and S^T */
            }
            for (int64_t k = 0; k < nnz; ++k) {
                mf[k] = rnd_from64(ldexp(m[k], -sM), rt);
                nf[k] = rnd_from64(ldexp(nv[k], -sN), rt);
                nft[k] = rnd_from64(ldexp(nvt[k], -sN), rt);
            }
            sigH = (float)ldexp(al, -sM);
            sigS = (float)ldexp(al, -sN);
        }
    }
    info->scale_exp_M = sM;
    info->scale_exp_N = sN;

    stop_state st = { or_matrix_norm_inf(n, rp, a), norm_inf64(n, b), 0.0, 0.0 };
    int status = OR_NOT_CONVERGED;
    int k = 0;
    for (;;) {
        /* step 1: residual in u_f = FP64 */
        or_residual(n, rp, ci, a, b, x, r);
        info->spmv_count++;
        int s = outer_test(n, r, x, P, &st, info, eta_hist, k);
        if (s == 1) { status = OR_OK; break; }
        if (s == -1) { status = OR_DIVERGED; break; }
        if (k >= P->max_outer) break;
        int64_t ih, is;
        double upd;    /* y_true = upd * y_stored */
        if (prec == OR_PREC_DOUBLE) {
            /* steps 2-3 in FP64 */
            memset(z, 0, szv);
            ih = or_cg(n, rp, ci, m, al, r, z, P->eps_inner, P->max_inner);
            if (ih < 0) { status = OR_DIVERGED; break; }
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) z[i] *= pfac;
            memset(y, 0, szv);
            is = or_cgnr(n, rp, ci, nv, rpt, cit, nvt, al, z, y, P->eps_inner, P->max_inner);
            if (is < 0) { status = OR_DIVERGED; break; }
            upd = 1.0;
            /* step 4: x = x + y */
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) x[i] += y[i];
        } else {
            int e = 0, ez = 0;
            if (!naive) {
                double rinf = norm_inf64(n, r);
                if (rinf > 0.0) e = ilog2_floor(rinf);
            }
            /* r^ = fl_r(r 2^-e) */
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) {
                double v = ldexp(r[i], -e);
                rf[i] = rnd_from64(v, rt);
            }
            ih = lp_cg(n, rp, ci, mf, sigH, rf, zf, P->eps_inner, P->max_inner, rt);
            if (ih < 0) { status = OR_DIVERGED; break; }
            if (naive) {
                /* (2-w) a z formed in the inner precision */
                float pf = (float)pfac;
                #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
                for (int64_t i = 0; i < n; ++i) zf[i] = rnd_store(pf * zf[i], rt);
                upd = 1.0;
            } else {
                float zinf = norm_inf32(n, zf);
                if (zinf > 0.0f && isfinite(zinf)) ez = ilog2_floor((double)zinf);
                #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
                for (int64_t i = 0; i < n; ++i) zf[i] = rnd_store(ldexpf(zf[i], -ez), rt);
                upd = ldexp(pfac, e - sM + ez - sN);
            }
            is = lp_cgnr(n, rp, ci, nf, rpt, cit, nft, sigS, zf, yf, P->eps_inner, P->max_inner, rt);
            if (is < 0) { status = OR_DIVERGED; break; }
            /* step 4 in u = FP64 */
            #pragma omp parallel for schedule(static) if (n > OR_PAR_MIN)
            for (int64_t i = 0; i < n; ++i) x[i] = fma(upd, (double)yf[i], x[i]);
        }
        info->inner_iters_H += ih;
        info->inner_iters_S += is;
        info->spmv_count += ih + 2 * is;
        if (itH) itH[k] = (int32_t)ih;
        if (itS) itS[k] = (int32_t)is;
        ++k;
    }
    info->outer_iters = k;
    info->status = status;
    free(m); free(nv); free(rpt); free(cit); free(nvt);
    free(r); free(z); free(y);
    free(mf); free(nf); free(nft); free(rf); free(zf); free(yf);
    return status;
}

int or_gadi_ir(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
               const double *b, double *x, const or_params *P, or_info *info,
               double *eta_hist, int32_t *itH, int32_t *itS)
{
    return or_gadi_ir_split(n, rp, ci, a, NULL, b, x, P, info, eta_hist, itH, itS);
}

/* One application of an operator of Algorithm 1 in a given inner precision,
 * with the same splitting, scaling and rounding as or_gadi_ir_split:
 *   which 0: y = A x (FP64)
 *   which 1: y = fl(H' x),  H' = 2^-sM (aI + M)
 *   which 2: y = fl(S' x),  S' = 2^-sN (aI + N)
 *   which 3: y = fl(S'^T x)
 * prec: OR_PREC_HALF, OR_PREC_HALF_NAIVE, OR_PREC_BF16, OR_PREC_E4M3,
 * OR_PREC_SINGLE or OR_PREC_DOUBLE;
 * x holds values of that precision (as doubles). The scale exponents used
 * are returned (zero in the naive mode, where alpha is rounded into the
 * stored FP16 diagonal as in or_gadi_ir_split). */
int or_lp_apply(int64_t n, const int32_t *rp, const int32_t *ci, const double *a,
                const double *m_user, double alpha, int which, int prec,
                const double *x, double *y, int32_t *sM_out, int32_t *sN_out)
{
    int64_t nnz = rp[n];
    size_t szm = (size_t)(nnz > 0 ? nnz : 1) * sizeof(double);
    double *m = (double *)malloc(szm), *nv = (double *)malloc(szm);
    if (m_user) {
        for (int64_t k = 0; k < nnz; ++k) { m[k] = m_user[k]; nv[k] = a[k] - m_user[k]; }
    } else if (or_hss_split(n, rp, ci, a, m, nv) != OR_OK) {
        free(m); free(nv); return OR_INVALID;
    }
    int32_t *rpt, *cit; double *nvt;
    transpose_csr(n, rp, ci, nv, &rpt, &cit, &nvt);
    const int naive = prec == OR_PREC_HALF_NAIVE;
    const int rt = (prec == OR_PREC_HALF || naive) ? RT_F16
                   : (prec == OR_PREC_BF16 ? RT_BF16 : (prec == OR_PREC_E4M3 ? RT_E4M3 : RT_F32));
    const int half = rt != RT_F32;
    int sM = 0, sN = 0;
    if (half && !naive) {
        sM = half_scale_exponent(n, rp, m, alpha);
        sN = half_scale_exponent(n, rp, nv, alpha);
        int sNt = half_scale_exponent(n, rpt, nvt, alpha);
        if (sNt > sN) sN = sNt;
    }
    if (sM_out) *sM_out = sM;
    if (sN_out) *sN_out = sN;
    if (which == 0) {
        or_spmv_shift(n, rp, ci, a, 0.0, x, y);
    } else if (prec == OR_PREC_DOUBLE) {
        if (which == 1) or_spmv_shift(n, rp, ci, m, alpha, x, y);
        else if (which == 2) or_spmv_shift(n, rp, ci, nv, alpha, x, y);
        else or_spmv_shift(n, rpt, cit, nvt, alpha, x, y);
    } else {
        size_t szmf = (size_t)(nnz > 0 ? nnz : 1) * sizeof(float);
        size_t szvf = (size_t)(n > 0 ? n : 1) * sizeof(float);
        float *vf = (float *)malloc(szmf), *xf = (float *)malloc(szvf), *yf = (float *)malloc(szvf);
        const double *src = which == 1 ? m : (which == 2 ? nv : nvt);
        const int32_t *rpx = which == 3 ? rpt : rp, *cix = which == 3 ? cit : ci;
        int s = which == 1 ? sM : sN;
        for (int64_t i = 0; i < n; ++i)
            for (int32_t k = rpx[i]; k < rpx[i + 1]; ++k) {
                /* naive: alpha rounded into the stored diagonal, nothing scaled */
                double v = naive ? src[k] + (cix[k] == i ? alpha : 0.0) : ldexp(src[k], -s);
                vf[k] = half ? rnd_from64(v, rt) : (float)src[k];
            }
        for (int64_t i = 0; i < n; ++i) xf[i] = (float)x[i];
        float sig = naive ? 0.0f : (float)ldexp(alpha, -s);
        if (which == 3) spmv32(n, rpt, cit, vf, sig, xf, yf, rt);
        else spmv32(n, rp, ci, vf, sig, xf, yf, rt);
        for (int64_t i = 0; i < n; ++i) y[i] = (double)yf[i];
        free(vf); free(xf); free(yf);
    }
    free(m); free(nv); free(rpt); free(cit); free(nvt);
    return OR_OK;
}

/* FP64 -> FP16 conversion (round to nearest even, direct from double), as
 * raw bits; used by the tests to pin the emulation against IEEE 754. */
void or_to_half_bits(int64_t n, const double *in, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        _Float16 h = (_Float16)in[i];
        memcpy(&out[i], &h, sizeof(uint16_t));
    }
}

/* FP64 -> bfloat16 (round to nearest even, one rounding), as raw bits. */
void or_to_bf16_bits(int64_t n, const double *in, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        float f = bf16_of_float(float_round_odd(in[i]));
        uint32_t u;
        memcpy(&u, &f, sizeof u);
        out[i] = (uint16_t)(u >> 16);
    }
}

/* FP64 -> FP8 E4M3 (round to nearest even, saturating), as the 8-bit
 * codes: sign << 7 | exponent field << 3 | fraction; NaN as 0x7f. */
void or_to_e4m3_bits(int64_t n, const double *in, uint8_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        const double r = e4m3_of_double(in[i]);
        if (r != r) { out[i] = 0x7f; continue; }
        const uint8_t sign = signbit(r) ? 0x80 : 0x00;
        const double a = fabs(r);
        uint8_t code;
        if (a < ldexp(1.0, -6)) {
            code = (uint8_t)(a / ldexp(1.0, -9));               /* subnormal: m 2^-9 */
        } else {
            int e = 0;
            frexp(a, &e);                                        /* a in [2^(e-1), 2^e) */
            const int ex = e - 1;
            const int frac = (int)(a / ldexp(1.0, ex - 3)) - 8;  /* a = (8 + frac) 2^(ex-3) */
            code = (uint8_t)(((ex + 7) << 3) | frac);
        }
        out[i] = sign | code;
    }
}

/* Single inner solves exposed for unit tests. */
int64_t or_cg_solve(int64_t n, const int32_t *rp, const int32_t *ci, const double *m, double sigma,
                    const double *rhs, double *v, double eps, int32_t maxit)
{
    return or_cg(n, rp, ci, m, sigma, rhs, v, eps, maxit);
}

int64_t or_cgnr_solve(int64_t n, const int32_t *rp, const int32_t *ci, const double *nv, double sigma,
                      const double *rhs, double *v, double eps, int32_t maxit)
{
    int32_t *rpt, *cit; double *nvt;
    if (transpose_csr(n, rp, ci, nv, &rpt, &cit, &nvt) != OR_OK) return -2;
    int64_t it = or_cgnr(n, rp, ci, nv, rpt, cit, nvt, sigma, rhs, v, eps, maxit);
    free(rpt); free(cit); free(nvt);
    return it;
}

/* Wall-clock seconds, for the CPU baseline timing. */
double or_wtime(void)
{
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return 0.0;
#endif
}

/* ------------------------------------------------------------------ */
/* GADI-AB: GADI-IR (Algorithm 1) for the Sylvester equation (§4.3)    */
/*     A X + X B = C,  A (m x m), B (n x n) tridiagonal, X, C (m x n) */
/* The operator L(X) = A X + X B is split into X -> A X and X -> X B   */
/* (the paper's GADI-AB: M, N of Algorithm 1 replaced by A, B). One   */
/* outer step:                                                         */
/*   R = C - A X - X B                         (FP64, u_f)              */
/*   e = floor(log2 max|R|), R^ = fl_r(2^-e R)                          */
/*   Z = H'^-1 R^,  H' = 2^-sA (aI + A)          columns of R^          */
/*   ez = floor(log2 max|Z|), Z^ = fl_r(2^-ez Z)                        */
/*   Y = Z^ S'^-1,  S' = 2^-sB (aI + B)          rows of Z^             */
/*   X = X + (2-w) a 2^(e - sA + ez - sB) Y      (FP64, u)              */
/* Readings: the residual sign follows R = C - A X - X B (the paper    */
/* writes both A X + X B + C = 0 and this residual); the inner systems */
/* are tridiagonal and, for a > 0 and these A, B, diagonally dominant, */
/* so each is solved directly (Thomas: no pivoting, stable here) in    */
/* the inner precision: factors from FP64, stored in FP32 (FP64 for    */
/* the FP64 inner path), every stored intermediate rounded to u_r.     */
/* Matrices: lo[i] = T[i][i-1] (lo[0] unused), dg[i] = T[i][i],        */
/* up[i] = T[i][i+1] (up[m-1] unused). X, C row-major.                 */
/* ------------------------------------------------------------------ */

/* (|sigma| + max row sum of |T|) 2^-s in (1, 2] */
static int tri_scale_exponent(int64_t m, const double *lo, const double *dg, const double *up, double sigma)
{
    double nrm = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double s = fabs(dg[i]);
        if (i > 0) s += fabs(lo[i]);
        if (i < m - 1) s += fabs(up[i]);
        if (s > nrm) nrm = s;
    }
    nrm += fabs(sigma);
    if (!(nrm > 0.0) || !isfinite(nrm)) return 0;
    int e;
    double mm = frexp(nrm, &e);
    return ((mm == 0.5) ? e - 1 : e) - 1;
}

/* Thomas factors of T = 2^-s (sigma I + tridiag(lo, dg, up)):
 * w_0 = t_00, w_i = t_ii - t_i,i-1 c_(i-1) (one fused multiply-add),
 * c_i = t_i,i+1 / w_i; returns ls = scaled lo, c, iw = 1 / w. */
static void tri_factor(int64_t m, const double *lo, const double *dg, const double *up, double sigma, int s,
                       double *ls, double *c, double *iw)
{
    double w = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double d = ldexp(sigma + dg[i], -s);
        ls[i] = i > 0 ? ldexp(lo[i], -s) : 0.0;
        w = i > 0 ? fma(-ls[i], c[i - 1], d) : d;
        iw[i] = 1.0 / w;
        c[i] = i < m - 1 ? ldexp(up[i], -s) / w : 0.0;
    }
}

/* Solve T v = rhs in place along a strided line, low precision: forward
 * y_i = fl(fl32(fmaf(-l_i, y_(i-1), v_i)) * iw_i), back
 * z_i = fl(fmaf(-c_i, z_(i+1), y_i)); fl = rounding to the storage type. */
static void tri_solve32(int64_t m, int64_t stride, const float *ls, const float *c, const float *iw, float *v, int rt)
{
    float y = rnd_store(v[0] * iw[0], rt);
    v[0] = y;
    for (int64_t i = 1; i < m; ++i) {
        y = rnd_store(fmaf(-ls[i], y, v[i * stride]) * iw[i], rt);
        v[i * stride] = y;
    }
    float z = y;
    for (int64_t i = m - 2; i >= 0; --i) {
        z = rnd_store(fmaf(-c[i], z, v[i * stride]), rt);
        v[i * stride] = z;
    }
}

static void tri_solve64(int64_t m, int64_t stride, const double *ls, const double *c, const double *iw, double *v)
{
    double y = v[0] * iw[0];
    v[0] = y;
    for (int64_t i = 1; i < m; ++i) {
        y = fma(-ls[i], y, v[i * stride]) * iw[i];
        v[i * stride] = y;
    }
    double z = y;
    for (int64_t i = m - 2; i >= 0; --i) {
        z = fma(-c[i], z, v[i * stride]);
        v[i * stride] = z;
    }
}

/* R = C - A X - X B, each entry one chain of fused multiply-adds in the
 * order A's (i-1, i, i+1), then B's (j-1, j, j+1) */
static void sylv_residual(int64_t m, int64_t n, const double *al, const double *ad, const double *au,
                          const double *bl, const double *bd, const double *bu, const double *C,
                          const double *X, double *R)
{
    #pragma omp parallel for schedule(static) if (m * n > OR_PAR_MIN)
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) {
            const double *x = X + i * n + j;
            double r = C[i * n + j];
            if (i > 0) r = fma(-al[i], x[-n], r);
            r = fma(-ad[i], x[0], r);
            if (i < m - 1) r = fma(-au[i], x[n], r);
            if (j > 0) r = fma(-bu[j - 1], x[-1], r);     /* B[j-1][j] */
            r = fma(-bd[j], x[0], r);
            if (j < n - 1) r = fma(-bl[j + 1], x[1], r);  /* B[j+1][j] */
            R[i * n + j] = r;
        }
}

/* ||L||_inf of X -> A X + X B on vec(X): the largest row sum of
 * I (x) A + B^T (x) I */
double or_sylv_norm_inf(int64_t m, int64_t n, const double *al, const double *ad, const double *au,
                        const double *bl, const double *bd, const double *bu)
{
    double best = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double sa = (i > 0 ? fabs(al[i]) : 0.0) + (i < m - 1 ? fabs(au[i]) : 0.0);
        for (int64_t j = 0; j < n; ++j) {
            double sb = (j > 0 ? fabs(bu[j - 1]) : 0.0) + (j < n - 1 ? fabs(bl[j + 1]) : 0.0);
            double s = sa + sb + fabs(ad[i] + bd[j]);
            if (s > best) best = s;
        }
    }
    return best;
}

/* GADI-AB to eta = max|R| / (||L||_inf max|X| + max|C|) <= tol. prec:
 * OR_PREC_DOUBLE, _SINGLE, _HALF or _BF16 (the FP16 and bfloat16 inner
 * paths scale H, S, R and Z by powers of two as the vector method does).
 * X holds x0 on entry. */
int or_sylv_gadi_ab(int64_t m, int64_t n, const double *al, const double *ad, const double *au,
                    const double *bl, const double *bd, const double *bu, const double *C, double *X,
                    double alpha, double omega, int prec, double tol, int32_t max_outer, or_info *info,
                    double *eta_hist)
{
    memset(info, 0, sizeof *info);
    if (m < 1 || n < 1 || !(alpha > 0.0) || !(omega >= 0.0 && omega < 2.0) || max_outer < 0 ||
        (prec != OR_PREC_DOUBLE && prec != OR_PREC_SINGLE && prec != OR_PREC_HALF && prec != OR_PREC_BF16)) {
        info->status = OR_INVALID;
        return OR_INVALID;
    }
    const int64_t mn = m * n;
    const int low = prec != OR_PREC_DOUBLE;
    const int rt = prec == OR_PREC_HALF ? RT_F16 : (prec == OR_PREC_BF16 ? RT_BF16 : RT_F32);
    const int scaled = prec == OR_PREC_HALF || prec == OR_PREC_BF16;
    /* the row solves use S'^T: sub-diagonal B[j-1][j] = bu[j-1], super B[j+1][j] = bl[j+1] */
    double *btl = (double *)calloc((size_t)n, sizeof(double)), *btu = (double *)calloc((size_t)n, sizeof(double));
    for (int64_t j = 0; j < n; ++j) {
        btl[j] = j > 0 ? bu[j - 1] : 0.0;
        btu[j] = j < n - 1 ? bl[j + 1] : 0.0;
    }
    const int sA = scaled ? tri_scale_exponent(m, al, ad, au, alpha) : 0;
    const int sB = scaled ? tri_scale_exponent(n, btl, bd, btu, alpha) : 0;
    info->scale_exp_M = sA;
    info->scale_exp_N = sB;
    double *la = (double *)malloc((size_t)m * sizeof(double)), *ca = (double *)malloc((size_t)m * sizeof(double));
    double *iwa = (double *)malloc((size_t)m * sizeof(double));
    double *lb = (double *)malloc((size_t)n * sizeof(double)), *cb = (double *)malloc((size_t)n * sizeof(double));
    double *iwb = (double *)malloc((size_t)n * sizeof(double));
    tri_factor(m, al, ad, au, alpha, sA, la, ca, iwa);
    tri_factor(n, btl, bd, btu, alpha, sB, lb, cb, iwb);
    float *laf = (float *)malloc((size_t)m * sizeof(float)), *caf = (float *)malloc((size_t)m * sizeof(float));
    float *iwaf = (float *)malloc((size_t)m * sizeof(float));
    float *lbf = (float *)malloc((size_t)n * sizeof(float)), *cbf = (float *)malloc((size_t)n * sizeof(float));
    float *iwbf = (float *)malloc((size_t)n * sizeof(float));
    for (int64_t i = 0; i < m; ++i) { laf[i] = (float)la[i]; caf[i] = (float)ca[i]; iwaf[i] = (float)iwa[i]; }
    for (int64_t j = 0; j < n; ++j) { lbf[j] = (float)lb[j]; cbf[j] = (float)cb[j]; iwbf[j] = (float)iwb[j]; }

    double *R = (double *)malloc((size_t)mn * sizeof(double));
    float *Zf = (float *)malloc((size_t)mn * sizeof(float));
    const double Ln = or_sylv_norm_inf(m, n, al, ad, au, bl, bd, bu);
    double cmax = 0.0;
    for (int64_t k = 0; k < mn; ++k) cmax = fmax(cmax, fabs(C[k]));
    const double pfac = (2.0 - omega) * alpha;
    int status = OR_NOT_CONVERGED, k = 0;
    for (;;) {
        sylv_residual(m, n, al, ad, au, bl, bd, bu, C, X, R);
        double rmax = 0.0, xmax = 0.0;
        for (int64_t q = 0; q < mn; ++q) {
            rmax = fmax(rmax, fabs(R[q]));
            xmax = fmax(xmax, fabs(X[q]));
        }
        if (!isfinite(rmax)) { status = OR_DIVERGED; break; }
        double den = Ln * xmax + cmax;
        info->eta_inf = den > 0.0 ? rmax / den : (rmax == 0.0 ? 0.0 : INFINITY);
        if (eta_hist) eta_hist[k] = info->eta_inf;
        if (info->eta_inf <= tol) { status = OR_OK; break; }
        if (k >= max_outer) break;
        double upd;
        if (!low) {
            for (int64_t i = 0; i < n; ++i) tri_solve64(m, n, la, ca, iwa, R + i);    /* columns */
            for (int64_t i = 0; i < m; ++i) tri_solve64(n, 1, lb, cb, iwb, R + i * n); /* rows */
            upd = pfac;
            for (int64_t q = 0; q < mn; ++q) X[q] = fma(upd, R[q], X[q]);
        } else {
            int e = rmax > 0.0 ? ilog2_floor(rmax) : 0;
            for (int64_t q = 0; q < mn; ++q) Zf[q] = rnd_from64(ldexp(R[q], -e), rt);
            for (int64_t j = 0; j < n; ++j) tri_solve32(m, n, laf, caf, iwaf, Zf + j, rt);
            float zmax = 0.0f;
            for (int64_t q = 0; q < mn; ++q) zmax = fmaxf(zmax, fabsf(Zf[q]));
            int ez = (zmax > 0.0f && isfinite(zmax)) ? ilog2_floor((double)zmax) : 0;
            for (int64_t q = 0; q < mn; ++q) Zf[q] = rnd_store(ldexpf(Zf[q], -ez), rt);
            for (int64_t i = 0; i < m; ++i) tri_solve32(n, 1, lbf, cbf, iwbf, Zf + i * n, rt);
            upd = ldexp(pfac, e - sA + ez - sB);
            for (int64_t q = 0; q < mn; ++q) X[q] = fma(upd, (double)Zf[q], X[q]);
        }
        info->spmv_count++;
        ++k;
    }
    info->outer_iters = k;
    info->status = status;
    free(btl); free(btu); free(la); free(ca); free(iwa); free(lb); free(cb); free(iwb);
    free(laf); free(caf); free(iwaf); free(lbf); free(cbf); free(iwbf); free(R); free(Zf);
    return status;
}
