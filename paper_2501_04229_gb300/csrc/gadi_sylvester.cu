// gadi_sylvester.cu -- GADI-AB: GADI-IR (Algorithm 1) for the Sylvester
// equation A X + X B = C with tridiagonal A (m x m) and B (n x n) (§4.3).
//
// The operator L(X) = A X + X B is split into X -> A X and X -> X B (the
// paper's GADI-AB). One outer step:
//   R  = C - A X - X B                            FP64 (u_f)
//   R^ = fl_r(2^-e R),  e = floor(log2 max|R|)
//   Z  = H'^-1 R^       H' = 2^-sA (aI + A)       one tridiagonal solve per column
//   Z^ = fl_r(2^-ez Z), ez = floor(log2 max|Z|)
//   Y  = Z^ S'^-1       S' = 2^-sB (aI + B)       one tridiagonal solve per row
//   X += (2-w) a 2^(e - sA + ez - sB) Y           FP64 (u)
// The inner systems are tridiagonal and (a > 0, the paper's A and B)
// diagonally dominant, so each is solved directly (Thomas, no pivoting) in
// the inner precision: factors computed on the host in FP64 (one fused
// multiply-add per pivot), stored in FP32 (FP64 for the FP64 inner path);
// every stored intermediate is rounded to the storage type.
//
// Layout: X, C, R row-major m x n (FP64). The column solves run one thread
// per column down the rows (consecutive threads read consecutive
// addresses); Z^ is then written transposed (32 x 32 shared-memory tiles)
// so that the row solves run the same way on Z^T, and the update reads Y^T
// back through tiles. max|R|, max|X| and max|Z| are reduced per block and
// combined with integer atomicMax on the bit patterns of the non-negative
// values (order-free, so deterministic); e and ez are formed on the device.
// The host reads max|R| and max|X| once per outer step for the stop test.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/gadi.h"
#include "gadi_device.cuh"

using namespace gadi;

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 32;

__device__ __forceinline__ double dmax_of(const unsigned long long *bits) { return __longlong_as_double((long long)*bits); }

__device__ __forceinline__ unsigned long long abs_bits(double v)
{
    return (unsigned long long)__double_as_longlong(fabs(v));
}

// R = C - A X - X B (fused multiply-adds in the order A's i-1, i, i+1, then
// B's j-1, j, j+1); maxima of |R| (NaN above everything) and |X|. With R32,
// also the round-to-odd FP32 copy of R: fl16(2^-e R) is then an exact FP32
// scaling and one rounding (same bits as from FP64, for -100 <= e <= 126),
// without FP64 work in the sequential solves.
__global__ void k_residual(int64_t m, int64_t n, const double *__restrict__ al, const double *__restrict__ ad,
                           const double *__restrict__ au, const double *__restrict__ bl,
                           const double *__restrict__ bd, const double *__restrict__ bu,
                           const double *__restrict__ C, const double *__restrict__ X, double *__restrict__ R,
                           float *__restrict__ R32, unsigned long long *maxbits)
{
    unsigned long long rm = 0, xm = 0;
    const int64_t mn = m * n;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < mn; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / n, j = q - i * n;
        const double *x = X + q;
        double r = C[q];
        if (i > 0) r = __fma_rn(-al[i], x[-n], r);
        r = __fma_rn(-ad[i], x[0], r);
        if (i < m - 1) r = __fma_rn(-au[i], x[n], r);
        if (j > 0) r = __fma_rn(-bu[j - 1], x[-1], r);
        r = __fma_rn(-bd[j], x[0], r);
        if (j < n - 1) r = __fma_rn(-bl[j + 1], x[1], r);
        R[q] = r;
        if (R32) R32[q] = __uint_as_float(float_bits_round_odd(r));
        rm = max(rm, abs_bits(r));
        xm = max(xm, abs_bits(x[0]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        rm = max(rm, __shfl_xor_sync(0xffffffffu, rm, o));
        xm = max(xm, __shfl_xor_sync(0xffffffffu, xm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxbits, rm);
        atomicMax(maxbits + 1, xm);
    }
}

__global__ void k_absmax(int64_t cnt, const double *__restrict__ v, unsigned long long *maxbits)
{
    unsigned long long m = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += (int64_t)gridDim.x * blockDim.x)
        m = max(m, abs_bits(v[q]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(maxbits, m);
}

// e = floor(log2 max|R|) for the reduced inner precisions, else 0
__device__ __forceinline__ int exp_of(const unsigned long long *bits, int low)
{
    const double v = dmax_of(bits);
    return (low && v > 0.0 && isfinite(v)) ? ilogb(v) : 0;
}

// Tridiagonal solves along `count` lines of length len, line t at
// base + t, elements stride apart (consecutive threads: consecutive
// lines). The right-hand side is fl_T(2^-e R): FROM = 1 from the FP64 array
// src, FROM = 2 from its round-to-odd FP32 copy src32 (FP16 T); FROM = 0:
// the line already holds it (in T). Results (in T) go to dst.
// The maximum |result| goes to zmax (as float bits) when asked.
template <class T, int FROM>
__global__ void k_tri_lines(int64_t len, int64_t count, int64_t stride, const double *__restrict__ src,
                            const float *__restrict__ src32,
                            T *__restrict__ dst, const typename Prec<T>::Acc *__restrict__ ls,
                            const typename Prec<T>::Acc *__restrict__ cf, const typename Prec<T>::Acc *__restrict__ iw,
                            const unsigned long long *rmaxbits, int low, unsigned *zmaxbits)
{
    using P = Prec<T>;
    using Acc = typename P::Acc;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float zm = 0.0f;
    if (t < count) {
        double sc = 1.0;
        if constexpr (FROM != 0) sc = ldexp(1.0, -exp_of(rmaxbits, low));
        const float sc32 = (float)sc;
        auto rhs = [&](int64_t i) -> Acc {
            if constexpr (FROM == 1) {
                const double v = src[t + i * stride];
                return P::ld(P::from64(sc == 1.0 ? v : v * sc));
            } else if constexpr (FROM == 2) {
                return P::rnd(__fmul_rn(src32[t + i * stride], sc32));
            } else {
                return P::ld(dst[t + i * stride]);
            }
        };
        // the recurrences run element by element; their operands are loaded
        // KB at a time first, so a line's loads overlap instead of each one
        // waiting for the previous step
        constexpr int KB = 16;
        Acc y = Acc(0);
        for (int64_t i0 = 0; i0 < len; i0 += KB) {
            Acc v[KB], l[KB], w[KB];
#pragma unroll
            for (int k = 0; k < KB; ++k)
                if (i0 + k < len) {
                    v[k] = rhs(i0 + k);
                    l[k] = ls[i0 + k];
                    w[k] = iw[i0 + k];
                }
#pragma unroll
            for (int k = 0; k < KB; ++k)
                if (i0 + k < len) {
                    y = i0 + k == 0 ? P::rnd(P::mul(v[k], w[k])) : P::rnd(P::mul(P::madd(v[k], -l[k], y), w[k]));
                    dst[t + (i0 + k) * stride] = P::st(y);
                }
        }
        Acc z = y;
        zm = fabsf((float)z);
        // back substitution over i = len-2 .. 0, in chunks [i1 - KB + 1, i1]
        for (int64_t i1 = len - 2; i1 >= 0; i1 -= KB) {
            Acc v[KB], c[KB];
#pragma unroll
            for (int k = 0; k < KB; ++k)
                if (i1 - k >= 0) {
                    v[k] = P::ld(dst[t + (i1 - k) * stride]);
                    c[k] = cf[i1 - k];
                }
#pragma unroll
            for (int k = 0; k < KB; ++k)
                if (i1 - k >= 0) {
                    z = P::rnd(P::madd(v[k], -c[k], z));
                    dst[t + (i1 - k) * stride] = P::st(z);
                    zm = fmaxf(zm, fabsf((float)z));
                }
        }
    }
    if (zmaxbits) {
        for (int o = 16; o > 0; o >>= 1) zm = fmaxf(zm, __shfl_xor_sync(0xffffffffu, zm, o));
        if ((threadIdx.x & 31) == 0) atomicMax(zmaxbits, __float_as_uint(zm));
    }
}

// dst (n x m) = fl_T(2^-ez src^T), src m x n; 32 x 32 tiles through shared memory
template <class T>
__global__ void k_transpose_scale(int64_t m, int64_t n, const T *__restrict__ src, T *__restrict__ dst,
                                  const unsigned *zmaxbits, int low)
{
    using P = Prec<T>;
    using Acc = typename P::Acc;
    __shared__ Acc tile[kTile][kTile + 1];
    const float zmax = __uint_as_float(*zmaxbits);
    const int ez = (low && zmax > 0.0f && isfinite(zmax)) ? ilogb(zmax) : 0;
    const Acc sc = (Acc)ldexp(1.0, -ez);
    const int64_t i0 = (int64_t)blockIdx.y * kTile, j0 = (int64_t)blockIdx.x * kTile;
    for (int r = threadIdx.y; r < kTile; r += blockDim.y) {
        const int64_t i = i0 + r, j = j0 + threadIdx.x;
        if (i < m && j < n) tile[r][threadIdx.x] = P::rnd(P::mul(P::ld(src[i * n + j]), sc));
    }
    __syncthreads();
    for (int r = threadIdx.y; r < kTile; r += blockDim.y) {
        const int64_t j = j0 + r, i = i0 + threadIdx.x;
        if (i < m && j < n) dst[j * m + i] = P::st(tile[threadIdx.x][r]);
    }
}

// X[i][j] += (2-w) a 2^(e - sA + ez - sB) Y[i][j], Y given transposed (n x m)
template <class T>
__global__ void k_update(int64_t m, int64_t n, const T *__restrict__ yt, double *__restrict__ X, double pfac,
                         int sA, int sB, const unsigned long long *rmaxbits, const unsigned *zmaxbits, int low)
{
    using P = Prec<T>;
    using Acc = typename P::Acc;
    __shared__ Acc tile[kTile][kTile + 1];
    const int e = exp_of(rmaxbits, low);
    const float zmax = __uint_as_float(*zmaxbits);
    const int ez = (low && zmax > 0.0f && isfinite(zmax)) ? ilogb(zmax) : 0;
    const double upd = ldexp(pfac, e - sA + ez - sB);
    const int64_t i0 = (int64_t)blockIdx.y * kTile, j0 = (int64_t)blockIdx.x * kTile;
    for (int r = threadIdx.y; r < kTile; r += blockDim.y) {
        const int64_t j = j0 + r, i = i0 + threadIdx.x;
        if (i < m && j < n) tile[threadIdx.x][r] = P::ld(yt[j * m + i]);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < kTile; r += blockDim.y) {
        const int64_t i = i0 + r, j = j0 + threadIdx.x;
        if (i < m && j < n) X[i * n + j] = __fma_rn(upd, P::to64(tile[r][threadIdx.x]), X[i * n + j]);
    }
}

unsigned grid_for(int64_t work, int threads = kThreads)
{
    int64_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

// host: (|sigma| + max row sum) 2^-s in (1, 2]
int tri_scale_exponent(const std::vector<double> &lo, const std::vector<double> &dg, const std::vector<double> &up,
                       double sigma)
{
    const size_t m = dg.size();
    double nrm = 0.0;
    for (size_t i = 0; i < m; ++i) {
        double s = std::fabs(dg[i]);
        if (i > 0) s += std::fabs(lo[i]);
        if (i + 1 < m) s += std::fabs(up[i]);
        nrm = std::max(nrm, s);
    }
    nrm += std::fabs(sigma);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return 0;
    int e;
    const double mm = std::frexp(nrm, &e);
    return ((mm == 0.5) ? e - 1 : e) - 1;
}

// host: Thomas factors of 2^-s (sigma I + tridiag(lo, dg, up)) in FP64
void tri_factor(const std::vector<double> &lo, const std::vector<double> &dg, const std::vector<double> &up,
                double sigma, int s, std::vector<double> &ls, std::vector<double> &c, std::vector<double> &iw)
{
    const size_t m = dg.size();
    ls.assign(m, 0.0);
    c.assign(m, 0.0);
    iw.assign(m, 0.0);
    double w = 0.0;
    for (size_t i = 0; i < m; ++i) {
        const double d = std::ldexp(sigma + dg[i], -s);
        ls[i] = i > 0 ? std::ldexp(lo[i], -s) : 0.0;
        w = i > 0 ? std::fma(-ls[i], c[i - 1], d) : d;
        iw[i] = 1.0 / w;
        c[i] = i + 1 < m ? std::ldexp(up[i], -s) / w : 0.0;
    }
}

}  // namespace

struct gadi_sylv {
    int64_t m = 0, n = 0;
    cudaStream_t stream = nullptr;
    std::vector<double> hal, had, hau, hbl, hbd, hbu;       // host copies
    std::vector<double> btl, btu;                           // S^T off-diagonals
    double *al = nullptr, *ad = nullptr, *au = nullptr, *bl = nullptr, *bd = nullptr, *bu = nullptr;
    double *R = nullptr;
    void *Z = nullptr, *Zt = nullptr;                       // m n elements of up to 8 bytes
    void *fac = nullptr;                                    // 3 (m + n) factors of up to 8 bytes
    unsigned long long *maxbits = nullptr;                  // [0] max|R|, [1] max|X|, [2] max|C|, [3] max|Z| (float bits)
    double Ln = 0.0;
    double alpha = 1.0, omega = 1.0;
    int u_r = GADI_F16;
    int sA = 0, sB = 0;
    std::string err;
};

namespace {

gadi_status sfail(gadi_sylv *s, gadi_status st, const char *msg)
{
    if (s) s->err = msg;
    return st;
}

#define SCK(call)                                                                 \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            if (s) s->err = std::string(#call) + ": " + cudaGetErrorString(e_);   \
            return GADI_ERR_CUDA;                                                 \
        }                                                                         \
    } while (0)

void release(gadi_sylv *s)
{
    void *ptrs[] = {s->al, s->ad, s->au, s->bl, s->bd, s->bu, s->R, s->Z, s->Zt, s->fac, s->maxbits};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

template <class T>
gadi_status run(gadi_sylv *s, const double *C, double *X, double tol, int max_outer, gadi_info *info)
{
    using Acc = typename Prec<T>::Acc;
    const int64_t m = s->m, n = s->n, mn = m * n;
    const int low = std::is_same<T, double>::value ? 0 : 1;
    const bool scaled = std::is_same<T, __half>::value || std::is_same<T, __nv_bfloat16>::value;
    s->sA = scaled ? tri_scale_exponent(s->hal, s->had, s->hau, s->alpha) : 0;
    s->sB = scaled ? tri_scale_exponent(s->btl, s->hbd, s->btu, s->alpha) : 0;
    std::vector<double> la, ca, iwa, lb, cb, iwb;
    tri_factor(s->hal, s->had, s->hau, s->alpha, s->sA, la, ca, iwa);
    tri_factor(s->btl, s->hbd, s->btu, s->alpha, s->sB, lb, cb, iwb);
    std::vector<Acc> f;
    f.reserve(3 * (m + n));
    for (auto *v : {&la, &ca, &iwa}) for (double d : *v) f.push_back((Acc)d);
    for (auto *v : {&lb, &cb, &iwb}) for (double d : *v) f.push_back((Acc)d);
    Acc *fd = (Acc *)s->fac;
    SCK(cudaMemcpyAsync(fd, f.data(), f.size() * sizeof(Acc), cudaMemcpyHostToDevice, s->stream));
    const Acc *fla = fd, *fca = fd + m, *fiwa = fd + 2 * m;
    const Acc *flb = fd + 3 * m, *fcb = flb + n, *fiwb = flb + 2 * n;
    T *Z = (T *)s->Z, *Zt = (T *)s->Zt;
    // FP16 only: below 2^-126 the FP32 copy is not exact, which bfloat16's range would show
    constexpr bool k16 = std::is_same<T, __half>::value;
    float *R32 = k16 ? reinterpret_cast<float *>(Zt) : nullptr;   // Zt is free until the transpose
    unsigned *zbits = reinterpret_cast<unsigned *>(s->maxbits + 3);
    const double pfac = (2.0 - s->omega) * s->alpha;

    SCK(cudaMemsetAsync(s->maxbits + 2, 0, sizeof(unsigned long long), s->stream));
    k_absmax<<<grid_for(mn), kThreads, 0, s->stream>>>(mn, C, s->maxbits + 2);
    const dim3 tb(kTile, 8), tg((unsigned)((n + kTile - 1) / kTile), (unsigned)((m + kTile - 1) / kTile));
    const auto t0 = std::chrono::steady_clock::now();
    int k = 0, status = GADI_ERR_NOT_CONVERGED;
    double eta = 0.0;
    for (;;) {
        SCK(cudaMemsetAsync(s->maxbits, 0, 2 * sizeof(unsigned long long), s->stream));   // max|R|, max|X|
        k_residual<<<grid_for(mn), kThreads, 0, s->stream>>>(m, n, s->al, s->ad, s->au, s->bl, s->bd, s->bu, C, X,
                                                            s->R, R32, s->maxbits);
        unsigned long long hb[3];
        SCK(cudaMemcpyAsync(hb, s->maxbits, sizeof hb, cudaMemcpyDeviceToHost, s->stream));
        SCK(cudaStreamSynchronize(s->stream));
        double rmax, xmax, cmax;
        std::memcpy(&rmax, &hb[0], 8);
        std::memcpy(&xmax, &hb[1], 8);
        std::memcpy(&cmax, &hb[2], 8);
        if (!std::isfinite(rmax)) { status = GADI_ERR_DIVERGED; break; }
        const double den = s->Ln * xmax + cmax;
        eta = den > 0.0 ? rmax / den : (rmax == 0.0 ? 0.0 : INFINITY);
        if (eta <= tol) { status = GADI_OK; break; }
        if (k >= max_outer) break;
        SCK(cudaMemsetAsync(zbits, 0, sizeof(unsigned), s->stream));
        // one warp per block: the lines spread over as many SMs as there are warps of lines
        const int e = (rmax > 0.0) ? std::ilogb(rmax) : 0;
        if (k16 && e >= -100 && e <= 126)
            k_tri_lines<T, 2><<<grid_for(n, 32), 32, 0, s->stream>>>(m, n, n, nullptr, R32, Z, fla, fca, fiwa,
                                                                     s->maxbits, low, zbits);
        else
            k_tri_lines<T, 1><<<grid_for(n, 32), 32, 0, s->stream>>>(m, n, n, s->R, nullptr, Z, fla, fca, fiwa,
                                                                     s->maxbits, low, zbits);
        k_transpose_scale<T><<<tg, tb, 0, s->stream>>>(m, n, Z, Zt, zbits, low);
        k_tri_lines<T, 0><<<grid_for(m, 32), 32, 0, s->stream>>>(n, m, m, nullptr, nullptr, Zt, flb, fcb, fiwb,
                                                                 nullptr, low, nullptr);
        k_update<T><<<tg, tb, 0, s->stream>>>(m, n, Zt, X, pfac, s->sA, s->sB, s->maxbits, zbits, low);
        SCK(cudaGetLastError());
        ++k;
    }
    SCK(cudaGetLastError());
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->outer_iters = k;
        info->status = status;
        info->eta_inf = eta;
        info->res_rel = eta;
        info->t_solve_s = secs;
        info->scale_exp_M = s->sA;
        info->scale_exp_N = s->sB;
        info->kernel = GADI_KERNEL_AUTO;
        info->block_threads = kThreads;
    }
    if (status == GADI_ERR_NOT_CONVERGED) return sfail(s, GADI_ERR_NOT_CONVERGED, "max_outer reached before the tolerance");
    if (status == GADI_ERR_DIVERGED) return sfail(s, GADI_ERR_DIVERGED, "the residual is not finite");
    return GADI_OK;
}

bool is_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

gadi_status gadi_sylv_create(int64_t m, int64_t n, const double *a_lo, const double *a_diag, const double *a_up,
                             const double *b_lo, const double *b_diag, const double *b_up, void *cuda_stream,
                             gadi_sylv **out)
{
    if (!out) return GADI_ERR_INVALID_ARG;
    *out = nullptr;
    if (m < 1 || n < 1 || m * n > ((int64_t)1 << 31) || !a_lo || !a_diag || !a_up || !b_lo || !b_diag || !b_up)
        return GADI_ERR_INVALID_ARG;
    gadi_sylv *s = new gadi_sylv;
    s->m = m;
    s->n = n;
    s->stream = (cudaStream_t)cuda_stream;
    s->hal.assign(a_lo, a_lo + m);
    s->had.assign(a_diag, a_diag + m);
    s->hau.assign(a_up, a_up + m);
    s->hbl.assign(b_lo, b_lo + n);
    s->hbd.assign(b_diag, b_diag + n);
    s->hbu.assign(b_up, b_up + n);
    s->hal[0] = 0.0;
    s->hau[m - 1] = 0.0;
    s->hbl[0] = 0.0;
    s->hbu[n - 1] = 0.0;
    for (int64_t i = 0; i < m; ++i)
        if (!std::isfinite(s->hal[i]) || !std::isfinite(s->had[i]) || !std::isfinite(s->hau[i])) {
            delete s;
            return GADI_ERR_INVALID_ARG;
        }
    for (int64_t j = 0; j < n; ++j)
        if (!std::isfinite(s->hbl[j]) || !std::isfinite(s->hbd[j]) || !std::isfinite(s->hbu[j])) {
            delete s;
            return GADI_ERR_INVALID_ARG;
        }
    // the row solves use S^T: sub-diagonal B[j-1][j] = b_up[j-1], super-diagonal B[j+1][j] = b_lo[j+1]
    s->btl.assign(n, 0.0);
    s->btu.assign(n, 0.0);
    for (int64_t j = 0; j < n; ++j) {
        s->btl[j] = j > 0 ? s->hbu[j - 1] : 0.0;
        s->btu[j] = j < n - 1 ? s->hbl[j + 1] : 0.0;
    }
    // ||L||_inf of vec(X) -> vec(A X + X B): the largest row sum of I (x) A + B^T (x) I
    std::vector<double> sa(m), sb(n);
    for (int64_t i = 0; i < m; ++i) sa[i] = std::fabs(s->hal[i]) + std::fabs(s->hau[i]);
    for (int64_t j = 0; j < n; ++j) sb[j] = std::fabs(s->btl[j]) + std::fabs(s->btu[j]);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = 0; j < n; ++j) s->Ln = std::max(s->Ln, sa[i] + sb[j] + std::fabs(s->had[i] + s->hbd[j]));
    const int64_t mn = m * n;
    bool ok = cudaMalloc(&s->al, m * 8) == cudaSuccess && cudaMalloc(&s->ad, m * 8) == cudaSuccess &&
              cudaMalloc(&s->au, m * 8) == cudaSuccess && cudaMalloc(&s->bl, n * 8) == cudaSuccess &&
              cudaMalloc(&s->bd, n * 8) == cudaSuccess && cudaMalloc(&s->bu, n * 8) == cudaSuccess &&
              cudaMalloc(&s->R, mn * 8) == cudaSuccess && cudaMalloc(&s->Z, mn * 8) == cudaSuccess &&
              cudaMalloc(&s->Zt, mn * 8) == cudaSuccess && cudaMalloc(&s->fac, 3 * (m + n) * 8) == cudaSuccess &&
              cudaMalloc(&s->maxbits, 4 * sizeof(unsigned long long)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release(s);
        delete s;
        return GADI_ERR_OUT_OF_MEMORY;
    }
    cudaError_t e = cudaSuccess;
    const std::pair<double *, const std::vector<double> *> up[] = {
        {s->al, &s->hal}, {s->ad, &s->had}, {s->au, &s->hau}, {s->bl, &s->hbl}, {s->bd, &s->hbd}, {s->bu, &s->hbu}};
    for (auto &u : up)
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(u.first, u.second->data(), u.second->size() * 8, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(s);
        delete s;
        return GADI_ERR_CUDA;
    }
    *out = s;
    return GADI_OK;
}

gadi_status gadi_sylv_set_params(gadi_sylv *s, double alpha, double omega, gadi_precision u_r)
{
    if (!s) return GADI_ERR_INVALID_ARG;
    if (!(alpha > 0.0) || !std::isfinite(alpha)) return sfail(s, GADI_ERR_INVALID_ARG, "alpha must be positive");
    if (!(omega >= 0.0 && omega < 2.0)) return sfail(s, GADI_ERR_INVALID_ARG, "omega must lie in [0, 2)");
    if (u_r < GADI_F64 || u_r > GADI_E4M3) return sfail(s, GADI_ERR_INVALID_ARG, "unknown precision");
    if (u_r == GADI_E4M3) return sfail(s, GADI_ERR_UNSUPPORTED, "no FP8 inner precision for the Sylvester solver");
    s->alpha = alpha;
    s->omega = omega;
    s->u_r = u_r;
    return GADI_OK;
}

gadi_status gadi_sylv_solve(gadi_sylv *s, const double *C, double *X, double tol, int32_t max_outer, gadi_info *info)
{
    if (!s) return GADI_ERR_INVALID_ARG;
    if (!C || !X || !is_device(C) || !is_device(X))
        return sfail(s, GADI_ERR_INVALID_ARG, "C and X must be device pointers");
    if (!(tol >= 0.0) || max_outer < 0) return sfail(s, GADI_ERR_INVALID_ARG, "tol >= 0 and max_outer >= 0");
    switch (s->u_r) {
    case GADI_F16: return run<__half>(s, C, X, tol, max_outer, info);
    case GADI_BF16: return run<__nv_bfloat16>(s, C, X, tol, max_outer, info);
    case GADI_F32: return run<float>(s, C, X, tol, max_outer, info);
    default: return run<double>(s, C, X, tol, max_outer, info);
    }
}

const char *gadi_sylv_last_error(const gadi_sylv *s)
{
    return s ? s->err.c_str() : "null handle";
}

void gadi_sylv_destroy(gadi_sylv *s)
{
    if (!s) return;
    release(s);
    delete s;
}

}  // extern "C"
