// gadi_ops.cuh -- the operators of GADI-IR for the persistent kernel, and the
// vector expressions they are applied to.
//
//   kOpA  : (A x)_i                       FP64 (outer residual, Alg. 1 step 1)
//   kOpH  : (H' x)_i = 2^-sM (aI + M) x   inner precision (Alg. 1 step 2)
//   kOpS  : (S' x)_i = 2^-sN (aI + N) x   inner precision (Alg. 1 step 3)
//   kOpST : (S'^T x)_i                    (CGNR's transpose product)
//
// Work is done in items of R consecutive rows (R = 1 for the general sparse
// operator; R = 4 or 8 for the stencil when the grid side is a multiple of
// R: one 8- or 16-byte FP16 load per vector and one coordinate computation
// per item).
//
// A row is evaluated as sigma*f(i) first, then the matrix entries in
// ascending column order (the CSR order), each term one fused multiply-add:
// in FP32 for the FP16 inner precision, in FP64 for the residual and the
// FP64 inner path. So a row equals, bit for bit, the same sum formed on the
// CPU.
//
// The vector argument is an expression object with one(j) (value at column
// j) and many<K>(j0, out) (values at j0..j0+K-1, j0 a multiple of K); the kernel
// passes expressions such as "r + beta p rounded to FP16" so that vector
// updates of a Krylov step fuse into the next operator application.
#pragma once

#include "gadi_device.cuh"

namespace gadi {

enum : int { kOpA = 0, kOpH = 1, kOpS = 2, kOpST = 3 };

// ---------------------------------------------------------------------------
// K-wide loads and stores of FP16 / FP64 vectors (K = 4 or 8; one 8- or
// 16-byte transaction per FP16 chunk)
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void ldv(const __half *p, int64_t j0, float (&o)[K])
{
    static_assert(K == 4 || K == 8, "chunk width");
    if constexpr (K == 8) {
        const uint4 u = *reinterpret_cast<const uint4 *>(p + j0);
        const __half2 *h = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __half22float2(h[k]);
            o[2 * k] = f.x;
            o[2 * k + 1] = f.y;
        }
    } else {
        const uint2 u = *reinterpret_cast<const uint2 *>(p + j0);
        const __half2 *h = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float2 f = __half22float2(h[k]);
            o[2 * k] = f.x;
            o[2 * k + 1] = f.y;
        }
    }
}

template <int K>
__device__ __forceinline__ void stv(__half *p, int64_t j0, const float (&v)[K])
{
    if constexpr (K == 8) {
        uint4 u;
        __half2 *h = reinterpret_cast<__half2 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = __float22half2_rn(make_float2(v[2 * k], v[2 * k + 1]));
        *reinterpret_cast<uint4 *>(p + j0) = u;
    } else {
        uint2 u;
        __half2 *h = reinterpret_cast<__half2 *>(&u);
#pragma unroll
        for (int k = 0; k < 2; ++k) h[k] = __float22half2_rn(make_float2(v[2 * k], v[2 * k + 1]));
        *reinterpret_cast<uint2 *>(p + j0) = u;
    }
}

template <int K>
__device__ __forceinline__ void ldv(const __nv_bfloat16 *p, int64_t j0, float (&o)[K])
{
    static_assert(K == 4 || K == 8, "chunk width");
    if constexpr (K == 8) {
        const uint4 u = *reinterpret_cast<const uint4 *>(p + j0);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __bfloat1622float2(h[k]);
            o[2 * k] = f.x;
            o[2 * k + 1] = f.y;
        }
    } else {
        const uint2 u = *reinterpret_cast<const uint2 *>(p + j0);
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float2 f = __bfloat1622float2(h[k]);
            o[2 * k] = f.x;
            o[2 * k + 1] = f.y;
        }
    }
}

template <int K>
__device__ __forceinline__ void stv(__nv_bfloat16 *p, int64_t j0, const float (&v)[K])
{
    if constexpr (K == 8) {
        uint4 u;
        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = __float22bfloat162_rn(make_float2(v[2 * k], v[2 * k + 1]));
        *reinterpret_cast<uint4 *>(p + j0) = u;
    } else {
        uint2 u;
        __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
        for (int k = 0; k < 2; ++k) h[k] = __float22bfloat162_rn(make_float2(v[2 * k], v[2 * k + 1]));
        *reinterpret_cast<uint2 *>(p + j0) = u;
    }
}

// FP8 E4M3 chunks: one 4- or 8-byte transaction; element j0 + k is byte k
// (little endian), pairs convert through FP16 (exact)
template <int K>
__device__ __forceinline__ void ldv(const __nv_fp8_e4m3 *p, int64_t j0, float (&o)[K])
{
    static_assert(K == 4 || K == 8, "chunk width");
    uint32_t w[K / 4];
    if constexpr (K == 8) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p + j0);
        w[0] = u.x;
        w[1] = u.y;
    } else {
        w[0] = *reinterpret_cast<const uint32_t *>(p + j0);
    }
#pragma unroll
    for (int k = 0; k < K / 2; ++k) {
        const __nv_fp8x2_storage_t q = (__nv_fp8x2_storage_t)(w[k / 2] >> (16 * (k % 2)));
        const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(q, __NV_E4M3)));
        o[2 * k] = f.x;
        o[2 * k + 1] = f.y;
    }
}

template <int K>
__device__ __forceinline__ void stv(__nv_fp8_e4m3 *p, int64_t j0, const float (&v)[K])
{
    uint32_t w[K / 4];
#pragma unroll
    for (int k = 0; k < K / 4; ++k) w[k] = 0u;
#pragma unroll
    for (int k = 0; k < K / 2; ++k) {
        const __nv_fp8x2_storage_t q =
            __nv_cvt_float2_to_fp8x2(make_float2(v[2 * k], v[2 * k + 1]), __NV_SATFINITE, __NV_E4M3);
        w[k / 2] |= (uint32_t)q << (16 * (k % 2));
    }
    if constexpr (K == 8) *reinterpret_cast<uint2 *>(p + j0) = make_uint2(w[0], w[1]);
    else *reinterpret_cast<uint32_t *>(p + j0) = w[0];
}

template <int K>
__device__ __forceinline__ void ldv(const float *p, int64_t j0, float (&o)[K])
{
    const float4 *q = reinterpret_cast<const float4 *>(p + j0);
#pragma unroll
    for (int k = 0; k < K / 4; ++k) {
        const float4 d = q[k];
        o[4 * k] = d.x;
        o[4 * k + 1] = d.y;
        o[4 * k + 2] = d.z;
        o[4 * k + 3] = d.w;
    }
}

template <int K>
__device__ __forceinline__ void stv(float *p, int64_t j0, const float (&v)[K])
{
    float4 *q = reinterpret_cast<float4 *>(p + j0);
#pragma unroll
    for (int k = 0; k < K / 4; ++k) q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
}

template <int K>
__device__ __forceinline__ void ldv(const double *p, int64_t j0, double (&o)[K])
{
    const double2 *q = reinterpret_cast<const double2 *>(p + j0);
#pragma unroll
    for (int k = 0; k < K / 2; ++k) {
        const double2 d = q[k];
        o[2 * k] = d.x;
        o[2 * k + 1] = d.y;
    }
}

template <int K>
__device__ __forceinline__ void stv(double *p, int64_t j0, const double (&v)[K])
{
    double2 *q = reinterpret_cast<double2 *>(p + j0);
#pragma unroll
    for (int k = 0; k < K / 2; ++k) q[k] = make_double2(v[2 * k], v[2 * k + 1]);
}

// Raw 8-element chunks: the load split from the conversion, so that a
// chunk can be requested one loop iteration before it is used (z-marching)
template <class T> struct Raw8;
template <> struct Raw8<__half> { uint4 u; };
template <> struct Raw8<float> { float4 a, b; };
template <> struct Raw8<double> { double2 a, b, c, d; };

__device__ __forceinline__ void ldraw8(const __half *p, int64_t j0, Raw8<__half> &r)
{
    r.u = *reinterpret_cast<const uint4 *>(p + j0);
}
__device__ __forceinline__ void ldraw8(const float *p, int64_t j0, Raw8<float> &r)
{
    const float4 *q = reinterpret_cast<const float4 *>(p + j0);
    r.a = q[0];
    r.b = q[1];
}
__device__ __forceinline__ void ldraw8(const double *p, int64_t j0, Raw8<double> &r)
{
    const double2 *q = reinterpret_cast<const double2 *>(p + j0);
    r.a = q[0];
    r.b = q[1];
    r.c = q[2];
    r.d = q[3];
}
__device__ __forceinline__ void cvt8(const Raw8<__half> &r, float (&o)[8])
{
    const __half2 *h = reinterpret_cast<const __half2 *>(&r.u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __half22float2(h[k]);
        o[2 * k] = f.x;
        o[2 * k + 1] = f.y;
    }
}
__device__ __forceinline__ void cvt8(const Raw8<float> &r, float (&o)[8])
{
    o[0] = r.a.x; o[1] = r.a.y; o[2] = r.a.z; o[3] = r.a.w;
    o[4] = r.b.x; o[5] = r.b.y; o[6] = r.b.z; o[7] = r.b.w;
}
__device__ __forceinline__ void cvt8(const Raw8<double> &r, double (&o)[8])
{
    o[0] = r.a.x; o[1] = r.a.y; o[2] = r.b.x; o[3] = r.b.y;
    o[4] = r.c.x; o[5] = r.c.y; o[6] = r.d.x; o[7] = r.d.y;
}

// own-row access of an item of R rows; values rounded to T on store
template <class T, int R>
struct ItemIO {
    using Acc = typename Prec<T>::Acc;
    static __device__ __forceinline__ void ld(const T *p, int64_t item, Acc (&o)[R])
    {
        if constexpr (R > 1) ldv<R>(p, item * R, o);
        else o[0] = Prec<T>::ld(p[item]);
    }
    static __device__ __forceinline__ void st(T *p, int64_t item, const Acc (&v)[R])
    {
        if constexpr (R > 1) stv<R>(p, item * R, v);
        else p[item] = Prec<T>::st(v[0]);
    }
};

template <int R>
struct ItemIO64 {
    static __device__ __forceinline__ void ld(const double *p, int64_t item, double (&o)[R])
    {
        if constexpr (R > 1) ldv<R>(p, item * R, o);
        else o[0] = p[item];
    }
    static __device__ __forceinline__ void st(double *p, int64_t item, const double (&v)[R])
    {
        if constexpr (R > 1) stv<R>(p, item * R, v);
        else p[item] = v[0];
    }
};

// ---------------------------------------------------------------------------
// Vector expressions (value of an inner-precision vector at column j)
// ---------------------------------------------------------------------------
template <class T>
struct XLoad {                       // a
    using Acc = typename Prec<T>::Acc;
    using Val = Acc;
    const T *a;
    __device__ __forceinline__ Acc one(int64_t j) const { return Prec<T>::ld(a[j]); }
    template <int K>
    __device__ __forceinline__ void many(int64_t j0, Acc (&o)[K]) const { ldv<K>(a, j0, o); }
    struct Raw { Raw8<T> v; };
    __device__ __forceinline__ void load8(int64_t j0, Raw &w) const { ldraw8(a, j0, w.v); }
    __device__ __forceinline__ void eval8(const Raw &w, Acc (&o)[8]) const { cvt8(w.v, o); }
};

template <class T>
struct XAxpy {                       // fl(a + c b)
    using Acc = typename Prec<T>::Acc;
    using Val = Acc;
    using P = Prec<T>;
    const T *a, *b;
    Acc c;
    __device__ __forceinline__ Acc one(int64_t j) const { return P::rnd(P::madd(P::ld(a[j]), c, P::ld(b[j]))); }
    template <int K>
    __device__ __forceinline__ void many(int64_t j0, Acc (&o)[K]) const
    {
        Acc x[K], y[K];
        ldv<K>(a, j0, x);
        ldv<K>(b, j0, y);
        P::madd_s(o, x, c, y);
        P::rndv(o);
    }
    struct Raw { Raw8<T> v[2]; };
    __device__ __forceinline__ void load8(int64_t j0, Raw &w) const
    {
        ldraw8(a, j0, w.v[0]);
        ldraw8(b, j0, w.v[1]);
    }
    __device__ __forceinline__ void eval8(const Raw &w, Acc (&o)[8]) const
    {
        Acc x[8], y[8];
        cvt8(w.v[0], x);
        cvt8(w.v[1], y);
        P::madd_s(o, x, c, y);
        P::rndv(o);
    }
};

template <class T>
struct XAxpy2 {                      // fl(a - c fl(b + d e))  (C-G residual update, fused)
    using Acc = typename Prec<T>::Acc;
    using Val = Acc;
    using P = Prec<T>;
    const T *a, *b, *e;
    Acc c, d;
    __device__ __forceinline__ Acc one(int64_t j) const
    {
        const Acc s = P::rnd(P::madd(P::ld(b[j]), d, P::ld(e[j])));
        return P::rnd(P::madd(P::ld(a[j]), -c, s));
    }
    template <int K>
    __device__ __forceinline__ void many(int64_t j0, Acc (&o)[K]) const
    {
        Acc x[K], y[K], w[K];
        ldv<K>(a, j0, x);
        ldv<K>(b, j0, y);
        ldv<K>(e, j0, w);
        P::madd_s(w, y, d, w);
        P::rndv(w);
        P::madd_s(o, x, -c, w);
        P::rndv(o);
    }
    struct Raw { Raw8<T> v[3]; };
    __device__ __forceinline__ void load8(int64_t j0, Raw &r) const
    {
        ldraw8(a, j0, r.v[0]);
        ldraw8(b, j0, r.v[1]);
        ldraw8(e, j0, r.v[2]);
    }
    __device__ __forceinline__ void eval8(const Raw &r, Acc (&o)[8]) const
    {
        Acc x[8], y[8], w[8];
        cvt8(r.v[0], x);
        cvt8(r.v[1], y);
        cvt8(r.v[2], w);
        P::madd_s(w, y, d, w);
        P::rndv(w);
        P::madd_s(o, x, -c, w);
        P::rndv(o);
    }
};

template <class T>
struct XScale {                      // fl(c a): c a power of two, or (2-w) a in the unscaled mode
    using Acc = typename Prec<T>::Acc;
    using Val = Acc;
    using P = Prec<T>;
    const T *a;
    Acc c;
    __device__ __forceinline__ Acc one(int64_t j) const { return P::rnd(P::mul(P::ld(a[j]), c)); }
    template <int K>
    __device__ __forceinline__ void many(int64_t j0, Acc (&o)[K]) const
    {
        Acc x[K];
        ldv<K>(a, j0, x);
        P::mul_s(o, c, x);
        P::rndv(o);
    }
    struct Raw { Raw8<T> v; };
    __device__ __forceinline__ void load8(int64_t j0, Raw &w) const { ldraw8(a, j0, w.v); }
    __device__ __forceinline__ void eval8(const Raw &w, Acc (&o)[8]) const
    {
        Acc x[8];
        cvt8(w.v, x);
        P::mul_s(o, c, x);
        P::rndv(o);
    }
};

template <class T>
struct XDemote {                     // fl_T(2^-e r), r in FP64 (Alg. 1: r^ = fl_r(s^))
    using Acc = typename Prec<T>::Acc;
    using Val = Acc;
    const double *r;
    double sc;                       // 2^-e
    struct Raw { Raw8<double> v; };
    __device__ __forceinline__ void load8(int64_t j0, Raw &w) const { ldraw8(r, j0, w.v); }
    __device__ __forceinline__ void eval8(const Raw &w, Acc (&o)[8]) const
    {
        double x[8];
        cvt8(w.v, x);
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = Prec<T>::ld(Prec<T>::from64(sc == 1.0 ? x[k] : x[k] * sc));
    }
    __device__ __forceinline__ Acc one(int64_t j) const
    {
        return Prec<T>::ld(Prec<T>::from64(sc == 1.0 ? r[j] : r[j] * sc));
    }
    template <int K>
    __device__ __forceinline__ void many(int64_t j0, Acc (&o)[K]) const
    {
        double x[K];
        ldv<K>(r, j0, x);
#pragma unroll
        for (int k = 0; k < K; ++k) o[k] = Prec<T>::ld(Prec<T>::from64(sc == 1.0 ? x[k] : x[k] * sc));
    }
};

// fl_T(2^-e r) (T = FP16 or FP8) from the round-to-odd FP32 copy of r: an
// exact FP32 scaling and one round-to-nearest-even conversion give the same
// value as the direct conversion from FP64 (valid for -100 <= e <= 126,
// where entries below the FP32 normal range round to zero either way)
template <class T>
struct XDemoteOdd {
    using Val = float;
    const float *r32;
    float sc;                        // 2^-e
    __device__ __forceinline__ float one(int64_t j) const
    {
        return Prec<T>::rnd(__fmul_rn(r32[j], sc));
    }
    template <int K>
    __device__ __forceinline__ void many(int64_t j0, float (&o)[K]) const
    {
        float x[K];
        ldv<K>(r32, j0, x);
        Prec<__half>::mul_s(x, sc, x);
        Prec<T>::rndv(x);
#pragma unroll
        for (int k = 0; k < K; ++k) o[k] = x[k];
    }
    struct Raw { Raw8<float> v; };
    __device__ __forceinline__ void load8(int64_t j0, Raw &w) const { ldraw8(r32, j0, w.v); }
    __device__ __forceinline__ void eval8(const Raw &w, float (&o)[8]) const
    {
        float x[8];
        cvt8(w.v, x);
        Prec<__half>::mul_s(x, sc, x);
        Prec<T>::rndv(x);
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = x[k];
    }
};

struct XLoad64 {
    using Val = double;
    const double *a;
    __device__ __forceinline__ double one(int64_t j) const { return a[j]; }
    template <int K>
    __device__ __forceinline__ void many(int64_t j0, double (&o)[K]) const { ldv<K>(a, j0, o); }
    struct Raw { Raw8<double> v; };
    __device__ __forceinline__ void load8(int64_t j0, Raw &w) const { ldraw8(a, j0, w.v); }
    __device__ __forceinline__ void eval8(const Raw &w, double (&o)[8]) const { cvt8(w.v, o); }
};

// ---------------------------------------------------------------------------
// General sparse matrix in row-major ELL form built from the CSR input:
// W slots per row (W = longest row rounded up to a multiple of 4), columns
// ascending, padding slots hold column = row and value 0 at the end of the
// row. M and N (the splitting) share A's pattern and column array.
// NT holds N^T's values on the same pattern when N is not skew-symmetric
// (user splitting); for HSS N^T = -N and NT is null.
// ---------------------------------------------------------------------------
template <class T>
struct EllOp {
    using Acc = typename Prec<T>::Acc;
    static constexpr int R = 1;
    static constexpr bool kZMarch = false;          // grid-stride rows only
    int64_t n;
    int W;
    const int *__restrict__ col;
    const double *__restrict__ a64;   // A values (FP64)
    const T *__restrict__ m;          // 2^-sM M in the inner precision
    const T *__restrict__ nv;         // 2^-sN N
    const T *__restrict__ nt;         // 2^-sN N^T, or null when N^T = -N
    Acc sigH, sigS;                   // 2^-sM alpha, 2^-sN alpha

    // the column indices of a row of the common width 8 (5- and 7-point
    // rows), two 16-byte loads
    __device__ __forceinline__ void cols8(const int *c, int (&cc)[8]) const
    {
        const int4 c0 = __ldg(reinterpret_cast<const int4 *>(c));
        const int4 c1 = __ldg(reinterpret_cast<const int4 *>(c) + 1);
        cc[0] = c0.x; cc[1] = c0.y; cc[2] = c0.z; cc[3] = c0.w;
        cc[4] = c1.x; cc[5] = c1.y; cc[6] = c1.z; cc[7] = c1.w;
    }

    // Rows of width 8 read their columns and values with vector loads and
    // issue all eight gathers before the first product; the products are
    // summed in the same (ascending column) order as for any other width.
    // kRes: start from init and subtract every product (init - A x, one
    // fused multiply-add per term); else A x from zero.
    template <bool kRes, class F>
    __device__ __forceinline__ void rowsA_t(int64_t i, const F &f, const double (&init)[1], double (&out)[1]) const
    {
        const int *c = col + i * W;
        const double *v = a64 + i * W;
        const double sg = kRes ? -1.0 : 1.0;
        double acc = kRes ? init[0] : 0.0;
        if (W == 8) {
            int cc[8];
            double vv[8], xv[8];
            cols8(c, cc);
            ldv<8>(v, 0, vv);
#pragma unroll
            for (int k = 0; k < 8; ++k) xv[k] = f.one(cc[k]);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc = __fma_rn(sg * vv[k], xv[k], acc);
        } else {
            for (int k = 0; k < W; ++k) acc = __fma_rn(sg * __ldg(v + k), f.one(__ldg(c + k)), acc);
        }
        out[0] = acc;
    }
    template <class F>
    __device__ __forceinline__ void rowsA(int64_t i, const F &f, double (&out)[1]) const
    {
        const double z[1] = {0.0};
        rowsA_t<false>(i, f, z, out);
    }
    // r = b - A x for the outer residual (Algorithm 1 step 1)
    template <class F>
    __device__ __forceinline__ void resid(int64_t i, const F &f, const double (&b)[1], double (&out)[1]) const
    {
        rowsA_t<true>(i, f, b, out);
    }

    template <class F>
    __device__ __forceinline__ void rows(int which, int64_t i, const F &f, Acc (&out)[1]) const
    {
        using P = Prec<T>;
        const int *c = col + i * W;
        const T *v;
        Acc sig, sgn = Acc(1);
        if (which == kOpH) { v = m; sig = sigH; }
        else if (which == kOpS) { v = nv; sig = sigS; }
        else if (nt) { v = nt; sig = sigS; }
        else { v = nv; sig = sigS; sgn = Acc(-1); }
        v += i * W;
        Acc acc = P::mul(sig, f.one(i));
        if (W == 8) {
            int cc[8];
            Acc vv[8], xv[8];
            cols8(c, cc);
            ldv<8>(v, 0, vv);
#pragma unroll
            for (int k = 0; k < 8; ++k) xv[k] = f.one(cc[k]);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc = P::madd(acc, sgn * vv[k], xv[k]);
        } else {
            for (int k = 0; k < W; ++k) acc = P::madd(acc, sgn * P::ld(v[k]), f.one(__ldg(c + k)));
        }
        out[0] = acc;
    }
};

// ---------------------------------------------------------------------------
// Matrix-free 5-point (2D) / 7-point (3D) convection-diffusion operator of
// §4.1 on an N^dim grid, x fastest; R > 1 needs N % R == 0 (an item is R
// nodes of one x-line). Constant-k form: scalar coefficients. Face form:
// per-node arrays of the diagonal and of the upper-face couplings per axis
// (M is symmetric, so the lower coupling of node i along d is the upper
// coupling of node i - e_d). N is the constant convection c in both forms.
// ---------------------------------------------------------------------------
// the multiplier of StencilOp::divide for side N
__host__ __device__ inline unsigned long long div_magic(unsigned N)
{
    return N <= 1 ? 0ull : ~0ull / N + 1;
}

template <class T, int DIM, int RR>
struct StencilOp {
    using Acc = typename Prec<T>::Acc;
    static constexpr int kDim = DIM;
    static constexpr int R = RR;
    int dim, N;
    int64_t n;
    // FP64 A for the residual: constant form (a_diag, a_lo, a_hi); face form
    // AD[i], AL[d][i] = a_{i,i-e_d}, AU[d][i] = a_{i,i+e_d}
    double a_diag, a_lo, a_hi;
    const double *__restrict__ AD;
    const double *__restrict__ AL[3];
    const double *__restrict__ AU[3];
    // inner: constant form (h_diag, h_off); face form HD[i] = 2^-sM m_ii,
    // HK[d][i] = 2^-sM m_{i,i+e_d}; S' coupling 2^-sN c rounded to T
    Acc h_diag, h_off, s_c;
    const T *__restrict__ HD;
    const T *__restrict__ HK[3];
    Acc sigH, sigS;
    // unscaled FP16 mode: alpha rounded to T as S's stored diagonal, added at
    // the diagonal's place in the row (zero otherwise: alpha is in sigS)
    Acc s_diag;

    unsigned long long divN;          // ceil(2^64 / N) (0 for N = 1): v / N = mulhi(v, divN)

    // v / N for v < 2^31: floor(v ceil(2^64/N) / 2^64) is exact, as the
    // error v (ceil(2^64/N) N - 2^64) / (N 2^64) < 2^-33 stays below 1/N
    __device__ __forceinline__ unsigned divide(unsigned v) const
    {
        return divN ? (unsigned)__umul64hi((unsigned long long)v, divN) : v;
    }

    // grid coordinates of node i (x fastest); n < 2^31 is enforced at create
    __device__ __forceinline__ void coords(int64_t i, unsigned (&cd)[3]) const
    {
        const unsigned ii = (unsigned)i, NN = (unsigned)N;
        const unsigned t = divide(ii);
        cd[0] = ii - t * NN;
        if (DIM == 3) {
            const unsigned u = divide(t);
            cd[1] = t - u * NN;
            cd[2] = u;
        } else {
            cd[1] = t;
            cd[2] = 0;
        }
    }

    __device__ __forceinline__ int64_t stride(int d) const
    {
        return d == 0 ? 1 : (d == 1 ? (int64_t)N : (int64_t)N * N);
    }

    // ---- z-marching rows (3D, constant coefficients, 8-row items) ------------
    // A thread marches along z through one column of items (the 8-row chunk
    // of an x-line at fixed y): the values of the planes below and above
    // (zl, zu) and its own (c) come from the march; only the y neighbours
    // and the two x ends are loaded. The terms and their order are those of
    // rows() and resid(), so every row has the same bits.
    static constexpr bool kZMarchCapable = DIM == 3 && RR == 8 && std::is_same<T, __half>::value;
    static constexpr bool kZMarch = false;          // grid-stride items (ZMarchOp marches)
    struct ZCol {                     // the column's boundary flags (fixed along z)
        bool hly, huy, hxm, hxp;
    };
    __device__ __forceinline__ ZCol zcol(int64_t col) const
    {
        const unsigned nx8 = (unsigned)N / 8;
        const unsigned y = (unsigned)col / nx8, xc = (unsigned)col - y * nx8;
        const unsigned last = (unsigned)N - 1;
        return ZCol{y > 0, y < last, xc > 0, xc * 8 + 8 <= last};
    }
    template <class F, class V>
    __device__ __forceinline__ void zm_gather(int64_t i0, const ZCol &zc, const F &f, V (&yl)[8], V (&yu)[8],
                                              V &xm, V &xp) const
    {
        if (zc.hly) {
            f.template many<8>(i0 - N, yl);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) yl[k] = V(0);
        }
        if (zc.huy) {
            f.template many<8>(i0 + N, yu);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) yu[k] = V(0);
        }
        xm = zc.hxm ? f.one(i0 - 1) : V(0);
        xp = zc.hxp ? f.one(i0 + 8) : V(0);
    }
    template <class F>
    __device__ __forceinline__ void rows_zm(int which, int64_t item, const F &f, const ZCol &zc, bool hlz, bool huz,
                                            const Acc (&c)[8], const Acc (&zl)[8], const Acc (&zu)[8],
                                            Acc (&out)[8]) const
    {
        using P = Prec<T>;
        const int64_t i0 = item * 8;
        Acc yl[8], yu[8], xm, xp, acc[8], sh[8];
        zm_gather(i0, zc, f, yl, yu, xm, xp);
        if (which == kOpH) {
            P::mul_s(acc, sigH, c);
            if (hlz) P::madd_s(acc, acc, h_off, zl);
            if (zc.hly) P::madd_s(acc, acc, h_off, yl);
#pragma unroll
            for (int k = 0; k < 8; ++k) sh[k] = k ? c[k - 1] : xm;
            P::madd_s(acc, acc, h_off, sh);
            P::madd_s(acc, acc, h_diag, c);
#pragma unroll
            for (int k = 0; k < 8; ++k) sh[k] = k < 7 ? c[k + 1] : xp;
            P::madd_s(acc, acc, h_off, sh);
            if (zc.huy) P::madd_s(acc, acc, h_off, yu);
            if (huz) P::madd_s(acc, acc, h_off, zu);
        } else {
            const Acc lo = which == kOpS ? -s_c : s_c;
            P::mul_s(acc, sigS, c);
            if (hlz) P::madd_s(acc, acc, lo, zl);
            if (zc.hly) P::madd_s(acc, acc, lo, yl);
#pragma unroll
            for (int k = 0; k < 8; ++k) sh[k] = k ? c[k - 1] : xm;
            P::madd_s(acc, acc, lo, sh);
            if (s_diag != Acc(0)) P::madd_s(acc, acc, s_diag, c);
#pragma unroll
            for (int k = 0; k < 8; ++k) sh[k] = k < 7 ? c[k + 1] : xp;
            P::madd_s(acc, acc, -lo, sh);
            if (zc.huy) P::madd_s(acc, acc, -lo, yu);
            if (huz) P::madd_s(acc, acc, -lo, zu);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) out[k] = acc[k];
    }
    // r = b - A x along the march (FP64 x values c, zl, zu)
    template <class F>
    __device__ __forceinline__ void resid_zm(int64_t item, const F &f, const ZCol &zc, bool hlz, bool huz,
                                             const double (&c)[8], const double (&zl)[8], const double (&zu)[8],
                                             const double (&b)[8], double (&out)[8]) const
    {
        const int64_t i0 = item * 8;
        double yl[8], yu[8], xm, xp, acc[8];
        zm_gather(i0, zc, f, yl, yu, xm, xp);
        const double clo = -a_lo, cdg = -a_diag, chi = -a_hi;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = b[k];
        if (hlz) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = __fma_rn(clo, zl[k], acc[k]);
        }
        if (zc.hly) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = __fma_rn(clo, yl[k], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k > 0 || zc.hxm) acc[k] = __fma_rn(clo, k ? c[k - 1] : xm, acc[k]);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = __fma_rn(cdg, c[k], acc[k]);
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k < 7 || zc.hxp) acc[k] = __fma_rn(chi, k < 7 ? c[k + 1] : xp, acc[k]);
        if (zc.huy) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = __fma_rn(chi, yu[k], acc[k]);
        }
        if (huz) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = __fma_rn(chi, zu[k], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) out[k] = acc[k];
    }

    // ---- scalar rows (R == 1) ------------------------------------------------
    // (A x)_i from zero, or (kRes) init - (A x)_i with every product
    // subtracted by one fused multiply-add, in the same term order
    template <bool kRes, class F>
    __device__ __forceinline__ double rowA1(int64_t i, const F &f, double init = 0.0) const
    {
        unsigned cd[3];
        coords(i, cd);
        const unsigned last = (unsigned)N - 1;
        const double sg = kRes ? -1.0 : 1.0;
        double acc = kRes ? init : 0.0;
        const bool face = AD != nullptr;
#pragma unroll
        for (int d = DIM - 1; d >= 0; --d)
            if (cd[d] > 0) acc = __fma_rn(sg * (face ? __ldg(AL[d] + i) : a_lo), f.one(i - stride(d)), acc);
        acc = __fma_rn(sg * (face ? __ldg(AD + i) : a_diag), f.one(i), acc);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            if (cd[d] < last) acc = __fma_rn(sg * (face ? __ldg(AU[d] + i) : a_hi), f.one(i + stride(d)), acc);
        return acc;
    }

    template <class F>
    __device__ __forceinline__ Acc row1(int which, int64_t i, const F &f) const
    {
        using P = Prec<T>;
        unsigned cd[3];
        coords(i, cd);
        const unsigned last = (unsigned)N - 1;
        const Acc fi = f.one(i);
        if (which == kOpH) {
            const bool face = HD != nullptr;
            Acc acc = P::mul(sigH, fi);
#pragma unroll
            for (int d = DIM - 1; d >= 0; --d)
                if (cd[d] > 0)
                    acc = P::madd(acc, face ? P::ld(HK[d][i - stride(d)]) : h_off, f.one(i - stride(d)));
            acc = P::madd(acc, face ? P::ld(HD[i]) : h_diag, fi);
#pragma unroll
            for (int d = 0; d < DIM; ++d)
                if (cd[d] < last) acc = P::madd(acc, face ? P::ld(HK[d][i]) : h_off, f.one(i + stride(d)));
            return acc;
        }
        const Acc lo = which == kOpS ? -s_c : s_c;
        Acc acc = P::mul(sigS, fi);
#pragma unroll
        for (int d = DIM - 1; d >= 0; --d)
            if (cd[d] > 0) acc = P::madd(acc, lo, f.one(i - stride(d)));
        if (s_diag != Acc(0)) acc = P::madd(acc, s_diag, fi);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            if (cd[d] < last) acc = P::madd(acc, -lo, f.one(i + stride(d)));
        return acc;
    }

    // ---- R-row items (R = 4 or 8) ----------------------------------------------
    // Items of R: neighbours along y and z are whole aligned chunks; along x
    // they are the item's own values shifted by one, with the two ends from
    // one(). Every neighbour value of an item is read before its first term
    // is formed: a neighbour outside the grid reads the item's own chunk (a
    // valid address) and its term is left out afterwards, so the item's
    // loads issue back to back and a pass waits for memory once per item
    // rather than once per neighbour. Terms and their order are unchanged.
    // The FP64 inner path (bound by the FP64 rate, and short of registers
    // for eight FP64 chunks) loads each neighbour where its term is formed.
    static constexpr bool kHoist = !std::is_same<T, double>::value;
    // kRes: init - A x (every coefficient negated, which is exact, so each
    // term is one fused multiply-add subtracting the product); else A x
    template <bool kRes, class F>
    __device__ __forceinline__ void rowsA_t(int64_t item, const F &f, const double (&init)[R], double (&out)[R]) const
    {
        if constexpr (R == 1) {
            out[0] = rowA1<kRes>(item, f, init[0]);
        } else {
            constexpr int NB = DIM - 1;
            const int64_t i0 = item * R;
            unsigned cd[3];
            coords(i0, cd);
            const unsigned last = (unsigned)N - 1;
            const bool face = AD != nullptr;
            bool hl[NB], hu[NB];
            double c[R], acc[R], cf[R], tl[NB][R], tu[NB][R];
            f.template many<R>(i0, c);
#pragma unroll
            for (int d = 1; d < DIM; ++d) {
                hl[d - 1] = cd[d] > 0;
                hu[d - 1] = cd[d] < last;
                if constexpr (kHoist) {
                    f.template many<R>(hl[d - 1] ? i0 - stride(d) : i0, tl[d - 1]);
                    f.template many<R>(hu[d - 1] ? i0 + stride(d) : i0, tu[d - 1]);
                }
            }
            const bool hxm = cd[0] > 0, hxp = cd[0] + R <= last;
            double xm = 0.0, xp = 0.0;
            if constexpr (kHoist) {
                xm = f.one(hxm ? i0 - 1 : i0);
                xp = f.one(hxp ? i0 + R : i0);
            } else {
                if (hxm) xm = f.one(i0 - 1);
                if (hxp) xp = f.one(i0 + R);
            }
            const double sg = kRes ? -1.0 : 1.0;
            const double clo = sg * a_lo, cdg = sg * a_diag, chi = sg * a_hi;
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] = kRes ? init[k] : 0.0;
#pragma unroll
            for (int d = DIM - 1; d >= 1; --d)
                if (hl[d - 1]) {
                    if constexpr (!kHoist) f.template many<R>(i0 - stride(d), tl[d - 1]);
                    if (face) ldv<R>(AL[d], i0, cf);
#pragma unroll
                    for (int k = 0; k < R; ++k) acc[k] = __fma_rn(face ? sg * cf[k] : clo, tl[d - 1][k], acc[k]);
                }
            {   // x lower
                if (face) ldv<R>(AL[0], i0, cf);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (k > 0 || hxm) acc[k] = __fma_rn(face ? sg * cf[k] : clo, k ? c[k - 1] : xm, acc[k]);
            }
            if (face) ldv<R>(AD, i0, cf);
#pragma unroll
            for (int k = 0; k < R; ++k) acc[k] = __fma_rn(face ? sg * cf[k] : cdg, c[k], acc[k]);
            {   // x upper
                if (face) ldv<R>(AU[0], i0, cf);
#pragma unroll
                for (int k = 0; k < R; ++k)
                    if (k < R - 1 || hxp) acc[k] = __fma_rn(face ? sg * cf[k] : chi, k < R - 1 ? c[k + 1] : xp, acc[k]);
            }
#pragma unroll
            for (int d = 1; d < DIM; ++d)
                if (hu[d - 1]) {
                    if constexpr (!kHoist) f.template many<R>(i0 + stride(d), tu[d - 1]);
                    if (face) ldv<R>(AU[d], i0, cf);
#pragma unroll
                    for (int k = 0; k < R; ++k) acc[k] = __fma_rn(face ? sg * cf[k] : chi, tu[d - 1][k], acc[k]);
                }
#pragma unroll
            for (int k = 0; k < R; ++k) out[k] = acc[k];
        }
    }

    template <class F>
    __device__ __forceinline__ void rowsA(int64_t item, const F &f, double (&out)[R]) const
    {
        double z[R];
#pragma unroll
        for (int k = 0; k < R; ++k) z[k] = 0.0;
        rowsA_t<false>(item, f, z, out);
    }
    // r = b - A x for the outer residual (Algorithm 1 step 1): b[k] is row
    // item * R + k of the right-hand side
    template <class F>
    __device__ __forceinline__ void resid(int64_t item, const F &f, const double (&b)[R], double (&out)[R]) const
    {
        rowsA_t<true>(item, f, b, out);
    }

    template <class F>
    __device__ __forceinline__ void rows(int which, int64_t item, const F &f, Acc (&out)[R]) const
    {
        using P = Prec<T>;
        if constexpr (R == 1) {
            out[0] = row1(which, item, f);
        } else {
            // element-wise over the item's R rows (packed pairs for FP16); the
            // x neighbours are the item's own values shifted by one, with a
            // zero term (value 0, so the sum keeps its value) where a row has
            // no neighbour
            constexpr int NB = DIM - 1;
            const int64_t i0 = item * R;
            unsigned cd[3];
            coords(i0, cd);
            const unsigned last = (unsigned)N - 1;
            bool hl[NB], hu[NB];
            Acc c[R], acc[R], cf[R], sh[R], tl[NB][R], tu[NB][R];
            f.template many<R>(i0, c);
#pragma unroll
            for (int d = 1; d < DIM; ++d) {
                hl[d - 1] = cd[d] > 0;
                hu[d - 1] = cd[d] < last;
                if constexpr (kHoist) {
                    f.template many<R>(hl[d - 1] ? i0 - stride(d) : i0, tl[d - 1]);
                    f.template many<R>(hu[d - 1] ? i0 + stride(d) : i0, tu[d - 1]);
                }
            }
            const bool hxm = cd[0] > 0, hxp = cd[0] + R <= last;
            Acc xm = Acc(0), xp = Acc(0);
            if constexpr (kHoist) {
                const Acc xm0 = f.one(hxm ? i0 - 1 : i0), xp0 = f.one(hxp ? i0 + R : i0);
                xm = hxm ? xm0 : Acc(0);
                xp = hxp ? xp0 : Acc(0);
            } else {
                if (hxm) xm = f.one(i0 - 1);
                if (hxp) xp = f.one(i0 + R);
            }
            if (which == kOpH) {
                const bool face = HD != nullptr;
                P::mul_s(acc, sigH, c);
#pragma unroll
                for (int d = DIM - 1; d >= 1; --d)
                    if (hl[d - 1]) {
                        if constexpr (!kHoist) f.template many<R>(i0 - stride(d), tl[d - 1]);
                        if (face) {
                            ldv<R>(HK[d], i0 - stride(d), cf);
                            P::madd_v(acc, acc, cf, tl[d - 1]);
                        } else {
                            P::madd_s(acc, acc, h_off, tl[d - 1]);
                        }
                    }
                {   // x lower: coupling of node i with i-1 is HK[0][i-1]
#pragma unroll
                    for (int k = 0; k < R; ++k) sh[k] = k ? c[k - 1] : xm;
                    if (face) {
                        Acc cs[R];
                        ldv<R>(HK[0], i0, cf);
                        cs[0] = hxm ? P::ld(HK[0][i0 - 1]) : Acc(0);
#pragma unroll
                        for (int k = 1; k < R; ++k) cs[k] = cf[k - 1];
                        P::madd_v(acc, acc, cs, sh);
                    } else {
                        P::madd_s(acc, acc, h_off, sh);
                    }
                }
                if (face) {
                    Acc dg[R];
                    ldv<R>(HD, i0, dg);
                    P::madd_v(acc, acc, dg, c);
                } else {
                    P::madd_s(acc, acc, h_diag, c);
                }
                {   // x upper: coupling HK[0][i]
#pragma unroll
                    for (int k = 0; k < R; ++k) sh[k] = k < R - 1 ? c[k + 1] : xp;
                    if (face) P::madd_v(acc, acc, cf, sh);
                    else P::madd_s(acc, acc, h_off, sh);
                }
#pragma unroll
                for (int d = 1; d < DIM; ++d)
                    if (hu[d - 1]) {
                        if constexpr (!kHoist) f.template many<R>(i0 + stride(d), tu[d - 1]);
                        if (face) {
                            ldv<R>(HK[d], i0, cf);
                            P::madd_v(acc, acc, cf, tu[d - 1]);
                        } else {
                            P::madd_s(acc, acc, h_off, tu[d - 1]);
                        }
                    }
            } else {
                const Acc lo = which == kOpS ? -s_c : s_c;
                P::mul_s(acc, sigS, c);
#pragma unroll
                for (int d = DIM - 1; d >= 1; --d)
                    if (hl[d - 1]) {
                        if constexpr (!kHoist) f.template many<R>(i0 - stride(d), tl[d - 1]);
                        P::madd_s(acc, acc, lo, tl[d - 1]);
                    }
                {
#pragma unroll
                    for (int k = 0; k < R; ++k) sh[k] = k ? c[k - 1] : xm;
                    P::madd_s(acc, acc, lo, sh);
                }
                if (s_diag != Acc(0)) P::madd_s(acc, acc, s_diag, c);
                {
#pragma unroll
                    for (int k = 0; k < R; ++k) sh[k] = k < R - 1 ? c[k + 1] : xp;
                    P::madd_s(acc, acc, -lo, sh);
                }
#pragma unroll
                for (int d = 1; d < DIM; ++d)
                    if (hu[d - 1]) {
                        if constexpr (!kHoist) f.template many<R>(i0 + stride(d), tu[d - 1]);
                        P::madd_s(acc, acc, -lo, tu[d - 1]);
                    }
            }
#pragma unroll
            for (int k = 0; k < R; ++k) out[k] = acc[k];
        }
    }
};

// The stencil operator with the z-marching traversal compiled in: its own
// instantiation of the solve kernel (the passes march along z and nothing
// else), so that the grid-stride instantiation keeps its own register
// allocation.
template <class Base>
struct ZMarchOp : Base {
    using BaseOp = Base;
    static_assert(Base::kZMarchCapable, "z-marching needs the 3D FP16 stencil with 8-row items");
    static constexpr bool kZMarch = true;
};

}  // namespace gadi
