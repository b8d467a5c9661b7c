// gadi_ops.cuh -- the operators of GADI-IR as row functions for the
// persistent kernel.
//
//   which = kOpA  : (A x)_i                       FP64 (outer residual, Alg. 1 step 1)
//   which = kOpH  : (H' x)_i = 2^-sM (aI + M) x   inner precision (Alg. 1 step 2)
//   which = kOpS  : (S' x)_i = 2^-sN (aI + N) x   inner precision (Alg. 1 step 3)
//   which = kOpST : (S'^T x)_i                    (CGNR's transpose product)
//
// A row is evaluated as sigma*f(i) first, then the matrix entries in
// ascending column order (the CSR order), with explicitly rounded products
// and sums. For FP16 values and vectors each product is exact in FP32, so a
// row equals the FP32 sum of the same terms in the same order on any device.
//
// f(j) supplies the vector value at column j as an Acc; the persistent
// kernel passes expressions (e.g. r_j + beta p_j rounded to storage) so that
// the vector update of a Krylov step can be fused into the next product
// without an extra grid barrier.
#pragma once

#include "gadi_device.cuh"

namespace gadi {

enum : int { kOpA = 0, kOpH = 1, kOpS = 2, kOpST = 3 };

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
    int64_t n;
    int W;
    const int *__restrict__ col;
    const double *__restrict__ a64;   // A values (FP64)
    const T *__restrict__ m;          // 2^-sM M in the inner precision
    const T *__restrict__ nv;         // 2^-sN N
    const T *__restrict__ nt;         // 2^-sN N^T, or null when N^T = -N
    Acc sigH, sigS;                   // 2^-sM alpha, 2^-sN alpha

    template <class F>
    __device__ __forceinline__ double rowA(int64_t i, F f) const
    {
        const int *c = col + i * W;
        const double *v = a64 + i * W;
        double acc = 0.0;
        for (int k = 0; k < W; ++k) acc = d_madd(acc, __ldg(v + k), f(__ldg(c + k)));
        return acc;
    }

    template <class F>
    __device__ __forceinline__ Acc row(int which, int64_t i, F f) const
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
        Acc acc = P::mul(sig, f(i));
        for (int k = 0; k < W; ++k) {
            Acc val = P::ld(v[k]);
            acc = P::add(acc, P::mul(sgn * val, f(__ldg(c + k))));
        }
        return acc;
    }
};

// ---------------------------------------------------------------------------
// Matrix-free 5-point (2D) / 7-point (3D) convection-diffusion operator of
// §4.1 on an N^dim grid, x fastest. Constant-k form: all coefficients are
// scalars. Face form: per-node arrays of the diagonal and of the upper-face
// couplings per axis, taken from the HSS split values (M symmetric, so the
// lower coupling of node i along d is the upper coupling of node i - e_d).
// The convection part N is the constant c = beta h / 2 in both forms.
// ---------------------------------------------------------------------------
template <class T, int DIM>
struct StencilOp {
    using Acc = typename Prec<T>::Acc;
    static constexpr int kDim = DIM;
    int dim, N;          // dim == DIM
    int64_t n;
    // FP64 A for the residual: constant form uses (a_diag, a_lo, a_hi);
    // face form uses AD[i] and AL[d][i] = a_{i,i-e_d}, AU[d][i] = a_{i,i+e_d}
    double a_diag, a_lo, a_hi;
    const double *__restrict__ AD;
    const double *__restrict__ AL[3];
    const double *__restrict__ AU[3];
    // inner operators: H' diagonal/off-diagonal (constant form) or arrays
    // HD[i] = 2^-sM m_ii, HK[d][i] = 2^-sM m_{i,i+e_d} (face form);
    // S': 2^-sN c rounded to T
    Acc h_diag, h_off, s_c;
    const T *__restrict__ HD;
    const T *__restrict__ HK[3];
    Acc sigH, sigS;

    // grid coordinates of node i (x fastest); n < 2^31 is enforced at create
    __device__ __forceinline__ void coords(int64_t i, unsigned (&cd)[3]) const
    {
        const unsigned ii = (unsigned)i, NN = (unsigned)N;
        const unsigned t = ii / NN;
        cd[0] = ii - t * NN;
        if (DIM == 3) {
            const unsigned u = t / NN;
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

    template <class F>
    __device__ __forceinline__ double rowA(int64_t i, F f) const
    {
        unsigned cd[3];
        coords(i, cd);
        const unsigned last = (unsigned)N - 1;
        double acc = 0.0;
        const bool face = AD != nullptr;
#pragma unroll
        for (int d = DIM - 1; d >= 0; --d)
            if (cd[d] > 0) acc = d_madd(acc, face ? __ldg(AL[d] + i) : a_lo, f(i - stride(d)));
        acc = d_madd(acc, face ? __ldg(AD + i) : a_diag, f(i));
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            if (cd[d] < last) acc = d_madd(acc, face ? __ldg(AU[d] + i) : a_hi, f(i + stride(d)));
        return acc;
    }

    template <class F>
    __device__ __forceinline__ Acc row(int which, int64_t i, F f) const
    {
        using P = Prec<T>;
        unsigned cd[3];
        coords(i, cd);
        const unsigned last = (unsigned)N - 1;
        const Acc fi = f(i);
        if (which == kOpH) {
            const bool face = HD != nullptr;
            Acc acc = P::mul(sigH, fi);
#pragma unroll
            for (int d = DIM - 1; d >= 0; --d)
                if (cd[d] > 0)
                    acc = P::add(acc, P::mul(face ? P::ld(HK[d][i - stride(d)]) : h_off, f(i - stride(d))));
            acc = P::add(acc, P::mul(face ? P::ld(HD[i]) : h_diag, fi));
#pragma unroll
            for (int d = 0; d < DIM; ++d)
                if (cd[d] < last) acc = P::add(acc, P::mul(face ? P::ld(HK[d][i]) : h_off, f(i + stride(d))));
            return acc;
        }
        // S' (lower -c, upper +c) or S'^T (lower +c, upper -c); N has a zero diagonal
        const Acc lo = which == kOpS ? -s_c : s_c;
        Acc acc = P::mul(sigS, fi);
#pragma unroll
        for (int d = DIM - 1; d >= 0; --d)
            if (cd[d] > 0) acc = P::add(acc, P::mul(lo, f(i - stride(d))));
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            if (cd[d] < last) acc = P::add(acc, P::mul(-lo, f(i + stride(d))));
        return acc;
    }
};

}  // namespace gadi
