// gadi_api.cu -- C ABI of libgadi.so: set-up kernels (CSR checks, HSS
// splitting into the ELL layout, FP16 demotion, stencil extraction) and the
// host logic around the persistent solve kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/gadi.h"
#include "gadi_solve.cuh"

using namespace gadi;

// ===========================================================================
// Set-up kernels
// ===========================================================================
namespace {

constexpr int kSetupThreads = 256;

inline unsigned grid_for(int64_t n, int threads = kSetupThreads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535LL * 32) g = 65535LL * 32;
    return (unsigned)g;
}

// flags in the set-up error word
enum : int {
    kBadRowPtr = 1, kBadCol = 2, kUnsorted = 4, kNonFinite = 8, kUnsymPattern = 16,
    kStencilPattern = 32, kStencilValue = 64
};

__global__ void k_check_csr(int64_t n, int64_t nnz, const int *rp, const int *ci, const double *v,
                            int *bad, int *maxlen)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int lo = rp[i], hi = rp[i + 1];
        int f = 0;
        if (i == 0 && lo != 0) f |= kBadRowPtr;
        if (i == n - 1 && (int64_t)hi != nnz) f |= kBadRowPtr;
        if (lo < 0 || hi < lo || (int64_t)hi > nnz) {
            atomicOr(bad, f | kBadRowPtr);
            continue;
        }
        atomicMax(maxlen, hi - lo);
        for (int k = lo; k < hi; ++k) {
            int c = ci[k];
            if (c < 0 || (int64_t)c >= n) f |= kBadCol;
            if (k > lo && c <= ci[k - 1]) f |= kUnsorted;
            if (!isfinite(v[k])) f |= kNonFinite;
        }
        if (f) atomicOr(bad, f);
    }
}

__device__ __forceinline__ int find_in_row(const int *rp, const int *ci, int64_t row, int64_t col)
{
    int lo = rp[row], hi = rp[row + 1] - 1;
    while (lo <= hi) {
        int mid = lo + ((hi - lo) >> 1);
        int c = ci[mid];
        if (c == col) return mid;
        if (c < col) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v)
{
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

// Splitting of A on its own pattern into the ELL arrays.
//   HSS:  m = (a_ij + a_ji)/2, n = (a_ij - a_ji)/2           (§4.1)
//   user: m = m_user_ij, n = a_ij - m_ij, n^T_ij = a_ji - m_ji
// norms[0..3] receive max row sums of |A|, |M|, |N|, |N^T|.
__global__ void k_split_ell(int64_t n, const int *rp, const int *ci, const double *a,
                            const double *mu, int W, int *ecol, double *ea, double *em,
                            double *en, double *ent, double *norms, int *bad)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t base = i * W;
        int t = 0;
        double sa = 0, sm = 0, sn = 0, snt = 0;
        for (int k = rp[i]; k < rp[i + 1]; ++k, ++t) {
            const int j = ci[k];
            const int kt = find_in_row(rp, ci, j, i);
            double aij = a[k], m, nv, ntv;
            if (kt < 0) {
                atomicOr(bad, kUnsymPattern);
                m = nv = ntv = 0.0;
            } else if (mu) {
                m = mu[k];
                nv = __dsub_rn(aij, m);
                ntv = __dsub_rn(a[kt], mu[kt]);
            } else {
                m = __dmul_rn(0.5, __dadd_rn(aij, a[kt]));
                nv = __dmul_rn(0.5, __dsub_rn(aij, a[kt]));
                ntv = -nv;
            }
            ecol[base + t] = j;
            ea[base + t] = aij;
            em[base + t] = m;
            en[base + t] = nv;
            if (ent) ent[base + t] = ntv;
            sa += fabs(aij);
            sm += fabs(m);
            sn += fabs(nv);
            snt += fabs(ntv);
        }
        for (; t < W; ++t) {
            ecol[base + t] = (int)i;
            ea[base + t] = 0.0;
            em[base + t] = 0.0;
            en[base + t] = 0.0;
            if (ent) ent[base + t] = 0.0;
        }
        atomic_max_nonneg(norms + 0, sa);
        atomic_max_nonneg(norms + 1, sm);
        atomic_max_nonneg(norms + 2, sn);
        atomic_max_nonneg(norms + 3, snt);
    }
}

// dst = fl_T(src * 2^-s), round to nearest even, directly from FP64
template <class TD>
__global__ void k_demote(int64_t cnt, const double *src, TD *dst, double scale)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = Prec<TD>::from64(__dmul_rn(src[i], scale));
}

// unscaled FP16 mode: dst = fl16(sign src + alpha) on the stored diagonal
// (the first slot of a row whose column is the row; padding slots come after
// the row's entries), fl16(sign src) elsewhere. W = 0: every entry is a
// diagonal. sign = -1 forms N^T = -N of a skew-symmetric N.
template <class TD>
__global__ void k_demote_diag(int64_t cnt, int W, const int *col, const double *src, TD *dst,
                              double alpha, double sign)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        bool diag = W == 0;
        if (!diag) {
            const int64_t row = i / W, k0 = row * W;
            diag = col[i] == row;
            for (int64_t k = k0; k < i && diag; ++k)
                if (col[k] == row) diag = false;
        }
        const double v = sign < 0.0 ? -src[i] : src[i];
        dst[i] = Prec<TD>::from64(diag ? __dadd_rn(v, alpha) : v);
    }
}

template <class TD>
__global__ void k_count_range(int64_t cnt, const double *src, const TD *dst, int *lost)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x) {
        float h = Prec<TD>::ld(dst[i]);
        if ((src[i] != 0.0 && h == 0.0f) || isinf(h)) atomicAdd(lost, 1);
    }
}

// Check the ELL arrays against the stencil description and extract the
// per-node values the face-coefficient kernels use.
__global__ void k_stencil_extract(int64_t n, int dim, int N, double c, int variable_k, int W,
                                  const int *ecol, const double *ea, const double *em,
                                  const double *en, double *AD, double *AL0, double *AL1,
                                  double *AL2, double *AU0, double *AU1, double *AU2, double *HD,
                                  double *HK0, double *HK1, double *HK2, int *bad)
{
    double *AL[3] = {AL0, AL1, AL2}, *AU[3] = {AU0, AU1, AU2}, *HK[3] = {HK0, HK1, HK2};
    const int64_t st[3] = {1, N, (int64_t)N * N};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int cd[3];
        int64_t t = i / N;
        cd[0] = (int)(i - t * N);
        if (dim == 3) { cd[1] = (int)(t % N); cd[2] = (int)(t / N); }
        else { cd[1] = (int)t; cd[2] = 0; }
        // expected columns, ascending: lower (z, y, x), diagonal, upper (x, y, z)
        int64_t cols[7];
        int kind[7];   // -1-d lower along d, 0 diagonal, 1+d upper along d
        int ne = 0;
        for (int d = dim - 1; d >= 0; --d)
            if (cd[d] > 0) { cols[ne] = i - st[d]; kind[ne++] = -1 - d; }
        cols[ne] = i; kind[ne++] = 0;
        for (int d = 0; d < dim; ++d)
            if (cd[d] < N - 1) { cols[ne] = i + st[d]; kind[ne++] = 1 + d; }
        int f = 0;
        for (int s = 0; s < W; ++s) {
            const int64_t idx = i * W + s;
            if (s >= ne) {
                if (ecol[idx] != (int)i || ea[idx] != 0.0) f |= kStencilPattern;
                continue;
            }
            if (ecol[idx] != cols[s]) { f |= kStencilPattern; continue; }
            const double av = ea[idx], mv = em[idx], nvv = en[idx];
            const int kd = kind[s];
            const double tol = 1e-12 * fmax(1.0, fabs(av));
            if (kd == 0) {
                if (fabs(nvv) > tol) f |= kStencilValue;
                if (!variable_k && fabs(av - 2.0 * dim) > tol) f |= kStencilValue;
                if (AD) { AD[i] = av; HD[i] = mv; }
            } else {
                const int d = (kd < 0 ? -kd : kd) - 1;
                const double want_n = kd < 0 ? -c : c;
                if (fabs(nvv - want_n) > tol) f |= kStencilValue;
                if (!variable_k && fabs(mv + 1.0) > tol) f |= kStencilValue;
                if (AD) {
                    if (kd < 0) AL[d][i] = av;
                    else { AU[d][i] = av; HK[d][i] = mv; }
                }
            }
        }
        if (AD) {
            for (int d = 0; d < dim; ++d) {
                if (cd[d] == 0) AL[d][i] = 0.0;
                if (cd[d] == N - 1) { AU[d][i] = 0.0; HK[d][i] = 0.0; }
            }
        }
        if (f) atomicOr(bad, f);
    }
}

// ||b||_inf and a non-finite flag
__global__ void k_vec_check(int64_t n, const double *b, double *out_max, int *nonfinite)
{
    double m = 0.0;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double v = b[i];
        if (!isfinite(v)) bad = 1;
        else m = fmax(m, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(out_max, m);
        if (bad) atomicOr(nonfinite, 1);
    }
}

}  // namespace

// ===========================================================================
// Handle
// ===========================================================================
struct gadi_solver {
    int dev = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    int64_t n = 0, nnz = 0;
    int W = 0;
    bool user_split = false;
    // ELL arrays (device)
    int *ecol = nullptr;
    double *ea = nullptr, *em = nullptr, *en = nullptr, *ent = nullptr;
    // 2-byte inner values (FP16, or bfloat16 in the same arrays) and FP32 ones
    __half *m16 = nullptr, *n16 = nullptr, *nt16 = nullptr;
    float *m32 = nullptr, *n32 = nullptr, *nt32 = nullptr;
    double anorm = 0, mnorm = 0, nnorm = 0, ntnorm = 0;
    // stencil
    bool has_stencil = false;
    int sdim = 0, sN = 0, variable_k = 0;
    double beta = 0, c = 0;
    // constant-coefficient values taken from the split (so the stencil
    // operators equal the sparse ones bit for bit): A's diagonal, lower and
    // upper couplings, M's off-diagonal and N's upper coupling
    double a_diag = 0, a_lo = 0, a_hi = 0, m_off = 0, n_up = 0;
    double *AD = nullptr, *AL[3] = {}, *AU[3] = {}, *HD64 = nullptr, *HK64[3] = {};
    __half *HD16 = nullptr, *HK16[3] = {};
    float *HD32 = nullptr, *HK32[3] = {};
    // parameters
    double alpha = 1.0, omega = 1.0;
    int u_r = GADI_F16;
    double eps = -1.0;
    int max_inner = 200, max_outer = 100000;
    int stop = GADI_STOP_ETA;
    int kernel = GADI_KERNEL_AUTO;
    int item_rows = 0;        // stencil rows per item: 0 = automatic, 1, 4 or 8
    int traversal = 0;        // 0: z-marching solves where available, 1: grid-stride items
    int blocks = 0, threads = 0;
    double wait_ms = 2000.0;
    int force_timeout = 0;
    // demoted operator state
    int sM = 0, sNs = 0;
    bool demoted = false;
    double demoted_alpha = 0.0;
    int scaling = 1;          // 0: unscaled FP16 inner mode (alpha rounded into the FP16 diagonal)
    int demoted_scaling = 1;
    int demoted_ur = -1;
    // work
    double *bdev = nullptr, *xdev = nullptr, *r64 = nullptr;
    double *x2 = nullptr;     // second iterate buffer (the iterates alternate with x)
    void *vec = nullptr;      // 9 vectors of n elements of the inner type (sized for FP64);
                              // with FP16 inner vectors, the FP32 residual copy follows them
    double *part = nullptr;
    int part_blocks = 0;
    Ctl *ctl = nullptr;
    double *scratch = nullptr;   // small device scratch (norms, flags)
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const gadi_model *models[2] = {nullptr, nullptr};   // MLP, GPR (not owned)
    std::string err;
};

namespace {

gadi_status fail(gadi_solver *h, gadi_status s, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return fail(h, e_ == cudaErrorMemoryAllocation ? GADI_ERR_OUT_OF_MEMORY           \
                                                          : GADI_ERR_CUDA,                    \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,     \
                        __LINE__);                                                            \
        }                                                                                     \
    } while (0)

template <class X>
cudaError_t dalloc(X **p, size_t count)
{
    return cudaMalloc((void **)p, (count ? count : 1) * sizeof(X));
}

// the inner work vectors (9 n FP64, or 9 n FP16 followed by the n-float
// round-to-odd residual copy at a 256-byte boundary)
size_t vec_bytes(int64_t n)
{
    const size_t half_path = ((size_t)9 * n * sizeof(__half) + 255) / 256 * 256 + (size_t)n * sizeof(float);
    return std::max((size_t)9 * n * sizeof(double), half_path);
}

float *r32_of(void *vec, int64_t n)
{
    return reinterpret_cast<float *>(static_cast<char *>(vec) + ((size_t)9 * n * sizeof(__half) + 255) / 256 * 256);
}

void release(gadi_solver *h)
{
    void *ptrs[] = {h->ecol, h->ea, h->em, h->en, h->ent, h->m16, h->n16, h->nt16, h->AD,
                    h->AL[0], h->AL[1], h->AL[2], h->AU[0], h->AU[1], h->AU[2], h->HD64,
                    h->HK64[0], h->HK64[1], h->HK64[2], h->HD16, h->HK16[0], h->HK16[1],
                    h->HK16[2], h->bdev, h->xdev, h->x2, h->r64, h->vec, h->part, h->ctl, h->scratch,
                    h->m32, h->n32, h->nt32, h->HD32, h->HK32[0], h->HK32[1], h->HK32[2]};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// s such that (|sigma| + norm) 2^-s lies in (1, 2]: keeps FP16 values of the
// scaled operator, and of K p and K K^T r for vectors of size O(1), in range
int half_scale_exponent(double norm, double sigma)
{
    double v = norm + std::fabs(sigma);
    if (!(v > 0.0) || !std::isfinite(v)) return 0;
    int e;
    double m = std::frexp(v, &e);
    int c = (m == 0.5) ? e - 1 : e;
    return c - 1;
}

bool use_stencil(const gadi_solver *h)
{
    if (h->kernel == GADI_KERNEL_STENCIL) return true;
    if (h->kernel == GADI_KERNEL_SPARSE) return false;
    return h->has_stencil;
}

// The inner operator values of storage type TD, demoted from FP64: scaled by
// 2^-sM / 2^-sN, or (unscaled FP16 mode) with alpha rounded into the stored
// diagonals and N^T in its own array.
template <class TD>
void demote_all(gadi_solver *h, TD *m, TD *nv, TD *nt, TD *hd, TD *const *hk, bool naive, double scM, double scN)
{
    const int64_t cnt = h->n * (int64_t)h->W;
    if (naive) {
        k_demote_diag<TD><<<grid_for(cnt), kSetupThreads, 0, h->stream>>>(cnt, h->W, h->ecol, h->em, m, h->alpha, 1.0);
        k_demote_diag<TD><<<grid_for(cnt), kSetupThreads, 0, h->stream>>>(cnt, h->W, h->ecol, h->en, nv, h->alpha, 1.0);
        // S^T = aI + N^T keeps +alpha on its diagonal
        k_demote_diag<TD><<<grid_for(cnt), kSetupThreads, 0, h->stream>>>(cnt, h->W, h->ecol, h->ent ? h->ent : h->en,
                                                                          nt, h->alpha, h->ent ? 1.0 : -1.0);
        if (h->HD64) {
            k_demote_diag<TD><<<grid_for(h->n), kSetupThreads, 0, h->stream>>>(h->n, 0, nullptr, h->HD64, hd,
                                                                               h->alpha, 1.0);
            for (int d = 0; d < h->sdim; ++d)
                k_demote<TD><<<grid_for(h->n), kSetupThreads, 0, h->stream>>>(h->n, h->HK64[d], hk[d], 1.0);
        }
        return;
    }
    k_demote<TD><<<grid_for(cnt), kSetupThreads, 0, h->stream>>>(cnt, h->em, m, scM);
    k_demote<TD><<<grid_for(cnt), kSetupThreads, 0, h->stream>>>(cnt, h->en, nv, scN);
    if (h->ent) k_demote<TD><<<grid_for(cnt), kSetupThreads, 0, h->stream>>>(cnt, h->ent, nt, scN);
    if (h->HD64) {
        k_demote<TD><<<grid_for(h->n), kSetupThreads, 0, h->stream>>>(h->n, h->HD64, hd, scM);
        for (int d = 0; d < h->sdim; ++d)
            k_demote<TD><<<grid_for(h->n), kSetupThreads, 0, h->stream>>>(h->n, h->HK64[d], hk[d], scM);
    }
}

// entries that flush to zero or overflow in the inner precision after scaling
template <class TD>
gadi_status count_lost(gadi_solver *h, const TD *m, const TD *nv, const char *name)
{
    const int64_t cnt = h->n * (int64_t)h->W;
    int *lost = (int *)h->scratch;
    CK(cudaMemsetAsync(lost, 0, sizeof(int), h->stream));
    k_count_range<TD><<<grid_for(cnt), kSetupThreads, 0, h->stream>>>(cnt, h->em, m, lost);
    k_count_range<TD><<<grid_for(cnt), kSetupThreads, 0, h->stream>>>(cnt, h->en, nv, lost);
    int nlost = 0;
    CK(cudaMemcpyAsync(&nlost, lost, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (nlost) return fail(h, GADI_ERR_RANGE, "%d matrix entries are out of %s range after scaling", nlost, name);
    return GADI_OK;
}

// Demote the inner operators for the current alpha and inner precision:
// FP16, bfloat16 and FP8 E4M3 with the power-of-two scaling (or FP16
// unscaled), FP32 unscaled; FP64 needs nothing.
gadi_status prepare_inner(gadi_solver *h)
{
    if (h->u_r == GADI_F64) {
        h->sM = h->sNs = 0;
        return GADI_OK;
    }
    const bool naive = h->scaling == 0 && h->u_r == GADI_F16;
    const bool scaled = h->u_r != GADI_F32 && !naive;
    int sM = scaled ? half_scale_exponent(h->mnorm, h->alpha) : 0;
    int sN = scaled ? half_scale_exponent(h->nnorm, h->alpha) : 0;
    if (h->demoted && h->demoted_ur == h->u_r && sM == h->sM && sN == h->sNs &&
        h->demoted_scaling == h->scaling && (!naive || h->demoted_alpha == h->alpha))
        return GADI_OK;
    h->demoted = false;
    const int64_t cnt = h->n * (int64_t)h->W;
    const double scM = std::ldexp(1.0, -sM), scN = std::ldexp(1.0, -sN);
    const bool own_nt = h->ent || naive;     // S^T needs its own array
    gadi_status st = GADI_OK;
    if (h->u_r == GADI_F32) {
        bool ok = (h->m32 || !dalloc(&h->m32, cnt)) && (h->n32 || !dalloc(&h->n32, cnt)) &&
                  (!own_nt || h->nt32 || !dalloc(&h->nt32, cnt));
        if (ok && h->HD64) {
            ok = h->HD32 || !dalloc(&h->HD32, h->n);
            for (int d = 0; d < h->sdim && ok; ++d) ok = h->HK32[d] || !dalloc(&h->HK32[d], h->n);
        }
        if (!ok) {
            cudaGetLastError();
            return fail(h, GADI_ERR_OUT_OF_MEMORY, "no memory for the FP32 inner values");
        }
        demote_all<float>(h, h->m32, h->n32, h->nt32, h->HD32, h->HK32, false, scM, scN);
        CK(cudaGetLastError());
    } else {
        if (own_nt && !h->nt16 && dalloc(&h->nt16, cnt) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, GADI_ERR_OUT_OF_MEMORY, "no memory for the S^T values");
        }
        if (h->u_r == GADI_F16) {
            demote_all<__half>(h, h->m16, h->n16, h->nt16, h->HD16, h->HK16, naive, scM, scN);
            CK(cudaGetLastError());
            st = count_lost<__half>(h, h->m16, h->n16, "FP16");
        } else if (h->u_r == GADI_BF16) {
            auto bf = [](__half *p) { return reinterpret_cast<__nv_bfloat16 *>(p); };
            __nv_bfloat16 *hk[3] = {bf(h->HK16[0]), bf(h->HK16[1]), bf(h->HK16[2])};
            demote_all<__nv_bfloat16>(h, bf(h->m16), bf(h->n16), bf(h->nt16), bf(h->HD16), hk, false, scM, scN);
            CK(cudaGetLastError());
            st = count_lost<__nv_bfloat16>(h, bf(h->m16), bf(h->n16), "bfloat16");
        } else {
            // one-byte values in the first half of the 2-byte arrays
            auto f8 = [](__half *p) { return reinterpret_cast<__nv_fp8_e4m3 *>(p); };
            __nv_fp8_e4m3 *hk[3] = {f8(h->HK16[0]), f8(h->HK16[1]), f8(h->HK16[2])};
            demote_all<__nv_fp8_e4m3>(h, f8(h->m16), f8(h->n16), f8(h->nt16), f8(h->HD16), hk, false, scM, scN);
            CK(cudaGetLastError());
            st = count_lost<__nv_fp8_e4m3>(h, f8(h->m16), f8(h->n16), "FP8 E4M3");
        }
    }
    if (st != GADI_OK) return st;
    h->sM = sM;
    h->sNs = sN;
    h->demoted = true;
    h->demoted_ur = h->u_r;
    h->demoted_alpha = h->alpha;
    h->demoted_scaling = h->scaling;
    return GADI_OK;
}

template <class T>
EllOp<T> make_ell(const gadi_solver *h)
{
    using Acc = typename Prec<T>::Acc;
    EllOp<T> op;
    op.n = h->n;
    op.W = h->W;
    op.col = h->ecol;
    op.a64 = h->ea;
    const bool naive = h->scaling == 0 && std::is_same<T, __half>::value;
    if constexpr (std::is_same<T, double>::value) {
        op.m = h->em;
        op.nv = h->en;
        op.nt = h->ent;
    } else if constexpr (std::is_same<T, float>::value) {
        op.m = h->m32;
        op.nv = h->n32;
        op.nt = h->ent ? h->nt32 : nullptr;
    } else {
        op.m = reinterpret_cast<const T *>(h->m16);
        op.nv = reinterpret_cast<const T *>(h->n16);
        op.nt = (h->ent || naive) ? reinterpret_cast<const T *>(h->nt16) : nullptr;
    }
    op.sigH = naive ? Acc(0) : (Acc)std::ldexp(h->alpha, -h->sM);
    op.sigS = naive ? Acc(0) : (Acc)std::ldexp(h->alpha, -h->sNs);
    return op;
}

float half_round(double v)
{
    return __half2float(__double2half(v));
}

// v rounded to the nearest FP8 E4M3 value: 3 fraction bits below the
// leading bit, whose exponent is at least -6 (the smallest normal exponent;
// below it the spacing stays 2^-9), ties to even; magnitudes at or above
// 448, the largest finite value, saturate to it
float e4m3_round(double v)
{
    if (std::isnan(v)) return (float)v;
    const double a = std::fabs(v);
    if (a >= 448.0) return (float)std::copysign(448.0, v);
    int ex = 0;
    std::frexp(a, &ex);                        // a = f 2^ex, f in [0.5, 1)
    const double q = std::ldexp(1.0, std::max(ex - 1, -6) - 3);
    return (float)std::copysign(std::nearbyint(a / q) * q, v);
}

// v rounded once to the inner storage type T (as an arithmetic value)
template <class T>
typename Prec<T>::Acc round_to(double v)
{
    if constexpr (std::is_same<T, __half>::value) return half_round(v);
    else if constexpr (std::is_same<T, __nv_bfloat16>::value) return __bfloat162float(__double2bfloat16(v));
    else if constexpr (std::is_same<T, __nv_fp8_e4m3>::value) return e4m3_round(v);
    else if constexpr (std::is_same<T, float>::value) return (float)v;
    else return v;
}

template <class T, int DIM, int R>
StencilOp<T, DIM, R> make_stencil(const gadi_solver *h)
{
    using Acc = typename Prec<T>::Acc;
    StencilOp<T, DIM, R> op{};
    op.dim = h->sdim;
    op.N = h->sN;
    op.divN = div_magic((unsigned)op.N);
    op.n = h->n;
    op.a_diag = h->a_diag;
    op.a_lo = h->a_lo;
    op.a_hi = h->a_hi;
    op.AD = h->AD;
    for (int d = 0; d < 3; ++d) {
        op.AL[d] = h->AL[d];
        op.AU[d] = h->AU[d];
    }
    const double scM = std::ldexp(1.0, -h->sM), scN = std::ldexp(1.0, -h->sNs);
    op.s_diag = Acc(0);
    if constexpr (std::is_same<T, __half>::value) {
        if (h->scaling == 0) {
            // unscaled: alpha rounded into the FP16 diagonals, added in the row's order
            op.h_diag = half_round(h->a_diag + h->alpha);
            op.h_off = half_round(h->m_off);
            op.s_c = half_round(h->n_up);
            op.s_diag = half_round(h->alpha);
            op.HD = h->HD16;
            for (int d = 0; d < 3; ++d) op.HK[d] = h->HK16[d];
            op.sigH = Acc(0);
            op.sigS = Acc(0);
            return op;
        }
    }
    if constexpr (std::is_same<T, double>::value) {
        op.h_diag = h->a_diag;
        op.h_off = h->m_off;
        op.s_c = h->n_up;
        op.HD = h->HD64;
        for (int d = 0; d < 3; ++d) op.HK[d] = h->HK64[d];
    } else {
        op.h_diag = round_to<T>(h->a_diag * scM);
        op.h_off = round_to<T>(h->m_off * scM);
        op.s_c = round_to<T>(h->n_up * scN);
        if constexpr (std::is_same<T, float>::value) {
            op.HD = h->HD32;
            for (int d = 0; d < 3; ++d) op.HK[d] = h->HK32[d];
        } else {
            op.HD = reinterpret_cast<const T *>(h->HD16);
            for (int d = 0; d < 3; ++d) op.HK[d] = reinterpret_cast<const T *>(h->HK16[d]);
        }
    }
    op.sigH = (Acc)std::ldexp(h->alpha, -h->sM);
    op.sigS = (Acc)std::ldexp(h->alpha, -h->sNs);
    return op;
}

// the operator object of family Op for the handle's current parameters
template <class Op, class T>
Op make_op(gadi_solver *h)
{
    if constexpr (std::is_same<Op, EllOp<T>>::value) {
        return make_ell<T>(h);
    } else if constexpr (Op::kZMarch) {
        Op op;
        static_cast<typename Op::BaseOp &>(op) = make_stencil<T, Op::kDim, Op::R>(h);
        return op;
    } else {
        return make_stencil<T, Op::kDim, Op::R>(h);
    }
}

// z-marching segment length for a launch of `lanes` threads on the N^3
// stencil: about one column segment (N/8 x N columns) per thread, at least
// 4 planes (0: the march does not pay; use grid-stride items)
inline int zmarch_len(int N, int64_t lanes)
{
    const int64_t cols = (int64_t)(N / 8) * N;
    const int64_t nseg = std::max<int64_t>(1, lanes / cols);
    const int zlen = (int)((N + nseg - 1) / nseg);
    return zlen >= 4 ? zlen : 0;
}

template <class Op, class T>
gadi_status run_solve(gadi_solver *h, const double *b, double *x, double tol, double bnorm,
                      gadi_info *info)
{
    Op op = make_op<Op, T>(h);
    const int64_t nitems = h->n / Op::R;

    auto kern = gadi_solve_kernel<Op, T>;
    int threads = h->threads;
    if (threads == 0) {
        // enough threads for one item each on every SM, between 128 and 1024
        const int64_t per_sm = (nitems + h->num_sms - 1) / h->num_sms;
        threads = 128;
        while (threads < max_threads<Op>() && threads < per_sm) threads = std::min(2 * threads, max_threads<Op>());
        if (nitems <= 16384) threads = max_threads<Op>();
    }
    if (threads > max_threads<Op>())
        return fail(h, GADI_ERR_INVALID_ARG, "block_threads %d exceeds %d for this kernel", threads,
                    max_threads<Op>());
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0));
    if (per_sm < 1)
        return fail(h, GADI_ERR_CUDA, "solve kernel cannot run with %d threads per block", threads);
    const int max_blocks = per_sm * h->num_sms;
    int blocks = h->blocks;
    if (blocks == 0) {
        int64_t need = (nitems + threads - 1) / threads;
        if (nitems <= 16384) need = 1;
        blocks = (int)std::min<int64_t>(need, max_blocks);
    }
    if (blocks > max_blocks)
        return fail(h, GADI_ERR_INVALID_ARG, "grid_blocks %d exceeds the co-resident maximum %d",
                    blocks, max_blocks);
    int zlen = 0;
    if constexpr (Op::kZMarch) {
        zlen = blocks > 1 ? zmarch_len(op.N, (int64_t)blocks * threads) : 0;
        if (zlen == 0) return run_solve<typename Op::BaseOp, T>(h, b, x, tol, bnorm, info);
    }
    if (blocks > h->part_blocks) {
        if (h->part) cudaFree(h->part);
        h->part = nullptr;
        h->part_blocks = 0;
        CK(dalloc(&h->part, (size_t)2 * kMaxSlots * blocks));
        h->part_blocks = blocks;
    }

    T *V = (T *)h->vec;
    const int64_t n = h->n;
    SolveArgs<Op, T> a;
    a.op = op;
    a.n = n;
    a.nitems = nitems;
    a.b = b;
    a.x = x;
    a.x2 = h->x2;
    a.r64 = h->r64;
    a.r32 = r32_of(h->vec, n);
    for (int j = 0; j < 9; ++j) a.v[j] = V + j * n;
    a.anorm = h->anorm;
    a.bnorm = bnorm;
    a.tol = tol;
    a.eps = h->eps > 0 ? h->eps : (h->u_r == GADI_F64 ? 1e-10 : (h->u_r == GADI_E4M3 ? 0.1 : 1e-2));
    a.pfac = (2.0 - h->omega) * h->alpha;
    a.sM = h->sM;
    a.sN = h->sNs;
    a.half = h->u_r != GADI_F64 ? 1 : 0;     // r and z scaled by powers of two below FP64
    a.naive = (h->u_r == GADI_F16 && h->scaling == 0) ? 1 : 0;
    a.stop_kind = h->stop;
    a.max_inner = h->max_inner;
    a.max_outer = h->max_outer;
    a.ctl = h->ctl;
    a.part = h->part;
    a.eta_hist = nullptr;
    a.race_bound = nullptr;
    a.wait_ns = (unsigned long long)(h->wait_ms * 1e6);
    a.extra = h->force_timeout ? 1u : 0u;
    a.zlen = zlen;

    CK(cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->stream));
    CK(cudaEventRecord(h->ev0, h->stream));
    void *args[] = {(void *)&a};
    if (blocks > 1)
        CK(cudaLaunchCooperativeKernel((const void *)kern, dim3(blocks), dim3(threads), args, 0,
                                       h->stream));
    else
        CK(cudaLaunchKernel((const void *)kern, dim3(1), dim3(threads), args, 0, h->stream));
    CK(cudaEventRecord(h->ev1, h->stream));
    Ctl c;
    CK(cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->ev0, h->ev1));
    gadi_status st = c.error ? (gadi_status)c.error : (gadi_status)c.status;
    if (info) {
        info->outer_iters = c.outer_iters;
        info->status = st;
        info->inner_iters_H = c.itH;
        info->inner_iters_S = c.itS;
        info->spmv_count = c.spmv;
        info->eta_inf = c.eta;
        info->res_rel = c.res;
        info->t_solve_s = ms * 1e-3;
        info->scale_exp_M = h->sM;
        info->scale_exp_N = h->sNs;
        info->kernel = std::is_same<Op, EllOp<T>>::value ? GADI_KERNEL_SPARSE : GADI_KERNEL_STENCIL;
        info->grid_blocks = blocks;
        info->block_threads = threads;
        info->zmarch_planes = zlen;
    }
    if (st == GADI_ERR_TIMEOUT) return fail(h, st, "a device-side grid-barrier wait expired");
    if (st == GADI_ERR_DIVERGED) return fail(h, st, "the iteration diverged (non-finite values, inner breakdown or residual growth)");
    if (st == GADI_ERR_NOT_CONVERGED) return fail(h, st, "max_outer reached before the tolerance");
    return st;
}

// ring slots (planes) of the staged stencil application
constexpr int kStagedSlots = 8;

template <class Op, class T>
gadi_status run_apply(gadi_solver *h, int which, const void *x, void *y)
{
    Op op = make_op<Op, T>(h);
    const int64_t nitems = h->n / Op::R;
    if constexpr (std::is_same<Op, StencilOp<__half, 3, 8>>::value) {
        // constant-coefficient FP16 stencil without a set launch shape: the
        // shared-memory staged kernel when a block can own ty >= 4 whole
        // y-lines (ty divides N, nx8 ty <= 512 threads), with z segments of
        // at least 4 planes and about two blocks per SM in all
        const int nx8 = op.N / 8;
        int ty = 0;
        if (nx8 <= 128)
            for (int t = 512 / nx8; t >= 4; --t)
                if (op.N % t == 0) { ty = t; break; }
        if (!h->threads && !h->blocks && op.HD == nullptr && which != kOpA && ty) {
            constexpr int S = kStagedSlots;
            const int ytiles = op.N / ty;
            const int64_t want = (2 * (int64_t)h->num_sms + ytiles - 1) / ytiles;
            const int nseg = (int)std::max<int64_t>(1, std::min<int64_t>(op.N / 4, want));
            const int zlen = (op.N + nseg - 1) / nseg;
            const int segs = (op.N + zlen - 1) / zlen;
            const size_t smem = (size_t)S * (ty + 2) * nx8 * sizeof(uint4);
            auto kern = gadi_apply_staged_kernel<Op, S>;
            CK(cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            kern<<<(unsigned)(ytiles * segs), (unsigned)(nx8 * ty), smem, h->stream>>>(
                op, which, ty, zlen, (const __half *)x, (__half *)y);
            CK(cudaGetLastError());
            return GADI_OK;
        }
    }
    // launch shape: gadi_set_launch's when given, else one item per thread
    const int threads = h->threads ? h->threads : kSetupThreads;
    const unsigned blocks = h->blocks ? (unsigned)h->blocks : grid_for(nitems, threads);
    if constexpr (Op::R == 8) gadi_apply_kernel_wide<Op, T><<<blocks, threads, 0, h->stream>>>(op, nitems, which, x, y);
    else gadi_apply_kernel<Op, T><<<blocks, threads, 0, h->stream>>>(op, nitems, which, x, y);
    CK(cudaGetLastError());
    return GADI_OK;
}

template <class X>
struct Tag {
    using type = X;
};

// stencil rows per item in use: the one set by gadi_set_item_rows when the
// grid side is a multiple of it, else 8 or 4 when the side allows, else 1
int item_rows(const gadi_solver *h)
{
    if (h->item_rows > 0 && h->sN % h->item_rows == 0) return h->item_rows;
    if (h->item_rows == 0) {
        if (h->sN % 8 == 0) return 8;
        if (h->sN % 4 == 0) return 4;
    }
    return 1;
}

// call fn(Tag<Op>, Tag<T>) with the operator family and inner type in use:
// the sparse operator, or the stencil for dim 2/3 with items of 1, 4 or 8
// rows of one grid line
template <class T, int DIM, class Fn>
gadi_status dispatch_rows(const gadi_solver *h, Fn &&fn, bool solve)
{
    switch (item_rows(h)) {
    case 8:
        if constexpr (StencilOp<T, DIM, 8>::kZMarchCapable) {
            // solves of the constant-coefficient operator: the z-marching family
            if (solve && h->traversal == 0 && !h->variable_k)
                return fn(Tag<ZMarchOp<StencilOp<T, DIM, 8>>>{}, Tag<T>{});
        }
        return fn(Tag<StencilOp<T, DIM, 8>>{}, Tag<T>{});
    case 4: return fn(Tag<StencilOp<T, DIM, 4>>{}, Tag<T>{});
    default: return fn(Tag<StencilOp<T, DIM, 1>>{}, Tag<T>{});
    }
}

template <class T, class Fn>
gadi_status dispatch_op(const gadi_solver *h, Fn &&fn, bool solve)
{
    if (!use_stencil(h)) return fn(Tag<EllOp<T>>{}, Tag<T>{});
    if (h->sdim == 3) return dispatch_rows<T, 3>(h, fn, solve);
    return dispatch_rows<T, 2>(h, fn, solve);
}

// solve = true: a solve, which may use the z-marching operator family
template <class Fn>
gadi_status dispatch(const gadi_solver *h, Fn &&fn, bool solve = false)
{
    switch (h->u_r) {
    case GADI_F16: return dispatch_op<__half>(h, fn, solve);
    case GADI_BF16: return dispatch_op<__nv_bfloat16>(h, fn, solve);
    case GADI_E4M3: return dispatch_op<__nv_fp8_e4m3>(h, fn, solve);
    case GADI_F32: return dispatch_op<float>(h, fn, solve);
    default: return dispatch_op<double>(h, fn, solve);
    }
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *gadi_status_str(gadi_status s)
{
    switch (s) {
    case GADI_OK: return "GADI_OK";
    case GADI_ERR_INVALID_ARG: return "GADI_ERR_INVALID_ARG";
    case GADI_ERR_OUT_OF_MEMORY: return "GADI_ERR_OUT_OF_MEMORY";
    case GADI_ERR_CUDA: return "GADI_ERR_CUDA";
    case GADI_ERR_RANGE: return "GADI_ERR_RANGE";
    case GADI_ERR_NOT_CONVERGED: return "GADI_ERR_NOT_CONVERGED";
    case GADI_ERR_DIVERGED: return "GADI_ERR_DIVERGED";
    case GADI_ERR_TIMEOUT: return "GADI_ERR_TIMEOUT";
    case GADI_ERR_NO_MODEL: return "GADI_ERR_NO_MODEL";
    case GADI_ERR_UNSUPPORTED: return "GADI_ERR_UNSUPPORTED";
    }
    return "unknown gadi_status";
}

const char *gadi_last_error(const gadi_solver *h)
{
    return h ? h->err.c_str() : "null handle";
}

void gadi_destroy(gadi_solver *h)
{
    if (!h) return;
    release(h);
    delete h;
}

gadi_status gadi_create(const gadi_csr *A, gadi_splitting split, const gadi_csr *M_user,
                        const gadi_stencil *structure, void *cuda_stream, gadi_solver **out)
{
    gadi_solver *h = nullptr;
    if (!out) return GADI_ERR_INVALID_ARG;
    *out = nullptr;
    if (!A || A->n < 1 || A->nnz < A->n || A->nnz > 0x7fffffffLL || !A->row_ptr || !A->col_idx || !A->val)
        return GADI_ERR_INVALID_ARG;
    if (split != GADI_SPLIT_HSS && split != GADI_SPLIT_USER) return GADI_ERR_INVALID_ARG;
    if (split == GADI_SPLIT_USER && (!M_user || M_user->n != A->n || M_user->nnz != A->nnz || !M_user->val ||
                                     M_user->on_device != A->on_device))
        return GADI_ERR_INVALID_ARG;
    if (structure) {
        const gadi_stencil &s = *structure;
        if ((s.dim != 2 && s.dim != 3) || s.N < 1 || !std::isfinite(s.beta) ||
            (s.variable_k && s.dim != 3) || split != GADI_SPLIT_HSS)
            return GADI_ERR_INVALID_ARG;
        int64_t nn = s.dim == 3 ? (int64_t)s.N * s.N * s.N : (int64_t)s.N * s.N;
        if (nn != A->n || nn >= (1LL << 31)) return GADI_ERR_INVALID_ARG;
    }
    h = new (std::nothrow) gadi_solver();
    if (!h) return GADI_ERR_OUT_OF_MEMORY;
    gadi_status st = GADI_OK;
    auto bail = [&](gadi_status s) {
        release(h);
        delete h;
        return s;
    };
    do {
        cudaError_t e;
        if ((e = cudaGetDevice(&h->dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->dev)) != cudaSuccess) {
            cudaGetLastError();
            return bail(GADI_ERR_CUDA);
        }
        h->stream = (cudaStream_t)cuda_stream;
        h->n = A->n;
        h->nnz = A->nnz;
        h->user_split = split == GADI_SPLIT_USER;
        const int64_t n = h->n, nnz = h->nnz;
        int *rp = nullptr, *ci = nullptr;
        double *va = nullptr, *vm = nullptr;
        bool own = !A->on_device;
        auto cleanup_in = [&]() {
            if (own) {
                if (rp) cudaFree(rp);
                if (ci) cudaFree(ci);
                if (va) cudaFree(va);
                if (vm) cudaFree(vm);
            }
        };
        if (own) {
            if (dalloc(&rp, n + 1) || dalloc(&ci, nnz) || dalloc(&va, nnz) ||
                (h->user_split && dalloc(&vm, nnz))) {
                cleanup_in();
                cudaGetLastError();
                return bail(GADI_ERR_OUT_OF_MEMORY);
            }
            cudaMemcpyAsync(rp, A->row_ptr, (n + 1) * sizeof(int), cudaMemcpyHostToDevice, h->stream);
            cudaMemcpyAsync(ci, A->col_idx, nnz * sizeof(int), cudaMemcpyHostToDevice, h->stream);
            cudaMemcpyAsync(va, A->val, nnz * sizeof(double), cudaMemcpyHostToDevice, h->stream);
            if (h->user_split)
                cudaMemcpyAsync(vm, M_user->val, nnz * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        } else {
            rp = (int *)A->row_ptr;
            ci = (int *)A->col_idx;
            va = (double *)A->val;
            vm = h->user_split ? (double *)M_user->val : nullptr;
        }
        if (dalloc(&h->scratch, 64) != cudaSuccess) { cleanup_in(); return bail(GADI_ERR_OUT_OF_MEMORY); }
        int *flags = (int *)h->scratch;          // [0] bad, [1] maxlen
        double *norms = h->scratch + 4;          // [0..3]
        cudaMemsetAsync(h->scratch, 0, 64 * sizeof(double), h->stream);
        k_check_csr<<<grid_for(n), kSetupThreads, 0, h->stream>>>(n, nnz, rp, ci, va, flags, flags + 1);
        if (h->user_split)
            k_check_csr<<<grid_for(n), kSetupThreads, 0, h->stream>>>(n, nnz, rp, ci, vm, flags, flags + 1);
        int hf[2] = {0, 0};
        e = cudaMemcpyAsync(hf, flags, sizeof hf, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) { cleanup_in(); cudaGetLastError(); return bail(GADI_ERR_CUDA); }
        if (hf[0]) { cleanup_in(); return bail(GADI_ERR_INVALID_ARG); }
        h->W = std::max(4, (hf[1] + 3) / 4 * 4);
        if (structure && h->W > 8) { cleanup_in(); return bail(GADI_ERR_INVALID_ARG); }
        const int64_t cell = n * (int64_t)h->W;
        if (dalloc(&h->ecol, cell) || dalloc(&h->ea, cell) || dalloc(&h->em, cell) ||
            dalloc(&h->en, cell) || (h->user_split && dalloc(&h->ent, cell)) ||
            dalloc(&h->m16, cell) || dalloc(&h->n16, cell) || (h->user_split && dalloc(&h->nt16, cell))) {
            cleanup_in();
            cudaGetLastError();
            return bail(GADI_ERR_OUT_OF_MEMORY);
        }
        k_split_ell<<<grid_for(n), kSetupThreads, 0, h->stream>>>(n, rp, ci, va, vm, h->W, h->ecol, h->ea,
                                                                  h->em, h->en, h->ent, norms, flags);
        double hn[4];
        e = cudaMemcpyAsync(hn, norms, sizeof hn, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, sizeof hf, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cleanup_in();
        if (e != cudaSuccess) { cudaGetLastError(); return bail(GADI_ERR_CUDA); }
        if (hf[0]) return bail(GADI_ERR_INVALID_ARG);
        h->anorm = hn[0];
        h->mnorm = hn[1];
        h->nnorm = std::max(hn[2], hn[3]);
        if (structure) {
            h->has_stencil = true;
            h->sdim = structure->dim;
            h->sN = structure->N;
            h->beta = structure->beta;
            h->variable_k = structure->variable_k;
            const double hh = 1.0 / (structure->N + 1);
            h->c = structure->beta * hh / 2.0;
            if (h->variable_k) {
                bool okm = !dalloc(&h->AD, n) && !dalloc(&h->HD64, n) && !dalloc(&h->HD16, n);
                for (int d = 0; d < 3 && okm; ++d)
                    okm = !dalloc(&h->AL[d], n) && !dalloc(&h->AU[d], n) && !dalloc(&h->HK64[d], n) &&
                          !dalloc(&h->HK16[d], n);
                if (!okm) { cudaGetLastError(); return bail(GADI_ERR_OUT_OF_MEMORY); }
            }
            cudaMemsetAsync(flags, 0, sizeof(int), h->stream);
            k_stencil_extract<<<grid_for(n), kSetupThreads, 0, h->stream>>>(
                n, h->sdim, h->sN, h->c, h->variable_k, h->W, h->ecol, h->ea, h->em, h->en, h->AD,
                h->AL[0], h->AL[1], h->AL[2], h->AU[0], h->AU[1], h->AU[2], h->HD64, h->HK64[0],
                h->HK64[1], h->HK64[2], flags);
            e = cudaMemcpyAsync(hf, flags, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) { cudaGetLastError(); return bail(GADI_ERR_CUDA); }
            if (hf[0]) return bail(GADI_ERR_INVALID_ARG);
            // constant-coefficient scalars from rows 0 and 1: row 0 stores
            // (diagonal, x+, ...), row 1 stores (x-, diagonal, ...)
            const int W = h->W;
            double row01[3][16] = {};
            const int cnt = (int)std::min<int64_t>(2 * W, n * W);
            e = cudaMemcpyAsync(row01[0], h->ea, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(row01[1], h->em, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(row01[2], h->en, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) { cudaGetLastError(); return bail(GADI_ERR_CUDA); }
            h->a_diag = row01[0][0];
            if (structure->N >= 2) {
                h->a_hi = row01[0][1];
                h->m_off = row01[1][1];
                h->n_up = row01[2][1];
                h->a_lo = row01[0][W];
            } else {
                h->a_hi = h->a_lo = h->m_off = h->n_up = 0.0;
            }
        }
        if (dalloc(&h->r64, n) || dalloc(&h->bdev, n) || dalloc(&h->xdev, n) || dalloc(&h->x2, n) ||
            cudaMalloc(&h->vec, vec_bytes(n)) || dalloc(&h->ctl, 1)) {
            cudaGetLastError();
            return bail(GADI_ERR_OUT_OF_MEMORY);
        }
        if (cudaEventCreate(&h->ev0) || cudaEventCreate(&h->ev1)) {
            cudaGetLastError();
            return bail(GADI_ERR_CUDA);
        }
    } while (0);
    *out = h;
    return st;
}

gadi_status gadi_set_params(gadi_solver *h, double alpha, double omega, gadi_precision u_r,
                            gadi_precision u, gadi_precision u_f)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (!(alpha > 0.0) || !std::isfinite(alpha))
        return fail(h, GADI_ERR_INVALID_ARG, "alpha must be positive and finite (Thm 1)");
    if (!(omega >= 0.0 && omega < 2.0))
        return fail(h, GADI_ERR_INVALID_ARG, "omega must lie in [0, 2) (Thm 1)");
    auto valid = [](int p) { return p >= GADI_F64 && p <= GADI_E4M3; };
    if (!valid(u_r) || !valid(u) || !valid(u_f))
        return fail(h, GADI_ERR_INVALID_ARG, "unknown precision");
    if (u != GADI_F64 || u_f != GADI_F64)
        return fail(h, GADI_ERR_UNSUPPORTED, "supported precision triples: u = u_f = F64, any u_r");
    if (u_r != h->u_r) h->demoted = false;
    h->alpha = alpha;
    h->omega = omega;
    h->u_r = u_r;
    return GADI_OK;
}

gadi_status gadi_set_inner(gadi_solver *h, double eps_inner, int32_t max_inner, int32_t max_outer)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (!(eps_inner > 0.0 && eps_inner < 1.0) || max_inner < 1 || max_outer < 0)
        return fail(h, GADI_ERR_INVALID_ARG, "need 0 < eps_inner < 1, max_inner >= 1, max_outer >= 0");
    h->eps = eps_inner;
    h->max_inner = max_inner;
    h->max_outer = max_outer;
    return GADI_OK;
}

gadi_status gadi_set_stop(gadi_solver *h, gadi_stop kind)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (kind != GADI_STOP_ETA && kind != GADI_STOP_RES) return fail(h, GADI_ERR_INVALID_ARG, "unknown stop kind");
    h->stop = kind;
    return GADI_OK;
}

gadi_status gadi_set_kernel(gadi_solver *h, gadi_kernel kind)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (kind < GADI_KERNEL_AUTO || kind > GADI_KERNEL_STENCIL)
        return fail(h, GADI_ERR_INVALID_ARG, "unknown kernel kind");
    if (kind == GADI_KERNEL_STENCIL && !h->has_stencil)
        return fail(h, GADI_ERR_INVALID_ARG, "the stencil kernels need a stencil descriptor at create");
    h->kernel = kind;
    return GADI_OK;
}

gadi_status gadi_set_scaling(gadi_solver *h, int32_t on)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (on != 0 && on != 1) return fail(h, GADI_ERR_INVALID_ARG, "scaling must be 0 or 1");
    h->scaling = on;
    return GADI_OK;
}

gadi_status gadi_set_traversal(gadi_solver *h, int32_t mode)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (mode != 0 && mode != 1)
        return fail(h, GADI_ERR_INVALID_ARG, "traversal must be 0 (automatic) or 1 (grid-stride items)");
    h->traversal = mode;
    return GADI_OK;
}

gadi_status gadi_set_item_rows(gadi_solver *h, int32_t rows)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (rows != 0 && rows != 1 && rows != 4 && rows != 8)
        return fail(h, GADI_ERR_INVALID_ARG, "rows per item must be 0 (automatic), 1, 4 or 8");
    h->item_rows = rows;
    return GADI_OK;
}

gadi_status gadi_set_launch(gadi_solver *h, int32_t grid_blocks, int32_t block_threads)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (grid_blocks < 0 || (block_threads != 0 && block_threads != 128 && block_threads != 256 &&
                            block_threads != 512 && block_threads != 1024))
        return fail(h, GADI_ERR_INVALID_ARG, "grid_blocks >= 0; block_threads in {0,128,256,512,1024}");
    h->blocks = grid_blocks;
    h->threads = block_threads;
    return GADI_OK;
}

gadi_status gadi_set_wait_limit(gadi_solver *h, double milliseconds)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (!(milliseconds > 0.0 && milliseconds <= 600000.0))
        return fail(h, GADI_ERR_INVALID_ARG, "wait limit must lie in (0, 600000] ms");
    h->wait_ms = milliseconds;
    return GADI_OK;
}

gadi_status gadi_debug_force_timeout(gadi_solver *h, int32_t on)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    h->force_timeout = on ? 1 : 0;
    return GADI_OK;
}

gadi_status gadi_get_scales(gadi_solver *h, int32_t *sM, int32_t *sN)
{
    if (!h || !sM || !sN) return GADI_ERR_INVALID_ARG;
    gadi_status st = prepare_inner(h);
    if (st != GADI_OK) return st;
    *sM = h->sM;
    *sN = h->sNs;
    return GADI_OK;
}

gadi_status gadi_solve(gadi_solver *h, const double *b, double *x, double tol, gadi_info *info)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (!b || !x) return fail(h, GADI_ERR_INVALID_ARG, "b and x must not be NULL");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(h, GADI_ERR_INVALID_ARG, "tol must be positive");
    const bool bd = is_device_ptr(b), xd = is_device_ptr(x);
    if (bd != xd) return fail(h, GADI_ERR_INVALID_ARG, "b and x must both be host or both be device pointers");
    const int64_t n = h->n;
    const double *bb = b;
    double *xx = x;
    if (!bd) {
        CK(cudaMemcpyAsync(h->bdev, b, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(h->xdev, x, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        bb = h->bdev;
        xx = h->xdev;
    }
    // ||b||_inf and finiteness of b and x0
    double *bn = h->scratch + 8;
    int *nf = (int *)(h->scratch + 9);
    CK(cudaMemsetAsync(h->scratch + 8, 0, 3 * sizeof(double), h->stream));
    k_vec_check<<<grid_for(n), kSetupThreads, 0, h->stream>>>(n, bb, bn, nf);
    k_vec_check<<<grid_for(n), kSetupThreads, 0, h->stream>>>(n, xx, h->scratch + 10, nf);
    CK(cudaGetLastError());
    double hb[2];
    CK(cudaMemcpyAsync(hb, h->scratch + 8, sizeof hb, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    int nonfinite;
    std::memcpy(&nonfinite, &hb[1], sizeof(int));
    if (nonfinite) return fail(h, GADI_ERR_INVALID_ARG, "b or x0 holds a NaN or Inf");
    gadi_status st = prepare_inner(h);
    if (st != GADI_OK) return st;
    st = dispatch(h, [&](auto opk, auto tk) {
        using Op = typename decltype(opk)::type;
        using T = typename decltype(tk)::type;
        return run_solve<Op, T>(h, bb, xx, tol, hb[0], info);
    }, true);
    if (st == GADI_ERR_CUDA || st == GADI_ERR_OUT_OF_MEMORY) return st;
    if (!xd) {
        std::string keep = h->err;
        CK(cudaMemcpyAsync(x, h->xdev, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        h->err = keep;
    }
    return st;
}

gadi_status gadi_apply(gadi_solver *h, int32_t which, const void *x, void *y)
{
    if (!h) return GADI_ERR_INVALID_ARG;
    if (which < kOpA || which > kOpST || !x || !y) return fail(h, GADI_ERR_INVALID_ARG, "bad apply arguments");
    gadi_status st = prepare_inner(h);
    if (st != GADI_OK) return st;
    return dispatch(h, [&](auto opk, auto tk) {
        using Op = typename decltype(opk)::type;
        using T = typename decltype(tk)::type;
        return run_apply<Op, T>(h, which, x, y);
    });
}

gadi_status gadi_set_model(gadi_solver *h, int32_t kind, const gadi_model *model)
{
    if (!h || (kind != GADI_MODEL_MLP && kind != GADI_MODEL_GPR)) return GADI_ERR_INVALID_ARG;
    h->models[kind] = model;
    return GADI_OK;
}

gadi_status gadi_predict_params(gadi_solver *h, const double *features, int32_t nfeat, int32_t kind,
                                double *alpha, double *omega)
{
    if (!h || !alpha || !omega || kind < GADI_MODEL_MLP || kind > GADI_MODEL_GRID) return GADI_ERR_INVALID_ARG;
    if (kind != GADI_MODEL_GRID) {
        if (!features || nfeat < 2) return fail(h, GADI_ERR_INVALID_ARG, "features need (log n, log beta)");
        if (!h->models[kind]) return fail(h, GADI_ERR_NO_MODEL, "no model of this kind attached");
        double y[2];
        gadi_status st = gadi_model_predict(h->models[kind], features, 1, y);
        if (st != GADI_OK) return fail(h, st, "model prediction failed");
        const double a = std::exp(y[0]);
        if (!(a > 0.0) || !std::isfinite(a)) return fail(h, GADI_ERR_RANGE, "predicted alpha out of range");
        *alpha = a;
        *omega = std::min(1.999, std::max(0.0, y[1]));
        return GADI_OK;
    }
    // grid search on the handle's own system: b = A 1, x0 = 0, each candidate
    // capped at the fewest outer steps of a converged candidate so far
    const int64_t n = h->n;
    double *ones = nullptr, *b = nullptr, *x = nullptr;
    auto cleanup = [&]() {
        if (ones) cudaFree(ones);
        if (b) cudaFree(b);
        if (x) cudaFree(x);
    };
    if (dalloc(&ones, n) || dalloc(&b, n) || dalloc(&x, n)) {
        cudaGetLastError();
        cleanup();
        return fail(h, GADI_ERR_OUT_OF_MEMORY, "grid search buffers");
    }
    std::vector<double> h1(n, 1.0);
    cudaError_t e = cudaMemcpyAsync(ones, h1.data(), n * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) { cleanup(); return fail(h, GADI_ERR_CUDA, "grid search upload"); }
    const double save_a = h->alpha, save_w = h->omega;
    const int save_outer = h->max_outer;
    gadi_status st = gadi_apply(h, kOpA, ones, b);
    if (st != GADI_OK) { cleanup(); return st; }
    long long best_cost = -1;
    int best_outer = save_outer;
    double ba = 0, bw = 0;
    for (int ia = 0; ia < 16; ++ia)
        for (int iw = 0; iw < 4; ++iw) {
            const double a = std::pow(10.0, -3.0 + 5.0 * ia / 15.0), w = 0.5 * iw;
            h->alpha = a;
            h->omega = w;
            h->max_outer = best_outer;
            if ((e = cudaMemsetAsync(x, 0, n * sizeof(double), h->stream)) != cudaSuccess) break;
            gadi_info info;
            gadi_status s2 = gadi_solve(h, b, x, 1e-10, &info);
            if (s2 == GADI_ERR_CUDA || s2 == GADI_ERR_OUT_OF_MEMORY || s2 == GADI_ERR_TIMEOUT) { st = s2; break; }
            if (s2 != GADI_OK) continue;
            if (best_cost < 0 || info.spmv_count < best_cost) {
                best_cost = info.spmv_count;
                best_outer = std::min(best_outer, info.outer_iters);
                ba = a;
                bw = w;
            }
        }
    h->alpha = save_a;
    h->omega = save_w;
    h->max_outer = save_outer;
    h->demoted = false;
    cleanup();
    if (e != cudaSuccess) return fail(h, GADI_ERR_CUDA, "grid search");
    if (st != GADI_OK) return st;
    if (best_cost < 0) return fail(h, GADI_ERR_NOT_CONVERGED, "no grid candidate converged");
    *alpha = ba;
    *omega = bw;
    return GADI_OK;
}

}  // extern "C"
