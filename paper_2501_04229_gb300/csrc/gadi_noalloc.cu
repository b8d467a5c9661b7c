// gadi_noalloc.cu -- gadi_solve_stencil_noalloc: a GADI-IR solve of the
// constant-coefficient convection-diffusion stencil that allocates no device
// memory. Its scratch (control block, reduction partials, FP64 residual, its
// FP32 copy, a second iterate and the FP16 inner vectors) lives in one
// file-scope __device__ array of fixed
// size, g_noalloc_scratch, which every GPU that loads the library holds until
// the process exits.
//
// The host never uses the array's name as an address: the first call on a
// device (with that device current) looks the address up once with
// cudaGetSymbolAddress and caches it per device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/gadi.h"
#include "gadi_solve.cuh"

using namespace gadi;

namespace {

constexpr int64_t kNoallocMaxN = GADI_NOALLOC_MAX_N;
constexpr int kNoallocMaxBlocks = 1024;
constexpr size_t kCtlBytes = 256;
constexpr size_t kPartBytes = (size_t)2 * kMaxSlots * kNoallocMaxBlocks * sizeof(double);
constexpr size_t kChkBytes = 256;
constexpr size_t kR64Bytes = (size_t)kNoallocMaxN * sizeof(double);
constexpr size_t kR32Bytes = (size_t)kNoallocMaxN * sizeof(float);
constexpr size_t kX2Bytes = (size_t)kNoallocMaxN * sizeof(double);
constexpr size_t kVecBytes = (size_t)9 * kNoallocMaxN * sizeof(__half);
constexpr size_t kScratchBytes = kCtlBytes + kPartBytes + kChkBytes + kR64Bytes + kR32Bytes + kX2Bytes + kVecBytes;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};

// ||b||_inf, ||x0||_inf and a non-finite flag, into the scratch check area
__global__ void k_noalloc_check(int64_t n, const double *b, const double *x, double *out, int *bad)
{
    double mb = 0.0, mx = 0.0;
    int f = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double vb = b[i], vx = x[i];
        if (!isfinite(vb) || !isfinite(vx)) f = 1;
        else {
            mb = fmax(mb, fabs(vb));
            mx = fmax(mx, fabs(vx));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mb = fmax(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        f |= __shfl_xor_sync(0xffffffffu, f, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax((unsigned long long *)out, (unsigned long long)__double_as_longlong(mb));
        atomicMax((unsigned long long *)(out + 1), (unsigned long long)__double_as_longlong(mx));
        if (f) atomicOr(bad, 1);
    }
}

// a failed CUDA call: clear the runtime's last-error state (a non-sticky
// error such as a rejected launch would otherwise surface in the caller's
// next CUDA or torch check) and report GADI_ERR_CUDA
gadi_status cuda_failure()
{
    cudaGetLastError();
    return GADI_ERR_CUDA;
}

// the address of g_noalloc_scratch on the current device (looked up once)
cudaError_t scratch_address(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = (unsigned char *)p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

int half_scale(double norm, double sigma)
{
    double v = norm + std::fabs(sigma);
    if (!(v > 0.0) || !std::isfinite(v)) return 0;
    int e;
    double m = std::frexp(v, &e);
    return ((m == 0.5) ? e - 1 : e) - 1;
}

// max over rows of sum_j |v_ij| for the stencil with lower coefficient lo,
// diagonal dg and upper coefficient hi, summed in ascending column order
double stencil_row_norm(int dim, int N, double lo, double dg, double hi)
{
    double best = 0.0;
    int classes = 1;
    for (int d = 0; d < dim; ++d) classes *= 3;
    for (int cls = 0; cls < classes; ++cls) {
        int pos[3] = {0, 0, 0}, t = cls;    // 0 first, 1 interior, 2 last
        bool ok = true;
        for (int d = 0; d < dim; ++d) {
            pos[d] = t % 3;
            t /= 3;
            if (pos[d] == 1 && N < 3) ok = false;
            if (pos[d] == 2 && N < 2) ok = false;
        }
        if (!ok) continue;
        double s = 0.0;
        for (int d = dim - 1; d >= 0; --d)
            if (pos[d] != 0) s += std::fabs(lo);
        s += std::fabs(dg);
        for (int d = 0; d < dim; ++d)
            if (pos[d] != 2 && N >= 2) s += std::fabs(hi);
        if (s > best) best = s;
    }
    return best;
}

float to_half_float(double v)
{
    return __half2float(__double2half(v));
}

template <int DIM, int R>
gadi_status launch(int dev, int num_sms, cudaStream_t stream, unsigned char *base, int N, double c,
                   double alpha, double omega, double eps, int max_inner, int max_outer,
                   const double *b, double *x, double tol, double bnorm, gadi_info *info)
{
    using Op = StencilOp<__half, DIM, R>;
    const int64_t n = DIM == 3 ? (int64_t)N * N * N : (int64_t)N * N;
    // coefficients exactly as the HSS split of the assembled operator gives them
    const double a_diag = 2.0 * DIM, a_lo = -1.0 - c, a_hi = -1.0 + c;
    const double m_off = 0.5 * (a_hi + a_lo), n_up = 0.5 * (a_hi - a_lo);
    const double anorm = stencil_row_norm(DIM, N, a_lo, a_diag, a_hi);
    const double mnorm = stencil_row_norm(DIM, N, m_off, a_diag, m_off);
    const double nnorm = stencil_row_norm(DIM, N, -n_up, 0.0, n_up);
    const int sM = half_scale(mnorm, alpha), sN = half_scale(nnorm, alpha);
    const double scM = std::ldexp(1.0, -sM), scN = std::ldexp(1.0, -sN);

    Op op{};
    op.dim = DIM;
    op.N = N;
    op.divN = div_magic((unsigned)op.N);
    op.n = n;
    op.a_diag = a_diag;
    op.a_lo = a_lo;
    op.a_hi = a_hi;
    op.h_diag = to_half_float(a_diag * scM);
    op.h_off = to_half_float(m_off * scM);
    op.s_c = to_half_float(n_up * scN);
    op.sigH = (float)std::ldexp(alpha, -sM);
    op.sigS = (float)std::ldexp(alpha, -sN);

    const int64_t nitems = n / R;
    auto kern = gadi_solve_kernel<Op, __half>;
    int threads = 128;
    {
        const int64_t per_sm = (nitems + num_sms - 1) / num_sms;
        while (threads < max_threads<Op>() && threads < per_sm) threads = std::min(2 * threads, max_threads<Op>());
        if (nitems <= 16384) threads = max_threads<Op>();
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
    if (e != cudaSuccess || per_sm < 1) return cuda_failure();
    int64_t need = (nitems + threads - 1) / threads;
    if (nitems <= 16384) need = 1;
    const int blocks = (int)std::min<int64_t>(std::min<int64_t>(need, (int64_t)per_sm * num_sms), kNoallocMaxBlocks);

    Ctl *ctl = (Ctl *)base;
    SolveArgs<Op, __half> a;
    a.op = op;
    a.n = n;
    a.nitems = nitems;
    a.b = b;
    a.x = x;
    a.r64 = (double *)(base + kCtlBytes + kPartBytes + kChkBytes);
    a.r32 = (float *)(base + kCtlBytes + kPartBytes + kChkBytes + kR64Bytes);
    a.x2 = (double *)(base + kCtlBytes + kPartBytes + kChkBytes + kR64Bytes + kR32Bytes);
    __half *V = (__half *)(base + kCtlBytes + kPartBytes + kChkBytes + kR64Bytes + kR32Bytes + kX2Bytes);
    for (int j = 0; j < 9; ++j) a.v[j] = V + j * n;
    a.anorm = anorm;
    a.bnorm = bnorm;
    a.tol = tol;
    a.eps = eps;
    a.pfac = (2.0 - omega) * alpha;
    a.sM = sM;
    a.sN = sN;
    a.half = 1;
    a.naive = 0;
    a.stop_kind = GADI_STOP_ETA;
    a.max_inner = max_inner;
    a.max_outer = max_outer;
    a.ctl = ctl;
    a.part = (double *)(base + kCtlBytes);
    a.eta_hist = nullptr;
    a.race_bound = nullptr;
    a.wait_ns = 2000000000ULL;
    a.extra = 0;
    a.zlen = 0;

    // the control block must start at zero; everything else is written
    // before it is read by the kernel itself
    if ((e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), stream)) != cudaSuccess) return cuda_failure();
    const auto t0 = std::chrono::steady_clock::now();   // host wall time (no CUDA events here)
    void *args[] = {(void *)&a};
    if (blocks > 1)
        e = cudaLaunchCooperativeKernel((const void *)kern, dim3(blocks), dim3(threads), args, 0, stream);
    else
        e = cudaLaunchKernel((const void *)kern, dim3(1), dim3(threads), args, 0, stream);
    if (e != cudaSuccess) return cuda_failure();
    Ctl hc;
    if ((e = cudaMemcpyAsync(&hc, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(stream)) != cudaSuccess)
        return cuda_failure();
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const gadi_status st = hc.error ? (gadi_status)hc.error : (gadi_status)hc.status;
    if (info) {
        info->outer_iters = hc.outer_iters;
        info->status = st;
        info->inner_iters_H = hc.itH;
        info->inner_iters_S = hc.itS;
        info->spmv_count = hc.spmv;
        info->eta_inf = hc.eta;
        info->res_rel = hc.res;
        info->t_solve_s = secs;
        info->scale_exp_M = sM;
        info->scale_exp_N = sN;
        info->kernel = GADI_KERNEL_STENCIL;
        info->grid_blocks = blocks;
        info->block_threads = threads;
        info->zmarch_planes = 0;
    }
    return st;
}

// p is managed memory, or device memory of device dev (the kernels read and
// write b and x in place on the current device; memory of another GPU is
// refused rather than dereferenced across devices)
bool device_pointer(const void *p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" gadi_status gadi_solve_stencil_noalloc(int32_t dim, int32_t N, double beta, double alpha,
                                                  double omega, double eps_inner, int32_t max_inner,
                                                  int32_t max_outer, const double *b, double *x,
                                                  double tol, void *cuda_stream, gadi_info *info)
{
    if (dim != 2 && dim != 3) return GADI_ERR_INVALID_ARG;
    if (N < 1 || !std::isfinite(beta)) return GADI_ERR_INVALID_ARG;
    const int64_t n = dim == 3 ? (int64_t)N * N * N : (int64_t)N * N;
    if (n > kNoallocMaxN) return GADI_ERR_INVALID_ARG;
    if (!(alpha > 0.0) || !std::isfinite(alpha) || !(omega >= 0.0 && omega < 2.0))
        return GADI_ERR_INVALID_ARG;
    if (!(eps_inner > 0.0 && eps_inner < 1.0) || max_inner < 1 || max_outer < 0)
        return GADI_ERR_INVALID_ARG;
    if (!(tol > 0.0) || !std::isfinite(tol) || !b || !x) return GADI_ERR_INVALID_ARG;
    int dev = 0, num_sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return GADI_ERR_CUDA;
    }
    if (!device_pointer(b, dev) || !device_pointer(x, dev)) return GADI_ERR_INVALID_ARG;
    unsigned char *base = nullptr;
    if (scratch_address(dev, &base) != cudaSuccess) {
        cudaGetLastError();
        return GADI_ERR_CUDA;
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // ||b||_inf and finiteness of b and x0
    double *chk = (double *)(base + kCtlBytes + kPartBytes);
    int *bad = (int *)(chk + 2);
    double hk[3];
    if (cudaMemsetAsync(chk, 0, 3 * sizeof(double), stream) != cudaSuccess) return cuda_failure();
    const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
    k_noalloc_check<<<g, 256, 0, stream>>>(n, b, x, chk, bad);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(hk, chk, sizeof hk, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return cuda_failure();
    int nonfinite;
    std::memcpy(&nonfinite, &hk[2], sizeof(int));
    if (nonfinite) return GADI_ERR_INVALID_ARG;
    const double c = beta * (1.0 / (N + 1)) / 2.0;
    const bool v8 = N % 8 == 0;
    if (dim == 3)
        return v8 ? launch<3, 8>(dev, num_sms, stream, base, N, c, alpha, omega, eps_inner, max_inner,
                                 max_outer, b, x, tol, hk[0], info)
                  : launch<3, 1>(dev, num_sms, stream, base, N, c, alpha, omega, eps_inner, max_inner,
                                 max_outer, b, x, tol, hk[0], info);
    return v8 ? launch<2, 8>(dev, num_sms, stream, base, N, c, alpha, omega, eps_inner, max_inner,
                             max_outer, b, x, tol, hk[0], info)
              : launch<2, 1>(dev, num_sms, stream, base, N, c, alpha, omega, eps_inner, max_inner,
                             max_outer, b, x, tol, hk[0], info);
}
