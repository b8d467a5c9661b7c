// gadi_predict.cu -- parameter predictors for (alpha, omega) (§3.3).
//
// Features x = (log n, log beta), targets y = (log alpha*, omega*); both are
// standardised (zero mean, unit variance per column) before fitting.
//
// GPR (§3.3.1): one Gaussian process per target, squared-exponential kernel
// sf^2 exp(-|x - x'|^2 / (2 ell^2)) with sf = 1 on standardised targets and
// noise sn^2; (ell, sn) chosen on a grid by the log marginal likelihood;
// posterior mean k*^T (K + sn^2 I)^-1 y. FP32 arithmetic, as the paper fits
// its GPR in FP32; small dense systems, so it runs on the host.
//
// MLP 2 -> 64 -> 64 -> 2, tanh hidden layers, linear output, loss
// 1/(2m) sum (y - t)^2, Adam. Trained and evaluated on the GPU: BF16
// weights and activations into tensor-core MMAs (mma.sync m16n8k16, FP32
// accumulation) for the 64 x 64 layer in the forward and both backward
// products, FP32 elsewhere; FP32 master weights. Per-block gradient
// partials are summed in a fixed order (deterministic training). One
// training step (forward + backward kernel, reduction + Adam kernel) is
// captured once in a CUDA graph and replayed for every epoch. Weights start
// from SplitMix64 (Glorot uniform), the stream the oracle uses.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gadi.h"

namespace {

constexpr int kH = 64;                       // hidden width
constexpr int kIn = 2, kOut = 2;
// flat parameter layout: W1 [64][2], b1 [64], W2 [64][64], b2 [64], W3 [2][64], b3 [2]
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kOut * kH, kNP = ob3 + kOut;
constexpr int kWarps = 2;                    // warps per block, 16 samples each
constexpr int kSamplesPerBlock = 16 * kWarps;

// ---------------------------------------------------------------------------
// SplitMix64 (the published 64-bit generator) for the initial weights
// ---------------------------------------------------------------------------
uint64_t splitmix_next(uint64_t &s)
{
    s += 0x9E3779B97F4A7C15ULL;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void glorot_init(uint64_t seed, std::vector<double> &p)
{
    p.assign(kNP, 0.0);
    uint64_t s = seed;
    const int off[3] = {oW1, oW2, oW3}, fo[3] = {kH, kH, kOut}, fi[3] = {kIn, kH, kH};
    for (int l = 0; l < 3; ++l) {
        const double a = std::sqrt(6.0 / (fi[l] + fo[l]));
        for (int k = 0; k < fo[l] * fi[l]; ++k) {
            const double u = (double)(splitmix_next(s) >> 11) * 0x1.0p-53;
            p[off[l] + k] = (2.0 * u - 1.0) * a;
        }
    }
}

// ---------------------------------------------------------------------------
// MLP kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct MlpDev {
    float *master;       // kNP FP32 master weights
    float *m1, *m2;      // Adam moments
    float *gpart;        // [blocks][kNP] gradient partials
    float *lpart;        // [blocks] loss partials
    float *loss_hist;    // [epochs]
    int *step;           // Adam step counter (device)
};

// One block: 2 warps x 16 samples. Forward for every sample; with T != null
// also the backward pass, each warp writing its own gradient partial.
__global__ void __launch_bounds__(64) mlp_fwd_bwd(const float *__restrict__ X, const float *__restrict__ T,
                                                   int m, const float *__restrict__ wmaster,
                                                   float *__restrict__ Y, float *__restrict__ gpart,
                                                   float *__restrict__ lpart)
{
    __shared__ float sW1[kH * kIn], sb1[kH], sb2[kH], sW3[kOut * kH], sb3[kOut];
    __shared__ __nv_bfloat16 sW2[kH * kH];      // W2[n][k] (row-major)
    __shared__ __nv_bfloat16 sW2t[kH * kH];     // W2^T[k][n]
    __shared__ float sH1[kWarps][16][kH], sH2[kWarps][16][kH], sD[kWarps][16][kH];
    __shared__ float sX[kWarps][16][kIn], sDY[kWarps][16][kOut];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const bool train = T != nullptr;
    // weights: BF16-rounded copies of the FP32 master
    for (int k = tid; k < kH * kIn; k += blockDim.x) sW1[k] = __bfloat162float(__float2bfloat16_rn(wmaster[oW1 + k]));
    for (int k = tid; k < kOut * kH; k += blockDim.x) sW3[k] = __bfloat162float(__float2bfloat16_rn(wmaster[oW3 + k]));
    for (int k = tid; k < kH * kH; k += blockDim.x) {
        const __nv_bfloat16 v = __float2bfloat16_rn(wmaster[oW2 + k]);
        sW2[k] = v;
        sW2t[(k % kH) * kH + k / kH] = v;
    }
    for (int k = tid; k < kH; k += blockDim.x) {
        sb1[k] = wmaster[ob1 + k];
        sb2[k] = wmaster[ob2 + k];
    }
    if (tid < kOut) sb3[tid] = wmaster[ob3 + tid];
    const int s0 = blockIdx.x * kSamplesPerBlock + warp * 16;
    for (int k = lane; k < 16 * kIn; k += 32) {
        const int s = s0 + k / kIn;
        sX[warp][k / kIn][k % kIn] = s < m ? X[(size_t)s * kIn + k % kIn] : 0.f;
    }
    __syncthreads();

    // layer 1 (FP32 SIMT): H1 = tanh(W1 x + b1)
    for (int k = lane; k < 16 * kH; k += 32) {
        const int s = k / kH, j = k % kH;
        float z = sb1[j];
#pragma unroll
        for (int i = 0; i < kIn; ++i) z = fmaf(sW1[j * kIn + i], sX[warp][s][i], z);
        sH1[warp][s][j] = tanhf(z);
    }
    __syncwarp();
    // layer 2 on tensor cores: Z2 = H1 W2^T (16 x 64 x 64), H2 = tanh(Z2 + b2)
    for (int nt = 0; nt < kH / 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < kH / 16; ++kt) {
            const int k0 = kt * 16 + 2 * tig;
            uint32_t a[4], b[2];
            a[0] = pack_bf16(sH1[warp][gid][k0], sH1[warp][gid][k0 + 1]);
            a[1] = pack_bf16(sH1[warp][gid + 8][k0], sH1[warp][gid + 8][k0 + 1]);
            a[2] = pack_bf16(sH1[warp][gid][k0 + 8], sH1[warp][gid][k0 + 9]);
            a[3] = pack_bf16(sH1[warp][gid + 8][k0 + 8], sH1[warp][gid + 8][k0 + 9]);
            const int n = nt * 8 + gid;   // B[k][n] = W2[n][k]
            b[0] = *reinterpret_cast<const uint32_t *>(&sW2[n * kH + k0]);
            b[1] = *reinterpret_cast<const uint32_t *>(&sW2[n * kH + k0 + 8]);
            mma_bf16(c, a, b);
        }
        const int n0 = nt * 8 + 2 * tig;
        sH2[warp][gid][n0] = tanhf(c[0] + sb2[n0]);
        sH2[warp][gid][n0 + 1] = tanhf(c[1] + sb2[n0 + 1]);
        sH2[warp][gid + 8][n0] = tanhf(c[2] + sb2[n0]);
        sH2[warp][gid + 8][n0 + 1] = tanhf(c[3] + sb2[n0 + 1]);
    }
    __syncwarp();
    // layer 3 (FP32 SIMT): Y = W3 H2 + b3; one (sample, output) per lane
    {
        const int s = lane >> 1, o = lane & 1;
        float y = sb3[o];
        for (int j = 0; j < kH; ++j) y = fmaf(sW3[o * kH + j], sH2[warp][s][j], y);
        const int gs = s0 + s;
        if (!train) {
            if (gs < m) Y[(size_t)gs * kOut + o] = y;
        } else {
            const float t = gs < m ? T[(size_t)gs * kOut + o] : y;
            const float dy = gs < m ? (y - t) / (float)m : 0.f;
            sDY[warp][s][o] = dy;
            float l = gs < m ? 0.5f * (y - t) * (y - t) / (float)m : 0.f;
            for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
            if (lane == 0) lpart[blockIdx.x * kWarps + warp] = l;
        }
    }
    if (!train) return;
    __syncwarp();
    float *g = gpart + ((size_t)blockIdx.x * kWarps + warp) * kNP;
    // dW3 = dY^T H2, db3 = sum dY; dZ2 = (dY W3) (1 - H2^2)
    for (int k = lane; k < kOut * kH; k += 32) {
        const int o = k / kH, j = k % kH;
        float a = 0.f;
        for (int s = 0; s < 16; ++s) a = fmaf(sDY[warp][s][o], sH2[warp][s][j], a);
        g[oW3 + k] = a;
    }
    if (lane < kOut) {
        float a = 0.f;
        for (int s = 0; s < 16; ++s) a += sDY[warp][s][lane];
        g[ob3 + lane] = a;
    }
    for (int k = lane; k < 16 * kH; k += 32) {
        const int s = k / kH, j = k % kH;
        float d = 0.f;
#pragma unroll
        for (int o = 0; o < kOut; ++o) d = fmaf(sDY[warp][s][o], sW3[o * kH + j], d);
        const float h = sH2[warp][s][j];
        sD[warp][s][j] = d * (1.f - h * h);
    }
    __syncwarp();
    // db2 = sum dZ2; dW2 = dZ2^T H1 on tensor cores (64 x 16 x 64)
    for (int j = lane; j < kH; j += 32) {
        float a = 0.f;
        for (int s = 0; s < 16; ++s) a += sD[warp][s][j];
        g[ob2 + j] = a;
    }
    for (int mt = 0; mt < kH / 16; ++mt) {
        uint32_t a[4];
        const int r = mt * 16 + gid, k0 = 2 * tig;   // A[r][s] = dZ2[s][r]
        a[0] = pack_bf16(sD[warp][k0][r], sD[warp][k0 + 1][r]);
        a[1] = pack_bf16(sD[warp][k0][r + 8], sD[warp][k0 + 1][r + 8]);
        a[2] = pack_bf16(sD[warp][k0 + 8][r], sD[warp][k0 + 9][r]);
        a[3] = pack_bf16(sD[warp][k0 + 8][r + 8], sD[warp][k0 + 9][r + 8]);
        for (int nt = 0; nt < kH / 8; ++nt) {
            uint32_t b[2];
            const int n = nt * 8 + gid;               // B[s][n] = H1[s][n]
            b[0] = pack_bf16(sH1[warp][k0][n], sH1[warp][k0 + 1][n]);
            b[1] = pack_bf16(sH1[warp][k0 + 8][n], sH1[warp][k0 + 9][n]);
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma_bf16(c, a, b);
            const int col = nt * 8 + 2 * tig;
            g[oW2 + r * kH + col] = c[0];
            g[oW2 + r * kH + col + 1] = c[1];
            g[oW2 + (r + 8) * kH + col] = c[2];
            g[oW2 + (r + 8) * kH + col + 1] = c[3];
        }
    }
    // dH1 = dZ2 W2 on tensor cores (16 x 64 x 64); dZ1 = dH1 (1 - H1^2)
    for (int nt = 0; nt < kH / 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < kH / 16; ++kt) {
            const int k0 = kt * 16 + 2 * tig;
            uint32_t a[4], b[2];
            a[0] = pack_bf16(sD[warp][gid][k0], sD[warp][gid][k0 + 1]);
            a[1] = pack_bf16(sD[warp][gid + 8][k0], sD[warp][gid + 8][k0 + 1]);
            a[2] = pack_bf16(sD[warp][gid][k0 + 8], sD[warp][gid][k0 + 9]);
            a[3] = pack_bf16(sD[warp][gid + 8][k0 + 8], sD[warp][gid + 8][k0 + 9]);
            const int n = nt * 8 + gid;   // B[k][n] = W2[k][n] = W2^T[n][k]
            b[0] = *reinterpret_cast<const uint32_t *>(&sW2t[n * kH + k0]);
            b[1] = *reinterpret_cast<const uint32_t *>(&sW2t[n * kH + k0 + 8]);
            mma_bf16(c, a, b);
        }
        const int n0 = nt * 8 + 2 * tig;
        // write dZ1 into sH2's space (H2 is no longer needed)
        const float h00 = sH1[warp][gid][n0], h01 = sH1[warp][gid][n0 + 1];
        const float h10 = sH1[warp][gid + 8][n0], h11 = sH1[warp][gid + 8][n0 + 1];
        sH2[warp][gid][n0] = c[0] * (1.f - h00 * h00);
        sH2[warp][gid][n0 + 1] = c[1] * (1.f - h01 * h01);
        sH2[warp][gid + 8][n0] = c[2] * (1.f - h10 * h10);
        sH2[warp][gid + 8][n0 + 1] = c[3] * (1.f - h11 * h11);
    }
    __syncwarp();
    // dW1 = dZ1^T X, db1 = sum dZ1
    for (int k = lane; k < kH * kIn; k += 32) {
        const int j = k / kIn, i = k % kIn;
        float a = 0.f;
        for (int s = 0; s < 16; ++s) a = fmaf(sH2[warp][s][j], sX[warp][s][i], a);
        g[oW1 + k] = a;
    }
    for (int j = lane; j < kH; j += 32) {
        float a = 0.f;
        for (int s = 0; s < 16; ++s) a += sH2[warp][s][j];
        g[ob1 + j] = a;
    }
}

// Sum the warp partials in order; Adam on the FP32 master weights (or just
// the summed gradient when grad_out is given). One block, so the step
// counter is read by all threads before thread 0 advances it.
__global__ void __launch_bounds__(1024) mlp_reduce_adam(MlpDev d, int nparts, float lr, float *grad_out)
{
    const int t = *d.step + 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (int k = threadIdx.x; k < kNP; k += blockDim.x) {
        float gk = 0.f;
        for (int b = 0; b < nparts; ++b) gk += d.gpart[(size_t)b * kNP + k];
        if (grad_out) {
            grad_out[k] = gk;
            continue;
        }
        const float m1 = b1 * d.m1[k] + (1.f - b1) * gk;
        const float m2 = b2 * d.m2[k] + (1.f - b2) * gk * gk;
        d.m1[k] = m1;
        d.m2[k] = m2;
        d.master[k] -= lr * (m1 / c1) / (sqrtf(m2 / c2) + eps);
    }
    __syncthreads();
    if (threadIdx.x == 0 && !grad_out) {
        float l = 0.f;
        for (int b = 0; b < nparts; ++b) l += d.lpart[b];
        d.loss_hist[t - 1] = l;
        *d.step = t;
    }
}

// ---------------------------------------------------------------------------
// GPR in FP32 (host)
// ---------------------------------------------------------------------------
struct GprCol {
    float ell, sn;
    std::vector<float> alpha;
};

bool cholesky(std::vector<float> &K, int m)
{
    for (int j = 0; j < m; ++j) {
        float d = K[j * m + j];
        for (int k = 0; k < j; ++k) d -= K[j * m + k] * K[j * m + k];
        if (!(d > 0.f)) return false;
        d = std::sqrt(d);
        K[j * m + j] = d;
        for (int i = j + 1; i < m; ++i) {
            float v = K[i * m + j];
            for (int k = 0; k < j; ++k) v -= K[i * m + k] * K[j * m + k];
            K[i * m + j] = v / d;
        }
    }
    return true;
}

void chol_solve(const std::vector<float> &L, int m, std::vector<float> &v)
{
    for (int i = 0; i < m; ++i) {
        float s = v[i];
        for (int k = 0; k < i; ++k) s -= L[i * m + k] * v[k];
        v[i] = s / L[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        float s = v[i];
        for (int k = i + 1; k < m; ++k) s -= L[k * m + i] * v[k];
        v[i] = s / L[i * m + i];
    }
}

float se(const float *a, const float *b, float ell)
{
    float d2 = 0.f;
    for (int i = 0; i < kIn; ++i) d2 += (a[i] - b[i]) * (a[i] - b[i]);
    return std::exp(-d2 / (2.f * ell * ell));
}

}  // namespace

struct gadi_model {
    int kind;
    double xmu[kIn], xsd[kIn], ymu[kOut], ysd[kOut];
    // GPR
    std::vector<float> X;        // standardised training inputs
    GprCol cols[kOut];
    // MLP
    float *dmaster = nullptr;    // device FP32 master weights
    std::vector<double> loss;    // training loss per epoch
};

namespace {

void standardize(const double *A, int m, int c, double *mu, double *sd)
{
    for (int j = 0; j < c; ++j) {
        double s = 0.0, q = 0.0;
        for (int i = 0; i < m; ++i) s += A[i * c + j];
        mu[j] = s / m;
        for (int i = 0; i < m; ++i) q += (A[i * c + j] - mu[j]) * (A[i * c + j] - mu[j]);
        sd[j] = std::sqrt(q / m);
        if (!(sd[j] > 0.0)) sd[j] = 1.0;
    }
}

gadi_status gpr_fit(gadi_model *M, const double *X, const double *Y, int m, const double *hyper, int nhyper)
{
    const float ells_def[] = {0.25f, 0.5f, 1.0f, 2.0f, 4.0f}, noises_def[] = {1e-3f, 1e-2f, 1e-1f};
    std::vector<float> ells(ells_def, ells_def + 5), noises(noises_def, noises_def + 3);
    if (hyper && nhyper >= 2) {
        ells.assign(1, (float)hyper[0]);
        noises.assign(1, (float)hyper[1]);
    }
    M->X.resize((size_t)m * kIn);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < kIn; ++j) M->X[i * kIn + j] = (float)((X[i * kIn + j] - M->xmu[j]) / M->xsd[j]);
    for (int c = 0; c < kOut; ++c) {
        std::vector<float> y(m);
        for (int i = 0; i < m; ++i) y[i] = (float)((Y[i * kOut + c] - M->ymu[c]) / M->ysd[c]);
        float best = -INFINITY;
        bool found = false;
        for (float ell : ells)
            for (float sn : noises) {
                std::vector<float> K((size_t)m * m);
                for (int i = 0; i < m; ++i)
                    for (int j = 0; j < m; ++j)
                        K[i * m + j] = se(&M->X[i * kIn], &M->X[j * kIn], ell) + (i == j ? sn * sn : 0.f);
                if (!cholesky(K, m)) continue;
                std::vector<float> a = y;
                chol_solve(K, m, a);
                float logdet = 0.f, yta = 0.f;
                for (int i = 0; i < m; ++i) {
                    logdet += 2.f * std::log(K[i * m + i]);
                    yta += y[i] * a[i];
                }
                const float lml = -0.5f * yta - 0.5f * logdet - 0.5f * m * std::log(2.f * 3.14159265f);
                if (!found || lml > best) {
                    best = lml;
                    found = true;
                    M->cols[c].ell = ell;
                    M->cols[c].sn = sn;
                    M->cols[c].alpha = a;
                }
            }
        if (!found) return GADI_ERR_RANGE;
    }
    return GADI_OK;
}

gadi_status run_mlp(gadi_model *M, const double *X, const double *Y, int m, int epochs, float lr,
                    uint64_t seed, cudaStream_t stream, const double *init_params, double *grad_out)
{
    const int nb = (m + kSamplesPerBlock - 1) / kSamplesPerBlock;
    std::vector<float> hx((size_t)m * kIn), hy((size_t)m * kOut);
    for (int i = 0; i < m; ++i) {
        for (int j = 0; j < kIn; ++j) hx[i * kIn + j] = (float)((X[i * kIn + j] - M->xmu[j]) / M->xsd[j]);
        for (int j = 0; j < kOut; ++j) hy[i * kOut + j] = (float)((Y[i * kOut + j] - M->ymu[j]) / M->ysd[j]);
    }
    std::vector<double> p0;
    if (init_params) p0.assign(init_params, init_params + kNP);
    else glorot_init(seed, p0);
    std::vector<float> p0f(p0.begin(), p0.end());
    float *dX = nullptr, *dY = nullptr, *buf = nullptr, *dgrad = nullptr;
    int *dstep = nullptr;
    auto cleanup = [&]() {
        if (dX) cudaFree(dX);
        if (dY) cudaFree(dY);
        if (buf) cudaFree(buf);
        if (dgrad) cudaFree(dgrad);
        if (dstep) cudaFree(dstep);
    };
    const int nparts = nb * kWarps;
    const size_t nbuf = 2 * kNP + (size_t)nparts * kNP + nparts + (size_t)std::max(epochs, 1);
    if (cudaMalloc(&dX, hx.size() * sizeof(float)) || cudaMalloc(&dY, hy.size() * sizeof(float)) ||
        cudaMalloc(&buf, nbuf * sizeof(float)) || cudaMalloc(&dstep, sizeof(int)) ||
        (!M->dmaster && cudaMalloc(&M->dmaster, kNP * sizeof(float))) ||
        (grad_out && cudaMalloc(&dgrad, kNP * sizeof(float)))) {
        cudaGetLastError();
        cleanup();
        return GADI_ERR_OUT_OF_MEMORY;
    }
    MlpDev d;
    d.master = M->dmaster;
    d.m1 = buf;
    d.m2 = buf + kNP;
    d.gpart = buf + 2 * kNP;
    d.lpart = d.gpart + (size_t)nparts * kNP;
    d.loss_hist = d.lpart + nparts;
    d.step = dstep;
    cudaError_t e = cudaMemcpyAsync(dX, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dY, hy.data(), hy.size() * sizeof(float), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.master, p0f.data(), kNP * sizeof(float), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, 2 * kNP * sizeof(float), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(dstep, 0, sizeof(int), stream);
    if (e != cudaSuccess) { cleanup(); return GADI_ERR_CUDA; }
    if (grad_out) {
        mlp_fwd_bwd<<<nb, 32 * kWarps, 0, stream>>>(dX, dY, m, d.master, nullptr, d.gpart, d.lpart);
        mlp_reduce_adam<<<1, 1024, 0, stream>>>(d, nparts, 0.f, dgrad);
        std::vector<float> g(kNP);
        e = cudaMemcpyAsync(g.data(), dgrad, kNP * sizeof(float), cudaMemcpyDeviceToHost, stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        cleanup();
        if (e != cudaSuccess) return GADI_ERR_CUDA;
        for (int k = 0; k < kNP; ++k) grad_out[k] = g[k];
        return GADI_OK;
    }
    // one training step captured as a graph, replayed for every epoch
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) { cleanup(); return GADI_ERR_CUDA; }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        mlp_fwd_bwd<<<nb, 32 * kWarps, 0, cap>>>(dX, dY, m, d.master, nullptr, d.gpart, d.lpart);
        mlp_reduce_adam<<<1, 1024, 0, cap>>>(d, nparts, lr, nullptr);
        e = cudaStreamEndCapture(cap, &graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) e = cudaGraphLaunch(exec, stream);
    std::vector<float> hl(std::max(epochs, 1));
    if (e == cudaSuccess && epochs > 0)
        e = cudaMemcpyAsync(hl.data(), d.loss_hist, epochs * sizeof(float), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    cleanup();
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GADI_ERR_CUDA;
    }
    M->loss.assign(hl.begin(), hl.begin() + epochs);
    return GADI_OK;
}

}  // namespace

extern "C" {

gadi_status gadi_model_fit(int32_t kind, const double *X, const double *Y, int32_t m, const double *hyper,
                           int32_t nhyper, void *cuda_stream, gadi_model **out)
{
    if (!out || !X || !Y || m < 1 || (kind != GADI_MODEL_MLP && kind != GADI_MODEL_GPR) || nhyper < 0)
        return GADI_ERR_INVALID_ARG;
    if (kind == GADI_MODEL_GPR && m > 4096) return GADI_ERR_INVALID_ARG;
    for (int i = 0; i < m * kIn; ++i)
        if (!std::isfinite(X[i])) return GADI_ERR_INVALID_ARG;
    for (int i = 0; i < m * kOut; ++i)
        if (!std::isfinite(Y[i])) return GADI_ERR_INVALID_ARG;
    *out = nullptr;
    gadi_model *M = new (std::nothrow) gadi_model();
    if (!M) return GADI_ERR_OUT_OF_MEMORY;
    M->kind = kind;
    standardize(X, m, kIn, M->xmu, M->xsd);
    standardize(Y, m, kOut, M->ymu, M->ysd);
    gadi_status st;
    if (kind == GADI_MODEL_GPR) {
        st = gpr_fit(M, X, Y, m, hyper, nhyper);
    } else {
        const int epochs = hyper && nhyper >= 1 ? (int)hyper[0] : 3000;
        const float lr = hyper && nhyper >= 2 ? (float)hyper[1] : 1e-2f;
        const uint64_t seed = hyper && nhyper >= 3 ? (uint64_t)hyper[2] : 1;
        if (epochs < 0 || epochs > 1000000 || !(lr > 0.f)) st = GADI_ERR_INVALID_ARG;
        else st = run_mlp(M, X, Y, m, epochs, lr, seed, (cudaStream_t)cuda_stream, nullptr, nullptr);
    }
    if (st != GADI_OK) {
        gadi_model_destroy(M);
        return st;
    }
    *out = M;
    return GADI_OK;
}

gadi_status gadi_model_predict(const gadi_model *M, const double *X, int32_t count, double *Y)
{
    if (!M || !X || !Y || count < 1) return GADI_ERR_INVALID_ARG;
    std::vector<float> xs((size_t)count * kIn);
    for (int i = 0; i < count; ++i)
        for (int j = 0; j < kIn; ++j) {
            if (!std::isfinite(X[i * kIn + j])) return GADI_ERR_INVALID_ARG;
            xs[i * kIn + j] = (float)((X[i * kIn + j] - M->xmu[j]) / M->xsd[j]);
        }
    std::vector<float> ys((size_t)count * kOut);
    if (M->kind == GADI_MODEL_GPR) {
        const int m = (int)(M->X.size() / kIn);
        for (int i = 0; i < count; ++i)
            for (int c = 0; c < kOut; ++c) {
                float s = 0.f;
                for (int k = 0; k < m; ++k) s += se(&xs[i * kIn], &M->X[k * kIn], M->cols[c].ell) * M->cols[c].alpha[k];
                ys[i * kOut + c] = s;
            }
    } else {
        float *dx = nullptr, *dy = nullptr;
        if (cudaMalloc(&dx, xs.size() * sizeof(float)) || cudaMalloc(&dy, ys.size() * sizeof(float))) {
            cudaGetLastError();
            if (dx) cudaFree(dx);
            return GADI_ERR_OUT_OF_MEMORY;
        }
        cudaError_t e = cudaMemcpy(dx, xs.data(), xs.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            mlp_fwd_bwd<<<(count + kSamplesPerBlock - 1) / kSamplesPerBlock, 32 * kWarps>>>(
                dx, nullptr, count, M->dmaster, dy, nullptr, nullptr);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(ys.data(), dy, ys.size() * sizeof(float), cudaMemcpyDeviceToHost);
        cudaFree(dx);
        cudaFree(dy);
        if (e != cudaSuccess) return GADI_ERR_CUDA;
    }
    for (int i = 0; i < count; ++i)
        for (int c = 0; c < kOut; ++c) Y[i * kOut + c] = ys[i * kOut + c] * M->ysd[c] + M->ymu[c];
    return GADI_OK;
}

gadi_status gadi_model_loss(const gadi_model *M, double *loss, int32_t cap, int32_t *count)
{
    if (!M || !count || cap < 0 || (cap > 0 && !loss)) return GADI_ERR_INVALID_ARG;
    *count = (int32_t)M->loss.size();
    for (int i = 0; i < cap && i < *count; ++i) loss[i] = M->loss[i];
    return GADI_OK;
}

gadi_status gadi_mlp_gradient(const double *params, const double *X, const double *T, int32_t m,
                              void *cuda_stream, double *grad)
{
    if (!params || !X || !T || !grad || m < 1) return GADI_ERR_INVALID_ARG;
    gadi_model M;
    M.kind = GADI_MODEL_MLP;
    for (int j = 0; j < kIn; ++j) { M.xmu[j] = 0.0; M.xsd[j] = 1.0; }
    for (int j = 0; j < kOut; ++j) { M.ymu[j] = 0.0; M.ysd[j] = 1.0; }
    gadi_status st = run_mlp(&M, X, T, m, 0, 0.f, 0, (cudaStream_t)cuda_stream, params, grad);
    if (M.dmaster) cudaFree(M.dmaster);
    return st;
}

int32_t gadi_mlp_param_count(void)
{
    return kNP;
}

void gadi_model_destroy(gadi_model *M)
{
    if (!M) return;
    if (M->dmaster) cudaFree(M->dmaster);
    delete M;
}

}  // extern "C"
