// gadi_device.cuh -- device primitives of the persistent GADI-IR solve kernel:
// precision traits, a bounded software grid barrier and deterministic
// all-block reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "gadi_bits.cuh"
#include <stdint.h>

namespace gadi {

// status codes shared with gadi.h
enum : int {
    kOk = 0, kErrInvalid = 1, kErrOom = 2, kErrCuda = 3, kErrRange = 4,
    kErrNotConverged = 5, kErrDiverged = 6, kErrTimeout = 7
};

__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// Precision traits. T is the storage type of the inner vectors and matrix
// values; Acc the arithmetic type (FP32 for FP16 storage, FP64 otherwise).
// Every rounding step is the one written in the source: a sum of products
// takes one fused multiply-add per term (madd) in FP32 and in FP64, which
// halves the instructions (and on this GPU's low FP64 rate matters most
// there); a lone product or sum is rounded on its own.
// ---------------------------------------------------------------------------
template <class T> struct Prec;

// Two FP32 values in one 64-bit register pair, operated on by the packed
// FP32 instructions (mul.rn.f32x2 / fma.rn.f32x2): each lane is an IEEE
// round-to-nearest-even operation, the same result as the scalar
// __fmul_rn / __fmaf_rn, at half the instruction count. (A packed multiply
// followed by a packed add is contracted into a fused multiply-add by the
// assembler even with .rn, so sums of products are written as fma here and
// everywhere in the FP32 arithmetic of the FP16 path.)
__device__ __forceinline__ unsigned long long f2_pack(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void f2_unpack(unsigned long long v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// a b + c per lane
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

template <> struct Prec<__half> {
    using Acc = float;
    static __device__ __forceinline__ float ld(__half v) { return __half2float(v); }
    static __device__ __forceinline__ __half st(float v) { return __float2half_rn(v); }
    // round an Acc value through the storage type
    static __device__ __forceinline__ float rnd(float v) { return __half2float(__float2half_rn(v)); }
    static __device__ __forceinline__ __half from64(double v) { return __double2half(v); }
    // the exact FP64 value of an FP32 value, by integer operations
    static __device__ __forceinline__ double to64(float v) { return double_of_float(v); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    // c + a b, one fused multiply-add (one rounding)
    static __device__ __forceinline__ float madd(float c, float a, float b) { return __fmaf_rn(a, b, c); }
    // element-wise, two lanes per packed instruction (outputs may alias inputs):
    // o = c + a b with a scalar; o = c + a b; o = a b with a scalar
    template <int K>
    static __device__ __forceinline__ void madd_s(float (&o)[K], const float (&c)[K], float a, const float (&b)[K])
    {
        if constexpr (K % 2 == 0) {
            const unsigned long long aa = f2_pack(a, a);
#pragma unroll
            for (int k = 0; k < K; k += 2)
                f2_unpack(f2_fma(aa, f2_pack(b[k], b[k + 1]), f2_pack(c[k], c[k + 1])), o[k], o[k + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) o[k] = madd(c[k], a, b[k]);
        }
    }
    template <int K>
    static __device__ __forceinline__ void madd_v(float (&o)[K], const float (&c)[K], const float (&a)[K],
                                                  const float (&b)[K])
    {
        if constexpr (K % 2 == 0) {
#pragma unroll
            for (int k = 0; k < K; k += 2)
                f2_unpack(f2_fma(f2_pack(a[k], a[k + 1]), f2_pack(b[k], b[k + 1]), f2_pack(c[k], c[k + 1])),
                          o[k], o[k + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) o[k] = madd(c[k], a[k], b[k]);
        }
    }
    template <int K>
    static __device__ __forceinline__ void mul_s(float (&o)[K], float a, const float (&b)[K])
    {
        if constexpr (K % 2 == 0) {
            const unsigned long long aa = f2_pack(a, a);
#pragma unroll
            for (int k = 0; k < K; k += 2) f2_unpack(f2_mul(aa, f2_pack(b[k], b[k + 1])), o[k], o[k + 1]);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) o[k] = mul(a, b[k]);
        }
    }
    // round an even number of values through FP16, two per conversion
    template <int K>
    static __device__ __forceinline__ void rndv(float (&v)[K])
    {
        if constexpr (K % 2 == 0) {
#pragma unroll
            for (int k = 0; k < K; k += 2) {
                const float2 f = __half22float2(__float22half2_rn(make_float2(v[k], v[k + 1])));
                v[k] = f.x;
                v[k + 1] = f.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = rnd(v[k]);
        }
    }
};

// FP32 storage and arithmetic (u_r = single): no rounding between steps
template <> struct Prec<float> {
    using Acc = float;
    static __device__ __forceinline__ float ld(float v) { return v; }
    static __device__ __forceinline__ float st(float v) { return v; }
    static __device__ __forceinline__ float rnd(float v) { return v; }
    static __device__ __forceinline__ float from64(double v) { return __double2float_rn(v); }
    static __device__ __forceinline__ double to64(float v) { return double_of_float(v); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float madd(float c, float a, float b) { return __fmaf_rn(a, b, c); }
    template <int K>
    static __device__ __forceinline__ void madd_s(float (&o)[K], const float (&c)[K], float a, const float (&b)[K])
    {
        Prec<__half>::madd_s(o, c, a, b);
    }
    template <int K>
    static __device__ __forceinline__ void madd_v(float (&o)[K], const float (&c)[K], const float (&a)[K],
                                                  const float (&b)[K])
    {
        Prec<__half>::madd_v(o, c, a, b);
    }
    template <int K>
    static __device__ __forceinline__ void mul_s(float (&o)[K], float a, const float (&b)[K])
    {
        Prec<__half>::mul_s(o, a, b);
    }
    template <int K>
    static __device__ __forceinline__ void rndv(float (&)[K]) {}
};

// BF16 storage with FP32 arithmetic (a precision variant of u_r)
template <> struct Prec<__nv_bfloat16> {
    using Acc = float;
    static __device__ __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float rnd(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    static __device__ __forceinline__ __nv_bfloat16 from64(double v) { return __double2bfloat16(v); }
    static __device__ __forceinline__ double to64(float v) { return double_of_float(v); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float madd(float c, float a, float b) { return __fmaf_rn(a, b, c); }
    template <int K>
    static __device__ __forceinline__ void madd_s(float (&o)[K], const float (&c)[K], float a, const float (&b)[K])
    {
        Prec<__half>::madd_s(o, c, a, b);
    }
    template <int K>
    static __device__ __forceinline__ void madd_v(float (&o)[K], const float (&c)[K], const float (&a)[K],
                                                  const float (&b)[K])
    {
        Prec<__half>::madd_v(o, c, a, b);
    }
    template <int K>
    static __device__ __forceinline__ void mul_s(float (&o)[K], float a, const float (&b)[K])
    {
        Prec<__half>::mul_s(o, a, b);
    }
    template <int K>
    static __device__ __forceinline__ void rndv(float (&v)[K])
    {
        if constexpr (K % 2 == 0) {
#pragma unroll
            for (int k = 0; k < K; k += 2) {
                const float2 f = __bfloat1622float2(__float22bfloat162_rn(make_float2(v[k], v[k + 1])));
                v[k] = f.x;
                v[k + 1] = f.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = rnd(v[k]);
        }
    }
};

// FP8 E4M3 storage with FP32 arithmetic (a precision variant of u_r below
// the paper's FP16): 3 fraction bits, exponent bias 7, largest finite value
// 448, subnormals down to 2^-9. Stores round to nearest even and saturate
// at +-448 (the format has no infinity).
template <> struct Prec<__nv_fp8_e4m3> {
    using Acc = float;
    static __device__ __forceinline__ float ld(__nv_fp8_e4m3 v)
    {
        return __half2float(__half(__nv_cvt_fp8_to_halfraw(v.__x, __NV_E4M3)));
    }
    static __device__ __forceinline__ __nv_fp8_e4m3 st(float v)
    {
        __nv_fp8_e4m3 o;
        o.__x = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        return o;
    }
    static __device__ __forceinline__ float rnd(float v) { return ld(st(v)); }
    // one rounding from FP64: round to odd at FP32 first (24 >= 4 + 2 bits)
    static __device__ __forceinline__ __nv_fp8_e4m3 from64(double v)
    {
        return st(__uint_as_float(float_bits_round_odd(v)));
    }
    static __device__ __forceinline__ double to64(float v) { return double_of_float(v); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float madd(float c, float a, float b) { return __fmaf_rn(a, b, c); }
    template <int K>
    static __device__ __forceinline__ void madd_s(float (&o)[K], const float (&c)[K], float a, const float (&b)[K])
    {
        Prec<__half>::madd_s(o, c, a, b);
    }
    template <int K>
    static __device__ __forceinline__ void madd_v(float (&o)[K], const float (&c)[K], const float (&a)[K],
                                                  const float (&b)[K])
    {
        Prec<__half>::madd_v(o, c, a, b);
    }
    template <int K>
    static __device__ __forceinline__ void mul_s(float (&o)[K], float a, const float (&b)[K])
    {
        Prec<__half>::mul_s(o, a, b);
    }
    // two values per conversion each way (FP8 pairs widen exactly to FP16)
    template <int K>
    static __device__ __forceinline__ void rndv(float (&v)[K])
    {
        if constexpr (K % 2 == 0) {
#pragma unroll
            for (int k = 0; k < K; k += 2) {
                const __nv_fp8x2_storage_t q =
                    __nv_cvt_float2_to_fp8x2(make_float2(v[k], v[k + 1]), __NV_SATFINITE, __NV_E4M3);
                const float2 f = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(q, __NV_E4M3)));
                v[k] = f.x;
                v[k + 1] = f.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = rnd(v[k]);
        }
    }
};

// storage types whose demotion of r (Alg. 1 step 2) starts from the
// round-to-odd FP32 copy of r: FP16 and FP8 (24 >= 11 + 2 and 24 >= 4 + 2)
template <class T>
constexpr bool kDemoteFromOdd = std::is_same<T, __half>::value || std::is_same<T, __nv_fp8_e4m3>::value;

template <> struct Prec<double> {
    using Acc = double;
    static __device__ __forceinline__ double ld(double v) { return v; }
    static __device__ __forceinline__ double st(double v) { return v; }
    static __device__ __forceinline__ double rnd(double v) { return v; }
    static __device__ __forceinline__ double from64(double v) { return v; }
    static __device__ __forceinline__ double to64(double v) { return v; }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double madd(double c, double a, double b) { return __fma_rn(a, b, c); }
    template <int K>
    static __device__ __forceinline__ void madd_s(double (&o)[K], const double (&c)[K], double a, const double (&b)[K])
    {
#pragma unroll
        for (int k = 0; k < K; ++k) o[k] = madd(c[k], a, b[k]);
    }
    template <int K>
    static __device__ __forceinline__ void madd_v(double (&o)[K], const double (&c)[K], const double (&a)[K],
                                                  const double (&b)[K])
    {
#pragma unroll
        for (int k = 0; k < K; ++k) o[k] = madd(c[k], a[k], b[k]);
    }
    template <int K>
    static __device__ __forceinline__ void mul_s(double (&o)[K], double a, const double (&b)[K])
    {
#pragma unroll
        for (int k = 0; k < K; ++k) o[k] = mul(a, b[k]);
    }
    template <int K>
    static __device__ __forceinline__ void rndv(double (&)[K]) {}
};


// ---------------------------------------------------------------------------
// Timers and ordered memory accesses (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_volatile_i32(const int *p)
{
    return *(const volatile int *)p;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Control block of one solve (device memory, zeroed before each launch).
struct Ctl {
    unsigned long long arrive;   // grid-barrier arrival counter (monotone within a launch)
    int error;                   // first error code raised on the device (0 = none)
    int status;                  // final gadi_status of the solve
    int outer_iters;
    int pad0;
    long long itH, itS, spmv;
    double eta, res, r0;
    int sM, sN;
};

// ---------------------------------------------------------------------------
// Reductions. Values are float (FP16 inner path) or double (FP64 residual
// phase, FP64 inner path); every order of operations is fixed, so results
// are deterministic and identical in every block.
// Block level: float goes through a shuffle tree in every warp, then one
// warp combines the warp results; double goes through shared memory and one
// warp with four accumulators per lane (few FP64 instructions, which matters
// on a GPU with a low FP64 rate).
// ---------------------------------------------------------------------------
constexpr int kMaxSlots = 3;
constexpr int kMaxThreads = 1024;
constexpr int kWordsPerSlot = 2;                 // a double needs two 32-bit payloads
constexpr int kMaxWords = kMaxSlots * kWordsPerSlot;
enum RedOp { kSum = 0, kMax = 1 };

template <class V>
__device__ __forceinline__ V red_op(V a, V b, int o)
{
    return o == kMax ? (a > b ? a : b) : a + b;   // maxima are over |values| >= 0
}

__device__ __forceinline__ double *red_scratch()
{
    __shared__ double sh[kMaxSlots * kMaxThreads + 2 * kMaxSlots + 2];
    return sh;
}

template <class V, int NS>
__device__ __forceinline__ void warp_tree(V (&v)[NS], const int (&ops)[NS])
{
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[s] = red_op(v[s], __shfl_xor_sync(0xffffffffu, v[s], o), ops[s]);
}

// block reduction; the result is valid in warp 0 (all its lanes)
template <int NS>
__device__ __forceinline__ void block_reduce_w0(float (&v)[NS], const int (&ops)[NS])
{
    float *sh = reinterpret_cast<float *>(red_scratch());
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    warp_tree(v, ops);
    if (lane == 0)
#pragma unroll
        for (int s = 0; s < NS; ++s) sh[s * 32 + warp] = v[s];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) v[s] = lane < nw ? sh[s * 32 + lane] : 0.0f;
        warp_tree(v, ops);
    }
}

template <int NS>
__device__ __forceinline__ void block_reduce_w0(double (&v)[NS], const int (&ops)[NS])
{
    double *sh = red_scratch();
#pragma unroll
    for (int s = 0; s < NS; ++s) sh[s * kMaxThreads + threadIdx.x] = v[s];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            double t0 = 0, t1 = 0, t2 = 0, t3 = 0;
            unsigned k = threadIdx.x;
            const unsigned nb = blockDim.x;
            for (; k + 96 < nb; k += 128) {
                t0 = red_op(t0, sh[s * kMaxThreads + k], ops[s]);
                t1 = red_op(t1, sh[s * kMaxThreads + k + 32], ops[s]);
                t2 = red_op(t2, sh[s * kMaxThreads + k + 64], ops[s]);
                t3 = red_op(t3, sh[s * kMaxThreads + k + 96], ops[s]);
            }
            for (; k < nb; k += 32) t0 = red_op(t0, sh[s * kMaxThreads + k], ops[s]);
            v[s] = red_op(red_op(t0, t1, ops[s]), red_op(t2, t3, ops[s]), ops[s]);
        }
        warp_tree(v, ops);
    }
}

// ---------------------------------------------------------------------------
// Grid all-reduce. Each block writes its block result to its own partial
// slots, then thread 0 arrives on a monotone 64-bit counter with a release
// add (which, after the preceding __syncthreads, publishes every write of
// the block) and spins with acquire loads until all blocks of this epoch
// have arrived. Warp 0 then reads all blocks' partials in one batch of
// independent loads and combines them in a fixed order (lane l takes blocks
// l, l+32, ... ascending, then a fixed shuffle tree), so every block holds
// bitwise identical results and takes identical branches. Partials
// alternate between two buffers by epoch parity, so a block that runs ahead
// never overwrites partials that a slower block has not read yet.
// The spin is bounded by wait_ns of %globaltimer: on expiry the block
// records kErrTimeout in ctl->error and every block leaves at its next
// exchange (a block that sees ctl->error stops waiting at once). One block
// needs no global memory at all.
// ---------------------------------------------------------------------------
// CH: blocks whose partials one lane loads per batch (32 CH blocks per
// batch); kernels with a 64-register budget use fewer
template <int CH>
struct GridExchangeT {
    Ctl *ctl;
    double *part;                  // [2][kMaxSlots][blocks of the team]
    unsigned epoch;
    unsigned long long wait_ns;
    unsigned extra;                // added to the arrival target (never reached: timeout test)
    bool block_only;               // the team is this block alone (no global memory used)
    // team of `team` blocks (0: the whole grid) in which this block is
    // number `rank`: the partials have one slot per team member
    unsigned team = 0, rank = 0;

    template <class V, int NS>
    __device__ __forceinline__ bool allreduce(V (&v)[NS], const int (&ops)[NS])
    {
        double *shd = red_scratch() + kMaxSlots * kMaxThreads;
        V *res = reinterpret_cast<V *>(shd);
        int *s_ok = reinterpret_cast<int *>(shd + 2 * kMaxSlots);
        block_reduce_w0(v, ops);
        const unsigned G = team ? team : gridDim.x;
        const unsigned me = team ? rank : blockIdx.x;
        if (block_only || G == 1) {
            if (threadIdx.x == 0)
#pragma unroll
                for (int s = 0; s < NS; ++s) res[s] = v[s];
            __syncthreads();
#pragma unroll
            for (int s = 0; s < NS; ++s) v[s] = res[s];
            __syncthreads();
            return true;
        }
        ++epoch;
        double *buf = part + (size_t)(epoch & 1u) * kMaxSlots * G;
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int ok = 1;
            if (lane == 0) {
#pragma unroll
                for (int s = 0; s < NS; ++s) buf[(size_t)s * G + me] = (double)v[s];
                red_release_add_u64(&ctl->arrive, 1ULL);
                const unsigned long long target = (unsigned long long)epoch * G + extra;
                const unsigned long long t0 = global_ns();
                unsigned spins = 0;
                while (ld_acquire_u64(&ctl->arrive) < target) {
                    if ((++spins & 15u) == 0) {
                        if (ld_volatile_i32(&ctl->error) != 0) { ok = 0; break; }
                        if (global_ns() - t0 > wait_ns) {
                            atomicCAS(&ctl->error, 0, kErrTimeout);
                            ok = 0;
                            break;
                        }
                    }
                }
            }
            __syncwarp();
            ok = __shfl_sync(0xffffffffu, ok, 0);
            V acc[NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) acc[s] = V(0);
            if (ok) {
                for (unsigned b0 = lane; b0 < G; b0 += 32 * CH) {
                    double w[CH][NS];
#pragma unroll
                    for (int c = 0; c < CH; ++c)
#pragma unroll
                        for (int s = 0; s < NS; ++s) {
                            const unsigned b = b0 + 32u * c;
                            w[c][s] = b < G ? __ldcg(buf + (size_t)s * G + b) : 0.0;
                        }
#pragma unroll
                    for (int c = 0; c < CH; ++c)
                        if (b0 + 32u * c < G)
#pragma unroll
                            for (int s = 0; s < NS; ++s) acc[s] = red_op(acc[s], (V)w[c][s], ops[s]);
                }
            }
            warp_tree(acc, ops);
            if (lane == 0) {
#pragma unroll
                for (int s = 0; s < NS; ++s) res[s] = acc[s];
                *s_ok = ok;
            }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < NS; ++s) v[s] = res[s];
        const bool good = *s_ok != 0;
        __syncthreads();
        return good;
    }

    // barrier without data
    __device__ __forceinline__ bool sync()
    {
        float v[1] = {0.0f};
        const int ops[1] = {kSum};
        return allreduce(v, ops);
    }
};

using GridExchange = GridExchangeT<4>;

}  // namespace gadi
