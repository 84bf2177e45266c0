// common.cuh -- shared definitions of the pPCA CUDA library (internal).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include "../../include/ppca.h"

namespace ppca {

// Device status word codes (written by kernels, read by ppca_sync).
enum DevStatus : int {
    kDevOk = 0,
    kDevCholeskyBreakdown = 1,   // non-positive pivot in CholeskyQR2
    kDevJacobiNoConverge = 2,    // Jacobi hit its sweep cap
    kDevWaitTimeout = 3,         // a bounded spin-wait ran out
    kDevBadArgument = 4,         // a kernel found an argument out of range
};

constexpr int kMaxM = 128;       // largest supported m = k + l

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// X as the kernels see it.
struct XView {
    const void* ptr = nullptr;
    int64_t n = 0, d = 0, ld = 0;
    ppca_dtype dtype = PPCA_F32;
    const float* scales = nullptr;   // FP8 per-row scales
};

__device__ __forceinline__ float load_x(const XView& x, int64_t r, int64_t j) {
    switch (x.dtype) {
    case PPCA_F32:
        return static_cast<const float*>(x.ptr)[r * x.ld + j];
    case PPCA_BF16:
        return __bfloat162float(static_cast<const __nv_bfloat16*>(x.ptr)[r * x.ld + j]);
    default: {
        __nv_fp8_e4m3 c;
        c.__x = static_cast<const uint8_t*>(x.ptr)[r * x.ld + j];
        return static_cast<float>(c) * x.scales[r];
    }
    }
}

// Error-free transformations for compensated ("double-float") FP32 sums.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    e = __fadd_rn(e, lo);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// Double-float ("df") numbers: an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, about 48 significand bits.  Knuth's TwoSum, the FMA-based
// TwoProduct and Dekker/Bailey-style normalisation; used where FP64 accuracy
// is needed but GB300's FP64 rate is too low.
struct dfloat {
    float hi, lo;
};

__device__ __forceinline__ dfloat df_make(double x) {
    dfloat r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

__device__ __forceinline__ dfloat df_norm(float s, float e) {
    dfloat r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ dfloat df_addx(dfloat a, dfloat b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return df_norm(s, e);
}

__device__ __forceinline__ dfloat df_neg(dfloat a) {
    a.hi = -a.hi;
    a.lo = -a.lo;
    return a;
}

__device__ __forceinline__ dfloat df_mulx(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_norm(p, e);
}

// a / b: one correction step of the float quotient.
__device__ __forceinline__ dfloat df_divx(dfloat a, dfloat b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dfloat r = df_addx(a, df_neg(df_mulx(df_norm(q1, 0.f), b)));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return df_norm(q1, q2);
}

// sqrt(a) for a > 0: one Newton correction of the float root.
__device__ __forceinline__ dfloat df_sqrtx(dfloat a) {
    const float s = __fsqrt_rn(a.hi);
    const float p = __fmul_rn(s, s);
    const float pe = __fmaf_rn(s, s, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
    return df_norm(s, __fdiv_rn(r, 2.0f * s));
}

__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Host-side count of kernel launches made by the library (measurement only).
void note_launch();
int64_t launches_so_far();

// Raises kernel `func`'s dynamic shared-memory limit on the current device to
// at least `bytes`, and never lowers it: a captured graph's kernel nodes keep
// the sizes they were captured with, so a later launch of the same kernel with
// less shared memory must not shrink the limit under them.
cudaError_t smem_at_least(const void* func, size_t bytes);

// Row sample of the pPCA step (the paper projects 10 % of the data in its
// large runs): 128-row block t is kept when the t-th output of the SplitMix64
// stream seeded with `seed` (Steele, Lea and Flood, 2014), as a 53-bit
// fraction, is below `fraction`.  Host and device evaluate the same integer
// arithmetic and the same exact double comparison.
constexpr uint64_t kSplitMixGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ inline uint64_t splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ inline uint64_t sample_block_u(uint64_t seed, int64_t t) {
    return splitmix64_mix(seed + (uint64_t)(t + 1) * kSplitMixGolden);
}

__host__ __device__ inline bool sample_block_kept(uint64_t u, double fraction) {
    return (double)(u >> 11) * 0x1p-53 < fraction;
}

}  // namespace ppca
