// Double-float ("df64") arithmetic on the FP32 pipe.  A value is an unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi); sums and products are carried with the
// error-free transformations TwoSum (Knuth) and TwoProd (one FMA), which keeps ~48 bits
// (relative rounding ~4e-15).  GB300 issues FP64 at ~1/64 of its FP32 rate, so FP64
// work whose accuracy target is above ~1e-13 runs several times faster this way.
//
// Every operation uses the _rn intrinsics so that the compiler cannot contract a product
// and a sum into an FMA (which would break the error-free transformations).  The
// conversions from and to FP64 work on the bit patterns with integer operations only.
// df_split gives x = hi + lo to 2^-46 relative for finite 2^-80 <= |x| < 2^128; for
// smaller |x| a remainder below the normal float range is flushed (absolute error < 2^-126,
// and |x| < 2^-126 splits to zero).  df_widen is exact for normal floats and zero.
#pragma once

#include <cstdint>
#include <cstring>

namespace zolo {

__host__ __device__ __forceinline__ uint32_t df_f2u(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float df_u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    std::memcpy(&x, &u, 4);
    return x;
#endif
}
__host__ __device__ __forceinline__ uint64_t df_d2u(double x) {
#ifdef __CUDA_ARCH__
    return ((uint64_t)(uint32_t)__double2hiint(x) << 32) | (uint32_t)__double2loint(x);
#else
    uint64_t u;
    std::memcpy(&u, &x, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double df_u2d(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __hiloint2double((int)(u >> 32), (int)(u & 0xFFFFFFFFu));
#else
    double x;
    std::memcpy(&x, &u, 8);
    return x;
#endif
}
__host__ __device__ __forceinline__ int df_clz32(uint32_t v) {
#ifdef __CUDA_ARCH__
    return __clz(v);
#else
    return v ? __builtin_clz(v) : 32;
#endif
}

// x = hi + lo (up to the flush of |lo| < 2^-126): hi keeps the top 24 bits of the mantissa
// (truncated), lo the leading 24 of the remaining 29 (truncated).
__host__ __device__ __forceinline__ void df_split(double x, float &hi, float &lo) {
    const uint64_t u = df_d2u(x);
    const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
    const int e = (int)((u >> 52) & 0x7FF);                 // biased FP64 exponent
    const uint64_t m = u & 0xFFFFFFFFFFFFFull;               // 52 mantissa bits
    const int ef = e - 896;                                  // biased FP32 exponent of hi
    if (ef <= 0) {                                           // below the normal float range
        hi = df_u2f(sign);
        lo = df_u2f(sign);
        return;
    }
    hi = df_u2f(sign | ((uint32_t)ef << 23) | (uint32_t)(m >> 29));
    const uint32_t r = (uint32_t)(m & 0x1FFFFFFFu);          // the 29 bits hi dropped
    if (r == 0) {
        lo = df_u2f(sign);
        return;
    }
    // r * 2^(e - 1075): leading bit of r at position p = 31 - clz(r)
    const int lz = df_clz32(r);
    const int el = e - 1075 + 127 + (31 - lz);               // biased FP32 exponent of lo
    if (el <= 0) {
        lo = df_u2f(sign);
        return;
    }
    const uint32_t mant = (lz + 1 < 32) ? ((r << (lz + 1)) >> 9) : 0u;   // 23 bits below the leading 1
    lo = df_u2f(sign | ((uint32_t)el << 23) | mant);
}

// float -> double exactly, by bits (normal floats and zero).
__host__ __device__ __forceinline__ double df_widen(float x) {
    const uint32_t u = df_f2u(x);
    const uint32_t sign = u & 0x80000000u, e = (u >> 23) & 0xFF, m = u & 0x7FFFFFu;
    if (e == 0) return df_u2d((uint64_t)sign << 32);
    return df_u2d(((uint64_t)(sign | ((e + 896u) << 20) | (m >> 3)) << 32) | ((uint64_t)(m & 7u) << 29));
}

#ifdef __CUDACC__
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float &s, float &e) {   // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// (sh, sl) += (ah, al) * (xh, xl)   (the al * xl term, ~2^-48 relative, is dropped)
__device__ __forceinline__ void df_fma(float &sh, float &sl, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    float t, f;
    df_two_sum(sh, p, t, f);
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(f, e));
}
// (sh, sl) += (bh, bl), renormalised
__device__ __forceinline__ void df_add(float &sh, float &sl, float bh, float bl) {
    float s, e;
    df_two_sum(sh, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(sl, bl));
    df_fast_two_sum(s, e, sh, sl);
}
__device__ __forceinline__ void df_norm(float &sh, float &sl) {
    float s, e;
    df_fast_two_sum(sh, sl, s, e);
    sh = s;
    sl = e;
}
#endif

}  // namespace zolo
