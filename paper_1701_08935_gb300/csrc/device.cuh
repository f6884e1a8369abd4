// Device-side helpers: complex arithmetic on (re, im) pairs and the job descriptors
// that drive the batched kernels.  Internal to the library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace zolo {

template <class T> struct alignas(2 * sizeof(T)) cx {
    T re, im;
};
using c64 = cx<float>;
using c128 = cx<double>;

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T r, T i) { return cx<T>{r, i}; }
template <class T> __host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> __host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T> __host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class T> __host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return {s * a.re, s * a.im}; }
template <class T> __host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return {a.re, -a.im}; }
template <class T> __host__ __device__ __forceinline__ T abs2(cx<T> a) { return a.re * a.re + a.im * a.im; }
// acc += a * b
template <class T> __host__ __device__ __forceinline__ void fma_acc(cx<T> &acc, cx<T> a, cx<T> b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
// a / b by Smith's algorithm (R. L. Smith, CACM 5(8), 1962)
template <class T> __host__ __device__ __forceinline__ cx<T> cdiv(cx<T> a, cx<T> b) {
    if (fabs(b.re) >= fabs(b.im)) {
        T r = b.im / b.re, d = b.re + b.im * r;
        return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
    } else {
        T r = b.re / b.im, d = b.im + b.re * r;
        return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
    }
}
template <class To, class Ti> __host__ __device__ __forceinline__ cx<To> cvt(cx<Ti> a) { return {(To)a.re, (To)a.im}; }

// One dense product C(m x n) (=|-=) op(A)(m x kk) op(B)(kk x n) on strided operands:
// A(i,l) = A[a + i*ars + l*acs], B(l,j) = B[b + l*brs + j*bcs], C(i,j) = C[c + i*crs + j*ccs].
struct GJob {
    int64_t a, b, c;
    int32_t m, n, k;
    int32_t ars, acs, brs, bcs, crs, ccs;
    int32_t tile0;      // first tile of this job inside its launch
    int32_t tm;         // tiles along m
    int32_t flags;      // GJ_CONJA | GJ_CONJB | GJ_SUB | GJ_ACC
    int32_t ks;         // split of the kk extent over ks CTAs (results added atomically)
    int64_t ps;         // GJ_PRESPLIT: float offset of A's pre-split tensor-core planes
};
// GJ_SUB: C -= AB, GJ_ACC: C += AB, neither: C = AB (never split).  GJ_PRESPLIT: A is also
// stored pre-split (see PJob); the tensor-core kernel loads those planes instead of A.
enum { GJ_CONJA = 1, GJ_CONJB = 2, GJ_SUB = 4, GJ_ACC = 8, GJ_PRESPLIT = 16 };

// One operand of the block solves (column-major, rows contiguous) kept pre-split for the
// tensor cores: per 128-row tile rt and k-step ks of 8, a 16 KB block at float offset
// ps + (rt * ceil(k / 8) + ks) * 4096 holding the four TF32 planes (re hi, re lo, im hi,
// im lo) of that 128 x 8 tile in the canonical no-swizzle K-major layout, zero-padded.
struct PJob {
    int64_t a;          // element offset of the operand's (0,0) entry
    int64_t ps;         // float offset of its blocks in the pre-split buffer
    int64_t blk0;       // its first block in the build launch
    int32_t acs;        // column stride
    int32_t m, k;       // rows, inner extent
    int32_t base;       // 0: front pool, 1: pivot-block inverses
};

// A diagonal block of a front: LU in place (FP64), inverses of L and U stored.
struct DJob {
    int64_t off;        // element offset of the block's (0,0) entry in the front pool
    int64_t inv;        // offset of Linv (nb x nb, ld NB); Uinv follows at + NB*NB
    int32_t ld, nb;
    int32_t front, pad;
};

// Row gathers / scatters between a global row-major block and front workspaces,
// and child-to-parent extend-adds.
struct RJob {
    int64_t src, dst;   // element offsets (meaning depends on the kernel)
    int64_t map;        // offset into an int32 row map
    int32_t rows;       // rows handled
    int32_t ld_src, ld_dst;  // matrix kernels: leading dimensions
    int32_t tile0, tr;  // tiling
    int32_t pad;
};

constexpr int NB = 64;          // panel width of the blocked front LU and solves
constexpr int MAX_INST = 8;     // batched instances per launch (poles x {K^-1, K^-H})

}  // namespace zolo
