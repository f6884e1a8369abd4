// Shift-invariant GMRES for Z_2r2(G; l2) X (the GMRES steps of Algorithm 2, eq. solve2) and the
// subspace iteration with Rayleigh-Ritz of Algorithm 1.
//
// GMRES: one Krylov basis per column c of X, shared by all 2 r2 shifts s = +-i sqrt(c_j):
//   (G + s I) V_m = V_{m+1} (Hbar_m + s Ibar)  (shift invariance), so every shifted system
//   is the small least-squares problem  min || beta_c e1 - (Hbar_m + s Ibar) z ||.
// Arnoldi uses classical Gram-Schmidt applied twice.  The least squares are solved by
// complex Givens rotations kept per (column, shift) and extended by one column per step;
// the step count m is the first one at which, for every column, the error bound
//   sum_s |omega_s| res_s / sqrt(l2^2 + |s|^2) <= gmres_tol * beta_c
// holds (same m for the whole block; G is B-normal with real spectrum outside (-l2, l2),
// so the bound follows from ||(G + s)^-1|| <= 1/dist(-s, spec G)).  Finally
//   Y = X/2 + sum_j V_j zeta_j,  zeta = sum_s omega_s z_s,  omega_s = M a_j / 4.
//
// Algorithm 1: Y = R(B^-1 A) Q, then the projected pencil (Y^H A Y, Y^H B Y) is solved by
// diagonalising the B-Gram matrix (dropping directions below drop_tol * max), a standard
// Hermitian eigenproblem in that basis, and Q = Y W Z.  Small Hermitian eigenproblems use
// a parallel cyclic Jacobi method (round-robin pairing, two launches per round).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include "factor.h"
#include "df64.cuh"

namespace zolo {

namespace {

constexpr int RED_CTAS = 304;     // fixed reduction grid (deterministic sums)
constexpr int JT = 8;             // basis vectors per pass of the multi-dot kernel

// ---------------------------------------------------------------- block kernels
// part[b][j][c] = sum over rows i = b, b+G, ... of conj(V_j[i,c]) W[i,c], j in [j0, j0+nj)
// FP64 -> FP32 by integer operations on the bit pattern (truncating the mantissa; values
// below 2^-126 become 0), so that reading FP64 operands costs no FP64-pipe instructions,
// which GB300 issues at ~1/64 of the FP32 rate.  Finite |x| < 2^128 only (the Krylov
// vectors it reads are normalised).
__device__ __forceinline__ float f64_to_f32_trunc(double x) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int32_t t = (int32_t)(hi & 0x7FFFFFFFu) - (int32_t)(896u << 20);    // rebias 1023 -> 127
    const uint32_t mag = t > 0 ? (((uint32_t)t << 3) | (lo >> 29)) : 0u;
    return __uint_as_float(mag | (hi & 0x80000000u));
}

// Krylov basis blocks are stored split: for V_j (n x k) the first n k float2 hold the
// complex64 "hi" parts and the next n k the remainders, V = hi + lo to ~2^-47 (df_split).
//
// part[b][t][c] = sum over this CTA's rows of conj(V_{j0+t}[i,c]) W[i,c], in FP32 on the hi
// parts.  The projection coefficients of classical Gram-Schmidt only need FP32 accuracy:
// the update W -= sum_j V_j h_j and the Hessenberg matrix use the same h, so the Arnoldi
// relation G V_m = V_{m+1} H_m stays exact to the update's rounding and the basis is
// orthonormal to ~1e-6, which keeps the least-squares residuals within 1e-4 of the true
// ones.  The partial sums are reduced in FP64 by k_multidot_sum.
__global__ void __launch_bounds__(256) k_multidot(int64_t n, int k, const float2 *const *__restrict__ V, int j0, int nj,
                                                  const c128 *__restrict__ W, double2 *__restrict__ part) {
    // rows in one contiguous chunk per CTA; for k <= 256 the threads form 256 / k row groups
    // of k consecutive columns (consecutive addresses of the row-major blocks), and the
    // groups' sums are added in a fixed order through shared memory
    __shared__ float2 red[JT][256];
    const int64_t rpc = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * rpc, r1 = r0 + rpc < n ? r0 + rpc : n;
    if (k <= 256) {
        const int rpp = 256 / k, c = threadIdx.x % k, rr = threadIdx.x / k;
        float ar[JT], ai[JT];
#pragma unroll
        for (int t = 0; t < JT; ++t) ar[t] = ai[t] = 0.f;
        if (rr < rpp)
            for (int64_t i = r0 + rr; i < r1; i += rpp) {
                const c128 w = W[i * k + c];
                const float wr = f64_to_f32_trunc(w.re), wi = f64_to_f32_trunc(w.im);
#pragma unroll
                for (int t = 0; t < JT; ++t)
                    if (t < nj) {
                        const float2 v = V[j0 + t][i * k + c];
                        ar[t] = fmaf(v.x, wr, fmaf(v.y, wi, ar[t]));        // conj(v) w
                        ai[t] = fmaf(v.x, wi, fmaf(-v.y, wr, ai[t]));
                    }
            }
#pragma unroll
        for (int t = 0; t < JT; ++t) red[t][threadIdx.x] = make_float2(ar[t], ai[t]);
        __syncthreads();
        for (int e = threadIdx.x; e < nj * k; e += 256) {
            const int t = e / k, cc = e - t * k;
            double sr = 0.0, si = 0.0;
            for (int q = 0; q < rpp; ++q) {
                const float2 v = red[t][q * k + cc];
                sr += v.x;
                si += v.y;
            }
            part[((int64_t)blockIdx.x * nj + t) * k + cc] = make_double2(sr, si);
        }
        return;
    }
    for (int c = threadIdx.x; c < k; c += 256) {
        float ar[JT], ai[JT];
#pragma unroll
        for (int t = 0; t < JT; ++t) ar[t] = ai[t] = 0.f;
        for (int64_t i = r0; i < r1; ++i) {
            const c128 w = W[i * k + c];
            const float wr = f64_to_f32_trunc(w.re), wi = f64_to_f32_trunc(w.im);
#pragma unroll
            for (int t = 0; t < JT; ++t)
                if (t < nj) {
                    const float2 v = V[j0 + t][i * k + c];
                    ar[t] = fmaf(v.x, wr, fmaf(v.y, wi, ar[t]));
                    ai[t] = fmaf(v.x, wi, fmaf(-v.y, wr, ai[t]));
                }
        }
#pragma unroll
        for (int t = 0; t < JT; ++t)
            if (t < nj) part[((int64_t)blockIdx.x * nj + t) * k + c] = make_double2(ar[t], ai[t]);
    }
}

// h[j0 + t][c] (+)= sum_b part[b][t][c];  also H(j0+t, col, c) += that value
__global__ void k_multidot_sum(int k, int nj, int parts, const double2 *__restrict__ part, c128 *__restrict__ h,
                               float4 *__restrict__ hs, int j0, c128 *__restrict__ H, int hld, int col) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nj * k) return;
    const int t = idx / k, c = idx - t * k;
    c128 s = mk<double>(0, 0);
    for (int b = 0; b < parts; ++b) {
        const double2 v = part[((int64_t)b * nj + t) * k + c];
        s.re += v.x;
        s.im += v.y;
    }
    h[(int64_t)(j0 + t) * k + c] = s;
    float4 sp;
    df_split(s.re, sp.x, sp.y);
    df_split(s.im, sp.z, sp.w);
    hs[(int64_t)(j0 + t) * k + c] = sp;
    c128 *e = H + ((int64_t)c * hld + col) * hld + (j0 + t);     // H[c][col][row], column-major per c
    *e = *e + s;
}

// W[i,c] -= sum_{j < nj} V_j[i,c] h[j][c]: the sum in double-float arithmetic on the FP32
// pipe (split basis and split h), one FP64 subtraction per element at the end.
__global__ void k_multiaxpy(int64_t n, int k, const float2 *const *__restrict__ V, int nj, const float4 *__restrict__ hs,
                            c128 *__restrict__ W) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nk = n * k;
    if (idx >= nk) return;
    const int c = (int)(idx % k);
    float srh = 0.f, srl = 0.f, sih = 0.f, sil = 0.f;
    for (int j = 0; j < nj; ++j) {
        const float4 hv = hs[(int64_t)j * k + c];
        const float2 vh = V[j][idx], vl = V[j][nk + idx];
        df_fma(srh, srl, vh.x, vl.x, hv.x, hv.y);            // vr hr
        df_fma(srh, srl, -vh.y, -vl.y, hv.z, hv.w);          // - vi hi
        df_fma(sih, sil, vh.x, vl.x, hv.z, hv.w);            // vr hi
        df_fma(sih, sil, vh.y, vl.y, hv.x, hv.y);            // vi hr
    }
    c128 w = W[idx];
    w.re = (w.re - df_widen(srh)) - df_widen(srl);
    w.im = (w.im - df_widen(sih)) - df_widen(sil);
    W[idx] = w;
}

// V = W / ||W_c|| per column c (norms[c] = sum of squares), stored split into the hi / lo
// planes of P; H(col+1, col, c) = ||W_c|| when H is given.
__global__ void k_normalize(int64_t n, int k, const double *__restrict__ nrm2, const c128 *__restrict__ W,
                            float2 *__restrict__ P, c128 *__restrict__ H, int hld, int col) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < (int64_t)k && H) {
        const double nv = sqrt(nrm2[idx]);
        H[((int64_t)idx * hld + col) * hld + col + 1] = mk<double>(nv, 0.0);
    }
    const int64_t nk = n * k;
    if (idx >= nk) return;
    const int c = (int)(idx % k);
    const double nv = sqrt(nrm2[c]);
    const double s = nv > 1e-300 ? 1.0 / nv : 0.0;
    const c128 v = s * W[idx];
    float2 hi, lo;
    df_split(v.re, hi.x, lo.x);
    df_split(v.im, hi.y, lo.y);
    P[idx] = hi;
    P[nk + idx] = lo;
}

// V (FP64, n x k) = hi + lo of a split basis block
__global__ void k_from_planes(int64_t n, int k, const float2 *__restrict__ P, c128 *__restrict__ V) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nk = n * k;
    if (idx >= nk) return;
    const float2 hi = P[idx], lo = P[nk + idx];
    V[idx] = mk<double>(df_widen(hi.x) + df_widen(lo.x), df_widen(hi.y) + df_widen(lo.y));
}

// Incremental Givens least squares for every (column c, shift s): append column `col`
// of (Hbar + s Ibar) for column c, rotate it by the stored rotations, make and store the
// new rotation, update g; res[c * ns + s] = |g_{col+1}|.
// Scratch per (c, s): rot c (double) and s (complex) per step, R (upper, m_max x m_max),
// g (m_max + 1).
struct LsqScratch {
    double *rc;    // [pairs][mmax]
    c128 *rs;      // [pairs][mmax]
    c128 *R;       // [pairs][mmax][mmax]  (column-major, R[col * mmax + row])
    c128 *g;       // [pairs][mmax + 1]
};
__global__ void k_lsq_step(int k, int ns, const c128 *__restrict__ shifts, const c128 *__restrict__ H, int hld, int col,
                           const double *__restrict__ beta, LsqScratch S, int mmax, double *__restrict__ res) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= k * ns) return;
    const int c = p / ns, s = p - c * ns;
    double *rc = S.rc + (int64_t)p * mmax;
    c128 *rs = S.rs + (int64_t)p * mmax;
    c128 *R = S.R + (int64_t)p * mmax * mmax;
    c128 *g = S.g + (int64_t)p * (mmax + 1);
    if (col == 0) {
        g[0] = mk<double>(beta[c], 0.0);
        for (int i = 1; i <= mmax; ++i) g[i] = mk<double>(0, 0);
    }
    const c128 *h = H + ((int64_t)c * hld + col) * hld;   // column `col` of Hbar for column c
    c128 *x = R + (int64_t)col * mmax;                    // rotated column, rows 0..col
    for (int i = 0; i <= col; ++i) x[i] = h[i];
    x[col] = x[col] + shifts[s];
    c128 xb = h[col + 1];                                  // sub-diagonal entry
    for (int t = 0; t < col; ++t) {                        // previous rotations on rows (t, t+1)
        const double cc = rc[t];
        const c128 ss = rs[t];
        const c128 a = x[t], b = x[t + 1];
        x[t] = cc * a + ss * b;
        x[t + 1] = cc * b - conj(ss) * a;
    }
    // new rotation zeroing xb against x[col]
    const double na = sqrt(abs2(x[col])), nb = sqrt(abs2(xb));
    double cc;
    c128 ss, r;
    if (nb == 0.0) {
        cc = 1.0; ss = mk<double>(0, 0); r = x[col];
    } else if (na == 0.0) {
        cc = 0.0; ss = (1.0 / nb) * conj(xb); r = mk<double>(nb, 0.0);
    } else {
        const double rho = hypot(na, nb);
        const c128 ph = (1.0 / na) * x[col];
        cc = na / rho;
        ss = (1.0 / rho) * (ph * conj(xb));
        r = rho * ph;
    }
    rc[col] = cc;
    rs[col] = ss;
    x[col] = r;
    const c128 g0 = g[col];
    g[col] = cc * g0;
    g[col + 1] = mk<double>(0, 0) - conj(ss) * g0;
    res[p] = sqrt(abs2(g[col + 1])) / fmax(beta[c], 1e-300);
}

// back substitution R z = g for every (c, s), then zeta[j][c] = sum_s omega_s z_s[j]
__global__ void k_lsq_solve(int k, int ns, int m, LsqScratch S, int mmax, const c128 *__restrict__ omega,
                            c128 *__restrict__ zall) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= k * ns) return;
    const c128 *R = S.R + (int64_t)p * mmax * mmax;
    const c128 *g = S.g + (int64_t)p * (mmax + 1);
    c128 *z = zall + (int64_t)p * mmax;
    for (int i = m - 1; i >= 0; --i) {
        c128 sum = g[i];
        for (int j = i + 1; j < m; ++j) sum = sum - R[(int64_t)j * mmax + i] * z[j];
        z[i] = cdiv(sum, R[(int64_t)i * mmax + i]);
    }
    const int s = p % ns;
    for (int i = 0; i < m; ++i) z[i] = omega[s] * z[i];
}
__global__ void k_zeta(int k, int ns, int m, int mmax, const c128 *__restrict__ zall, c128 *__restrict__ zeta) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= k * m) return;
    const int j = idx / k, c = idx - j * k;
    c128 s = mk<double>(0, 0);
    for (int t = 0; t < ns; ++t) s = s + zall[((int64_t)c * ns + t) * mmax + j];
    zeta[(int64_t)j * k + c] = s;
}
// Y[i,c] = X[i,c]/2 + sum_{j<m} V_j[i,c] zeta[j][c]
// (real_out: the real part only, for the real blocks of a real pencil, where the conjugate
// shift pairs give conjugate z_s and a real sum up to rounding)
__global__ void k_combine(int64_t n, int k, const c128 *__restrict__ X, int64_t ldx, const float2 *const *__restrict__ V,
                          int m, const c128 *__restrict__ zeta, c128 *__restrict__ Y, int64_t ldy, int real_out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nk = n * k;
    if (idx >= nk) return;
    const int64_t i = idx / k;
    const int c = (int)(idx - i * k);
    c128 y = 0.5 * X[i * ldx + c];
    for (int j = 0; j < m; ++j) {
        const float2 hi = V[j][idx], lo = V[j][nk + idx];
        const c128 v = mk<double>(df_widen(hi.x) + df_widen(lo.x), df_widen(hi.y) + df_widen(lo.y));
        fma_acc(y, v, zeta[(int64_t)j * k + c]);
    }
    if (real_out) y.im = 0.0;
    Y[i * ldy + c] = y;
}

// ---------------------------------------------------------------- small dense kernels
// C[i][j] = sum_b part[b][i][j]   (k x k, reduction of split-N Gram products)
__global__ void k_sum_parts(int64_t cnt, int parts, const c128 *__restrict__ part, c128 *__restrict__ C) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= cnt) return;
    c128 s = mk<double>(0, 0);
    for (int b = 0; b < parts; ++b) s = s + part[(int64_t)b * cnt + idx];
    C[idx] = s;
}
// Hermitian part in place: M = (M + M^H)/2, column-major k x k
__global__ void k_hermitize(int k, c128 *M) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= k * k) return;
    const int i = idx % k, j = idx / k;
    if (i > j) return;
    const c128 a = M[i + (int64_t)j * k], b = M[j + (int64_t)i * k];
    const c128 v = 0.5 * (a + conj(b));
    M[i + (int64_t)j * k] = v;
    M[j + (int64_t)i * k] = conj(v);
}
__global__ void k_eye(int k, c128 *V) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= k * k) return;
    V[idx] = mk<double>((idx % k) == (idx / k) ? 1.0 : 0.0, 0.0);
}

// Jacobi: pair t of round r (circle method, player 0 fixed, kk even)
__device__ __forceinline__ void jpair(int t, int r, int kk, int &p, int &q) {
    auto P = [&](int j) { return ((j + r) % (kk - 1)) + 1; };
    int a = (t == 0) ? 0 : P(t), b = (t == 0) ? P(0) : P(kk - 1 - t);
    p = min(a, b);
    q = max(a, b);
}
struct Rot {
    double c;
    c128 s, e;     // J = [[c, s], [-s e, c e]] with e = exp(-i phi)
};
// columns p, q of A and V: A <- A J, V <- V J (rotation computed from the pair's own columns)
__global__ void __launch_bounds__(128) k_jacobi_cols(int k, int kk, int r, c128 *A, c128 *V, Rot *rot) {
    const int t = blockIdx.x;
    int p, q;
    jpair(t, r, kk, p, q);
    __shared__ Rot R;
    if (q >= k) return;                        // the padding player
    if (threadIdx.x == 0) {
        const double app = A[p + (int64_t)p * k].re, aqq = A[q + (int64_t)q * k].re;
        const c128 apq = A[p + (int64_t)q * k];
        const double b = sqrt(abs2(apq));
        Rot x;
        if (b < 1e-300 || b <= 1e-18 * (fabs(app) + fabs(aqq))) {
            x.c = 1.0; x.s = mk<double>(0, 0); x.e = mk<double>(1, 0);
        } else {
            const c128 e = (1.0 / b) * conj(apq);
            const double tau = (aqq - app) / (2.0 * b);
            const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            const double c = 1.0 / sqrt(1.0 + tt * tt);
            x.c = c; x.s = mk<double>(tt * c, 0.0); x.e = e;
        }
        R = x;
        rot[t] = x;
    }
    __syncthreads();
    const Rot x = R;
    const c128 jpp = mk<double>(x.c, 0.0), jpq = x.s, jqp = mk<double>(0, 0) - x.s * x.e, jqq = x.c * x.e;
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const c128 a = A[i + (int64_t)p * k], b = A[i + (int64_t)q * k];
        A[i + (int64_t)p * k] = a * jpp + b * jqp;
        A[i + (int64_t)q * k] = a * jpq + b * jqq;
        const c128 u = V[i + (int64_t)p * k], v = V[i + (int64_t)q * k];
        V[i + (int64_t)p * k] = u * jpp + v * jqp;
        V[i + (int64_t)q * k] = u * jpq + v * jqq;
    }
}
// rows p, q of A: A <- J^H A
__global__ void __launch_bounds__(128) k_jacobi_rows(int k, int kk, int r, c128 *A, const Rot *rot) {
    const int t = blockIdx.x;
    int p, q;
    jpair(t, r, kk, p, q);
    if (q >= k) return;
    const Rot x = rot[t];
    const c128 jpp = mk<double>(x.c, 0.0), jpq = x.s, jqp = mk<double>(0, 0) - x.s * x.e, jqq = x.c * x.e;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        const c128 a = A[p + (int64_t)j * k], b = A[q + (int64_t)j * k];
        A[p + (int64_t)j * k] = conj(jpp) * a + conj(jqp) * b;
        A[q + (int64_t)j * k] = conj(jpq) * a + conj(jqq) * b;
    }
    if (threadIdx.x == 0) {                      // keep the 2 x 2 block exactly diagonal
        A[q + (int64_t)p * k] = mk<double>(0, 0);
        A[p + (int64_t)q * k] = mk<double>(0, 0);
        A[p + (int64_t)p * k].im = 0.0;
        A[q + (int64_t)q * k].im = 0.0;
    }
}
// off[0] = sum_{i != j} |A_ij|^2, off[1] = sum_i |A_ii|^2 (single CTA)
__global__ void k_offnorm(int k, const c128 *A, double *off) {
    __shared__ double s0[256], s1[256];
    double a = 0.0, d = 0.0;
    for (int64_t idx = threadIdx.x; idx < (int64_t)k * k; idx += 256) {
        const int i = (int)(idx % k), j = (int)(idx / k);
        const double v = abs2(A[idx]);
        if (i == j) d += v; else a += v;
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = d;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s0[threadIdx.x] += s0[threadIdx.x + w];
            s1[threadIdx.x] += s1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[0] = s0[0];
        off[1] = s1[0];
    }
}
__global__ void k_diag(int k, const c128 *A, double *d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) d[i] = A[i + (int64_t)i * k].re;
}
// W[:, t] = V[:, idx[t]] * scale[t]   (column-major k x kt)
__global__ void k_gather_cols(int k, int kt, const c128 *V, const int *idx, const double *scale, c128 *W) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= k * kt) return;
    const int i = e % k, t = e / k;
    W[e] = scale[t] * V[i + (int64_t)idx[t] * k];
}
// R = AQ - BQ diag(lam)  (n x m, ld m)
__global__ void k_resid_block(int64_t n, int m, const c128 *AQ, const c128 *BQ, const double *lam, c128 *R) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * m) return;
    const int c = (int)(idx % m);
    R[idx] = AQ[idx] - lam[c] * BQ[idx];
}
// D[i, t] = S[i, t] for t < nc  (row-major blocks, ld ldd / lds)
__global__ void k_copy_cols(int64_t n, int nc, const c128 *S, int64_t lds, c128 *D, int64_t ldd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nc) return;
    const int64_t i = idx / nc;
    const int t = (int)(idx - i * nc);
    D[i * ldd + t] = S[i * lds + t];
}
// E[i, t] = Q[i, sel[t]]  (row-major blocks, ld lde / ldq)
__global__ void k_select_cols(int64_t n, int nf, const c128 *Q, int64_t ldq, const int *sel, c128 *E, int64_t lde) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * nf) return;
    const int64_t i = idx / nf;
    const int t = (int)(idx - i * nf);
    E[i * lde + t] = Q[i * ldq + sel[t]];
}
// seeded starting block: SplitMix64 counter stream -> uniforms -> Box-Muller, (N + iN)/sqrt 2
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
// (real_only: N(0,1) real entries, the real starting block of a real pencil)
__global__ void k_randn(int64_t cnt, uint64_t seed, c128 *X, int real_only) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= cnt) return;
    const uint64_t a = splitmix64(seed ^ (2 * (uint64_t)idx)), b = splitmix64(seed ^ (2 * (uint64_t)idx + 1));
    const double u1 = ((a >> 11) + 1.0) * 0x1.0p-53, u2 = (b >> 11) * 0x1.0p-53;
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    X[idx] = real_only ? mk<double>(rad * cs, 0.0) : mk<double>(rad * cs * 0.7071067811865476, rad * sn * 0.7071067811865476);
}

inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ================================================================ device helpers (host side)
namespace {

int grow(zolo_factor_s *h, Buf &b, size_t bytes) {
    if (b.bytes >= bytes) return ZOLO_OK;
    dev_release(h, b);
    void *p = nullptr;
    int rc = dev_alloc(h, bytes, &p);
    if (rc) return rc;
    b = Buf{p, bytes};
    return ZOLO_OK;
}

// one strided complex GEMM on the device (job uploaded synchronously on the stream)
int gemm1(zolo_factor_s *h, cudaStream_t st, Buf &jobbuf, const c128 *A, const c128 *B, c128 *C, GJob j) {
    j.tm = (j.m + 63) / 64;
    j.tile0 = 0;
    const int tiles = j.tm * ((j.n + 63) / 64);
    if (tiles == 0 || j.k == 0) return ZOLO_OK;
    int rc = grow(h, jobbuf, sizeof(GJob));
    if (rc) return rc;
    rc = cuda_check(cudaMemcpyAsync(jobbuf.p, &j, sizeof(GJob), cudaMemcpyHostToDevice, st), "job");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "job");
    if (rc) return rc;
    GemmArgs<double> g;
    std::memset(&g, 0, sizeof(g));
    g.bm = 64;
    g.jobs[0] = (const GJob *)jobbuf.p;
    g.njobs[0] = 1;
    g.ntiles[0] = tiles;
    g.A[0] = A;
    g.B[0] = B;
    g.C[0] = C;
    launch_gemm<double>(g, 1, st, 8.0 * j.m * j.n * j.k);
    return cuda_check(cudaGetLastError(), "gemm1");
}

GJob job(int64_t a, int ars, int acs, int64_t b, int brs, int bcs, int64_t c, int crs, int ccs, int m, int n, int k,
         int flags) {
    GJob j;
    std::memset(&j, 0, sizeof(j));
    j.a = a; j.ars = ars; j.acs = acs;
    j.b = b; j.brs = brs; j.bcs = bcs;
    j.c = c; j.crs = crs; j.ccs = ccs;
    j.m = m; j.n = n; j.k = k; j.flags = flags;
    j.ks = 1;
    return j;
}

}  // namespace

// persistent work buffers of the Krylov / Rayleigh-Ritz layer
struct KrylovWork {
    std::vector<Buf> vblocks;          // Krylov basis blocks V_0, V_1, ... (allocated on demand)
    std::vector<c128 *> vhost;
    Buf vptr;                          // device copy of the block pointers
    int64_t vblk = 0;                  // elements per block the blocks were sized for
    Buf H, h, hs, part, nrm, beta, shifts, omega, res, lsq, zall, zeta;
    Buf wcur, vcur;                    // FP64 n x k blocks: the vector being orthogonalised, and V_i
    Buf gram_part, At, Bt, U, Vt, W, Ah, Z, Qt, rot, dvec, off, idx, scl, jobs;
    Buf Y, AY, BY, Q, R;
};

// the buffers themselves are device allocations owned (and freed) by the factor handle
void krylov_free(KrylovWork *w) { delete w; }

static KrylovWork &work(zolo_factor_s *h) {
    if (!h->kw) h->kw = new KrylovWork();
    return *h->kw;
}

// ---------------------------------------------------------------- GMRES driver
static int gmres_block(zolo_factor_s *h, int64_t k, const c128 *X, int64_t ldx, c128 *Y, int64_t ldy,
                       cudaStream_t st, zolo_stats *stats) {
    KrylovWork &w = work(h);
    const int64_t n = h->n;
    const int mmax = std::max(1, h->opts.gmres_m_max > 0 ? h->opts.gmres_m_max : 100);
    const double tol = h->gmres_tol_now > 0 ? h->gmres_tol_now : (h->opts.gmres_tol > 0 ? h->opts.gmres_tol : 1e-12);
    const int r2 = h->fi.r2, ns = 2 * r2;
    const int hld = mmax + 1;
    const int64_t blk = n * k;
    if (w.vblk < blk) {                            // blocks sized for a smaller block width: drop them
        for (Buf &b : w.vblocks) dev_release(h, b);
        w.vblocks.clear();
        w.vhost.clear();
        w.vblk = blk;
    }
    int rc = grow(h, w.vptr, (size_t)(mmax + 1) * sizeof(c128 *));
    auto ensure_block = [&](int j) -> int {       // make V_0 .. V_j exist
        while ((int)w.vblocks.size() <= j) {
            Buf b;
            int r = grow(h, b, (size_t)w.vblk * sizeof(c128));
            if (r) return r;
            w.vblocks.push_back(b);
            w.vhost.push_back((c128 *)b.p);
            r = cuda_check(cudaMemcpyAsync(w.vptr.p, w.vhost.data(), w.vhost.size() * sizeof(c128 *),
                                           cudaMemcpyHostToDevice, st), "vptr");
            if (!r) r = cuda_check(cudaStreamSynchronize(st), "vptr");
            if (r) return r;
        }
        return ZOLO_OK;
    };
    if (!rc) rc = ensure_block(1);
    if (!rc) rc = grow(h, w.H, (size_t)k * hld * hld * sizeof(c128));
    if (!rc) rc = grow(h, w.h, (size_t)(mmax + 1) * k * sizeof(c128));
    if (!rc) rc = grow(h, w.part, (size_t)RED_CTAS * JT * k * sizeof(double2));
    if (!rc) rc = grow(h, w.nrm, (size_t)2 * k * sizeof(double));
    if (!rc) rc = grow(h, w.beta, (size_t)k * sizeof(double));
    if (!rc) rc = grow(h, w.shifts, (size_t)ns * sizeof(c128));
    if (!rc) rc = grow(h, w.omega, (size_t)ns * sizeof(c128));
    if (!rc) rc = grow(h, w.res, (size_t)k * ns * sizeof(double));
    const size_t pairs = (size_t)k * ns;
    const size_t lsq_bytes = pairs * (mmax * sizeof(double) + mmax * sizeof(c128) + (size_t)mmax * mmax * sizeof(c128) +
                                      (mmax + 1) * sizeof(c128));
    if (!rc) rc = grow(h, w.lsq, lsq_bytes);
    if (!rc) rc = grow(h, w.zall, pairs * mmax * sizeof(c128));
    if (!rc) rc = grow(h, w.zeta, (size_t)mmax * k * sizeof(c128));
    if (!rc) rc = grow(h, w.hs, (size_t)(mmax + 1) * k * sizeof(float4));
    if (!rc) rc = grow(h, w.wcur, (size_t)blk * sizeof(c128));
    if (!rc) rc = grow(h, w.vcur, (size_t)blk * sizeof(c128));
    if (rc) return rc;
    const float2 *const *Vp = (const float2 *const *)w.vptr.p;      // split basis blocks
    c128 *Wc = (c128 *)w.wcur.p, *Vc = (c128 *)w.vcur.p;
    float4 *hsp = (float4 *)w.hs.p;
    auto plane = [&](int j) { return (float2 *)w.vhost[j]; };
    c128 *H = (c128 *)w.H.p;
    c128 *hv = (c128 *)w.h.p;
    double *nrm = (double *)w.nrm.p, *beta = (double *)w.beta.p, *res = (double *)w.res.p;
    LsqScratch S;
    {
        char *p = (char *)w.lsq.p;
        S.rc = (double *)p;
        p += pairs * mmax * sizeof(double);
        S.rs = (c128 *)p;
        p += pairs * mmax * sizeof(c128);
        S.R = (c128 *)p;
        p += pairs * (size_t)mmax * mmax * sizeof(c128);
        S.g = (c128 *)p;
    }
    // shifts +- i sqrt(c_j) and weights M a_j / 4 (eq. solve2, the combination step of Algorithm 2)
    std::vector<c128> sh(ns), om(ns);
    for (int j = 0; j < r2; ++j) {
        const double sq = std::sqrt(h->fi.c[j]);
        sh[2 * j] = c128{0.0, sq};
        sh[2 * j + 1] = c128{0.0, -sq};
        om[2 * j] = om[2 * j + 1] = c128{h->fi.M * h->fi.a[j] / 4.0, 0.0};
    }
    rc = cuda_check(cudaMemcpyAsync(w.shifts.p, sh.data(), ns * sizeof(c128), cudaMemcpyHostToDevice, st), "shifts");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(w.omega.p, om.data(), ns * sizeof(c128), cudaMemcpyHostToDevice, st), "omega");
    if (!rc) rc = cuda_check(cudaMemsetAsync(H, 0, (size_t)k * hld * hld * sizeof(c128), st), "H");
    if (rc) return rc;
    // V_0 = X / beta
    {
        LinArgs a;
        std::memset(&a, 0, sizeof(a));
        a.n = n; a.k = k; a.ldy = k; a.Y = Wc; a.nterm = 1;
        a.coef[0] = c128{1.0, 0.0}; a.X[0] = X; a.ldx[0] = ldx;
        launch_lincomb(a, st);
        rc = colnorm2(h, k, Wc, k, nrm, st);
        if (rc) return rc;
        k_normalize<<<nblk(blk), 256, 0, st>>>(n, (int)k, nrm, Wc, plane(0), nullptr, hld, 0);
        count_launch();
        // beta = sqrt(nrm): reuse the normalise kernel's formula on a k-vector
    }
    {
        std::vector<double> hn(k);
        rc = cuda_check(cudaMemcpyAsync(hn.data(), nrm, k * sizeof(double), cudaMemcpyDeviceToHost, st), "beta");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "beta");
        if (rc) return rc;
        for (auto &x : hn) x = std::sqrt(x);
        if (h->opts.verbose)
            std::fprintf(stderr, "[zolo] gmres block k=%lld ldx=%lld: ||x_c|| in [%.3e, %.3e]\n", (long long)k,
                         (long long)ldx, *std::min_element(hn.begin(), hn.end()),
                         *std::max_element(hn.begin(), hn.end()));
        rc = cuda_check(cudaMemcpyAsync(beta, hn.data(), k * sizeof(double), cudaMemcpyHostToDevice, st), "beta");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "beta");
        if (rc) return rc;
    }
    int m = 0;
    double worst = 0.0;
    std::vector<double> hres(pairs), hnorm(2 * k);
    // Relaxed inner accuracy (inexact Krylov: Simoncini & Szyld 2003, Bouras & Fraysse 2005):
    // an error e_i in the i-th product G v_i enters the GMRES solution weighted by the LSQ
    // coefficient of v_i, which is of the size of the residual before step i.  So the
    // mixed-precision solves of step i are refined to 1e-2 tol / (error bound after step
    // i - 1), clamped to [refine_tol, 1e-3], instead of refine_tol throughout.
    const double rtol = h->opts.refine_tol > 0 ? h->opts.refine_tol : 1e-12;
    struct ResetRelax {
        zolo_factor_s *h;
        ~ResetRelax() { h->refine_tol_now = 0.0; }
    } reset_relax{h};
    for (int i = 0; i < mmax; ++i) {
        rc = ensure_block(i + 1);
        if (rc) return rc;
        c128 *Wv = Wc;
        if (h->prec == ZOLO_PREC_MIXED) {
            const double prev = (i == 0) ? 1.0 : std::max(worst, 1e-300);
            h->refine_tol_now = std::min(1e-3, std::max(rtol, 1e-2 * tol / prev));
        }
        k_from_planes<<<nblk(blk), 256, 0, st>>>(n, (int)k, plane(i), Vc);
        count_launch();
        rc = apply_inner(h, k, Vc, k, Wv, k, st, plane(i));
        if (rc) {                                          // a failed inner solve is not a short GMRES
            h->inner_failed = true;
            return rc;
        }
        // classical Gram-Schmidt with selective re-orthogonalisation (Kahan-Parlett / DGKS):
        // the second pass runs when some column lost more than 1/sqrt(2) of its norm
        rc = colnorm2(h, k, Wv, k, nrm + k, st);
        if (rc) return rc;
        for (int pass = 0; pass < 2; ++pass) {
            for (int j0 = 0; j0 <= i; j0 += JT) {
                const int nj = std::min(JT, i + 1 - j0);
                k_multidot<<<RED_CTAS, 256, 0, st>>>(n, (int)k, Vp, j0, nj, Wv, (double2 *)w.part.p);
                count_launch();
                k_multidot_sum<<<nblk((int64_t)nj * k), 256, 0, st>>>((int)k, nj, RED_CTAS, (const double2 *)w.part.p,
                                                                     hv, hsp, j0, H, hld, i);
                count_launch();
            }
            k_multiaxpy<<<nblk(blk), 256, 0, st>>>(n, (int)k, Vp, i + 1, hsp, Wv);
            count_launch();
            if (pass == 0) {
                rc = colnorm2(h, k, Wv, k, nrm, st);
                if (!rc) rc = cuda_check(cudaMemcpyAsync(hnorm.data(), nrm, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, st),
                                "cgs norms");
                if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "cgs norms");
                if (rc) return rc;
                bool again = false;
                for (int64_t c = 0; c < k && !again; ++c) again = hnorm[c] < 0.5 * hnorm[k + c];   // squared norms
                if (!again) break;
            }
        }
        rc = colnorm2(h, k, Wv, k, nrm, st);
        if (rc) return rc;
        k_normalize<<<nblk(blk), 256, 0, st>>>(n, (int)k, nrm, Wv, plane(i + 1), H, hld, i);
        count_launch();
        k_lsq_step<<<nblk((int64_t)pairs, 128), 128, 0, st>>>((int)k, ns, (const c128 *)w.shifts.p, H, hld, i, beta, S, mmax,
                                                         res);
        count_launch();
        rc = cuda_check(cudaMemcpyAsync(hres.data(), res, pairs * sizeof(double), cudaMemcpyDeviceToHost, st), "res");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "gmres step");
        if (rc) return rc;
        // error bound of the filtered column: || sum_s omega_s (G + s)^-1 r_s || <=
        // sum_s |omega_s| res_s / dist(-s, spec G), spec G real outside (-l2, l2), s imaginary
        worst = 0.0;
        for (int64_t c = 0; c < k; ++c) {
            double e = 0.0;
            for (int t = 0; t < ns; ++t) {
                const double v = hres[c * ns + t];
                e += std::hypot(om[t].re, om[t].im) * (std::isfinite(v) ? v : 1e300) /
                     std::sqrt(h->fi.ell2 * h->fi.ell2 + sh[t].im * sh[t].im);
            }
            worst = std::max(worst, e);
        }
        m = i + 1;
        if (h->opts.verbose && (i < 3 || worst <= tol))
            std::fprintf(stderr, "[zolo]   step %d: error bound %.3e (tol %.1e)\n", i + 1, worst, tol);
        if (worst <= tol) break;
    }
    k_lsq_solve<<<nblk((int64_t)pairs, 128), 128, 0, st>>>((int)k, ns, m, S, mmax, (const c128 *)w.omega.p,
                                                      (c128 *)w.zall.p);
    count_launch();
    k_zeta<<<nblk((int64_t)k * m), 256, 0, st>>>((int)k, ns, m, mmax, (const c128 *)w.zall.p, (c128 *)w.zeta.p);
    count_launch();
    k_combine<<<nblk(blk), 256, 0, st>>>(n, (int)k, X, ldx, Vp, m, (const c128 *)w.zeta.p, Y, ldy, h->realx ? 1 : 0);
    count_launch();
    rc = cuda_check(cudaGetLastError(), "gmres");
    if (rc) return rc;
    h->stats.n_gmres = m;
    h->stats.gmres_res = worst;
    if (stats) {
        stats->n_gmres = m;
        stats->gmres_res = worst;
        stats->n_solv = (int64_t)h->r1 * k * m;
    }
    if (worst > tol) return set_error(ZOLO_ENOCONV, "GMRES reached gmres_m_max without meeting gmres_tol");
    return ZOLO_OK;
}

// The columns of X are independent GMRES problems: process them in chunks whose Krylov
// basis, (m_max + 1) n x chunk complex128 blocks, fits a memory budget (100 GiB, or 60%
// of the free device memory plus the basis blocks this handle already holds, which are
// reused, if that is smaller), and of at most opts.gmres_chunk columns.
int gmres_apply(zolo_factor_s *h, int64_t k, const c128 *X, int64_t ldx, c128 *Y, int64_t ldy, cudaStream_t st,
                zolo_stats *stats) {
    const int mmax = std::max(1, h->opts.gmres_m_max > 0 ? h->opts.gmres_m_max : 100);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    double held = 0.0;
    for (const Buf &b : work(h).vblocks) held += (double)b.bytes;
    const double budget = std::min(100.0 * (1ull << 30), 0.6 * ((double)fr + held));
    const double per_col = (double)(mmax + 1) * h->n * sizeof(c128);
    int64_t chunk = std::max<int64_t>(1, (int64_t)(budget / per_col));
    if (chunk >= 32) chunk = chunk / 32 * 32;
    if (h->opts.gmres_chunk > 0) chunk = std::min<int64_t>(chunk, h->opts.gmres_chunk);
    chunk = std::min(chunk, k);
    const int64_t nch = (k + chunk - 1) / chunk;
    chunk = (k + nch - 1) / nch;                        // balance the chunks
    int worst_rc = ZOLO_OK, m_all = 0;
    double res_all = 0.0;
    h->inner_failed = false;
    for (int64_t c0 = 0; c0 < k; c0 += chunk) {
        const int64_t kc = std::min(chunk, k - c0);
        int rc = gmres_block(h, kc, X + c0, ldx, Y + c0, ldy, st, stats);
        if (rc && (rc != ZOLO_ENOCONV || h->inner_failed)) return rc;
        if (rc) worst_rc = rc;
        m_all = std::max(m_all, h->stats.n_gmres);
        res_all = std::max(res_all, h->stats.gmres_res);
    }
    h->stats.n_gmres = m_all;
    h->stats.gmres_res = res_all;
    if (stats) {
        stats->n_gmres = m_all;
        stats->gmres_res = res_all;
        stats->n_solv = (int64_t)h->r1 * k * m_all;
    }
    if (worst_rc) return set_error(worst_rc, "GMRES reached gmres_m_max without meeting gmres_tol");
    return ZOLO_OK;
}

// ---------------------------------------------------------------- small Hermitian eigensolver
// eigenvalues ascending in d (host), eigenvectors as columns of V (device, column-major k x k);
// A (device, column-major) is destroyed.
static int jacobi_eig(zolo_factor_s *h, KrylovWork &w, int k, c128 *A, c128 *V, std::vector<double> &d,
                      cudaStream_t st) {
    const int kk = k + (k & 1);
    int rc = grow(h, w.rot, (size_t)(kk / 2) * sizeof(Rot));
    if (!rc) rc = grow(h, w.off, 2 * sizeof(double));
    if (!rc) rc = grow(h, w.dvec, (size_t)k * sizeof(double));
    if (rc) return rc;
    k_hermitize<<<nblk((int64_t)k * k), 256, 0, st>>>(k, A);
    count_launch();
    k_eye<<<nblk((int64_t)k * k), 256, 0, st>>>(k, V);
    count_launch();
    double off[2] = {0, 0};
    for (int sweep = 0; sweep < 30; ++sweep) {
        k_offnorm<<<1, 256, 0, st>>>(k, A, (double *)w.off.p);
        count_launch();
        rc = cuda_check(cudaMemcpyAsync(off, w.off.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "off");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "jacobi");
        if (rc) return rc;
        if (!(std::isfinite(off[0]) && std::isfinite(off[1])))
            return set_error(ZOLO_ENOCONV, "non-finite entries in a projected matrix");
        if (off[0] <= 1e-30 * std::max(off[1], 1e-300) || k == 1) break;
        for (int r = 0; r < kk - 1; ++r) {
            k_jacobi_cols<<<kk / 2, 128, 0, st>>>(k, kk, r, A, V, (Rot *)w.rot.p);
            count_launch();
            k_jacobi_rows<<<kk / 2, 128, 0, st>>>(k, kk, r, A, (const Rot *)w.rot.p);
            count_launch();
        }
    }
    if (off[0] > 1e-24 * std::max(off[1], 1e-300) && k > 1)
        return set_error(ZOLO_ENOCONV, "Jacobi eigensolver did not converge");
    k_diag<<<nblk(k), 256, 0, st>>>(k, A, (double *)w.dvec.p);
    count_launch();
    d.assign(k, 0.0);
    rc = cuda_check(cudaMemcpyAsync(d.data(), w.dvec.p, k * sizeof(double), cudaMemcpyDeviceToHost, st), "eig");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "eig");
    return rc;
}

// W[:, t] = V[:, idx[t]] * scale[t]
static int gather_cols(zolo_factor_s *h, KrylovWork &w, int k, const c128 *V, const std::vector<int> &idx,
                       const std::vector<double> &scale, c128 *W, cudaStream_t st) {
    const int kt = (int)idx.size();
    int rc = grow(h, w.idx, std::max(1, kt) * sizeof(int));
    if (!rc) rc = grow(h, w.scl, std::max(1, kt) * sizeof(double));
    if (rc) return rc;
    rc = cuda_check(cudaMemcpyAsync(w.idx.p, idx.data(), kt * sizeof(int), cudaMemcpyHostToDevice, st), "idx");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(w.scl.p, scale.data(), kt * sizeof(double), cudaMemcpyHostToDevice, st), "scl");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "gather");
    if (rc) return rc;
    k_gather_cols<<<nblk((int64_t)k * kt), 256, 0, st>>>(k, kt, V, (const int *)w.idx.p, (const double *)w.scl.p, W);
    count_launch();
    return cuda_check(cudaGetLastError(), "gather");
}

// C (k x k, column-major) = Y^H Z for n x k row-major blocks, split over row chunks
static int gram(zolo_factor_s *h, KrylovWork &w, int64_t n, int k, const c128 *Y, const c128 *Z, c128 *C,
                cudaStream_t st) {
    const int64_t chunk = std::max<int64_t>(4096, (n + 127) / 128);
    const int parts = (int)((n + chunk - 1) / chunk);
    int rc = grow(h, w.gram_part, (size_t)parts * k * k * sizeof(c128));
    if (!rc) rc = grow(h, w.jobs, (size_t)parts * sizeof(GJob));
    if (rc) return rc;
    std::vector<GJob> js;
    int tiles = 0;
    for (int b = 0; b < parts; ++b) {
        const int64_t r0 = b * chunk;
        const int rows = (int)std::min<int64_t>(chunk, n - r0);
        // C_b(i, j) = sum_l conj(Y[r0 + l, i]) Z[r0 + l, j]
        GJob j = job(r0 * k, 1, k, r0 * k, k, 1, (int64_t)b * k * k, 1, k, k, k, rows, GJ_CONJA);
        j.tm = (k + 63) / 64;
        j.tile0 = tiles;
        tiles += j.tm * ((k + 63) / 64);
        js.push_back(j);
    }
    rc = cuda_check(cudaMemcpyAsync(w.jobs.p, js.data(), js.size() * sizeof(GJob), cudaMemcpyHostToDevice, st), "jobs");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "jobs");
    if (rc) return rc;
    GemmArgs<double> g;
    std::memset(&g, 0, sizeof(g));
    g.bm = 64;
    g.jobs[0] = (const GJob *)w.jobs.p;
    g.njobs[0] = parts;
    g.ntiles[0] = tiles;
    g.A[0] = Y;
    g.B[0] = Z;
    g.C[0] = (c128 *)w.gram_part.p;
    launch_gemm<double>(g, 1, st, 8.0 * k * k * (double)n);
    k_sum_parts<<<nblk((int64_t)k * k), 256, 0, st>>>((int64_t)k * k, parts, (const c128 *)w.gram_part.p, C);
    count_launch();
    return cuda_check(cudaGetLastError(), "gram");
}

// Y = R(B^-1 A) X for the handle's filter: Algorithm 2 (inner operator + shift-invariant
// GMRES) for the Zolotarev filter, the inner operator alone for a contour-integral filter
// (its quadrature points are all factored poles: r2 = 0).
int filter_apply(zolo_factor_s *h, int64_t k, const c128 *X, int64_t ldx, c128 *Y, int64_t ldy, cudaStream_t st,
                 zolo_stats *stats) {
    if (h->fi.r2 > 0) return gmres_apply(h, k, X, ldx, Y, ldy, st, stats);
    h->inner_failed = false;
    const int rc = apply_inner(h, k, X, ldx, Y, ldy, st);
    if (rc) h->inner_failed = true;
    h->stats.n_gmres = 1;
    h->stats.gmres_res = 0.0;
    if (stats) {
        stats->n_gmres = 1;
        stats->gmres_res = 0.0;
        stats->n_solv = (int64_t)h->r1 * k;
    }
    return rc;
}

// ---------------------------------------------------------------- Algorithm 1
// Subspace iteration with Rayleigh-Ritz.  Real pencils with opts.real_block keep every block
// real (one solve per pole).  With opts.lock, the pairs in (a, b) whose residual is <= tol
// after an iteration are locked: they move to the front of the block and are not filtered
// again, while every Rayleigh-Ritz step still runs on [locked | filtered] (the footnote of
// Algorithm 1).  A converged Ritz value inside a declared eigengap returns ZOLO_EGAP.
static int eigs_factored(zolo_factor_s *h, double a, double b, int64_t k0, const c128 *X0, double *evals, c128 *evecs,
                         int64_t ldv, int64_t cap, int64_t *n_found, double *resid, zolo_stats *stats,
                         cudaStream_t st) {
    KrylovWork &w = work(h);
    const int64_t n = h->n;
    int k = (int)k0;
    const int64_t blk = n * k;
    int rc = grow(h, w.Q, blk * sizeof(c128));
    if (!rc) rc = grow(h, w.Y, blk * sizeof(c128));
    if (!rc) rc = grow(h, w.AY, blk * sizeof(c128));
    if (!rc) rc = grow(h, w.BY, blk * sizeof(c128));
    if (!rc) rc = grow(h, w.R, blk * sizeof(c128));
    const size_t kk2 = (size_t)k * k * sizeof(c128);
    if (!rc) rc = grow(h, w.At, kk2);
    if (!rc) rc = grow(h, w.Bt, kk2);
    if (!rc) rc = grow(h, w.U, kk2);
    if (!rc) rc = grow(h, w.W, kk2);
    if (!rc) rc = grow(h, w.Ah, kk2);
    if (!rc) rc = grow(h, w.Z, kk2);
    if (!rc) rc = grow(h, w.Qt, kk2);
    if (!rc) rc = grow(h, w.dvec, (size_t)k * sizeof(double));
    if (!rc) rc = grow(h, w.idx, (size_t)k * sizeof(int));
    if (rc) return rc;
    c128 *Y = (c128 *)w.Y.p, *AY = (c128 *)w.AY.p, *BY = (c128 *)w.BY.p;
    c128 *At = (c128 *)w.At.p, *Bt = (c128 *)w.Bt.p, *U = (c128 *)w.U.p, *Wm = (c128 *)w.W.p;
    c128 *Ah = (c128 *)w.Ah.p, *Zm = (c128 *)w.Z.p, *Qt = (c128 *)w.Qt.p;
    const bool real_pencil = pencil_is_real(h) && h->opts.real_block;
    bool rx = false;
    if (X0) {
        rc = cuda_check(cudaMemcpyAsync(w.Q.p, X0, blk * sizeof(c128), cudaMemcpyDeviceToDevice, st), "X0");
        if (!rc && real_pencil) rc = block_is_real(h, k, (const c128 *)w.Q.p, k, st, &rx);
    } else {
        k_randn<<<nblk(blk), 256, 0, st>>>(blk, h->opts.seed, (c128 *)w.Q.p, real_pencil ? 1 : 0);
        count_launch();
        rc = cuda_check(cudaGetLastError(), "randn");
        rx = real_pencil;
    }
    if (rc) return rc;
    struct ResetReal {
        zolo_factor_s *h;
        ~ResetReal() { h->realx = false; }
    } reset_real{h};
    h->realx = rx;
    const int itmax = std::max(1, h->opts.n_iter_max);
    const double tol = h->opts.tol > 0 ? h->opts.tol : 1e-10;
    const double drop = h->opts.drop_tol > 0 ? h->opts.drop_tol : 1e-14;
    const bool lock = h->opts.lock != 0;
    std::vector<double> lam, res_all, mu;
    std::vector<int> sel;
    int kq = k;           // columns of the current block
    int nl = 0;           // locked columns at its front
    int it = 0;
    bool converged = false;
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    float t_apply = 0.f, t_rr = 0.f;
    int n_gm = 0;
    int64_t n_solv = 0;
    bool gmres_short = false;
    bool empty_before = false;
    for (it = 1; it <= itmax; ++it) {
        c128 *Q = (c128 *)w.Q.p, *R = (c128 *)w.R.p;
        cudaEventRecord(e0, st);
        // The first application starts from a random block: its filtered output is re-filtered
        // by the next iteration, so a loose GMRES tolerance (1e-6) is enough there; later
        // applications start from Ritz vectors and use gmres_tol.
        const double gt = h->opts.gmres_tol > 0 ? h->opts.gmres_tol : 1e-12;
        h->gmres_tol_now = (it == 1 && itmax > 1) ? std::max(gt, 1e-6) : gt;
        // Y = [Q_locked | R(B^-1 A) Q_rest]
        if (nl > 0) {
            k_copy_cols<<<nblk(n * nl), 256, 0, st>>>(n, nl, Q, kq, Y, kq);
            count_launch();
        }
        rc = filter_apply(h, kq - nl, Q + nl, kq, Y + nl, kq, st, nullptr);
        h->gmres_tol_now = 0.0;
        if (rc == ZOLO_ENOCONV && !h->inner_failed) {               // GMRES step cap: use the block
            gmres_short = true;
            rc = ZOLO_OK;
        }
        if (rc) break;
        n_gm += h->stats.n_gmres;
        n_solv += (int64_t)h->r1 * (kq - nl) * h->stats.n_gmres;
        cudaEventRecord(e1, st);
        launch_spmm(h->A, kq, Y, kq, AY, kq, c128{1.0, 0.0}, false, st);
        launch_spmm(h->B, kq, Y, kq, BY, kq, c128{1.0, 0.0}, false, st);
        rc = gram(h, w, n, kq, Y, AY, At, st);
        if (!rc) rc = gram(h, w, n, kq, Y, BY, Bt, st);
        if (rc) break;
        // B-Gram diagonalisation and drop (SVQB-style basis W = U_kept mu^-1/2)
        rc = jacobi_eig(h, w, kq, Bt, U, mu, st);
        if (rc) break;
        double mumax = 0.0;
        for (double x : mu) mumax = std::max(mumax, x);
        // directions whose B-norm is at the level of the filtered block's own error are
        // noise: drop below max(drop_tol, (10 * GMRES tolerance of this pass)^2) * max mu
        const double tol_it = (it == 1 && itmax > 1) ? std::max(gt, 1e-6) : gt;
        const double drop_it = std::max(drop, 100.0 * tol_it * tol_it);
        std::vector<int> keep;
        std::vector<double> scl;
        for (int i = 0; i < kq; ++i)
            if (mu[i] > drop_it * mumax) {
                keep.push_back(i);
                scl.push_back(1.0 / std::sqrt(mu[i]));
            }
        const int kt = (int)keep.size();
        if (h->opts.verbose)
            std::fprintf(stderr, "[zolo] iteration %d: %d locked, GMRES steps %d, B-Gram mu in [%.3e, %.3e], kept %d of %d\n",
                         it, nl, h->stats.n_gmres, *std::min_element(mu.begin(), mu.end()), mumax, kt, kq);
        if (kt == 0) {
            rc = set_error(ZOLO_ENOCONV, "filtered block vanished (no eigenvalues in the interval?)");
            break;
        }
        rc = gather_cols(h, w, kq, U, keep, scl, Wm, st);
        if (rc) break;
        // Ah = W^H At W  (kt x kt), via Z = At W then Ah = W^H Z
        rc = gemm1(h, st, w.jobs, At, Wm, Zm, job(0, 1, kq, 0, 1, kq, 0, 1, kq, kq, kt, kq, 0));
        if (!rc) rc = gemm1(h, st, w.jobs, Wm, Zm, Ah, job(0, kq, 1, 0, 1, kq, 0, 1, kt, kt, kt, kq, GJ_CONJA));
        if (!rc) rc = jacobi_eig(h, w, kt, Ah, Zm, lam, st);
        if (rc) break;
        // Qt = W Z (kq x kt), Q = Y Qt (n x kt, row-major)
        rc = gemm1(h, st, w.jobs, Wm, Zm, Qt, job(0, 1, kq, 0, 1, kt, 0, 1, kq, kq, kt, kt, 0));
        if (!rc) rc = gemm1(h, st, w.jobs, Y, Qt, Q, job(0, kq, 1, 0, 1, kq, 0, kt, 1, (int)n, kt, kq, 0));
        if (rc) break;
        // the Ritz pairs ascending (a host order of the columns of Q)
        std::vector<int> ord(kt);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return lam[x] < lam[y]; });
        // residuals r_i = ||A q_i - lam_i B q_i|| / (||A||_inf ||q_i||)
        kq = kt;
        launch_spmm(h->A, kq, Q, kq, AY, kq, c128{1.0, 0.0}, false, st);
        launch_spmm(h->B, kq, Q, kq, BY, kq, c128{1.0, 0.0}, false, st);
        rc = grow(h, w.dvec, (size_t)kq * sizeof(double));
        if (rc) break;
        rc = cuda_check(cudaMemcpyAsync(w.dvec.p, lam.data(), kq * sizeof(double), cudaMemcpyHostToDevice, st), "lam");
        if (rc) break;
        k_resid_block<<<nblk(n * kq), 256, 0, st>>>(n, kq, AY, BY, (const double *)w.dvec.p, R);
        count_launch();
        rc = grow(h, w.nrm, (size_t)3 * kq * sizeof(double));
        if (rc) break;
        double *nr = (double *)w.nrm.p;
        rc = colnorm2(h, kq, R, kq, nr, st);
        if (!rc) rc = colnorm2(h, kq, Q, kq, nr + kq, st);
        if (!rc) rc = colnorm2(h, kq, BY, kq, nr + 2 * kq, st);
        if (rc) break;
        std::vector<double> hn(3 * kq);
        rc = cuda_check(cudaMemcpyAsync(hn.data(), nr, 3 * kq * sizeof(double), cudaMemcpyDeviceToHost, st), "res");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "res");
        if (rc) break;
        cudaEventRecord(e2, st);
        cudaEventSynchronize(e2);
        float ta = 0.f, tr = 0.f;
        cudaEventElapsedTime(&ta, e0, e1);
        cudaEventElapsedTime(&tr, e1, e2);
        t_apply += ta;
        t_rr += tr;
        res_all.assign(kq, 0.0);
        double relerr = 0.0;
        const double ab = std::max(std::fabs(a), std::fabs(b));
        for (int i = 0; i < kq; ++i) res_all[i] = std::sqrt(hn[i]) / (h->normA_inf * std::sqrt(std::max(hn[kq + i], 1e-300)));
        sel.clear();
        double worst = 0.0;
        for (int t = 0; t < kq; ++t) {
            const int i = ord[t];
            if (lam[i] > a && lam[i] < b) {
                sel.push_back(i);
                worst = std::max(worst, res_all[i]);
                relerr = std::max(relerr, std::sqrt(hn[i]) / (ab * std::sqrt(std::max(hn[2 * kq + i], 1e-300))));
            }
        }
        h->stats.max_resid = worst;
        h->stats.relerr = relerr;
        if (h->opts.verbose)
            std::fprintf(stderr, "[zolo] iteration %d: Ritz values in [%.6f, %.6f], %d inside (a, b), worst residual %.3e\n",
                         it, *std::min_element(lam.begin(), lam.end()), *std::max_element(lam.begin(), lam.end()),
                         (int)sel.size(), worst);
        // An empty selection after the first application is not convergence: a random start
        // block leaves the filter's equiripple tail on every direction outside (a, b), which
        // drags the Rayleigh quotients of a narrow interval's pairs outside it; accept "no
        // eigenvalue in (a, b)" only when two applications in a row find none.
        if (sel.empty()) {
            if (empty_before) {
                converged = true;
                break;
            }
            empty_before = true;
            nl = 0;
            continue;
        }
        empty_before = false;
        if (worst <= tol) {
            converged = true;
            break;
        }
        if (lock && it < itmax) {
            // locked first (converged pairs in (a, b), ascending), then the rest ascending
            std::vector<int> perm;
            for (int t = 0; t < kq; ++t) {
                const int i = ord[t];
                if (lam[i] > a && lam[i] < b && res_all[i] <= tol) perm.push_back(i);
            }
            const int nlock = (int)perm.size();
            for (int t = 0; t < kq; ++t) {
                const int i = ord[t];
                if (!(lam[i] > a && lam[i] < b && res_all[i] <= tol)) perm.push_back(i);
            }
            rc = cuda_check(cudaMemcpyAsync(w.idx.p, perm.data(), kq * sizeof(int), cudaMemcpyHostToDevice, st), "perm");
            if (rc) break;
            k_select_cols<<<nblk(n * kq), 256, 0, st>>>(n, kq, Q, kq, (const int *)w.idx.p, R, kq);
            count_launch();
            rc = cuda_check(cudaStreamSynchronize(st), "perm");
            if (rc) break;
            std::swap(w.Q, w.R);                          // the permuted block becomes Q
            std::vector<double> l2(kq), r2(kq);
            for (int t = 0; t < kq; ++t) {
                l2[t] = lam[perm[t]];
                r2[t] = res_all[perm[t]];
            }
            lam.swap(l2);
            res_all.swap(r2);
            nl = nlock;
        } else {
            nl = 0;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    if (rc) return rc;
    c128 *Q = (c128 *)w.Q.p;
    h->stats.n_iter = std::min(it, itmax);
    h->stats.t_apply_ms = t_apply;
    h->stats.t_rr_ms = t_rr;
    h->stats.n_gmres = n_gm;
    h->stats.n_solv = n_solv;
    const int nf = (int)sel.size();
    h->stats.n_found = nf;
    *n_found = nf;
    if (nf > cap) return set_error(ZOLO_EINVAL, "cap too small for the eigenpairs found");
    for (int t = 0; t < nf; ++t) {
        evals[t] = lam[sel[t]];
        if (resid) resid[t] = res_all[sel[t]];
    }
    if (nf > 0 && evecs) {
        rc = cuda_check(cudaMemcpyAsync(w.idx.p, sel.data(), nf * sizeof(int), cudaMemcpyHostToDevice, st), "sel");
        if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "sel");
        if (rc) return rc;
        k_select_cols<<<nblk(n * nf), 256, 0, st>>>(n, nf, Q, kq, (const int *)w.idx.p, evecs, ldv);
        count_launch();
        rc = cuda_check(cudaGetLastError(), "evecs");
        if (rc) return rc;
    }
    rc = cuda_check(cudaStreamSynchronize(st), "eigs");
    if (rc) return rc;
    if (stats) *stats = h->stats;
    // a converged Ritz value strictly inside a declared eigengap (a-, a+) or (b-, b+)
    // contradicts the gaps the filter was built on: the pairs near that end may be missing
    if (h->fi.kind == ZOLO_FILTER_ZOLO) {
        const double m = 1e-9 * (b - a);
        const double *g = h->fi.gap;
        for (int i = 0; i < kq; ++i) {
            if (!(res_all[i] <= tol)) continue;
            const double x = lam[i];
            if ((x > g[0] + m && x < g[1] - m) || (x > g[2] + m && x < g[3] - m))
                return set_error(ZOLO_EGAP, "converged Ritz value " + std::to_string(x) + " lies inside a declared eigengap");
        }
    }
    if (!converged)
        return set_error(ZOLO_ENOCONV, gmres_short ? "eigenpair residuals above tol (GMRES also hit gmres_m_max)"
                                                   : "eigenpair residuals above tol after n_iter_max iterations");
    return ZOLO_OK;
}

}  // namespace zolo

using namespace zolo;

extern "C" {

int zolo_apply(zolo_factor_h h, int64_t k, const void *X, int64_t ldx, void *Y, int64_t ldy, zolo_stats *stats,
               void *stream) {
    clear_error();
    if (!h || !X || !Y || k <= 0 || ldx < k || ldy < k) return set_error(ZOLO_EINVAL, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    h->stats.n_refine_max = 0;
    bool rx = false;
    int rc = ZOLO_OK;
    if (pencil_is_real(h) && h->opts.real_block) rc = block_is_real(h, k, (const c128 *)X, ldx, st, &rx);
    h->realx = rx;
    if (!rc) rc = filter_apply(h, k, (const c128 *)X, ldx, (c128 *)Y, ldy, st, stats);
    h->realx = false;
    cudaEventRecord(e1, st);
    if (rc == ZOLO_OK || rc == ZOLO_ENOCONV) {
        int rc2 = cuda_check(cudaStreamSynchronize(st), "apply");
        if (rc2) rc = rc2;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        h->stats.t_apply_ms = ms;
        if (stats) {
            stats->t_apply_ms = ms;
            stats->n_refine_max = h->stats.n_refine_max;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

int zolo_eigs_factored(zolo_factor_h h, double a, double b, int64_t k0, const void *X0, double *evals, void *evecs,
                       int64_t ldv, int64_t cap, int64_t *n_found, double *resid, zolo_stats *stats, void *stream) {
    clear_error();
    if (!h || !evals || !n_found || k0 <= 0 || k0 > h->n || !(a < b) || cap < 0 || (evecs && ldv < cap))
        return set_error(ZOLO_EINVAL, "bad argument");
    *n_found = 0;
    return eigs_factored(h, a, b, k0, (const c128 *)X0, evals, (c128 *)evecs, ldv, cap, n_found, resid, stats,
                         (cudaStream_t)stream);
}

int zolo_eigs(const zolo_csr *A, const zolo_csr *B, double a, double b, int64_t n_est, const zolo_filter_spec *spec,
              const zolo_opts *opts, double *evals, void *evecs, int64_t ldv, int64_t cap, int64_t *n_found,
              double *resid, zolo_stats *stats, void *stream) {
    clear_error();
    if (!A || !B || !evals || !n_found || !(a < b) || n_est < 0) return set_error(ZOLO_EINVAL, "bad argument");
    CsrHost ha, hb;
    int rc0 = csr_host_view(A, ha, &A);
    if (!rc0) rc0 = csr_host_view(B, hb, &B);
    if (rc0) return rc0;
    zolo_opts o;
    if (opts) o = *opts; else zolo_opts_default(&o);
    zolo_filter_spec fs;
    if (spec) {
        fs = *spec;
    } else {
        const double g = (o.gap_rel > 0 ? o.gap_rel : 1e-2) * (b - a);
        fs.a_minus = a - g;
        fs.a_plus = a;
        fs.b_minus = b;
        fs.b_plus = b + g;
        fs.r1 = o.r1 > 0 ? o.r1 : 2;
        fs.r2 = o.r2 > 0 ? o.r2 : 2;
        fs.eps = 0.0;
    }
    zolo_filter f = nullptr;
    int rc = zolo_filter_build(&fs, &f);
    if (rc) return rc;
    zolo_factor_h h = nullptr;
    rc = zolo_factor(A, B, f, nullptr, &o, stream, &h);
    if (rc) {
        zolo_filter_destroy(f);
        return rc;
    }
    int64_t k = o.k > 0 ? o.k : (int64_t)std::ceil(1.5 * (double)n_est) + 8;
    k = std::min<int64_t>(k, A->n);
    const double tf = h->stats.t_factor_ms;
    rc = zolo_eigs_factored(h, a, b, k, nullptr, evals, evecs, ldv, cap, n_found, resid, stats, stream);
    if (stats) {
        stats->t_factor_ms = tf;
        stats->t_total_ms = tf + stats->t_apply_ms + stats->t_rr_ms;
    }
    zolo_factor_destroy(h);
    zolo_filter_destroy(f);
    return rc;
}

}  // extern "C"
