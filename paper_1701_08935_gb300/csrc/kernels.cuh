// Launch arguments and launchers of the device kernels.  Internal to the library.
#pragma once
#include <algorithm>
#include "device.cuh"

namespace zolo {

template <class T> struct GemmArgs {
    int bm;                              // tile height of this launch (64, or 128 for complex64)
    int bn;                              // tile width: 64 or 128 (bm = bn = 128: complex64 tensor cores)
    int real;                            // complex128 launches: all operands real (one FMA per product)
    int wmax;                            // tensor-core launches: widest C tile of any job (<= 128)
    const GJob *jobs[MAX_INST];
    const int32_t *tmap[MAX_INST];       // job of every tile of the launch, or null (binary search)
    int njobs[MAX_INST];
    int ntiles[MAX_INST];
    const cx<T> *A[MAX_INST];
    const cx<T> *B[MAX_INST];
    cx<T> *C[MAX_INST];
    const float *ps[MAX_INST];           // pre-split A planes of GJ_PRESPLIT jobs, or null
};

template <class T> struct DiagArgs {
    const DJob *jobs;
    int njobs;
    cx<T> *pool[MAX_INST];
    cx<T> *inv[MAX_INST];
    int *err;
    double *minpiv;          // [ninst * njobs]
    int *negcnt;             // optional [ninst]: pivots with negative real part
};

template <class T> struct AsmArgs {
    const int64_t *src, *dst;
    int64_t count;
    const c128 *val;
    c128 scale[MAX_INST];
    cx<T> *pool[MAX_INST];
};

template <class T> struct EaddArgs {
    const RJob *jobs;
    const int32_t *tmap;                 // job of every tile, or null (binary search)
    int njobs, ntiles;
    const int32_t *rel;
    cx<T> *pool[MAX_INST];
};

enum { ROW_GATHER = 0, ROW_SCATTER = 1, ROW_EADD = 2, ROW_ZERO = 3 };
// rows per CTA of the row kernels: about 2048 elements (8 per thread) for a block width k
inline int rows_per_tile(int64_t k) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, 2048 / std::max<int64_t>(1, k))); }

template <class T> struct RowArgs {
    const RJob *jobs;
    const int32_t *tmap;                 // job of every tile, or null (binary search)
    int njobs, ntiles;
    const int32_t *map;
    int mode, k;
    int rpt;                             // rows per CTA tile (the schedule's rows_per_tile(k))
    int64_t ldw, ldx;
    cx<T> *W[MAX_INST];
    c128 *X[MAX_INST];
};

struct DevCSR {
    int64_t n = 0, nnz = 0;
    int64_t *rp = nullptr;
    int32_t *ci = nullptr;
    c128 *v = nullptr;          // values as complex128
    double *vr = nullptr;       // the same values when all are real (else nullptr)
    float4 *vdf = nullptr;      // double-float split (re hi, re lo, im hi, im lo), mixed precision only
    float2 *vrdf = nullptr;     // double-float split of vr (hi, lo), when all values are real
};

// R_z = B_z - A X_z + s_z (M X_z) for up to MAX_INST instances (refinement residuals of
// K = A - sigma M and K^H = A - conj(sigma) M), all blocks n x k with their own ld
struct ResidArgs {
    int ninst, k;
    const c128 *Bz[MAX_INST];
    const c128 *Xz[MAX_INST];
    c128 *Rz[MAX_INST];
    c128 s[MAX_INST];
    int64_t ldb, ldx, ldr;
};
void launch_refine_resid(const DevCSR &A, const DevCSR &M, const ResidArgs &r, cudaStream_t st);
// The same residuals in double-float arithmetic on the FP32 pipe (relative rounding ~1e-14
// of sum |K||x|; used for refinement tolerances >= 1e-8).  Xs_z are the solutions split by
// launch_split_df; s_z is given as (re hi, re lo, im hi, im lo).  R_z gets FP32-accurate
// values (all a complex64 correction solve and a residual norm need).
struct ResidDfArgs {
    int ninst, k;
    const c128 *Bz[MAX_INST];
    const float4 *Xs[MAX_INST];
    c128 *Rz[MAX_INST];
    float4 s[MAX_INST];
    int64_t ldb, ldr;
};
void launch_refine_resid_df(const DevCSR &A, const DevCSR &M, const ResidDfArgs &r, cudaStream_t st);
// Y = M X with X given as double-float planes (n k float2 hi parts, then n k remainders,
// ld = k), in df64 on the FP32 pipe; Y (n x k, ld = k) gets FP64 values.
void launch_spmm_df(const DevCSR &M, int64_t k, const float2 *Xs, c128 *Y, cudaStream_t st);
// Xs[i k + c] = double-float split of X[i ldx + c] (n x k)
void launch_split_df(int64_t n, int64_t k, const c128 *X, int64_t ldx, float4 *Xs, cudaStream_t st);

constexpr int LIN_MAX = 8;
struct LinArgs {
    int64_t n, k, ldy;
    int nterm;
    int real_out;                        // 1: keep the real part of the sum only
    c128 coef[LIN_MAX];
    const c128 *X[LIN_MAX];
    int64_t ldx[LIN_MAX];
    c128 *Y;
};

// Every launch helper counts its launches; GEMM launches can also be bracketed by
// events (profiling on) so that a caller can read their summed device time.
struct LaunchCounters {
    int64_t launches = 0;          // all kernels of the library
    int64_t gemm_launches = 0;     // timed GEMM launches
    double gemm_flops = 0.0;       // executed flops of the timed GEMM jobs (8 m n k each)
    int64_t tc_launches = 0;       // the tensor-core subset of the timed GEMM launches,
    double tc_ms = 0.0;            // its summed device time (filled by prof_collect_ms)
    double tc_flops = 0.0;         // and its executed flops
    double gemm_bytes = 0.0;       // algorithmic bytes of the timed GEMM launches
    double tc_bytes = 0.0;         // ... of their tensor-core subset
};
LaunchCounters &counters();
void count_launch(int64_t n = 1);
void prof_set(int mask);          // bit 0: complex64 GEMMs, bit 1: complex128 GEMMs
double prof_collect_ms();          // synchronises the recorded events, returns the summed time
                                   // (and adds the tensor-core share to counters().tc_*)
template <class T>
void launch_gemm(const GemmArgs<T> &g, int ninst, cudaStream_t st, double flops = 0.0, double bytes = 0.0);
// complex64 tcgen05 GEMM (tiles 128 x <= 128, bm = bn = 128 in the job tiling)
void launch_gemm_tc(const GemmArgs<float> &g, dim3 grid, cudaStream_t st);
// Build the pre-split tensor-core planes of every PJob (one 16 KB block per CTA, grid.z =
// instances): instance z reads pool[z] / finv[z] and writes out[z].
struct PresplitArgs {
    const PJob *jobs;
    int njobs;
    const cx<float> *pool[MAX_INST];
    const cx<float> *finv[MAX_INST];
    float *out[MAX_INST];
};
void launch_presplit(const PresplitArgs &g, int64_t nblocks, int ninst, cudaStream_t st);
// device status word of the tensor-core GEMM: 0, or ZOLO_ETIMEOUT after an expired
// mbarrier wait (ZOLO_ECUDA when it cannot be read); `reset` clears a non-zero word
int gemm_tc_status(bool reset);
template <class T> void launch_diag_lu(const DiagArgs<T> &g, int ninst, cudaStream_t st);
template <class T> void launch_assemble(const AsmArgs<T> &g, int ninst, cudaStream_t st);
template <class T> void launch_extend_add(const EaddArgs<T> &g, int ninst, cudaStream_t st);
template <class T> void launch_rows(const RowArgs<T> &g, int ninst, cudaStream_t st);
// unit diagonals: for each job, P[dst + i (rows + 1)] = 1 and P[dst + rows^2 + i (rows + 1)] = 1
template <class T> struct EyeArgs {
    const RJob *jobs;
    const int32_t *tmap;                 // job of every tile, or null (binary search)
    int njobs, ntiles;
    cx<T> *P[MAX_INST];
};
template <class T> void launch_eye(const EyeArgs<T> &g, int ninst, cudaStream_t st);
// in-place transposes of square blocks: for each job, the rows x rows block at P[dst] (ld = rows);
// the job's CTAs (tr = tiles per side, tile0 its first CTA) take the 32 x 32 tile pairs
// (bi, bj), bi <= bj, in row order
template <class T> void launch_transpose_sq(const EyeArgs<T> &g, int ninst, cudaStream_t st);
void launch_spmm(const DevCSR &M, int64_t k, const c128 *X, int64_t ldx, c128 *Y, int64_t ldy, c128 s, bool acc,
                 cudaStream_t st);
void launch_lincomb(const LinArgs &a, cudaStream_t st);
// out[c] = sum_i |X[i, c]|^2 for an n x k block (imag_only: sum_i Im(X[i, c])^2), by a
// deterministic two-stage reduction through `part` (COLNORM_PARTS * k doubles, device)
constexpr int COLNORM_PARTS = 304;
void launch_colnorm2(int64_t n, int64_t k, const c128 *X, int64_t ldx, double *out, double *part, cudaStream_t st,
                     bool imag_only = false);

}  // namespace zolo
