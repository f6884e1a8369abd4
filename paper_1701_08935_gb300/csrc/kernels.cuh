// Launch arguments and launchers of the device kernels.  Internal to the library.
#pragma once
#include "device.cuh"

namespace zolo {

template <class T> struct GemmArgs {
    const GJob *jobs[MAX_INST];
    int njobs[MAX_INST];
    int ntiles[MAX_INST];
    const cx<T> *A[MAX_INST];
    const cx<T> *B[MAX_INST];
    cx<T> *C[MAX_INST];
};

template <class T> struct DiagArgs {
    const DJob *jobs;
    int njobs;
    cx<T> *pool[MAX_INST];
    cx<T> *inv[MAX_INST];
    int *err;
    double *minpiv;          // [ninst * njobs]
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
    int njobs, ntiles;
    const int32_t *rel;
    cx<T> *pool[MAX_INST];
};

enum { ROW_GATHER = 0, ROW_SCATTER = 1, ROW_EADD = 2 };
constexpr int ROWS_PER_TILE = 8;

template <class T> struct RowArgs {
    const RJob *jobs;
    int njobs, ntiles;
    const int32_t *map;
    int mode, k;
    int64_t ldw, ldx;
    cx<T> *W[MAX_INST];
    c128 *X[MAX_INST];
};

struct DevCSR {
    int64_t n = 0, nnz = 0;
    int64_t *rp = nullptr;
    int32_t *ci = nullptr;
    c128 *v = nullptr;
};

constexpr int LIN_MAX = 8;
struct LinArgs {
    int64_t n, k, ldy;
    int nterm;
    c128 coef[LIN_MAX];
    const c128 *X[LIN_MAX];
    int64_t ldx[LIN_MAX];
    c128 *Y;
};

template <class T> void launch_gemm(const GemmArgs<T> &g, int ninst, cudaStream_t st);
template <class T> void launch_diag_lu(const DiagArgs<T> &g, int ninst, cudaStream_t st);
template <class T> void launch_assemble(const AsmArgs<T> &g, int ninst, cudaStream_t st);
template <class T> void launch_extend_add(const EaddArgs<T> &g, int ninst, cudaStream_t st);
template <class T> void launch_rows(const RowArgs<T> &g, int ninst, cudaStream_t st);
void launch_spmm(const DevCSR &M, int64_t k, const c128 *X, int64_t ldx, c128 *Y, int64_t ldy, c128 s, bool acc,
                 cudaStream_t st);
void launch_lincomb(const LinArgs &a, cudaStream_t st);
// out[c] = sum_i |X[i, c]|^2 for an n x k block (deterministic two-stage reduction)
void launch_colnorm2(int64_t n, int64_t k, const c128 *X, int64_t ldx, double *out, cudaStream_t st);

}  // namespace zolo
