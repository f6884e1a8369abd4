// The factor handle: device copies of the pencil, the multifrontal fronts of the r1
// shifted matrices and the launch schedules that drive them.  Internal.
#pragma once
#include <vector>
#include "zolo_internal.h"
#include "kernels.cuh"

namespace zolo {

struct Launch {
    int64_t off = 0;     // first job in the device job array
    int cnt = 0;         // jobs
    int ntiles = 0;      // CTAs
    double flops = 0.0;  // executed flops of a GEMM launch (8 m n k summed over jobs)
    double bytes = 0.0;  // algorithmic bytes of its jobs: A, B read once, C written (and read if
                         // accumulated), at the launch's element size
    int bm = 64;         // GEMM tile height of the launch
    int bn = 64;         // GEMM tile width
    bool tc = false;     // complex64 tensor-core kernel (bm = bn = 128)
    int wmax = 128;      // tensor-core launches: widest C tile of any job
    int64_t tmoff = -1;  // first entry of the launch's tile -> job map (-1: none)
};

// one step of a level's factorisation: diagonal blocks, the two panels, Schur update
struct FStep {
    Launch diag, panelL, panelU, schur;
};

struct FLevel {
    int64_t pool_lo = 0, pool_hi = 0;              // the level's fronts are contiguous
    int64_t finv_lo = 0, finv_hi = 0;              // ... and so are their pivot-block inverses
    Launch eye;                                     // identity start of those inverses
    Launch tpose;                                   // their in-place transposes (row- to column-major)
    std::vector<Launch> linv, uinv;                // (apply, update) pairs per panel step
    int64_t asmA_lo = 0, asmA_hi = 0, asmB_lo = 0, asmB_hi = 0;
    std::vector<Launch> eadd;                      // one per child slot
    std::vector<FStep> steps;
};

// operand bases of a GEMM launch
enum { BK_POOL = 0, BK_INVBLK = 1, BK_INVFULL = 2, BK_W = 3, BK_YP = 4 };

// one launch of the block solve: rows kernel or GEMM
struct SOp {
    int kind = 0;        // SOP_*
    int abase = 0, bbase = BK_W, cbase = BK_W;      // GEMM operand bases (BK_*)
    Launch L;            // rows jobs, or GEMM jobs for K^-1
    Launch LH;           // GEMM jobs for K^-H
};
enum { SOP_GATHER_IN = 0, SOP_EADD = 1, SOP_GEMM = 2, SOP_GATHER_OUT = 3, SOP_SCATTER_OUT = 4, SOP_ZERO = 5 };

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct KrylovWork;                                 // GMRES / Rayleigh-Ritz buffers (krylov.cu)
void krylov_free(KrylovWork *w);
}  // namespace zolo

struct zolo_factor_s {
    int device = 0;
    int prec = ZOLO_PREC_FP64;
    int64_t n = 0;
    int r1 = 0;
    bool cplx = false;
    zolo_opts opts;
    zolo_filter_info fi;
    zolo_symbolic_s sym;
    zolo::DevCSR A, B;
    double normA_inf = 0.0;
    std::vector<zolo::Buf> owned;                  // every device allocation

    // front layout (per node)
    std::vector<int64_t> f_off, f_inv, f_wrow, f_rows, f_rel, f_finv;
    int64_t pool_elems = 0, inv_elems = 0, wrows = 0, finv_elems = 0;
    void *pool[ZOLO_MAX_R] = {};                   // per pole: fronts (T)
    void *inv[ZOLO_MAX_R] = {};                    // per pole: diagonal-block inverses (T)
    void *finv[ZOLO_MAX_R] = {};                   // per pole: full pivot-block inverses, L then U
                                                   // (np x np each, column-major once formed)
    // pre-split solve operands (MIXED): per front, the float offsets of the tensor-core planes
    // of its [Linv, Uinv, L_up, U_pu] (-1: none), one buffer per pole, rebuilt by every
    // factorisation
    std::vector<int64_t> f_ps;
    int64_t ps_floats = 0, ps_blocks = 0;
    int n_psjobs = 0;
    void *presplit[ZOLO_MAX_R] = {};
    zolo::PJob *d_psjobs = nullptr;
    int32_t *d_rows = nullptr, *d_rel = nullptr;
    int64_t *d_asm = nullptr;                      // [srcA | dstA | srcB | dstB]
    int64_t nA_asm = 0, nB_asm = 0;

    // factorisation schedule
    std::vector<zolo::FLevel> flev;
    zolo::DJob *d_djobs = nullptr;
    zolo::GJob *d_fjobs = nullptr;
    int32_t *d_ftmap = nullptr;                    // tile -> job maps of the factorisation launches
    zolo::RJob *d_ejobs = nullptr;
    int64_t n_djobs = 0;
    double *d_minpiv = nullptr;
    int *d_err = nullptr;

    // solve schedule (built for one k at a time)
    int64_t k_sched = -1;
    std::vector<zolo::SOp> fwd, bwd;
    zolo::GJob *d_sjobs = nullptr;
    int32_t *d_stmap = nullptr;                    // tile -> job maps of the solve launches
    zolo::RJob *d_rjobs = nullptr;
    zolo::Buf sched_buf;
    void *W[zolo::MAX_INST] = {};                  // front workspaces (T), wrows x k each
    void *Yp[zolo::MAX_INST] = {};                 // pivot-row intermediates (T), n x k each
    zolo::Buf w_buf;

    // scratch for the inner operator and for refinement (complex128, n x k blocks)
    zolo::Buf scratch, rscratch;
    double *d_norms = nullptr;                     // column norms, 2 * MAX_INST * kmax
    int64_t norms_k = 0;
    zolo::Buf colpart;                             // partial sums of the column-norm reduction
    bool realx = false;                            // the current filter application works on real
                                                   // blocks of a real pencil: one solve per pole

    zolo::KrylovWork *kw = nullptr;
    double gmres_tol_now = 0.0;                    // tolerance of the current filter application
    double refine_tol_now = 0.0;                   // relaxed refinement tolerance of the current
                                                   // inner application (0: opts.refine_tol)
    bool inner_failed = false;                     // an inner solve of the current GMRES failed
    int *d_negcnt = nullptr;                       // inertia: negative pivots per pole
    bool count_neg = false;
    bool real_fac = false;                         // real matrices (real pencil, real shifts)
    zolo_stats stats;
};

namespace zolo {
int dev_alloc(zolo_factor_s *h, size_t bytes, void **out);
void dev_release(zolo_factor_s *h, Buf &b);        // frees b if the handle owns it
int cuda_check(cudaError_t e, const char *what);
int factor_numeric(zolo_factor_s *h, cudaStream_t st);
int ensure_solve_schedule(zolo_factor_s *h, int64_t k);
// Batched block solves: for instance z < ninst, Xout[z] = K_{pole[z]}^{-1} Xin[z] (herm 0)
// or K^{-H} Xin[z] (herm 1), on the stored factors (no refinement).
int solve_batch(zolo_factor_s *h, int ninst, const int *pole, const int *herm, int64_t k, const c128 *const *Xin,
                int64_t ldin, c128 *const *Xout, int64_t ldout, cudaStream_t st);
// Same with FP64 iterative refinement when the factors are complex64.
int solve_refined(zolo_factor_s *h, int ninst, const int *pole, const int *herm, int64_t k, const c128 *const *Xin,
                  int64_t ldin, c128 *const *Xout, int64_t ldout, cudaStream_t st, int *n_refine);
int refine_loop(zolo_factor_s *h, int ninst, const int *pole, const int *herm, int64_t k, const c128 *const *Xin,
                int64_t ldin, c128 *const *Xout, int64_t ldout, cudaStream_t st, int *n_refine);
// Y = G X (eq. solve).  When Xs (the double-float planes of X: n k float2 hi parts, then
// n k remainders, ld = k) is given and the pencil has double-float values, B X is formed
// from them on the FP32 pipe.
int apply_inner(zolo_factor_s *h, int64_t k, const c128 *X, int64_t ldx, c128 *Y, int64_t ldy, cudaStream_t st,
                const float2 *Xs = nullptr);
// scratch block of complex128 with at least `blocks` n x k blocks
int ensure_scratch(zolo_factor_s *h, int64_t k, int blocks, c128 **out);
// partial-sum buffer of launch_colnorm2 for blocks of up to k columns
int ensure_colpart(zolo_factor_s *h, int64_t k, double **out);
// sum of squared column norms of X (n x k) into out[0..k) on the device
int colnorm2(zolo_factor_s *h, int64_t k, const c128 *X, int64_t ldx, double *out, cudaStream_t st,
             bool imag_only = false);
// true when the pencil's values are all real (A and B)
inline bool pencil_is_real(const zolo_factor_s *h) { return h->A.vr && h->B.vr; }
// whether every entry of the n x k device block X has a zero imaginary part (synchronises)
int block_is_real(zolo_factor_s *h, int64_t k, const c128 *X, int64_t ldx, cudaStream_t st, bool *real);
}  // namespace zolo
