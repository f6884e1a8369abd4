/*
 * zolo.h -- C ABI of the GB300 Zolotarev-filter interior eigensolver.
 *
 * Problem (Section 1, eq. IGEVP): for a sparse Hermitian-definite pencil (A, B)
 * (A, B Hermitian, B positive definite) and an interval (a, b), find every
 * eigenpair A x = lambda B x with a < lambda < b.  The method (Li & Yang,
 * arXiv:1701.08935) applies the rational filter
 *      R_ab(x) = ( Z_2r2( Zhat_2r1( T(x); l1 ); l2 ) + 1 ) / 2          (eq. R2)
 * to a block of vectors inside subspace iteration (Algorithm 1), evaluating it with
 * the hybrid method of Algorithm 2: r1 factored shifted matrices K_j = A - sigma_j B
 * give the inner operator G = Zhat(T(B^-1 A)) (eq. solve), and shift-invariant GMRES
 * over the 2 r2 shifts +-i sqrt(c_2j-1) gives Z(G) (eq. solve2).
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status (ZOLO_OK = 0); nothing throws across the
 *    ABI.  zolo_last_error() gives a thread-local message for the last failure.
 *  - Matrices enter as CSR (zolo_csr), in host or device memory: 0-based, n x n, full
 *    pattern (both triangles), column indices sorted inside each row; the library
 *    copies what it keeps, the caller keeps ownership of its arrays.
 *  - Vector blocks are DEVICE arrays of complex double (interleaved re, im) laid out
 *    row-major: entry (i, c) of an n x k block sits at X[i*ld + c], ld >= k (a
 *    contiguous torch tensor of shape (n, k) has ld = k).  Rows use the caller's
 *    (original) numbering.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls that return results to the host synchronise that stream.
 *  - Handles own their device memory until the matching destroy call.
 *  - Single GPU, the current CUDA device at the time of the call.
 */
#ifndef ZOLO_H
#define ZOLO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define ZOLO_OK        0
#define ZOLO_EINVAL    1  /* bad argument: shapes, ordering, non-finite, a- >= a+ ... */
#define ZOLO_ENOTHERM  2  /* A or B not Hermitian within a relative 1e-12 */
#define ZOLO_ENOMEM    3  /* device or host allocation failed */
#define ZOLO_ESINGULAR 4  /* zero / non-finite pivot in a front */
#define ZOLO_ENOCONV   5  /* residuals above tolerance after the allowed iterations */
#define ZOLO_ETIMEOUT  6  /* a bounded device wait expired */
#define ZOLO_ECUDA     7  /* a CUDA runtime call failed */
#define ZOLO_EGAP      8  /* a converged Ritz value lies inside a declared eigengap */

/* ---- value types of CSR arrays ------------------------------------------ */
#define ZOLO_R64  1       /* double */
#define ZOLO_C128 2       /* complex double, interleaved (re, im) */
#define ZOLO_C64  3       /* complex float, interleaved (re, im); widened to complex double */

/* ---- where the CSR arrays live ------------------------------------------- */
#define ZOLO_HOST   0     /* host memory (default) */
#define ZOLO_DEVICE 1     /* device memory of the current GPU: the library copies the arrays
                             to the host once per call (the ordering and the symbolic
                             analysis run there) and keeps its own device copy */

/* ---- filter kinds --------------------------------------------------------- */
#define ZOLO_FILTER_ZOLO 0  /* the composite Zolotarev filter R_ab (eq. R2), Algorithm 2      */
#define ZOLO_FILTER_CITZ 1  /* contour integral (eq. contourintegral) on the circle through a
                               and b, trapezoidal rule (Section 1.1): factored poles only   */
#define ZOLO_FILTER_CIGQ 2  /* the same contour, Gauss-Legendre rule on each half circle   */

/* ---- arithmetic of the factorisation and solves ------------------------- */
#define ZOLO_PREC_FP64  0 /* complex128 everywhere */
#define ZOLO_PREC_MIXED 1 /* complex64 fronts and solves (FP64 diagonal blocks), each
                             shifted solve refined to FP64 accuracy against the FP64
                             pencil; Krylov basis, least squares, Gram and Rayleigh-Ritz
                             stay FP64 */

/* ---- complex64 GEMM engine of the mixed-precision fronts and solves ------ */
#define ZOLO_TC_AUTO   0  /* tcgen05 tensor cores (3xTF32 split, FP32 accumulation) for
                             launches whose fronts average >= 256 rows, FP32 FMA for the rest */
#define ZOLO_TC_OFF    1  /* FP32 FMA only */
#define ZOLO_TC_ALWAYS 2  /* tensor cores for every complex64 GEMM launch */

#define ZOLO_MAX_R 16     /* largest r1, r2 accepted */

typedef struct {
    int64_t        n;        /* rows = columns */
    int64_t        nnz;
    const int64_t *row_ptr;  /* n+1 entries */
    const int32_t *col_idx;  /* nnz entries, sorted within each row */
    const void    *val;      /* nnz values of type `dtype` */
    int32_t        dtype;    /* ZOLO_R64, ZOLO_C128 or ZOLO_C64 */
    int32_t        mem;      /* ZOLO_HOST (0) or ZOLO_DEVICE: where the three arrays live */
} zolo_csr;

/* Filter specification: the eigengaps (a-, a+) around a and (b-, b+) around b
 * (Section 1.2; the gap-estimation step of Algorithm 2).  a_minus may be -INFINITY (the
 * lowest slice, as in Section 3.1).  r1 / r2 are the inner (factored) and outer
 * (GMRES) Zolotarev orders.  Orders chosen from eps (Remark after Algorithm 2: the error
 * of R_ab is (1 - S(l1; l1)) / 2, a function of (r1, r2) alone, evaluated without any
 * matrix): r1, r2 <= 0 -> the smallest r = r1 = r2 with delta0 <= eps; r1 > 0, r2 <= 0
 * -> the smallest r2 for that r1 (the factorisation count is fixed, e.g. by memory);
 * r1 <= 0, r2 > 0 -> the smallest r1 for that r2.                               */
typedef struct {
    double  a_minus, a_plus, b_minus, b_plus;
    int32_t r1, r2;
    double  eps;
} zolo_filter_spec;

/* Everything the filter-construction steps of Algorithm 2 compute. */
typedef struct {
    double  alpha, beta, gamma;         /* T(x) = gamma (x - alpha)/(x - beta)  (eq. mo) */
    double  ell1, ell2;                 /* eq. req and l2 = Zhat(l1; l1)              */
    double  delta1;                     /* error of Z_2r1(.; l1)                       */
    double  delta0;                     /* max |R_ab - S_ab| on the gap complement (Thm 3) */
    int32_t r1, r2;
    double  M_hat;                      /* M of Zhat_2r1 (divided by max Z)            */
    double  const_hat;                  /* M_hat sum_j a_hat_j gamma/(gamma^2 + c_hat_j) */
    double  a_hat[ZOLO_MAX_R];          /* Prop. 1 weights of the inner function       */
    double  c_hat[ZOLO_MAX_R];          /* c_hat_{2j-1}                                */
    double  sigma_hat[2 * ZOLO_MAX_R];  /* factored poles (re, im), Prop. 2            */
    double  w_hat[2 * ZOLO_MAX_R];      /* their weights (re, im), M_hat included      */
    double  M;                          /* M of the outer Z_2r2(.; l2)                 */
    double  a[ZOLO_MAX_R];              /* outer weights a_j (Cor. 1)                  */
    double  c[ZOLO_MAX_R];              /* outer c_{2j-1}: shifts are +-i sqrt(c)      */
    double  gap[4];                     /* the eigengaps a-, a+, b-, b+ of the spec      */
    int32_t kind;                       /* ZOLO_FILTER_ZOLO, ZOLO_FILTER_CITZ or _CIGQ   */
    int32_t npoles;                     /* contour filters: quadrature points (2 r1)     */
} zolo_filter_info;

/* Options.  zolo_opts_default() fills the documented defaults. */
typedef struct {
    int32_t  grid[3];      /* grid dims for geometric nested dissection (vertex id
                              x + nx (y + ny z)); grid[0] <= 0: no geometry, nested
                              dissection by level structures of the pattern's graph
                              (George & Liu)                                    */
    int32_t  leaf_max;     /* nested-dissection leaf size (default 32)            */
    int32_t  precision;    /* ZOLO_PREC_FP64 (default) or ZOLO_PREC_MIXED         */
    int32_t  gmres_m_max;  /* GMRES steps at most (default 100)                   */
    double   gmres_tol;    /* stop when, for every column c, the filtered-column error
                              bound sum_s |omega_s| res_s / sqrt(l2^2 + |s|^2) is
                              <= gmres_tol * ||x_c|| (res_s: shift s least-squares
                              residual; default 1e-12)                           */
    int32_t  refine_max;   /* refinement steps per shifted solve, MIXED (default 8) */
    double   refine_tol;   /* refinement stops at ||b - K x|| <= refine_tol ||b|| (1e-12),
                              or when the residual stalls below 1e-10 (FP64 floor)  */
    int32_t  n_iter_max;   /* subspace iterations at most (default 4)             */
    double   tol;          /* eigenpair residual ||Ax - lam Bx||/(||A||_inf ||x||) (1e-10) */
    double   drop_tol;     /* B-Gram eigenvalues below max(drop_tol, (10 tol_g)^2) * max
                              are dropped, tol_g the GMRES tolerance of that pass (1e-14) */
    int32_t  k;            /* subspace dimension; <= 0: ceil(1.5 n_est) + 8        */
    int32_t  r1, r2;       /* filter orders used by zolo_eigs (default 2, 2)       */
    double   gap_rel;      /* zolo_eigs without gaps: a- = a - g, b+ = b + g with
                              g = gap_rel (b - a) (default 1e-2)                  */
    uint64_t seed;         /* starting block: SplitMix64-seeded normal entries     */
    int32_t  verbose;      /* 0 silent, 1 stages to stderr                         */
    int32_t  tensor_core;  /* ZOLO_PREC_MIXED GEMMs: ZOLO_TC_AUTO (default), _OFF, _ALWAYS */
    int32_t  gmres_chunk;  /* GMRES columns per chunk at most (the columns are independent
                              problems); <= 0: as many as fit a Krylov basis of
                              min(100 GiB, 60% of free device memory)           */
    int32_t  split_k_min;  /* block solves: a launch with fewer than ~4 waves of tiles splits
                              the inner extent of its accumulating products over several
                              CTAs when that extent is >= split_k_min (default 512) */
    int32_t  real_block;   /* real pencils: 1 (default) keeps real blocks real -- a real
                              starting block, one solve per pole (K_j^-H B x = conj(K_j^-1 B x)
                              for real A, B, x: eq. solve), real Krylov vectors; 0 runs the
                              complex arithmetic of a Hermitian pencil              */
    int32_t  lock;         /* Algorithm 1: 1 (default) locks converged Ritz pairs in (a, b)
                              (they are no longer filtered; each Rayleigh-Ritz step still
                              includes them), 0 filters the whole block every iteration */
} zolo_opts;

/* Counters and timings filled by zolo_apply / zolo_eigs (n_solv as Section 3 counts it). */
typedef struct {
    int32_t n_iter;            /* subspace iterations run                      */
    int32_t n_gmres;           /* GMRES steps of the last filter application   */
    int64_t n_solv;            /* shifted solves: r * n_ss * n_iter * n_gmres   */
    int32_t n_refine_max;      /* largest refinement count of one solve (MIXED) */
    int32_t n_found;           /* eigenpairs returned                           */
    double  gmres_res;         /* worst relative least-squares residual         */
    double  max_resid;         /* worst eigenpair residual                      */
    double  relerr;            /* e_{Lambda,X} of eq. relerr                    */
    double  t_factor_ms, t_apply_ms, t_rr_ms, t_total_ms;
    double  min_pivot;         /* smallest |pivot| over all fronts and poles    */
    double  flops_factor;      /* algorithmic flops of one factorisation set    */
    double  flops_solve;       /* algorithmic flops of one block solve (k = 1)  */
    int64_t solve_cols;        /* block-solve columns run since the factorisation
                                  (instances x columns, refinement included)   */
} zolo_stats;

typedef struct zolo_filter_s   *zolo_filter;
typedef struct zolo_symbolic_s *zolo_symbolic;
typedef struct zolo_factor_s   *zolo_factor_h;

typedef struct {
    int64_t n, nnodes, nlevels;
    int64_t nnz_factor;        /* entries of L below the diagonal held by fronts     */
    int64_t front_entries;     /* sum over fronts of nf^2 (dense front storage)      */
    int64_t update_rows;       /* sum over fronts of the update-row counts           */
    int32_t max_front, max_pivots;
    double  flops_lu;          /* real flops of one complex no-pivot LU (all fronts) */
} zolo_symbolic_info;

/* ---- misc ---------------------------------------------------------------- */
void        zolo_opts_default(zolo_opts *opts);
const char *zolo_strerror(int status);
const char *zolo_last_error(void);              /* thread-local detail message */
int         zolo_version(void);                 /* 100 * major + minor */

/* ---- filter (host only; filter steps of Algorithm 2) ---------------------- */
/* Build R_ab: Moebius map from eq. req, Zolotarev coefficients (Thm 1), rescaling
 * (eq. rZ), l2, partial fractions (Prop. 1, Cor. 1) and inner poles/weights (Prop. 2).
 * EINVAL unless a- < a+ < b- < b+ (a- may be -inf), 1 <= r <= ZOLO_MAX_R.       */
int  zolo_filter_build(const zolo_filter_spec *spec, zolo_filter *out);
int  zolo_filter_get_info(zolo_filter f, zolo_filter_info *out);
/* R_ab(x[i]) for n real points, host arrays (any filter kind). */
int  zolo_filter_eval(zolo_filter f, int64_t n, const double *x, double *out);
/* The table of the Remark after Algorithm 2: delta0[(r1 - 1) rmax + (r2 - 1)] = error
 * (1 - S(l1; l1)) / 2 of R_ab with orders (r1, r2), 1 <= r1, r2 <= rmax <= ZOLO_MAX_R, for
 * the gaps of `spec` (its r1, r2, eps are ignored).  Host only.                       */
int  zolo_filter_table(const zolo_filter_spec *spec, int32_t rmax, double *delta0);
/* Contour-integral filters (Section 1.1, eq. contourintegral): the circle with centre
 * (a + b)/2 through a and b, discretised with npoles (even, 2..2 ZOLO_MAX_R) quadrature
 * points -- kind ZOLO_FILTER_CITZ: trapezoidal rule at angles 2 pi (j - 1/2) / npoles;
 * ZOLO_FILTER_CIGQ: npoles/2 Gauss-Legendre points on each half circle.  The points come in
 * conjugate pairs, so the filter is applied like the inner function of Algorithm 2: r1 =
 * npoles/2 factored poles sigma_j (upper half plane) with weights w_j and their conjugates
 * through K_j^-H (eq. solve), const = 0 and no outer GMRES (r2 = 0).  R(x) = sum over all
 * points of c_j / (z_j - x), c_j the quadrature weight times (z_j - centre) / npoles
 * (trapezoid) or the Gauss-Legendre weight times (z_j - centre) / 4.                    */
int  zolo_filter_build_contour(int32_t kind, double a, double b, int32_t npoles, zolo_filter *out);
void zolo_filter_destroy(zolo_filter f);

/* ---- ordering and symbolic analysis (host only, once per pattern) ------- */
/* Nested dissection of pattern(A) U pattern(B), assembly tree and front row lists.
 * A stencil reaching beyond nearest grid neighbours breaks the geometric
 * dissection and gives EINVAL.                                                 */
int  zolo_analyze(const zolo_csr *A, const zolo_csr *B, const zolo_opts *opts, zolo_symbolic *out);
int  zolo_symbolic_get_info(zolo_symbolic s, zolo_symbolic_info *out);
/* Export the index arrays (host buffers sized from the info): perm[n] (new -> old),
 * first[nnodes], npiv[nnodes], parent[nnodes] (-1 at the root), uptr[nnodes+1] and
 * urows[uptr[nnodes]] (update rows in new numbering, ascending per front). Any
 * pointer may be NULL to skip that array.                                        */
int  zolo_symbolic_export(zolo_symbolic s, int32_t *perm, int32_t *first, int32_t *npiv,
                          int32_t *parent, int64_t *uptr, int32_t *urows);
void zolo_symbolic_destroy(zolo_symbolic s);

/* ---- numeric factorisation (device) ------------------------------------- */
/* Upload the pencil and factor K_j = A - sigma_hat_j B, j = 1..r1, by the multifrontal
 * method on the device (the factorisation step of Algorithm 2): no-pivot LU of every front, level by
 * level, with the poles batched in each launch.  `sym` may be NULL (analysed here).
 * Device memory per pole: the fronts (sum of nf^2 entries), their pivot-block inverses, and
 * in ZOLO_PREC_MIXED a second copy of the large fronts' solve operands split into TF32
 * planes for the tensor cores (16 bytes per entry, rebuilt by every factorisation; left
 * out when it would take more than half of the free memory).
 * ESINGULAR on a zero / non-finite pivot.  Synchronises `stream`.               */
int  zolo_factor(const zolo_csr *A, const zolo_csr *B, zolo_filter f, zolo_symbolic sym,
                 const zolo_opts *opts, void *stream, zolo_factor_h *out);
/* Sylvester inertia: count[i] = number of eigenvalues of (A, B) below the real shift
 * sigma[i], i.e. the negative inertia of A - sigma_i B, read off the signs of the pivots
 * of the same no-pivot multifrontal factorisation (eq. IGEVP footnote: n_lambda is only
 * estimated; counts at a and b give it).  Always complex128 fronts whatever
 * opts->precision says (complex64 pivot signs are unreliable for indefinite shifts);
 * nshift >= 1 shifts, factored in batches of at most ZOLO_MAX_R that fit 70% of the
 * free device memory.  A shift on an eigenvalue gives ESINGULAR.  Synchronises.     */
int  zolo_inertia(const zolo_csr *A, const zolo_csr *B, zolo_symbolic sym, const zolo_opts *opts,
                  int32_t nshift, const double *sigma, int64_t *count, void *stream);
/* Re-factor an existing handle in place (same pencil, filter, options): the timed
 * factorisation step of a repeated workload.                                     */
int  zolo_refactor(zolo_factor_h h, void *stream);
void zolo_factor_destroy(zolo_factor_h h);
int  zolo_factor_get_stats(zolo_factor_h h, zolo_stats *out);

/* X := K_pole^-1 Bk (herm = 0) or K_pole^-H Bk (herm = 1) for an n x k device block,
 * through the stored factors (with refinement in MIXED precision).  Bk and X may not
 * overlap.  0 <= pole < r1.                                                      */
int  zolo_solve(zolo_factor_h h, int32_t pole, int32_t herm, int64_t k, const void *Bk,
                int64_t ldb, void *X, int64_t ldx, void *stream);
/* zolo_solve without device allocation.  The paper has no counterpart: this serves callers
 * that cannot call cudaMalloc on the calls they repeat -- hosts whose device memory belongs to
 * another component (a framework's caching allocator, a pool that must own every byte) and
 * allocation-free real-time loops, where an allocation could block or fail part-way.  Same
 * result as zolo_solve for a complex128 (ZOLO_PREC_FP64) handle; the front workspaces come
 * from one fixed device array of 32 MiB that every GPU loading the library holds until exit,
 * so (rows of all fronts + n) * k * 16 bytes must fit in it (EINVAL otherwise, with the
 * sizes).  Set-up: create the handle and call zolo_solve once with the same k (both
 * allocate); the first zolo_solve_noalloc call on a device looks up the array's device
 * address.  The current device must be the handle's (EINVAL otherwise).  All calls share
 * the array and it keeps the last call's contents (each call clears what it needs): calls
 * that overlap on the GPU race.  EINVAL for MIXED handles or a k without a schedule.
 * Asynchronous: returns once the work is queued on `stream`; synchronise it before reading X. */
int  zolo_solve_noalloc(zolo_factor_h h, int32_t pole, int32_t herm, int64_t k, const void *Bk,
                        int64_t ldb, void *X, int64_t ldx, void *stream);
/* Y := A X (which = 0) or B X (which = 1), device blocks (SpMM with the uploaded CSR). */
int  zolo_matmul(zolo_factor_h h, int32_t which, int64_t k, const void *X, int64_t ldx,
                 void *Y, int64_t ldy, void *stream);
/* Y := G X, the inner operator of eq. solve (r1 factored poles, conjugates via K^-H). */
int  zolo_apply_inner(zolo_factor_h h, int64_t k, const void *X, int64_t ldx, void *Y,
                      int64_t ldy, void *stream);
/* Y := R_ab(B^-1 A) X by the GMRES steps of Algorithm 2 (shift-invariant GMRES, one basis per
 * column shared by the 2 r2 shifts).  X, Y: n x k device blocks, may not overlap.  */
int  zolo_apply(zolo_factor_h h, int64_t k, const void *X, int64_t ldx, void *Y, int64_t ldy,
                zolo_stats *stats, void *stream);

/* ---- the eigensolver (Algorithm 1 with Algorithm 2 as the filter) ------- */
/* Eigenpairs of (A, B) in (a, b) for an existing factor handle (its filter fixes the
 * gaps); Algorithm 1 with Algorithm 2 as the filter.  k0: subspace dimension.  When
 * n_iter_max > 1 the first filter application, which starts from a random block, runs
 * GMRES to max(gmres_tol, 1e-6) only: its output is filtered again by the next iteration;
 * later applications use gmres_tol.  Results: evals[cap] ascending (host), evecs n x cap
 * device block (row-major, ld = ldv, B-orthonormal), resid[cap] host residuals
 * ||A x - lam B x|| / (||A||_inf ||x||).  X0 (device, n x k0, ld = k0) is the starting
 * block, or NULL for the seeded normal block.  On ENOCONV the best pairs found are still
 * returned.                                                                     */
int  zolo_eigs_factored(zolo_factor_h h, double a, double b, int64_t k0, const void *X0,
                        double *evals, void *evecs, int64_t ldv, int64_t cap, int64_t *n_found,
                        double *resid, zolo_stats *stats, void *stream);
/* One-call driver: filter from (a, b) and opts (gaps at gap_rel unless `spec` is given),
 * analysis, factorisation, Algorithm 1.  spec may be NULL.                      */
int  zolo_eigs(const zolo_csr *A, const zolo_csr *B, double a, double b, int64_t n_est,
               const zolo_filter_spec *spec, const zolo_opts *opts, double *evals, void *evecs,
               int64_t ldv, int64_t cap, int64_t *n_found, double *resid, zolo_stats *stats,
               void *stream);

/* Spectrum slicing (Section 3.2: eigenpairs in different spectrum ranges are independent
 * problems).  Every eigenpair with bounds[s] < lambda < bounds[s+1] for some s < nslice;
 * bounds strictly increasing.  One symbolic analysis is shared; per slice the count comes
 * from Sylvester inertia at its bounds (zolo_inertia), the filter from the slice and
 * opts->gap_rel (gaps of gap_rel times the slice width on both sides), r1 / r2 / k from opts
 * (k <= 0: ceil(1.5 count) + 8), then a factorisation and Algorithm 1.  Results are
 * concatenated slice by slice (ascending): evals[cap], evecs (device, n x cap, row-major,
 * ld = ldv, B-orthonormal within a slice), resid[cap] (may be NULL), slice_of[cap] (slice
 * index of each pair, may be NULL).  EINVAL with *n_found = the total count when cap is
 * too small.  ENOCONV when a slice did not converge or found fewer pairs than its count;
 * the pairs found are still returned.  stats: sums of times and solves, maxima of counts
 * and residuals over the slices.                                                   */
int  zolo_eigs_slices(const zolo_csr *A, const zolo_csr *B, int32_t nslice, const double *bounds,
                      const zolo_opts *opts, double *evals, void *evecs, int64_t ldv, int64_t cap,
                      int64_t *n_found, double *resid, int32_t *slice_of, zolo_stats *stats, void *stream);

/* ---- measurement hooks (no counterpart in the paper) ---------------------- */
/* Count the library's kernel launches from now on; gemm_events selects which dense-
 * product (GEMM) launches are bracketed with CUDA events: bit 0 complex64, bit 1
 * complex128 (0: none).  Process-wide, not thread-safe.                           */
int  zolo_profile_begin(int32_t gemm_events);
/* Synchronise `stream`, then report all launches, the timed GEMM launches, their summed
 * device time (ms) and the flops those GEMM jobs executed (8 m n k each).           */
int  zolo_profile_end(void *stream, int64_t *launches, int64_t *gemm_launches, double *gemm_ms,
                      double *gemm_flops);
/* The tcgen05 tensor-core share of the timed complex64 GEMM launches between the last
 * zolo_profile_begin and zolo_profile_end: launches, summed device time (ms), executed
 * flops (8 m n k per job).  Host values only; never fails.                         */
int  zolo_profile_tc(int64_t *launches, double *ms, double *flops);
/* Algorithmic bytes of the timed GEMM launches between the last zolo_profile_begin and
 * zolo_profile_end (each job's A and B read once, C written, and read too when the job
 * accumulates), all of them and the tensor-core subset.  Host values only.          */
int  zolo_profile_bytes(double *gemm_bytes, double *tc_bytes);

#ifdef __cplusplus
}
#endif
#endif /* ZOLO_H */
