// Spectrum slicing: the eigenpairs of (A, B) in a union of contiguous intervals, one
// filtered subspace iteration per slice.  Eigenpairs in different spectrum ranges are
// independent problems (Section 3.2 computes slices separately); a slice keeps only the
// eigenvalues of its own interval, so no pair is returned twice.
//
// Host driver over the public entry points: one symbolic analysis shared by every slice,
// exact per-slice counts from Sylvester inertia at the slice boundaries (FP64 fronts), then
// per slice a filter, a factorisation and Algorithm 1 writing into its own column range of
// the caller's eigenvector block.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "zolo.h"
#include "zolo_internal.h"

using namespace zolo;

extern "C" int zolo_eigs_slices(const zolo_csr *A, const zolo_csr *B, int32_t nslice, const double *bounds,
                                const zolo_opts *opts, double *evals, void *evecs, int64_t ldv, int64_t cap,
                                int64_t *n_found, double *resid, int32_t *slice_of, zolo_stats *stats,
                                void *stream) {
    clear_error();
    if (!A || !B || !bounds || !evals || !evecs || !n_found || nslice <= 0 || ldv < cap || cap < 0)
        return set_error(ZOLO_EINVAL, "bad argument");
    for (int s = 0; s <= nslice; ++s)
        if (!std::isfinite(bounds[s]) || (s > 0 && !(bounds[s - 1] < bounds[s])))
            return set_error(ZOLO_EINVAL, "slice bounds must be finite and strictly increasing");
    *n_found = 0;
    CsrHost ha, hb;                                 // one host copy for every slice
    int rc0 = csr_host_view(A, ha, &A);
    if (!rc0) rc0 = csr_host_view(B, hb, &B);
    if (rc0) return rc0;
    zolo_opts o;
    if (opts) o = *opts; else zolo_opts_default(&o);

    zolo_symbolic sym = nullptr;
    int rc = zolo_analyze(A, B, &o, &sym);
    if (rc) return rc;
    // eigenvalue counts below every boundary (exact, from the pivots' signs)
    std::vector<int64_t> below(nslice + 1);
    rc = zolo_inertia(A, B, sym, &o, nslice + 1, bounds, below.data(), stream);
    if (rc) {
        zolo_symbolic_destroy(sym);
        return rc;
    }
    const int64_t total = below[nslice] - below[0];
    if (total > cap) {
        *n_found = total;
        zolo_symbolic_destroy(sym);
        return set_error(ZOLO_EINVAL, "cap " + std::to_string(cap) + " is below the " + std::to_string(total) +
                                          " eigenvalues in the slices");
    }
    zolo_stats acc;
    std::memset(&acc, 0, sizeof(acc));
    int worst_rc = ZOLO_OK;
    int64_t off = 0;
    const size_t esz = 2 * sizeof(double);                  // complex128 entries of evecs
    for (int s = 0; s < nslice; ++s) {
        const int64_t ns = below[s + 1] - below[s];
        if (ns == 0) continue;
        const double a = bounds[s], b = bounds[s + 1];
        const double g = (o.gap_rel > 0 ? o.gap_rel : 1e-2) * (b - a);
        zolo_filter_spec fs;
        std::memset(&fs, 0, sizeof(fs));
        fs.a_minus = a - g;
        fs.a_plus = a;
        fs.b_minus = b;
        fs.b_plus = b + g;
        fs.r1 = o.r1 > 0 ? o.r1 : 2;
        fs.r2 = o.r2 > 0 ? o.r2 : 2;
        zolo_filter f = nullptr;
        rc = zolo_filter_build(&fs, &f);
        if (rc) break;
        zolo_factor_h h = nullptr;
        rc = zolo_factor(A, B, f, sym, &o, stream, &h);
        if (rc) {
            zolo_filter_destroy(f);
            break;
        }
        const int64_t k = std::min<int64_t>(o.k > 0 ? o.k : (int64_t)std::ceil(1.5 * (double)ns) + 8, A->n);
        int64_t nf = 0;
        zolo_stats st;
        std::memset(&st, 0, sizeof(st));
        rc = zolo_eigs_factored(h, a, b, k, nullptr, evals + off, (char *)evecs + off * esz, ldv, cap - off, &nf,
                                resid ? resid + off : nullptr, &st, stream);
        zolo_stats fst;
        if (zolo_factor_get_stats(h, &fst) == ZOLO_OK) st.t_factor_ms = fst.t_factor_ms;
        zolo_factor_destroy(h);
        zolo_filter_destroy(f);
        if (rc == ZOLO_ENOCONV) {
            worst_rc = ZOLO_ENOCONV;
            rc = ZOLO_OK;
        }
        if (rc) break;
        if (slice_of)
            for (int64_t i = 0; i < nf; ++i) slice_of[off + i] = s;
        off += nf;
        acc.n_iter = std::max(acc.n_iter, st.n_iter);
        acc.n_gmres = std::max(acc.n_gmres, st.n_gmres);
        acc.n_solv += st.n_solv;
        acc.n_refine_max = std::max(acc.n_refine_max, st.n_refine_max);
        acc.gmres_res = std::max(acc.gmres_res, st.gmres_res);
        acc.max_resid = std::max(acc.max_resid, st.max_resid);
        acc.relerr = std::max(acc.relerr, st.relerr);
        acc.t_factor_ms += st.t_factor_ms;
        acc.t_apply_ms += st.t_apply_ms;
        acc.t_rr_ms += st.t_rr_ms;
        acc.min_pivot = (acc.min_pivot == 0.0) ? st.min_pivot : std::min(acc.min_pivot, st.min_pivot);
        acc.flops_factor += st.flops_factor;
        acc.solve_cols += st.solve_cols;
    }
    zolo_symbolic_destroy(sym);
    *n_found = off;
    acc.n_found = (int32_t)off;
    acc.t_total_ms = acc.t_factor_ms + acc.t_apply_ms + acc.t_rr_ms;
    if (stats) *stats = acc;
    if (rc) return rc;
    if (worst_rc) return set_error(worst_rc, "some slice did not converge; its best pairs are returned");
    if (off != total)
        return set_error(ZOLO_ENOCONV, "found " + std::to_string(off) + " eigenpairs where inertia counts " +
                                           std::to_string(total));
    return ZOLO_OK;
}
