// Internal declarations shared by the host (.cpp) and device (.cu) parts of the
// library.  Not part of the ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>
#include <complex>
#include "../../include/zolo.h"

namespace zolo {

using cplx = std::complex<double>;

// thread-local last-error message; returns `status` for chaining
int set_error(int status, const std::string &msg);
void clear_error();

// ------------------------------------------------------------------ filter
struct Zolo {            // Z_2r(x; l) of Theorem 1
    int r = 0;
    double ell = 0, M = 0, delta = 0, zmax = 0;
    std::vector<double> c;      // c_1 .. c_{2r-1}
    std::vector<double> a;      // partial-fraction weights a_1..a_r (Prop. 1)
    double operator()(double x) const;    // M * product form
};
int zolo_build(int r, double ell, Zolo &z);

}  // namespace zolo

struct zolo_filter_s {
    zolo_filter_spec spec;
    int kind = ZOLO_FILTER_ZOLO;
    zolo::Zolo inner, outer;
    double alpha = 0, beta = 0, gamma = 0, ell1 = 0, ell2 = 0, delta0 = 0;
    zolo_filter_info info;
    double eval(double x) const;
};

// ------------------------------------------------------------------ symbolic
struct zolo_symbolic_s {
    int64_t n = 0;
    int32_t nnodes = 0, nlevels = 0;
    std::vector<int32_t> perm, iperm;     // new -> old, old -> new
    std::vector<int32_t> first, npiv, parent, level, lo;   // lo: smallest node of subtree
    std::vector<int64_t> uptr;            // update rows of node s: urows[uptr[s]..uptr[s+1])
    std::vector<int32_t> urows;           // new numbering, ascending
    std::vector<std::vector<int32_t>> children;
    std::vector<int32_t> by_level;        // nodes sorted by (level, id)
    std::vector<int32_t> level_ptr;       // nodes of level L: by_level[level_ptr[L]..level_ptr[L+1])
    zolo_symbolic_info info;
    int32_t nf(int s) const { return npiv[s] + (int32_t)(uptr[s + 1] - uptr[s]); }
    int32_t nu(int s) const { return (int32_t)(uptr[s + 1] - uptr[s]); }
    // position of new index t inside the rows of front s (pivots first, then update rows)
    int32_t pos_in(int s, int32_t t) const;
};

namespace zolo {
// Host copy of a CSR given in device memory or with complex64 values.
struct CsrHost {
    zolo_csr c;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> v;
};
// *use = `in` itself when it is a host CSR of double / complex double values, else a host
// complex128 / double copy held by `buf`.  EINVAL for an unknown mem or dtype, ECUDA when a
// device copy fails.
int csr_host_view(const zolo_csr *in, CsrHost &buf, const zolo_csr **use);
// Validate a host CSR; fills `complex_` with whether it carries complex values.
int check_csr(const zolo_csr *M, const char *name, bool &complex_);
// Build the symbolic analysis of pattern(A) U pattern(B).
int analyze(const zolo_csr *A, const zolo_csr *B, const zolo_opts &opts, zolo_symbolic_s &S);
}  // namespace zolo
