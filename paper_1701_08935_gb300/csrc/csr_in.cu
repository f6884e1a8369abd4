// CSR inputs in any memory space and value type, brought to the host form the ordering,
// the symbolic analysis and the assembly maps read: host arrays, double or complex double
// values.  A host CSR of those types is used in place; anything else is copied once.
#include <cuda_runtime.h>
#include <string>
#include "zolo_internal.h"

namespace zolo {

int csr_host_view(const zolo_csr *in, CsrHost &buf, const zolo_csr **use) {
    *use = in;
    if (!in) return ZOLO_OK;                         // null is diagnosed by check_csr
    if (in->mem != ZOLO_HOST && in->mem != ZOLO_DEVICE) return set_error(ZOLO_EINVAL, "csr: mem must be ZOLO_HOST or ZOLO_DEVICE");
    if (in->dtype != ZOLO_R64 && in->dtype != ZOLO_C128 && in->dtype != ZOLO_C64)
        return set_error(ZOLO_EINVAL, "csr: dtype must be ZOLO_R64, ZOLO_C128 or ZOLO_C64");
    if (in->mem == ZOLO_HOST && in->dtype != ZOLO_C64) return ZOLO_OK;
    if (in->n <= 0 || in->nnz < 0 || !in->row_ptr || !in->col_idx || !in->val)
        return set_error(ZOLO_EINVAL, "csr: bad size or null array");
    const int64_t n = in->n, nnz = in->nnz;
    const size_t vb = in->dtype == ZOLO_R64 ? 8 : (in->dtype == ZOLO_C128 ? 16 : 8);
    buf.rp.resize(n + 1);
    buf.ci.resize(nnz);
    std::vector<unsigned char> raw(nnz * vb);
    if (in->mem == ZOLO_DEVICE) {
        cudaError_t e = cudaMemcpy(buf.rp.data(), in->row_ptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(buf.ci.data(), in->col_idx, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(raw.data(), in->val, nnz * vb, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_error(ZOLO_ECUDA, std::string("csr: copy of a device array failed: ") + cudaGetErrorString(e));
        }
    } else {
        std::copy(in->row_ptr, in->row_ptr + n + 1, buf.rp.begin());
        std::copy(in->col_idx, in->col_idx + nnz, buf.ci.begin());
        std::copy((const unsigned char *)in->val, (const unsigned char *)in->val + nnz * vb, raw.begin());
    }
    int dtype = in->dtype;
    if (dtype == ZOLO_C64) {                         // widen complex float to complex double
        buf.v.resize(2 * nnz);
        const float *f = (const float *)raw.data();
        for (int64_t p = 0; p < 2 * nnz; ++p) buf.v[p] = (double)f[p];
        dtype = ZOLO_C128;
    } else {
        buf.v.resize(dtype == ZOLO_R64 ? nnz : 2 * nnz);
        std::copy((const double *)raw.data(), (const double *)raw.data() + buf.v.size(), buf.v.begin());
    }
    buf.c.n = n;
    buf.c.nnz = nnz;
    buf.c.row_ptr = buf.rp.data();
    buf.c.col_idx = buf.ci.data();
    buf.c.val = buf.v.data();
    buf.c.dtype = dtype;
    buf.c.mem = ZOLO_HOST;
    *use = &buf.c;
    return ZOLO_OK;
}

}  // namespace zolo
