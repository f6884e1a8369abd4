// zolo_solve_noalloc: the block solve of zolo_solve with its front workspaces taken from a
// fixed, file-scope device array instead of device allocations.
//
// Who needs it: callers that cannot call cudaMalloc on the calls they repeat -- hosts whose
// device memory is managed by another component (a framework's caching allocator or a
// memory pool that must own every byte), and allocation-free real-time loops, where an
// allocation could block or fail part-way through.  They create the factor handle and run
// one zolo_solve with their block width at set-up (both allocate); afterwards this entry
// point allocates nothing.
//
// Limits: complex128 (ZOLO_PREC_FP64) handles only (the mixed-precision path needs
// refinement buffers); (rows of all fronts + n) * k * 16 bytes must fit NOALLOC_BYTES.
// The array is shared by every call and keeps the last call's contents: the workspaces are
// cleared at the start of each call, and calls that overlap on the GPU (different streams,
// or the same handle from several threads) race on it.  The call is asynchronous: it
// returns once its work is queued on `stream`; synchronise that stream before reading X.
#include <cstring>
#include "factor.h"

namespace zolo {
namespace {

constexpr size_t NOALLOC_BYTES = size_t(32) << 20;      // 32 MiB, held by every GPU that loads the library
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEV = 64;
void *g_scratch_dev[NOALLOC_MAX_DEV] = {};               // device address of the array, per device

// Device address of the array on the current device (looked up once per device; the
// symbol name is only a host-side stand-in and must not be passed to kernels).
int scratch_address(void **out) {
    int dev = 0;
    int rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= NOALLOC_MAX_DEV) return set_error(ZOLO_EINVAL, "device ordinal out of range");
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        rc = cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
        if (rc) return rc;
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return ZOLO_OK;
}

}  // namespace
}  // namespace zolo

using namespace zolo;

extern "C" int zolo_solve_noalloc(zolo_factor_h h, int32_t pole, int32_t herm, int64_t k, const void *Bk, int64_t ldb,
                                  void *X, int64_t ldx, void *stream) {
    clear_error();
    if (!h || !Bk || !X || k <= 0 || ldb < k || ldx < k || pole < 0 || pole >= h->r1 || (herm != 0 && herm != 1))
        return set_error(ZOLO_EINVAL, "bad argument");
    if (h->prec != ZOLO_PREC_FP64)
        return set_error(ZOLO_EINVAL, "zolo_solve_noalloc supports complex128 (ZOLO_PREC_FP64) handles only");
    if (h->k_sched != k)
        return set_error(ZOLO_EINVAL, "no solve schedule for this block width: call zolo_solve once with k = " +
                                          std::to_string(k) + " at set-up");
    const size_t wbytes = (size_t)h->wrows * k * sizeof(c128);
    const size_t ybytes = (size_t)h->n * k * sizeof(c128);
    if (wbytes + ybytes > NOALLOC_BYTES)
        return set_error(ZOLO_EINVAL, "workspace of " + std::to_string(wbytes + ybytes) +
                                          " bytes exceeds the fixed no-allocation array of " +
                                          std::to_string(NOALLOC_BYTES) + " bytes");
    int cur = -1;
    int rc = cuda_check(cudaGetDevice(&cur), "cudaGetDevice");
    if (rc) return rc;
    if (cur != h->device)           // the array is per device; the factors live on h->device
        return set_error(ZOLO_EINVAL, "current device " + std::to_string(cur) + " is not the handle's device " +
                                          std::to_string(h->device));
    void *base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    c128 *W = (c128 *)base;
    c128 *Yp = (c128 *)((char *)base + wbytes);
    rc = cuda_check(cudaMemsetAsync(W, 0, wbytes, st), "clear W");
    if (!rc) rc = cuda_check(cudaMemsetAsync(Yp, 0, ybytes, st), "clear Y");
    if (rc) return rc;
    // the handle's forward / backward launch lists, with the workspaces redirected
    auto run = [&](const std::vector<SOp> &ops) {
        for (const SOp &o : ops) {
            if (o.kind == SOP_GEMM) {
                GemmArgs<double> g;
                std::memset(&g, 0, sizeof(g));
                g.bm = o.L.bm;
                g.bn = o.L.bn;
                const Launch &L = herm ? o.LH : o.L;
                auto basep = [&](int kind) -> c128 * {
                    switch (kind) {
                        case BK_POOL: return (c128 *)h->pool[pole];
                        case BK_INVBLK: return (c128 *)h->inv[pole];
                        case BK_INVFULL: return (c128 *)h->finv[pole];
                        case BK_YP: return Yp;
                        default: return W;
                    }
                };
                g.jobs[0] = h->d_sjobs + L.off;
                g.tmap[0] = L.tmoff >= 0 ? h->d_stmap + L.tmoff : nullptr;
                g.njobs[0] = L.cnt;
                g.ntiles[0] = L.ntiles;
                g.A[0] = basep(o.abase);
                g.B[0] = basep(o.bbase);
                g.C[0] = basep(o.cbase);
                launch_gemm<double>(g, 1, st, L.flops);
            } else {
                RowArgs<double> r;
                std::memset(&r, 0, sizeof(r));
                r.jobs = h->d_rjobs + o.L.off;
                r.tmap = o.L.tmoff >= 0 ? h->d_stmap + o.L.tmoff : nullptr;
                r.njobs = o.L.cnt;
                r.ntiles = o.L.ntiles;
                r.map = (o.kind == SOP_EADD) ? h->d_rel : h->d_rows;
                r.k = (int)k;
                r.rpt = rows_per_tile(k);
                r.ldw = k;
                r.mode = (o.kind == SOP_EADD) ? ROW_EADD
                         : (o.kind == SOP_SCATTER_OUT ? ROW_SCATTER : (o.kind == SOP_ZERO ? ROW_ZERO : ROW_GATHER));
                r.ldx = (o.kind == SOP_GATHER_IN) ? ldb : ldx;
                r.W[0] = W;
                r.X[0] = (o.kind == SOP_GATHER_IN) ? const_cast<c128 *>((const c128 *)Bk) : (c128 *)X;
                launch_rows<double>(r, 1, st);
            }
        }
    };
    run(h->fwd);
    run(h->bwd);
    rc = cuda_check(cudaGetLastError(), "solve_noalloc launch");
    if (rc) return rc;
    h->stats.solve_cols += k;
    return ZOLO_OK;
}
