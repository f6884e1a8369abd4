// Status codes, thread-local error messages and option defaults of the C ABI.
#include <cstring>
#include <string>
#include "zolo_internal.h"

namespace zolo {
namespace {
thread_local std::string g_last_error;
}
int set_error(int status, const std::string &msg) {
    g_last_error = msg;
    return status;
}
void clear_error() { g_last_error.clear(); }
const char *last_error_cstr() { return g_last_error.c_str(); }
}  // namespace zolo

extern "C" {

void zolo_opts_default(zolo_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->leaf_max = 32;
    o->precision = ZOLO_PREC_FP64;
    o->gmres_m_max = 100;
    o->gmres_tol = 1e-12;
    o->refine_max = 8;
    o->refine_tol = 1e-12;
    o->n_iter_max = 4;
    o->tol = 1e-10;
    o->drop_tol = 1e-14;
    o->k = 0;
    o->r1 = 2;
    o->r2 = 2;
    o->gap_rel = 1e-2;
    o->seed = 0x5eed;
    o->gmres_chunk = 0;
    o->split_k_min = 512;
    o->real_block = 1;
    o->lock = 1;
}

const char *zolo_strerror(int s) {
    switch (s) {
        case ZOLO_OK: return "ok";
        case ZOLO_EINVAL: return "invalid argument";
        case ZOLO_ENOTHERM: return "matrix not Hermitian";
        case ZOLO_ENOMEM: return "out of memory";
        case ZOLO_ESINGULAR: return "singular front pivot";
        case ZOLO_ENOCONV: return "not converged";
        case ZOLO_ETIMEOUT: return "device wait timed out";
        case ZOLO_ECUDA: return "CUDA error";
        case ZOLO_EGAP: return "Ritz value inside an eigengap";
        default: return "unknown status";
    }
}

const char *zolo_last_error(void) { return zolo::last_error_cstr(); }

int zolo_version(void) { return 100; }

}  // extern "C"
