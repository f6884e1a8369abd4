// placeholder, replaced by the Krylov / Rayleigh-Ritz implementation
#include "factor.h"
extern "C" {
int zolo_apply(zolo_factor_h, int64_t, const void *, int64_t, void *, int64_t, zolo_stats *, void *) {
    return zolo::set_error(ZOLO_EINVAL, "not built yet");
}
int zolo_eigs_factored(zolo_factor_h, double, double, int64_t, const void *, double *, void *, int64_t, int64_t,
                       int64_t *, double *, zolo_stats *, void *) {
    return zolo::set_error(ZOLO_EINVAL, "not built yet");
}
int zolo_eigs(const zolo_csr *, const zolo_csr *, double, double, int64_t, const zolo_filter_spec *,
              const zolo_opts *, double *, void *, int64_t, int64_t, int64_t *, double *, zolo_stats *, void *) {
    return zolo::set_error(ZOLO_EINVAL, "not built yet");
}
}
