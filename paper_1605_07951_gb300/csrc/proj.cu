// placeholder, replaced by the projection stage
#include "rsrr_handle.h"
extern "C" rsrr_status rsrr_project(rsrr_t *hh, void *stream) {
    (void)stream;
    rsrr::Handle *h = reinterpret_cast<rsrr::Handle *>(hh);
    if (!h) return RSRR_EINVAL;
    return h->fail(RSRR_ESTATE, "rsrr_project: not available");
}
extern "C" rsrr_status rsrr_solve(rsrr_t *hh, rsrr_result *out) {
    (void)out;
    rsrr::Handle *h = reinterpret_cast<rsrr::Handle *>(hh);
    if (!h) return RSRR_EINVAL;
    return h->fail(RSRR_ESTATE, "rsrr_solve: not available");
}
extern "C" rsrr_status rsrr_get_Q(rsrr_t *hh, rsrr_c128 *, int32_t, void *) { return RSRR_ESTATE; }
extern "C" rsrr_status rsrr_get_projected(rsrr_t *hh, rsrr_c128 *, int32_t, void *) { return RSRR_ESTATE; }
