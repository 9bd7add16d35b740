// sfh_serve.cu -- serving runtime (placeholder until the runtime lands).
#include "../../include/sfhad.h"

extern "C" sfh_status sfh_server_create(const sfh_server_opts *, sfh_server **out) {
    if (out) *out = nullptr;
    return SFH_EUNSUPPORTED;
}
extern "C" sfh_status sfh_serve_submit(sfh_server *, const sfh_request *, uint64_t *) { return SFH_EUNSUPPORTED; }
extern "C" sfh_status sfh_serve_poll(sfh_server *, uint64_t, sfh_result *) { return SFH_EUNSUPPORTED; }
extern "C" sfh_status sfh_serve_drain(sfh_server *, int) { return SFH_EUNSUPPORTED; }
extern "C" sfh_status sfh_server_destroy(sfh_server *) { return SFH_OK; }
