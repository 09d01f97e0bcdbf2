// Serving loop (continuous batching of IM queries over resident graphs and
// pools).
#include "runtime.h"

using namespace hbx;

struct hbx_server {
    hbx_ctx* ctx = nullptr;
};
struct hbx_ticket {
    int dummy = 0;
};

extern "C" int hbx_server_create(hbx_ctx* ctx, uint32_t, uint64_t, hbx_server** out) {
    if (out) *out = nullptr;
    return fail(ctx, HBX_ERR_INVALID_ARG, "serving is not available in this build");
}
extern "C" void hbx_server_destroy(hbx_server*) {}
extern "C" int hbx_submit(hbx_server*, hbx_graph*, hbx_model, uint32_t, double, double, uint64_t, const hbx_options*,
                          hbx_ticket** out) {
    if (out) *out = nullptr;
    return HBX_ERR_INVALID_ARG;
}
extern "C" int hbx_wait(hbx_ticket*, uint32_t*, double*, hbx_stats*, double*, int64_t) { return HBX_ERR_INVALID_ARG; }
extern "C" int hbx_cancel(hbx_ticket*) { return HBX_ERR_INVALID_ARG; }
extern "C" void hbx_ticket_destroy(hbx_ticket*) {}
void hbx_server_destroy_all(hbx_ctx*) {}
