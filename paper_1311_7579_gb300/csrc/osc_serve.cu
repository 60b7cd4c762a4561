// osc_serve.cu -- continuous-batching serving loop (placeholder until built out).
#include "osc_ctx.h"

using namespace osc;

extern "C" {

osc_status osc_serve_start(osc_ctx *ctx, int32_t max_slots, double lo, double hi, int32_t nbins) {
    (void)max_slots; (void)lo; (void)hi; (void)nbins;
    return ctx ? fail(ctx, OSC_E_STATE, "serving not available") : OSC_E_ARG;
}
osc_status osc_submit(osc_ctx *ctx, int32_t sample_id, const osc_point *pt, osc_precision prec, uint64_t *ticket) {
    (void)sample_id; (void)pt; (void)prec; (void)ticket;
    return ctx ? fail(ctx, OSC_E_STATE, "serving not running") : OSC_E_ARG;
}
osc_status osc_wait(osc_ctx *ctx, uint64_t ticket, double *out_hist, int32_t timeout_ms, double *latency_us) {
    (void)ticket; (void)out_hist; (void)timeout_ms; (void)latency_us;
    return ctx ? fail(ctx, OSC_E_STATE, "serving not running") : OSC_E_ARG;
}
osc_status osc_serve_stop(osc_ctx *ctx) { return ctx ? OSC_OK : OSC_E_ARG; }

}  // extern "C"
