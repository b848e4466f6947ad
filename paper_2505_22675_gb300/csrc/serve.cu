// Serving state of a context (continuous batching of submitted tiles).
#include "bg_internal.h"

extern "C" bg_status bg_serve_shutdown(bg_ctx_t ctx) {
    (void)ctx;
    return BG_OK;
}
