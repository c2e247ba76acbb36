// Serving loop (placeholder until the scheduler lands).
#include "lf_ctx.h"

extern "C" {
lf_status lf_serve_create(lf_ctx*, size_t, int, int, lf_serve**) { return LF_ERR_INVALID; }
lf_status lf_serve_submit(lf_serve*, const lf_request*, uint64_t*) { return LF_ERR_INVALID; }
lf_status lf_serve_poll(lf_serve*, uint64_t, int*, float*, size_t, lf_timing*) { return LF_ERR_INVALID; }
lf_status lf_serve_wait(lf_serve*, uint64_t, int) { return LF_ERR_INVALID; }
lf_status lf_serve_destroy(lf_serve*) { return LF_ERR_INVALID; }
}
