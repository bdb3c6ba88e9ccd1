// Serving state (hht_serve.cu): requests queued by hht_submit(), advanced by
// hht_progress(), collected by hht_poll().
#pragma once

#include <cstdint>

#include "../../include/hht.h"

namespace hht {
struct ServeState;
void serve_destroy(ServeState* s);
}  // namespace hht

// Runs a batch through the level loop (defined in hht_api.cu).
int hht_internal_run_job(hht_ctx* c, const hht_image* im, int count, hht_result* outs);
hht::ServeState** hht_internal_serve_slot(hht_ctx* c);
