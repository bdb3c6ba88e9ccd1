// Serving entry points: hht_submit / hht_progress / hht_poll.
//
// Requests are copied into library-owned host memory at submit time.  Each
// hht_progress() call takes every queued request and runs them together as
// one batch through the level loop; results wait in a table until polled.
#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/hht.h"
#include "hht_serve.h"

namespace hht {

struct Request {
    std::vector<hht_point> pts;
    hht_image im{};
    bool done = false;
    int status = HHT_E_PENDING;
    hht_result res{};
    std::vector<hht_leaf> leaves;
};

struct ServeState {
    uint64_t next_ticket = 1;
    std::map<uint64_t, Request> reqs;
    std::vector<uint64_t> queue;
    std::mutex mu;
};

void serve_destroy(ServeState* s) { delete s; }

}  // namespace hht

using namespace hht;

namespace {
ServeState* serve_of(hht_ctx* c) {
    ServeState** slot = hht_internal_serve_slot(c);
    if (!*slot) *slot = new ServeState();
    return *slot;
}
}  // namespace

extern "C" {

int hht_submit(hht_ctx* c, const hht_image* image, uint64_t* ticket) {
    if (!c || !image || !ticket) return HHT_E_ARG;
    const hht_image& im = *image;
    if (im.n < 0 || im.n > INT32_MAX || (im.n > 0 && !im.points) || im.W < 1 || im.H < 1 || im.W > HHT_MAX_SIDE ||
        im.H > HHT_MAX_SIDE || im.depth < 1 || im.depth > HHT_MAX_DEPTH || im.T < 1)
        return HHT_E_ARG;
    ServeState* s = serve_of(c);
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t t = s->next_ticket++;
    Request& r = s->reqs[t];
    r.pts.resize((size_t)im.n);
    if (im.n > 0 && cudaMemcpy(r.pts.data(), im.points, (size_t)im.n * sizeof(hht_point), cudaMemcpyDefault) != cudaSuccess) {
        s->reqs.erase(t);
        return HHT_E_CUDA;
    }
    r.im = im;
    r.im.points = r.pts.data();
    s->queue.push_back(t);
    *ticket = t;
    return HHT_OK;
}

int hht_progress(hht_ctx* c) {
    if (!c) return HHT_E_ARG;
    ServeState* s = serve_of(c);
    std::vector<uint64_t> batch;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        batch.swap(s->queue);
    }
    if (batch.empty()) return 0;
    std::vector<hht_image> ims(batch.size());
    std::vector<hht_result> outs(batch.size());
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t k = 0; k < batch.size(); ++k) {
            Request& r = s->reqs[batch[k]];
            ims[k] = r.im;
            // leaf capacity: every leaf is a cell of one of the two K x K grids
            const uint64_t K = 1ull << r.im.depth;
            const uint64_t cap = std::min<uint64_t>(2 * K * K, 1ull << 26);
            r.leaves.resize((size_t)cap);
            outs[k].leaves = r.leaves.data();
            outs[k].leaf_capacity = cap;
        }
    }
    hht_internal_run_job(c, ims.data(), (int)ims.size(), outs.data());
    std::lock_guard<std::mutex> lk(s->mu);
    for (size_t k = 0; k < batch.size(); ++k) {
        Request& r = s->reqs[batch[k]];
        r.res = outs[k];
        r.status = outs[k].status;
        r.done = true;
    }
    return 0;
}

int hht_poll(hht_ctx* c, uint64_t ticket, hht_result* out) {
    if (!c || !out) return HHT_E_ARG;
    ServeState* s = serve_of(c);
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HHT_E_UNKNOWN_TICKET;
    Request& r = it->second;
    if (!r.done) return HHT_E_PENDING;
    hht_leaf* dst = out->leaves;
    const uint64_t cap = out->leaf_capacity;
    hht_result res = r.res;
    res.leaves = dst;
    res.leaf_capacity = cap;
    int rc = r.status;
    if (rc == HHT_OK) {
        if (res.n_leaves > cap || (res.n_leaves > 0 && !dst)) {
            out->n_leaves = res.n_leaves;
            return HHT_E_CAPACITY;  // the ticket stays valid: poll again with a larger buffer
        }
        if (res.n_leaves && cudaMemcpy(dst, r.leaves.data(), res.n_leaves * sizeof(hht_leaf), cudaMemcpyDefault) != cudaSuccess)
            rc = HHT_E_CUDA;
    }
    *out = res;
    out->status = rc;
    s->reqs.erase(it);
    return rc;
}

}  // extern "C"
