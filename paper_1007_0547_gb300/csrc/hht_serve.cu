// Serving: hht_submit / hht_progress / hht_poll with continuous batching.
//
// The engine keeps a level loop running on the device.  Every unit (one half
// of one request) carries the loop step t0 at which it was admitted and is at
// level (step - t0); the stage / select / pass kernels read that per unit, so
// units of different ages share every launch.  One hht_progress() call is one
// step:
//   1. admit waiting requests while request slots and the memory budget allow
//      (by a projection of every request's bounds over the steps to come):
//      their level-0 regions, vote counters and voter streams are appended to
//      the current step's (stage kernel);
//   2. select: children of every current region (or leaves, for units that
//      reach their depth now);
//   3. pass: the next step's voter stream and vote counters;
//   4. requests whose units reached their depth at this step are complete:
//      their leaves (one block per unit, in the paper's depth-first order) are
//      copied into a device buffer of their own until polled, their statistics
//      are read back, and their slot is released (their bounds leave the
//      projection as the steps pass).
// Requests that arrive while others run are admitted at the next step and
// overlap with them on the device; results do not depend on the mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/hht.h"
#include "hht_ctx.h"
#include "hht_internal.h"
#include "hht_serve.h"

namespace hht {

struct Request {
    std::vector<hht_point> pts;
    hht_image im{};
    int slot = -1;
    int64_t t0 = 0;
    int64_t blocked_since = -1;  // first step at which it did not fit the budget
    bool done = false;
    bool range_error = false;
    int status = HHT_E_PENDING;
    // a finished request's leaves stay in device memory until it is polled
    void* dev_leaves = nullptr;
    uint64_t dev_bytes = 0;
    hht_result res{};
};

struct ServeState {
    static constexpr int kSlots = 1024;  // requests in flight at most (two units each)
    // A waiting request that does not fit the memory budget is passed over by
    // later ones that do for at most this many steps; after that nothing is
    // admitted until it fits (the running requests finish within 24 steps).
    static constexpr int64_t kBypassSteps = 12;
    static constexpr size_t kAdmitScan = 256;  // waiting requests examined per step

    std::mutex mu;
    uint64_t next_ticket = 1;
    std::map<uint64_t, Request> reqs;
    std::deque<uint64_t> waiting;
    std::deque<uint64_t> finished;  // tickets done and not yet listed by hht_done_tickets

    // engine
    bool init = false;
    std::vector<int> free_slots;
    std::vector<uint64_t> order;  // tickets in flight, in admission order (= record order)
    uint64_t budget = 0;
    // Projected voter records of the engine's two streams: stream[k] is the
    // stream read at step (step + k), held in vox[par ^ (k & 1)] (the one
    // written at step + k is stream[k + 1]): the sum over the requests in
    // flight of their bounds at the level each will then be at.
    static constexpr int kHorizon = kMaxDepth + 3;
    uint64_t stream[kHorizon] = {};
    // the same for the regions of each step (the parents: every one sizes a
    // pass record, four children's records, counters and cursors, or four
    // leaves)
    uint64_t regions[kHorizon] = {};
    static constexpr uint64_t kRegionBytes = sizeof(PassRegion) + 4 * (sizeof(Region) + 16 + 8 + sizeof(DevLeaf));
    int n_i64 = 0;
    int64_t step = 0;
    int par = 0;
    uint64_t P = 0, NV = 0;  // regions and voters of the current step
    DevBuf units, stats, infos, status, leaf_total, img_err, scan, pts, img_start, img_unit;
    DevBuf rec[2], preg[2], cnt[2], vox[2], cursors, leaves, sel_flags, sel_data;
    hht_ctx* ctx = nullptr;  // for the per-request leaf buffers
    // hht_poll's copies run here, so that a poll does not wait for the step
    // running on the context's stream
    cudaStream_t poll_stream = nullptr;
};

// Device memory for one finished request's leaves: the caller's allocator
// when the context has one, else the device's stream-ordered pool.
void* result_alloc(hht_ctx* c, size_t bytes) {
    void* p = nullptr;
    if (c->has_allocator) {
        p = c->allocator.alloc(bytes, (void*)c->stream, c->allocator.user);
        return p;
    }
    if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
void result_free(hht_ctx* c, void* p, size_t bytes) {
    if (!p) return;
    if (c->has_allocator)
        c->allocator.free(p, bytes, (void*)c->stream, c->allocator.user);
    else
        cudaFreeAsync(p, c->stream);
}

void serve_destroy(ServeState* s) {
    if (!s) return;
    if (s->ctx)
        for (auto& kv : s->reqs) result_free(s->ctx, kv.second.dev_leaves, kv.second.dev_bytes);
    if (s->ctx) cudaStreamSynchronize(s->ctx->stream);
    if (s->poll_stream) cudaStreamDestroy(s->poll_stream);
    delete s;
}

}  // namespace hht

using namespace hht;

namespace {

ServeState* serve_of(hht_ctx* c) {
    ServeState** slot = hht_internal_serve_slot(c);
    if (!*slot) {
        *slot = new ServeState();
        (*slot)->ctx = c;
    }
    return *slot;
}

// Upper bound on a request's voter records at level l, both halves: a list
// is kept for the levels up to depth - 2, and at level l a line votes in at
// most 2^l + (W_h - 1) 2^l / (2L) + 2 cells (and no more than the 4^l the
// level has), W_h the half's x extent (the image's width for half 0, its
// height for half 1).
uint64_t stream_bound(const hht_image& im, int l) {
    if (im.depth < 2 || l > im.depth - 2) return 0;
    if (l == 0) return 2 * (uint64_t)im.n;
    const uint64_t L = 1ull << ceil_log2_i(std::max(im.W, im.H));
    const uint64_t col = 1ull << l;
    uint64_t total = 0;
    for (int h = 0; h < 2; ++h) {
        const uint64_t Wh = (uint64_t)(h ? im.H : im.W);
        total += (uint64_t)im.n * std::min(col + (Wh - 1) * col / (2 * L) + 2, col * col);
    }
    return total;
}

// Upper bound on a request's regions at level l, both halves (the parents
// of step t0 + l, for l up to depth - 1; the last ones' children are the
// leaves, four per parent): the level's cells, and no more than its votes
// allow at T votes each.
uint64_t region_bound(const hht_image& im, int l) {
    if (l >= im.depth) return 0;
    if (l == 0) return 2;
    const uint64_t L = 1ull << ceil_log2_i(std::max(im.W, im.H));
    const uint64_t col = 1ull << l;
    uint64_t total = 0;
    for (int h = 0; h < 2; ++h) {
        const uint64_t Wh = (uint64_t)(h ? im.H : im.W);
        const uint64_t votes = (uint64_t)im.n * std::min(col + (Wh - 1) * col / (2 * L) + 2, col * col);
        total += std::min(col * col, votes / (uint64_t)im.T);
    }
    return total;
}

#define SV_CK(call)                     \
    do {                                \
        cudaError_t e_ = (call);        \
        if (e_ != cudaSuccess) {        \
            cudaGetLastError();         \
            return HHT_E_CUDA;          \
        }                               \
    } while (0)
#define SV_RK(call)                  \
    do {                             \
        int r_ = (call);             \
        if (r_ != HHT_OK) return r_; \
    } while (0)

int engine_init(hht_ctx* c, ServeState* S) {
    const int U = 2 * ServeState::kSlots;
    SV_RK(ensure(c, S->units, U * sizeof(Unit), true));
    SV_RK(ensure(c, S->stats, (size_t)U * (kMaxDepth + 1) * 4 * sizeof(uint64_t), true));
    SV_RK(ensure(c, S->infos, 2 * sizeof(LevelInfo), true));
    SV_RK(ensure(c, S->status, sizeof(DeviceStatus), true));
    SV_RK(ensure(c, S->leaf_total, sizeof(uint64_t), true));
    SV_RK(ensure(c, S->img_err, ServeState::kSlots * sizeof(uint32_t), true));  // range flags per request slot
    SV_RK(ensure(c, S->scan, sizeof(ScanState), true));
    for (int s = ServeState::kSlots - 1; s >= 0; --s) S->free_slots.push_back(s);
    // the context's budget, but no more than the device has: admission
    // counts on every byte of it
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const uint64_t room = (uint64_t)(0.85 * (double)fr);
    S->budget = c->budget ? std::min<uint64_t>(c->budget, room) : room;
    S->init = true;
    return HHT_OK;
}

// The most the projection asks of the stream buffer that is vox[par ^ odd]
// now (odd = 0: the one read at this step).
uint64_t projected(const ServeState* S, int odd) {
    uint64_t m = 0;
    for (int k = odd; k < ServeState::kHorizon; k += 2) m = std::max(m, S->stream[k]);
    return m;
}

// Admit waiting requests into the current step.
int engine_admit(hht_ctx* c, ServeState* S) {
    // Waiting requests are taken in arrival order while they fit the budget
    // (the first one always fits an idle engine).  One that does not fit is
    // passed over by later ones that do, so that a large request at the head
    // does not hold small ones back, until it has waited kBypassSteps steps.
    //
    // A request fits when, with its bounds added to the projection, the two
    // stream buffers (each at least its present size: a buffer does not
    // shrink) and the region buffers of the largest step to come need at
    // most 90 % of the budget (the rest: selection tiles, slack).
    std::vector<uint64_t> adm;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        const uint64_t have[2] = {S->vox[S->par].bytes / sizeof(Voter), S->vox[S->par ^ 1].bytes / sizeof(Voter)};
        uint64_t have_reg = S->cursors.bytes + S->leaves.bytes + S->sel_flags.bytes + S->sel_data.bytes;
        for (int k = 0; k < 2; ++k) have_reg += S->rec[k].bytes + S->cnt[k].bytes + S->preg[k].bytes;
        auto fits = [&](const hht_image& im) {
            uint64_t need[2] = {have[0], have[1]}, reg = 0;
            for (int k = 0; k < ServeState::kHorizon; ++k) {
                need[k & 1] = std::max(need[k & 1], S->stream[k] + stream_bound(im, k));
                reg = std::max(reg, S->regions[k] + region_bound(im, k));
            }
            return (double)(need[0] + need[1]) * sizeof(Voter) +
                       std::max((double)have_reg, (double)reg * ServeState::kRegionBytes) <=
                   0.9 * (double)S->budget;
        };
        size_t seen = 0;
        for (auto it = S->waiting.begin();
             it != S->waiting.end() && adm.size() < S->free_slots.size() && seen < ServeState::kAdmitScan; ++seen) {
            Request& r = S->reqs[*it];
            if ((S->order.empty() && adm.empty()) || fits(r.im)) {
                adm.push_back(*it);
                for (int k = 0; k < ServeState::kHorizon; ++k) {
                    S->stream[k] += stream_bound(r.im, k);
                    S->regions[k] += region_bound(r.im, k);
                }
                it = S->waiting.erase(it);
                continue;
            }
            if (r.blocked_since < 0) r.blocked_since = S->step;
            if (S->step - r.blocked_since >= ServeState::kBypassSteps) break;
            ++it;
        }
    }
    if (adm.empty()) return HHT_OK;
    cudaStream_t st = c->stream;
    const int m = (int)adm.size();
    std::vector<Unit> nu(2 * m);
    std::vector<uint64_t> img_start(m + 1);
    std::vector<uint32_t> img_unit(m);
    std::vector<Region> roots(2 * m);
    std::vector<hht_point> pts;
    uint64_t total = 0, v0 = 0;
    for (int k = 0; k < m; ++k) {
        Request& r = S->reqs[adm[k]];
        r.slot = S->free_slots.back();
        S->free_slots.pop_back();
        r.t0 = S->step;
        const int lL = ceil_log2_i(std::max(r.im.W, r.im.H));
        if (lL + r.im.depth > 27) ++S->n_i64;
        img_start[k] = total;
        img_unit[k] = (uint32_t)(2 * r.slot);
        for (int h = 0; h < 2; ++h) {
            Unit& U = nu[2 * k + h];
            std::memset(&U, 0, sizeof U);
            U.lL = lL; U.D = r.im.depth; U.T = r.im.T; U.image = k; U.n = r.im.n;
            U.W = r.im.W; U.H = r.im.H; U.half = h; U.t0 = (int32_t)S->step;
            U.root_rec = (uint32_t)(S->P + 2 * k + h);
            U.v0_off = S->NV + v0;
            if (U.D >= 2) v0 += (uint64_t)r.im.n;
            roots[2 * k + h] = Region{(uint32_t)(2 * r.slot + h), 0u, 0u, (uint32_t)r.im.n};
        }
        pts.insert(pts.end(), r.pts.begin(), r.pts.end());
        total += (uint64_t)r.im.n;
        S->order.push_back(adm[k]);
    }
    img_start[m] = total;
    // device buffers: the current step's records, counters and stream grow in place
    const int cp = S->par;
    SV_RK(ensure_keep(c, S->rec[cp], (S->P + 2 * m) * sizeof(Region), S->P * sizeof(Region)));
    SV_RK(ensure_keep(c, S->cnt[cp], (S->P + 2 * m) * 16, S->P * 16));
    SV_RK(ensure_sized(c, S->vox[cp], std::max<uint64_t>(S->NV + v0, 1) * sizeof(Voter), S->NV * sizeof(Voter),
                       projected(S, 0) * sizeof(Voter)));
    SV_RK(ensure(c, S->pts, std::max<uint64_t>(total, 1) * sizeof(hht_point)));
    SV_RK(ensure(c, S->img_start, (m + 1) * sizeof(uint64_t)));
    SV_RK(ensure(c, S->img_unit, m * sizeof(uint32_t)));
    for (int k = 0; k < m; ++k) {
        const Request& r = S->reqs[adm[k]];
        SV_CK(cudaMemcpyAsync((Unit*)S->units.p + 2 * r.slot, &nu[2 * k], 2 * sizeof(Unit), cudaMemcpyHostToDevice, st));
        // statistics rows of the two units: level 0 tested 1, passed 1, n codes
        std::vector<uint64_t> rows(2 * (kMaxDepth + 1) * 4, 0);
        for (int h = 0; h < 2; ++h) {
            rows[(size_t)h * (kMaxDepth + 1) * 4 + 0] = 1;
            rows[(size_t)h * (kMaxDepth + 1) * 4 + 1] = 1;
            rows[(size_t)h * (kMaxDepth + 1) * 4 + 3] = (uint64_t)r.im.n;
        }
        SV_CK(cudaMemcpyAsync((uint64_t*)S->stats.p + (size_t)2 * r.slot * (kMaxDepth + 1) * 4, rows.data(),
                              rows.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    }
    if (total > 0)
        SV_CK(cudaMemcpyAsync(S->pts.p, pts.data(), total * sizeof(hht_point), cudaMemcpyHostToDevice, st));
    SV_CK(cudaMemcpyAsync(S->img_start.p, img_start.data(), (m + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    SV_CK(cudaMemcpyAsync(S->img_unit.p, img_unit.data(), m * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    for (int k = 0; k < m; ++k)
        SV_CK(cudaMemsetAsync((uint32_t*)S->img_err.p + S->reqs[adm[k]].slot, 0, sizeof(uint32_t), st));
    SV_CK(cudaMemcpyAsync((Region*)S->rec[cp].p + S->P, roots.data(), 2 * m * sizeof(Region), cudaMemcpyHostToDevice, st));
    SV_CK(cudaMemsetAsync((char*)S->cnt[cp].p + S->P * 16, 0, 2 * m * 16, st));
    if (launch_stage((const int16_t*)S->pts.p, total, (const Unit*)S->units.p, m, (const uint64_t*)S->img_start.p,
                     (const uint32_t*)S->img_unit.p, (Voter*)S->vox[cp].p, (uint32_t*)S->cnt[cp].p,
                     (uint64_t*)S->stats.p, (uint32_t*)S->img_err.p, (DeviceStatus*)S->status.p, S->n_i64 > 0,
                     st) != 0)
        return HHT_E_CUDA;
    // range errors are read when the request completes (no synchronisation here)
    S->P += 2 * (uint64_t)m;
    S->NV += v0;
    return HHT_OK;
}

// Copy out the requests whose units reached their depth in the step just run.
int engine_complete(hht_ctx* c, ServeState* S, uint64_t step_leaves) {
    cudaStream_t st = c->stream;
    std::vector<uint64_t> fin;
    for (uint64_t t : S->order) {
        const Request& r = S->reqs[t];
        if (r.t0 + r.im.depth == S->step) fin.push_back(t);
    }
    if (fin.empty()) return HHT_OK;
    std::vector<std::vector<uint64_t>> rows(fin.size(), std::vector<uint64_t>(2 * (kMaxDepth + 1) * 4));
    for (size_t k = 0; k < fin.size(); ++k) {
        const Request& r = S->reqs[fin[k]];
        SV_CK(cudaMemcpyAsync(rows[k].data(), (uint64_t*)S->stats.p + (size_t)2 * r.slot * (kMaxDepth + 1) * 4,
                              rows[k].size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    }
    std::vector<uint32_t> slot_err(ServeState::kSlots, 0);
    SV_CK(cudaMemcpyAsync(slot_err.data(), S->img_err.p, ServeState::kSlots * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                          st));
    SV_CK(cudaStreamSynchronize(st));
    for (uint64_t t : fin) {
        Request& r = S->reqs[t];
        if (slot_err[r.slot]) r.range_error = true;
    }
    // the step's leaves are one block per finishing unit, in record (= admission)
    // order; each request's block is copied on the device into its own buffer
    // (polled later straight into the caller's), so no host copy holds the loop
    uint64_t off = 0;
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t k = 0; k < fin.size(); ++k) {
        Request& r = S->reqs[fin[k]];
        const int D = r.im.depth;
        hht_result& res = r.res;
        std::memset(&res, 0, sizeof res);
        res.depth = D;
        res.L = 1 << ceil_log2_i(std::max(r.im.W, r.im.H));
        uint64_t nl = 0;
        for (int h = 0; h < 2; ++h) {
            const uint64_t* su = rows[k].data() + (size_t)h * (kMaxDepth + 1) * 4;
            for (int l = 0; l <= D; ++l) {
                res.stats[h][l].tested = su[4 * l + 0];
                res.stats[h][l].passed = su[4 * l + 1];
                res.stats[h][l].votes = su[4 * l + 2];
                res.stats[h][l].tests = su[4 * l + 3];
            }
            nl += su[4 * D + 1];
        }
        res.n_leaves = nl;
        if (off + nl > step_leaves) return HHT_E_CUDA;
        r.status = r.range_error ? HHT_E_RANGE : HHT_OK;
        if (nl > 0 && r.status == HHT_OK) {
            r.dev_bytes = nl * sizeof(hht_leaf);
            r.dev_leaves = result_alloc(c, r.dev_bytes);
            if (!r.dev_leaves) {
                r.dev_bytes = 0;
                r.status = HHT_E_NOMEM;
            } else {
                SV_CK(cudaMemcpyAsync(r.dev_leaves, (const DevLeaf*)S->leaves.p + off, r.dev_bytes,
                                      cudaMemcpyDeviceToDevice, st));
            }
        }
        off += nl;
        r.done = true;
        S->finished.push_back(fin[k]);
        r.pts.clear();
        r.pts.shrink_to_fit();
        S->free_slots.push_back(r.slot);
        if (ceil_log2_i(std::max(r.im.W, r.im.H)) + D > 27) --S->n_i64;
    }
    // the copies are done before any poll reads them (on any stream)
    SV_CK(cudaStreamSynchronize(st));
    if (off != step_leaves) return HHT_E_CUDA;
    std::vector<uint64_t> keep;
    for (uint64_t t : S->order)
        if (!S->reqs[t].done) keep.push_back(t);
    S->order.swap(keep);
    return HHT_OK;
}

int engine_step(hht_ctx* c, ServeState* S) {
    cudaStream_t st = c->stream;
    if (!S->init) SV_RK(engine_init(c, S));
    SV_RK(engine_admit(c, S));
    if (S->order.empty()) return HHT_OK;
    const int cp = S->par, np = cp ^ 1;
    const uint64_t P = S->P;
    LevelInfo* d_infos = (LevelInfo*)S->infos.p;
    // the parents' totals (after admission) for the kernels
    SV_CK(cudaMemcpyAsync(&d_infos[cp].n_regions, &S->P, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    SV_CK(cudaMemcpyAsync(&d_infos[cp].n_voters, &S->NV, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    SV_CK(cudaMemsetAsync(&d_infos[np], 0, sizeof(LevelInfo), st));
    SV_CK(cudaMemsetAsync(S->leaf_total.p, 0, sizeof(uint64_t), st));
    LevelInfo h_next{};
    if (4 * P > kMaxLevelRecords) return HHT_E_NOMEM;
    if (P > 0) {
        const uint64_t sel_tiles = (P + 1023) / 1024;
        SV_RK(ensure(c, S->preg[cp], P * sizeof(PassRegion)));
        SV_RK(ensure(c, S->rec[np], 4 * P * sizeof(Region)));
        SV_RK(ensure(c, S->cnt[np], 4 * P * 16));
        SV_RK(ensure(c, S->cursors, 4 * P * sizeof(unsigned long long)));
        SV_RK(ensure(c, S->leaves, 4 * P * sizeof(DevLeaf)));
        if ((sel_tiles + 1) * 4 > S->sel_flags.bytes) SV_RK(ensure(c, S->sel_flags, (sel_tiles + 1) * 4, true));
        SV_RK(ensure(c, S->sel_data, (sel_tiles + 1) * 2 * 3 * sizeof(uint64_t)));
        LevelArgs a{};
        a.units = (const Unit*)S->units.p;
        a.parents = (const Region*)S->rec[cp].p;
        a.pregions = (PassRegion*)S->preg[cp].p;
        a.parent_cnt = (const uint32_t*)S->cnt[cp].p;
        a.children = (Region*)S->rec[np].p;
        a.child_cnt = (uint32_t*)S->cnt[np].p;
        a.cursor = (unsigned long long*)S->cursors.p;
        a.leaves = (DevLeaf*)S->leaves.p;
        a.stats = (uint64_t*)S->stats.p;
        a.info_prev = d_infos + cp;
        a.info = d_infos + np;
        a.leaf_total = (uint64_t*)S->leaf_total.p;
        a.scan = (ScanState*)S->scan.p;
        a.tile_flags = (uint32_t*)S->sel_flags.p;
        a.tile_data = (uint64_t*)S->sel_data.p;
        a.status = (DeviceStatus*)S->status.p;
        a.img_err = (const uint32_t*)S->img_err.p;
        a.cap_children = 4 * P;
        a.cap_leaves = 4 * P;
        a.cap_voters = UINT64_MAX;
        a.level = (int32_t)(S->step + 1);
        a.num_sms = c->num_sms;
        const int sel_grid = (int)std::min<uint64_t>(sel_tiles, (uint64_t)c->num_sms * c->occ_select);
        if (launch_select(a, 256, std::max(sel_grid, 1), st) != 0) return HHT_E_CUDA;
        DeviceStatus hs{};
        SV_CK(cudaMemcpyAsync(&h_next, d_infos + np, sizeof h_next, cudaMemcpyDeviceToHost, st));
        SV_CK(cudaMemcpyAsync(&hs, S->status.p, sizeof hs, cudaMemcpyDeviceToHost, st));
        SV_CK(cudaStreamSynchronize(st));
        if (hs.err & kErrTimeout) return HHT_E_TIMEOUT;
        if (hs.err) return HHT_E_CUDA;
        if (S->NV > 0) {
            SV_RK(ensure_sized(c, S->vox[np], std::max<uint64_t>(h_next.n_voters, 1) * sizeof(Voter), 0,
                               projected(S, 1) * sizeof(Voter)));
            a.vin = (const Voter*)S->vox[cp].p;
            a.vout = (Voter*)S->vox[np].p;
            a.cap_voters = h_next.n_voters;
            const bool i64 = S->n_i64 > 0;
            const uint64_t want = (S->NV + 2047) / 2048;
            const int grid = (int)std::min<uint64_t>(want, (uint64_t)c->num_sms * (i64 ? c->occ_pass64 : c->occ_pass32));
            if (launch_pass(a, i64, std::max(grid, 1), st) != 0) return HHT_E_CUDA;
        }
    }
    S->step += 1;
    SV_RK(engine_complete(c, S, h_next.n_leaves));
    S->P = h_next.n_regions;
    S->NV = h_next.n_voters;
    S->par = np;
    // the projection moves with the steps
    for (int k = 0; k + 1 < ServeState::kHorizon; ++k) {
        S->stream[k] = S->stream[k + 1];
        S->regions[k] = S->regions[k + 1];
    }
    S->stream[ServeState::kHorizon - 1] = 0;
    S->regions[ServeState::kHorizon - 1] = 0;
    return HHT_OK;
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
    std::vector<hht_point> pts((size_t)im.n);
    if (im.n > 0) {
        cudaSetDevice(c->device);
        if (cudaMemcpy(pts.data(), im.points, (size_t)im.n * sizeof(hht_point), cudaMemcpyDefault) != cudaSuccess) {
            cudaGetLastError();
            return HHT_E_CUDA;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t t = s->next_ticket++;
    Request& r = s->reqs[t];
    r.pts.swap(pts);
    r.im = im;
    r.im.points = r.pts.data();
    s->waiting.push_back(t);
    *ticket = t;
    return HHT_OK;
}

int hht_progress(hht_ctx* c) {
    if (!c) return HHT_E_ARG;
    ServeState* s = serve_of(c);
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    const int rc = engine_step(c, s);
    if (rc != HHT_OK) {
        // the running loop is lost: fail every request in it and start afresh
        std::lock_guard<std::mutex> lk2(s->mu);
        for (uint64_t t : s->order) {
            Request& r = s->reqs[t];
            r.done = true;
            r.status = rc;
            s->free_slots.push_back(r.slot);
            s->finished.push_back(t);
        }
        s->order.clear();
        std::fill(std::begin(s->stream), std::end(s->stream), 0ull);
        std::fill(std::begin(s->regions), std::end(s->regions), 0ull);
        s->n_i64 = 0;
        s->P = s->NV = 0;
        cudaMemsetAsync(s->status.p, 0, sizeof(DeviceStatus), c->stream);
        return rc;
    }
    std::lock_guard<std::mutex> lk2(s->mu);
    return (int)(s->order.size() + s->waiting.size());
}

int hht_done_tickets(hht_ctx* c, uint64_t* tickets, uint64_t capacity, uint64_t* count) {
    if (!c || !count || (capacity > 0 && !tickets)) return HHT_E_ARG;
    ServeState* s = serve_of(c);
    std::lock_guard<std::mutex> lk(s->mu);
    uint64_t n = 0;
    while (n < capacity && !s->finished.empty()) {
        const uint64_t t = s->finished.front();
        s->finished.pop_front();
        if (s->reqs.find(t) == s->reqs.end()) continue;  // already polled
        tickets[n++] = t;
    }
    *count = n;
    return HHT_OK;
}

int hht_poll(hht_ctx* c, uint64_t ticket, hht_result* out) {
    if (!c || !out) return HHT_E_ARG;
    ServeState* s = serve_of(c);
    hht_leaf* dst = out->leaves;
    const uint64_t cap = out->leaf_capacity;
    hht_result res{};
    int rc = HHT_OK;
    void* src = nullptr;
    uint64_t src_bytes = 0;
    cudaStream_t ps = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return HHT_E_UNKNOWN_TICKET;
        Request& r = it->second;
        if (!r.done) return HHT_E_PENDING;
        res = r.res;
        res.leaves = dst;
        res.leaf_capacity = cap;
        rc = r.status;
        if (rc == HHT_OK && (res.n_leaves > cap || (res.n_leaves > 0 && !dst))) {
            out->n_leaves = res.n_leaves;
            return HHT_E_CAPACITY;  // the ticket stays valid: poll again with a larger buffer
        }
        src = r.dev_leaves;
        src_bytes = r.dev_bytes;
        if (rc == HHT_OK && res.n_leaves && !s->poll_stream) {
            cudaSetDevice(c->device);
            if (cudaStreamCreateWithFlags(&s->poll_stream, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                s->poll_stream = nullptr;
                return HHT_E_CUDA;  // nothing released: the poll can be repeated
            }
        }
        ps = s->poll_stream;
        // the ticket is released here; its leaf buffer now belongs to this call
        s->reqs.erase(it);
        // A client that polls without draining hht_done_tickets leaves polled
        // tickets on the completion list: drop them once they outnumber the
        // live requests two to one, so the list stays bounded (amortised
        // O(log n) per request, since after a pass it holds live tickets only).
        if (s->finished.size() > 2 * s->reqs.size() + 64) {
            std::deque<uint64_t> live;
            for (uint64_t t : s->finished)
                if (s->reqs.count(t)) live.push_back(t);
            s->finished.swap(live);
        }
    }
    // The copy needs no lock: the engine finished writing the buffer (and
    // synchronised) before it marked the request done.
    if (src) cudaSetDevice(c->device);
    if (rc == HHT_OK && res.n_leaves) {
        if (copy_out_on(c, dst, src, src_bytes, ps) != HHT_OK || cudaStreamSynchronize(ps) != cudaSuccess) {
            cudaGetLastError();
            rc = HHT_E_CUDA;
        }
    }
    if (src) result_free(c, src, src_bytes);
    *out = res;
    out->status = rc;
    return rc;
}

}  // extern "C"
