// C ABI of libhht.so (declared in include/hht.h): contexts, device memory,
// and the level loop that drives the stage / select / pass kernels.
//
// A job is a set of images; each image contributes two units (its two
// halves).  All units of a job advance level by level through the same
// launches: select(s) turns the level-s vote counters into passed regions or
// leaves, pass(s) reads the level-(s-1) voter stream once and produces the
// level-s stream and the level-(s+1) counters.  Buffers are sized exactly
// from the per-level totals that select() writes; a batch that does not fit
// the memory budget is split into waves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/hht.h"
#include "hht_internal.h"
#include "hht_ctx.h"
#include "hht_serve.h"
#include "hht_trace.h"

using namespace hht;

namespace hht {

int cuda_fail(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return HHT_E_NOMEM;
    return HHT_E_CUDA;
}

// Device memory of the context: the caller's allocator when it gave one
// (hht_create_with_allocator), else cudaMalloc / cudaFree.  Frees happen
// after the context's stream has been synchronised.
static cudaError_t dev_alloc(hht_ctx* c, void** p, size_t bytes) {
    if (c->has_allocator) {
        *p = c->allocator.alloc(bytes, (void*)c->stream, c->allocator.user);
        return (*p && ((uintptr_t)*p % 256) == 0) ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
static void dev_free(hht_ctx* c, void* p, size_t bytes) {
    if (!p) return;
    if (c->has_allocator)
        c->allocator.free(p, bytes, (void*)c->stream, c->allocator.user);
    else
        cudaFree(p);
}

// Grow a device buffer to at least `bytes` (contents are not preserved).
int ensure(hht_ctx* c, DevBuf& b, size_t bytes, bool zero) {
    if (bytes <= b.bytes && b.p) return HHT_OK;
    size_t want = std::max<size_t>(bytes, b.bytes + b.bytes / 4);
    want = (want + 4095) & ~size_t(4095);
    if (want < 4096) want = 4096;
    if (c->budget && c->held - b.bytes + want > c->budget) {
        want = bytes;
        if (c->held - b.bytes + want > c->budget) return HHT_E_NOMEM;
    }
    if (b.p) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, b.p, b.bytes);
        c->held -= b.bytes;
        b.p = nullptr;
        b.bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = dev_alloc(c, &p, want);
    if (e != cudaSuccess && want > bytes) {
        // the growth margin did not fit: the exact size may
        cudaGetLastError();
        if (p) dev_free(c, p, want);
        p = nullptr;
        want = std::max<size_t>((bytes + 4095) & ~size_t(4095), 4096);
        e = dev_alloc(c, &p, want);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (p) dev_free(c, p, want);  // an allocator's block without the needed alignment
        if (c->debug)
            fprintf(stderr, "[hht] allocation of %.3f GB failed (context holds %.3f GB)\n", want / 1e9, c->held / 1e9);
        return HHT_E_NOMEM;
    }
    b.p = p;
    b.bytes = want;
    c->held += want;
    if (zero) {
        e = cudaMemsetAsync(p, 0, want, c->stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return HHT_OK;
}

// Grow a device buffer keeping its first `keep` bytes.
int ensure_keep(hht_ctx* c, DevBuf& b, size_t bytes, size_t keep) {
    if (bytes <= b.bytes && b.p) return HHT_OK;
    if (!b.p || keep == 0) return ensure(c, b, bytes);
    size_t want = std::max<size_t>(bytes, b.bytes + b.bytes / 2);
    want = (want + 4095) & ~size_t(4095);
    if (c->budget && c->held + want > c->budget) {
        want = bytes;
        if (c->held + want > c->budget) return HHT_E_NOMEM;
    }
    void* p = nullptr;
    cudaError_t e0 = dev_alloc(c, &p, want);
    if (e0 != cudaSuccess && want > bytes) {
        cudaGetLastError();  // the growth margin did not fit: try the exact size
        if (p) dev_free(c, p, want);
        p = nullptr;
        want = (bytes + 4095) & ~size_t(4095);
        e0 = dev_alloc(c, &p, want);
    }
    if (e0 != cudaSuccess) {
        cudaGetLastError();
        if (p) dev_free(c, p, want);
        return HHT_E_NOMEM;
    }
    c->held += want;
    cudaError_t e = cudaMemcpyAsync(p, b.p, std::min(keep, b.bytes), cudaMemcpyDeviceToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    dev_free(c, b.p, b.bytes);
    c->held -= b.bytes;
    b.p = p;
    b.bytes = want;
    return e == cudaSuccess ? HHT_OK : cuda_fail(e);
}

int ensure_sized(hht_ctx* c, DevBuf& b, size_t bytes, size_t keep, size_t target) {
    if (bytes <= b.bytes && b.p) return HHT_OK;
    size_t want = std::max<size_t>((std::max(bytes, target) + 4095) & ~size_t(4095), 4096);
    if (want > bytes) {
        // the target is a projection: when it does not fit, the present need does
        const uint64_t held = c->held - (keep == 0 ? b.bytes : 0);
        size_t fr = 0, tot = 0;
        const bool over_budget = c->budget && held + want > c->budget;
        if (over_budget || (cudaMemGetInfo(&fr, &tot) == cudaSuccess && want > fr + (keep == 0 ? b.bytes : 0)))
            want = std::max<size_t>((bytes + 4095) & ~size_t(4095), 4096);
    }
    if (!b.p || keep == 0) {
        if (b.p) {
            cudaStreamSynchronize(c->stream);
            dev_free(c, b.p, b.bytes);
            c->held -= b.bytes;
            b.p = nullptr;
            b.bytes = 0;
        }
        if (c->budget && c->held + want > c->budget) return HHT_E_NOMEM;
        void* p = nullptr;
        if (dev_alloc(c, &p, want) != cudaSuccess) {
            cudaGetLastError();
            if (p) dev_free(c, p, want);
            return HHT_E_NOMEM;
        }
        b.p = p;
        b.bytes = want;
        c->held += want;
        return HHT_OK;
    }
    if (c->budget && c->held + want > c->budget) return HHT_E_NOMEM;
    void* p = nullptr;
    if (dev_alloc(c, &p, want) != cudaSuccess) {
        cudaGetLastError();
        if (p) dev_free(c, p, want);
        return HHT_E_NOMEM;
    }
    c->held += want;
    cudaError_t e = cudaMemcpyAsync(p, b.p, std::min(keep, b.bytes), cudaMemcpyDeviceToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    dev_free(c, b.p, b.bytes);
    c->held -= b.bytes;
    b.p = p;
    b.bytes = want;
    return e == cudaSuccess ? HHT_OK : cuda_fail(e);
}

void release(hht_ctx* c, DevBuf& b) {
    if (b.p) {
        dev_free(c, b.p, b.bytes);
        c->held -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

}  // namespace hht

namespace {

// ---- kernel timing helpers: event pairs are resolved after the job's last sync
cudaEvent_t take_event(hht_ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

struct ProfScope {
    hht_ctx* c;
    int kind;
    cudaEvent_t a = nullptr;
    ProfScope(hht_ctx* c_, int kind_) : c(c_), kind(kind_) {
        if (c->profile) {
            a = take_event(c);
            cudaEventRecord(a, c->stream);
        }
    }
    ~ProfScope() {
        if (c->profile && a) {
            cudaEvent_t b = take_event(c);
            cudaEventRecord(b, c->stream);
            c->pending.push_back({a, b, kind});
        }
    }
};

void resolve_profile(hht_ctx* c) {
    for (auto& p : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        switch (p.kind) {
            case 0: c->prof.stage_ms += ms; break;
            case 1: c->prof.select_ms += ms; break;
            case 3: c->prof.edges_ms += ms; break;
            default: c->prof.pass_ms += ms; break;
        }
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    c->pending.clear();
}

int check_image(const hht_image& im) {
    if (im.n < 0 || im.n > INT32_MAX) return HHT_E_ARG;
    if (im.n > 0 && !im.points) return HHT_E_ARG;
    if (im.W < 1 || im.H < 1 || im.W > HHT_MAX_SIDE || im.H > HHT_MAX_SIDE) return HHT_E_ARG;
    if (im.depth < 1 || im.depth > HHT_MAX_DEPTH) return HHT_E_ARG;
    if (im.T < 1) return HHT_E_ARG;
    return HHT_OK;
}

// The circle test is built on int32 corner arithmetic: log2 L + depth <= 27.
int check_predicate(const hht_ctx* c, const hht_image& im) {
    if (c->predicate != HHT_PREDICATE_FHT) return HHT_OK;
    return hht::ceil_log2_i(std::max(im.W, im.H)) + im.depth <= 27 ? HHT_OK : HHT_E_ARG;
}

constexpr int kSelTile = 1024;   // parents per select tile

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)
#define RK(call)                     \
    do {                             \
        int r_ = (call);             \
        if (r_ != HHT_OK) return r_; \
    } while (0)

// Copy `bytes` of leaves from device memory to a caller's buffer on the
// context's stream.  A large copy into pinned host memory is written by the
// SMs through the buffer's device mapping: on a GB300 they reach host memory
// over NVLink-C2C at a steadier rate than a copy engine gave (whose device ->
// host copies of a few GB ran at about 200 GB/s on some calls and at a tenth
// of that on others).  $HHT_COPY_ENGINE=1 keeps every copy on the copy
// engines.  Anything else (device memory, pageable host memory, unaligned or
// small copies) goes through cudaMemcpyAsync.
}  // namespace

namespace {
// 1: copied by copy16_kernel, 0: by cudaMemcpyAsync, < 0: an error code
int copy_out_impl(hht_ctx* c, void* dst, const void* src, size_t bytes, cudaStream_t st) {
    constexpr size_t kKernelMin = 1u << 20;
    if (bytes >= kKernelMin && !c->copy_engine_only && ((uintptr_t)dst % 16) == 0 && ((uintptr_t)src % 16) == 0 &&
        bytes % 16 == 0) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
            if (launch_copy16(src, at.devicePointer, bytes / 16, c->num_sms * 4, st) != 0) return HHT_E_CUDA;
            return 1;
        }
        cudaGetLastError();
    }
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return 0;
}
}  // namespace

int hht::copy_out(hht_ctx* c, void* dst, const void* src, size_t bytes) {
    const int r = copy_out_impl(c, dst, src, bytes, c->stream);
    if (r < 0) return r;
    c->prof.launches += (uint64_t)r;
    return HHT_OK;
}

int hht::copy_out_on(hht_ctx* c, void* dst, const void* src, size_t bytes, cudaStream_t stream) {
    const int r = copy_out_impl(c, dst, src, bytes, stream);
    return r < 0 ? r : HHT_OK;
}

namespace {

// Host-side description of one wave of a job: its units (two per image),
// where each image's points start, and the sizes every form needs.
struct Wave {
    int count = 0, n_units = 0, Dmax = 0;
    bool i64 = false, fht = false;
    uint64_t total = 0, v0_len = 0;  // points of all images; level-0 voter records
    size_t stats_words = 0;
    std::vector<Unit> units;
    std::vector<uint64_t> img_start;
    std::vector<uint32_t> img_unit;
    uint64_t leaf_base = 0;  // leaves of the job's earlier waves (this wave's follow them)
};

void describe_wave(hht_ctx* c, const hht_image* im, int count, int job_first, Wave& w) {
    w.count = count;
    w.n_units = 2 * count;
    w.fht = c->predicate == HHT_PREDICATE_FHT;
    w.units.assign(w.n_units, Unit{});
    w.img_start.assign(count + 1, 0);
    w.img_unit.assign(count, 0);
    for (int g = 0; g < count; ++g) {
        const int lL = ceil_log2_i(std::max(im[g].W, im[g].H));
        w.Dmax = std::max(w.Dmax, im[g].depth);
        // int32 corner arithmetic is exact while lL + depth <= 27: then
        // |G| <= 4LK = 2^29 at every vertex of the parameter space, and the
        // level kernel's partial sums (u0 = dJ - 1 - G(SW) built as
        // W0 - x*A + (x + y)*K, with |x*A|, (x + y)*K < 2^28, and its column
        // steps of at most 4x*S/4 < 2^28) stay within 1.5 * 2^30; the FHT's
        // 2G values stay within 8LK = 2^30.  Both sides of the switch (27 and
        // 28, on 32767^2 and 16^2 frames, points at the far corners and on
        // lines through one vertex) are checked against the oracle on the GPU.
        if (lL + im[g].depth > 27) w.i64 = true;
        w.img_start[g] = w.total;
        w.img_unit[g] = (uint32_t)(2 * g);
        for (int h = 0; h < 2; ++h) {
            Unit& U = w.units[2 * g + h];
            U.lL = lL;
            U.D = im[g].depth;
            U.T = im[g].T;
            U.image = g;
            U.n = im[g].n;
            U.W = im[g].W;
            U.H = im[g].H;
            U.half = h;
            U.t0 = 0;
            U.root_rec = (uint32_t)(2 * g + h);
            // front-end split images: ALPHA points enter half 0 only, BETA half 1 only
            const bool on = !c->job_halves || ((c->job_halves[job_first + g] >> h) & 1u);
            U.inactive = on ? 0u : 1u;
            if (!on) U.n = 0;
            U.pad2 = 0;
            U.v0_off = w.v0_len;
            if (U.D >= 2 && on) w.v0_len += (uint64_t)im[g].n;
        }
        w.total += (uint64_t)im[g].n;
    }
    w.img_start[count] = w.total;
    w.stats_words = (size_t)w.n_units * (kMaxDepth + 1) * 4;
    w.leaf_base = c->job_leaves;
}

// Inputs and job state on the device, common to both forms: points, units,
// image table, statistics (level 0 filled in), level totals, the level-0
// region records and counters, status, leaf count.
int upload_wave(hht_ctx* c, const hht_image* im, const Wave& w) {
    cudaStream_t st = c->stream;
    const int count = w.count, n_units = w.n_units;
    RK(ensure(c, c->pts, std::max<uint64_t>(w.total, 1) * sizeof(hht_point)));
    for (int g = 0; g < count; ++g)
        if (im[g].n > 0)
            CK(cudaMemcpyAsync((char*)c->pts.p + w.img_start[g] * sizeof(hht_point), im[g].points,
                               (size_t)im[g].n * sizeof(hht_point), cudaMemcpyDefault, st));
    RK(ensure(c, c->units, n_units * sizeof(Unit)));
    RK(ensure(c, c->img_start, (count + 1) * sizeof(uint64_t)));
    RK(ensure(c, c->img_unit, count * sizeof(uint32_t)));
    RK(ensure(c, c->img_err, count * sizeof(uint32_t)));
    RK(ensure(c, c->stats, w.stats_words * sizeof(uint64_t)));
    RK(ensure(c, c->infos, (kMaxDepth + 1) * sizeof(LevelInfo)));
    RK(ensure(c, c->status, sizeof(DeviceStatus)));
    RK(ensure(c, c->leaf_total, sizeof(uint64_t)));
    RK(ensure(c, c->dims, sizeof(JobDims)));
    RK(ensure(c, c->rec[0], n_units * sizeof(Region)));
    RK(ensure(c, c->cnt[0], n_units * 4 * sizeof(uint32_t)));
    RK(ensure(c, c->vox[0], std::max<uint64_t>(w.v0_len, 1) * sizeof(Voter)));

    c->h_stats.assign(w.stats_words, 0);
    for (int u = 0; u < n_units; ++u) {
        uint64_t* s0 = &c->h_stats[(size_t)u * (kMaxDepth + 1) * 4];
        s0[0] = 1;                       // level 0: one region tested
        s0[1] = 1;                       // ... and always split
        s0[3] = (uint64_t)w.units[u].n;  // one code per point
    }
    c->h_infos.assign(kMaxDepth + 1, LevelInfo{});
    c->h_infos[0].n_regions = (uint64_t)n_units;
    c->h_infos[0].n_voters = w.v0_len;
    c->h_roots.resize(n_units);
    for (int u = 0; u < n_units; ++u) c->h_roots[u] = Region{(uint32_t)u, 0u, 0u, (uint32_t)w.units[u].n};
    c->h_dims = JobDims{w.total, count, 0};
    CK(cudaMemcpyAsync(c->units.p, w.units.data(), n_units * sizeof(Unit), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->img_start.p, w.img_start.data(), (count + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice,
                       st));
    CK(cudaMemcpyAsync(c->img_unit.p, w.img_unit.data(), count * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->stats.p, c->h_stats.data(), w.stats_words * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->infos.p, c->h_infos.data(), (kMaxDepth + 1) * sizeof(LevelInfo), cudaMemcpyHostToDevice,
                       st));
    CK(cudaMemcpyAsync(c->rec[0].p, c->h_roots.data(), n_units * sizeof(Region), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->dims.p, &c->h_dims, sizeof(JobDims), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(c->cnt[0].p, 0, n_units * 4 * sizeof(uint32_t), st));
    CK(cudaMemsetAsync(c->status.p, 0, sizeof(DeviceStatus), st));
    CK(cudaMemcpyAsync(c->leaf_total.p, &c->job_leaves, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(c->img_err.p, 0, count * sizeof(uint32_t), st));
    return HHT_OK;
}

// The level form's and the graph form's arguments of step s, apart from the
// capacities and the voter streams, which each form sets.
LevelArgs level_args(hht_ctx* c, int s) {
    const int pi = (s - 1) & 1, ci = s & 1;
    LevelArgs a{};
    a.units = (const Unit*)c->units.p;
    a.parents = (const Region*)c->rec[pi].p;
    a.pregions = (PassRegion*)c->preg[pi].p;
    a.parent_cnt = (const uint32_t*)c->cnt[pi].p;
    a.children = (Region*)c->rec[ci].p;
    a.child_cnt = (uint32_t*)c->cnt[ci].p;
    a.cursor = (unsigned long long*)c->cursors.p;
    a.leaves = (DevLeaf*)c->leaves.p;
    a.stats = (uint64_t*)c->stats.p;
    a.info_prev = (LevelInfo*)c->infos.p + (s - 1);
    a.info = (LevelInfo*)c->infos.p + s;
    a.leaf_total = (uint64_t*)c->leaf_total.p;
    a.status = (DeviceStatus*)c->status.p;
    a.level = s;
    a.num_sms = c->num_sms;
    a.scan = (ScanState*)c->scan_states.p;
    a.tile_flags = (uint32_t*)c->sel_flags.p;
    a.tile_data = (uint64_t*)c->sel_data.p;
    a.withhold_tile_plus1 = c->inject_tile >= 0 ? (uint32_t)(c->inject_tile + 1) : 0u;
    a.keep = c->job_keep;
    a.img_err = (const uint32_t*)c->img_err.p;
    a.keep_level = c->job_keep_level;
    return a;
}

// The level form: stage, then per level one selection and one pass launch,
// every buffer sized exactly from the selection's totals (one host
// synchronisation per level).  On return *leaf_total holds the leaf count
// after the wave and *err the device status bits.
int run_levels(hht_ctx* c, const Wave& w, uint64_t* leaf_total, uint32_t* err) {
    cudaStream_t st = c->stream;
    DeviceStatus* d_status = (DeviceStatus*)c->status.p;
    LevelInfo* d_infos = (LevelInfo*)c->infos.p;
    *leaf_total = w.leaf_base;
    *err = 0;
    {
        TraceRange tr_k("stage");
        ProfScope ps(c, 0);
        if (launch_stage((const int16_t*)c->pts.p, w.total, (const Unit*)c->units.p, w.count,
                         (const uint64_t*)c->img_start.p, (const uint32_t*)c->img_unit.p, (Voter*)c->vox[0].p,
                         (uint32_t*)c->cnt[0].p, (uint64_t*)c->stats.p, (uint32_t*)c->img_err.p, d_status, w.i64,
                         st, w.fht) != 0)
            return HHT_E_CUDA;
        if (w.total > 0) c->prof.launches += 1;
    }
    for (int s = 1; s <= w.Dmax; ++s) {
        TraceRange tr_level(level_name(s));
        const int pi = (s - 1) & 1, ci = s & 1;
        const uint64_t P = c->h_infos[s - 1].n_regions;
        if (P == 0) break;
        if (4 * P > kMaxLevelRecords) return HHT_E_NOMEM;
        RK(ensure(c, c->preg[pi], P * sizeof(PassRegion)));
        RK(ensure(c, c->rec[ci], 4 * P * sizeof(Region)));
        RK(ensure(c, c->cnt[ci], 4 * P * 4 * sizeof(uint32_t)));
        const uint64_t cap_leaves = *leaf_total + 4 * P;
        RK(ensure_keep(c, c->leaves, cap_leaves * sizeof(DevLeaf), *leaf_total * sizeof(DevLeaf)));
        const uint64_t sel_tiles = (P + kSelTile - 1) / kSelTile;
        if ((sel_tiles + 1) * 4 > c->sel_flags.bytes) RK(ensure(c, c->sel_flags, (sel_tiles + 1) * 4, true));
        RK(ensure(c, c->sel_data, (sel_tiles + 1) * 2 * 3 * sizeof(uint64_t)));
        RK(ensure(c, c->cursors, 4 * P * sizeof(unsigned long long)));

        LevelArgs a = level_args(c, s);
        a.cap_children = 4 * P;
        a.cap_leaves = cap_leaves;
        a.cap_tiles = sel_tiles;
        // select's capacity test on the voter stream is re-done below with the exact size
        a.cap_voters = UINT64_MAX;
        const int sel_grid = (int)std::min<uint64_t>(sel_tiles, (uint64_t)c->num_sms * c->occ_select);
        {
            TraceRange tr_k("select");
            ProfScope ps(c, 1);
            if (launch_select(a, 256, std::max(sel_grid, 1), st) != 0) return HHT_E_CUDA;
        }
        c->prof.launches += 1;
        c->prof.select_launches += 1;

        CK(cudaMemcpyAsync(&c->h_infos[s], d_infos + s, sizeof(LevelInfo), cudaMemcpyDeviceToHost, st));
        DeviceStatus hs{};
        CK(cudaMemcpyAsync(&hs, d_status, sizeof hs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *err = hs.err;
        if (c->debug)
            fprintf(stderr, "[hht]   step %d: parents %llu, regions %llu, voters in %llu, out %llu, leaves %llu, held %.2f GB\n",
                    s, (unsigned long long)P, (unsigned long long)c->h_infos[s].n_regions,
                    (unsigned long long)c->h_infos[s - 1].n_voters, (unsigned long long)c->h_infos[s].n_voters,
                    (unsigned long long)c->h_infos[s].n_leaves, c->held / 1e9);
        if (*err) break;
        *leaf_total += c->h_infos[s].n_leaves;
        if (s == w.Dmax) break;

        const uint64_t nin = c->h_infos[s - 1].n_voters;
        if (nin == 0) continue;  // no unit needs level s+1 counts
        const uint64_t nout = c->h_infos[s].n_voters;
        RK(ensure(c, c->vox[ci], std::max<uint64_t>(nout, 1) * sizeof(Voter)));
        a.vin = (const Voter*)c->vox[pi].p;
        a.vout = (Voter*)c->vox[ci].p;
        a.cap_voters = nout;
        const int shape = (w.i64 || w.fht) ? 0 : c->pass_shape;
        const int occ = w.fht ? c->occ_pass_fht : (w.i64 ? c->occ_pass64 : c->occ_shape[shape]);
        // enough warp slices to fill the device, no more than the stream needs
        const uint64_t tile = 8ull * (uint64_t)(w.fht ? 256 : pass_threads(w.i64, shape));
        const uint64_t want_blocks = (nin + tile - 1) / tile;
        const int pass_grid = (int)std::min<uint64_t>(want_blocks, (uint64_t)c->num_sms * occ);
        {
            TraceRange tr_k("pass");
            ProfScope ps(c, 2);
            if (launch_pass(a, w.i64, std::max(pass_grid, 1), st, shape, w.fht) != 0) return HHT_E_CUDA;
        }
        c->prof.launches += 1;
        c->prof.pass_launches += 1;
        c->prof.voters_read += nin;
        c->prof.voters_written += nout;
        c->prof.pass_bytes += 8 * (nin + nout);
    }
    return HHT_OK;
}

// Capacities of the graph form, from hard upper bounds of the wave's sizes.
// At level l a region is a cell of a 2^l x 2^l grid.  A line's voting cells
// in column i are the j with G(i, j) < 0 <= G(i + 1, j + 1), an interval of
// ceil(b_i) - ceil(b_{i+1}) + 1 cells where b_i = j at which G(i, j) = 0;
// summed over the 2^l columns this telescopes to at most
// 2^l + x * 2^l / (2L) + 1 cells, and x < W (half 0) or x < H (half 1).  So a
// half's voters at level l (the votes of its regions) are at most
// n * (2^l + (W_h - 1) 2^l / (2L) + 2), its passed regions at most that / T
// (each holds T votes or more) and 4^l, and its leaves likewise at its depth.
struct GraphCaps {
    uint64_t vox[2] = {1, 1};  // voter records per stream (even / odd levels)
    uint64_t rec[2] = {1, 1};  // region records per level (even / odd levels)
    uint64_t cursors = 1, tiles = 1, leaves = 0;
    uint64_t bytes = 0;
    std::vector<uint64_t> lvl_vox, lvl_rec;  // the bounds of each level
};

uint64_t sat_add(uint64_t a, uint64_t b) { return a > UINT64_MAX - b ? UINT64_MAX : a + b; }

bool graph_caps(const Wave& w, GraphCaps& cap) {
    std::vector<uint64_t> vox(w.Dmax + 1, 0), rec(w.Dmax + 1, 0);
    uint64_t leaves = 0;
    for (int u = 0; u < w.n_units; ++u) {
        const Unit& U = w.units[u];
        const uint64_t n = (uint64_t)U.n;
        const uint64_t L = 1ull << U.lL;
        const uint64_t Wh = (uint64_t)(U.half ? U.H : U.W);
        // votes of all level-l regions (n lines of at most per_line cells,
        // and no more cells than the level has): below 2^56 for D <= 24
        auto votes = [&](int l) {
            const uint64_t col = 1ull << l;
            const uint64_t per_line = col + (Wh - 1) * col / (2 * L) + 2;
            return n * std::min(per_line, col * col);
        };
        for (int l = 0; l <= U.D; ++l) {
            if (l <= U.D - 2) vox[l] = sat_add(vox[l], votes(l));
            if (l == 0) rec[0] = sat_add(rec[0], 1);  // the level-0 region of every unit
            else if (l < U.D) rec[l] = sat_add(rec[l], std::min<uint64_t>(1ull << (2 * l), votes(l) / (uint64_t)U.T));
        }
        leaves = sat_add(leaves, std::min<uint64_t>(1ull << (2 * U.D), votes(U.D) / (uint64_t)U.T));
    }
    cap.lvl_vox = vox;
    cap.lvl_rec = rec;
    for (int l = 0; l <= w.Dmax; ++l) {
        cap.vox[l & 1] = std::max(cap.vox[l & 1], vox[l]);
        cap.rec[l & 1] = std::max(cap.rec[l & 1], rec[l]);
        if (l >= 1) cap.cursors = std::max(cap.cursors, rec[l]);
    }
    // 32-bit region indices, and sizes far beyond any device
    if (std::max(cap.rec[0], cap.rec[1]) > kMaxLevelRecords) return false;
    if (std::max(cap.vox[0], cap.vox[1]) > (1ull << 40) || leaves > (1ull << 40)) return false;
    cap.tiles = (std::max(cap.rec[0], cap.rec[1]) + kSelTile - 1) / kSelTile + 1;
    cap.leaves = leaves;
    cap.bytes = 8 * (cap.vox[0] + cap.vox[1]) +
                (cap.rec[0] + cap.rec[1]) * (sizeof(Region) + sizeof(PassRegion) + 4 * sizeof(uint32_t)) +
                cap.cursors * sizeof(unsigned long long) + cap.tiles * (4 + 2 * 3 * sizeof(uint64_t)) +
                (w.leaf_base + leaves) * sizeof(DevLeaf) + 64 * w.total;
    return true;
}

// Allocate the graph form's buffers; false when they do not fit the budget
// (the wave then runs level by level).
bool size_graph_buffers(hht_ctx* c, const Wave& w, GraphCaps& cap) {
    if (!graph_caps(w, cap)) return false;
    uint64_t budget = c->budget;
    if (!budget) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        budget = (uint64_t)((double)(fr + c->held) * 0.8);
    }
    if (cap.bytes > budget) return false;
    for (int k = 0; k < 2; ++k) {
        if (ensure(c, c->vox[k], cap.vox[k] * sizeof(Voter)) != HHT_OK) return false;
        if (ensure(c, c->rec[k], cap.rec[k] * sizeof(Region)) != HHT_OK) return false;
        if (ensure(c, c->preg[k], cap.rec[k] * sizeof(PassRegion)) != HHT_OK) return false;
        if (ensure(c, c->cnt[k], cap.rec[k] * 4 * sizeof(uint32_t)) != HHT_OK) return false;
    }
    if (ensure(c, c->cursors, cap.cursors * sizeof(unsigned long long)) != HHT_OK) return false;
    if (cap.tiles * 4 > c->sel_flags.bytes && ensure(c, c->sel_flags, cap.tiles * 4, true) != HHT_OK) return false;
    if (ensure(c, c->sel_data, cap.tiles * 2 * 3 * sizeof(uint64_t)) != HHT_OK) return false;
    if (ensure_keep(c, c->leaves, std::max<uint64_t>(w.leaf_base + cap.leaves, 1) * sizeof(DevLeaf),
                    w.leaf_base * sizeof(DevLeaf)) != HHT_OK)
        return false;
    // the kernels are told the room the buffers have (at least the bounds):
    // a later job that fits the same buffers then replays the same graph
    const uint64_t cur = c->cursors.bytes / sizeof(unsigned long long);
    for (int k = 0; k < 2; ++k) {
        cap.vox[k] = c->vox[k].bytes / sizeof(Voter);
        cap.rec[k] = std::min({c->rec[k].bytes / sizeof(Region), c->preg[k].bytes / sizeof(PassRegion),
                               c->cnt[k].bytes / (4 * sizeof(uint32_t)), cur, (uint64_t)kMaxLevelRecords});
    }
    cap.tiles = std::min<uint64_t>(c->sel_flags.bytes / 4, c->sel_data.bytes / (2 * 3 * sizeof(uint64_t)));
    return true;
}

// Grids of the graph form's launches, from each level's bounds: a level's
// selection needs no more blocks than its parents fill tiles, and its pass
// no more warps than the parents' voter stream holds grabs, so the launches
// of a small job (or of a large job's first levels) are small.  Every kernel
// takes its work dynamically, so any grid of at least these sizes gives the
// same result: a captured graph whose grids cover a job's is replayed for
// it, and a new one is captured with each grid rounded up to a power of two
// (at most the full grid), so that jobs of similar size share it.
// Layout: [stage, sel[1..Dmax], pass[1..Dmax]].
std::vector<int> graph_grids(const hht_ctx* c, const Wave& w, const GraphCaps& cap) {
    const int shape = w.i64 ? 0 : c->pass_shape;
    const uint64_t occ = (uint64_t)(w.i64 ? c->occ_pass64 : c->occ_shape[shape]);
    const uint64_t warps_per_block = (uint64_t)pass_threads(w.i64, shape) / 32;
    auto fit = [](uint64_t want, uint64_t most) {
        uint64_t p = 1;
        while (p < want && p < most) p <<= 1;
        return (int)std::min(p, most);
    };
    std::vector<int> g(1 + 2 * (size_t)w.Dmax, 1);
    g[0] = fit((w.total + 255) / 256, (uint64_t)c->num_sms * 8);
    for (int s = 1; s <= w.Dmax; ++s) {
        g[s] = fit((cap.lvl_rec[s - 1] + kSelTile - 1) / kSelTile, (uint64_t)c->num_sms * c->occ_select);
        const uint64_t grabs = (cap.lvl_vox[s - 1] + kPassMinGrab - 1) / kPassMinGrab;
        g[w.Dmax + s] = fit((grabs + warps_per_block - 1) / warps_per_block, (uint64_t)c->num_sms * occ);
    }
    return g;
}

bool grids_cover(const std::vector<int>& have, const std::vector<int>& need) {
    if (have.size() != need.size()) return false;
    for (size_t k = 0; k < need.size(); ++k)
        if (have[k] < need[k]) return false;
    return true;
}

// Launch the graph form's kernels on the context's stream: the stage kernel
// (sizes from the JobDims in device memory), then for every level the
// selection and the pass, all with fixed arguments; every kernel reads the
// sizes of its level from the level totals that the previous selection wrote.
// With `evs`, a pair of events (recorded as graph nodes when capturing)
// brackets every kernel for hht_profile_*.
int launch_graph_kernels(hht_ctx* c, const Wave& w, const GraphCaps& cap, const std::vector<int>& grids,
                         cudaStream_t st, bool capturing, std::vector<hht_ctx::GraphEvent>* evs) {
    const int shape = w.i64 ? 0 : c->pass_shape;
    auto record = [&]() -> cudaEvent_t {
        cudaEvent_t e = take_event(c);
        if (capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else cudaEventRecord(e, st);
        return e;
    };
    cudaEvent_t e0 = nullptr;
    auto open = [&]() { e0 = evs ? record() : nullptr; };
    auto close = [&](int kind) {
        if (evs) evs->push_back({e0, record(), kind});
    };
    open();
    if (launch_stage((const int16_t*)c->pts.p, w.total, (const Unit*)c->units.p, w.count,
                     (const uint64_t*)c->img_start.p, (const uint32_t*)c->img_unit.p, (Voter*)c->vox[0].p,
                     (uint32_t*)c->cnt[0].p, (uint64_t*)c->stats.p, (uint32_t*)c->img_err.p,
                     (DeviceStatus*)c->status.p, w.i64, st, false, (const JobDims*)c->dims.p, grids[0]) != 0)
        return HHT_E_CUDA;
    close(0);
    for (int s = 1; s <= w.Dmax; ++s) {
        const int pi = (s - 1) & 1, ci = s & 1;
        LevelArgs a = level_args(c, s);
        a.cap_children = cap.rec[ci];
        a.cap_leaves = c->leaves.bytes / sizeof(DevLeaf);
        a.cap_tiles = cap.tiles;
        a.cap_voters = cap.vox[ci];
        a.vin = (const Voter*)c->vox[pi].p;
        a.vout = (Voter*)c->vox[ci].p;
        open();
        if (launch_select(a, 256, grids[s], st) != 0) return HHT_E_CUDA;
        close(1);
        if (s == w.Dmax) break;
        open();
        if (launch_pass(a, w.i64, grids[w.Dmax + s], st, shape, false) != 0) return HHT_E_CUDA;
        close(2);
    }
    return HHT_OK;
}

// The graph form: every kernel of the wave's level loop in one CUDA graph,
// captured once per argument set and replayed, so that a job is one graph
// launch and one host synchronisation.  On the legacy default stream, where
// capture is impossible, or if capture failed once, the same kernels are
// launched directly (still with no host synchronisation between levels).
// Event pairs captured into the graph stay with it; those of a direct launch
// go back to the pool once read.
int run_graph(hht_ctx* c, const Wave& w, const GraphCaps& cap, uint64_t* leaf_total, uint32_t* err) {
    // The legacy default stream cannot be captured: the graph then runs on the
    // context's own blocking stream, which the legacy stream orders against in
    // both directions (its earlier work runs first, its later work waits).
    if (!c->stream && !c->own_stream) {
        if (cudaStreamCreate(&c->own_stream) != cudaSuccess) {
            cudaGetLastError();
            c->own_stream = nullptr;
        }
    }
    cudaStream_t st = c->stream ? c->stream : c->own_stream;
    const bool events = c->profile;
    // everything the captured kernels take as arguments
    std::vector<unsigned char> key;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        key.insert(key.end(), b, b + n);
    };
    const void* ptrs[] = {c->pts.p,  c->units.p, c->img_start.p, c->img_unit.p, c->img_err.p, c->stats.p,
                          c->infos.p, c->status.p, c->leaf_total.p, c->dims.p, c->rec[0].p, c->rec[1].p,
                          c->preg[0].p, c->preg[1].p, c->cnt[0].p, c->cnt[1].p, c->vox[0].p, c->vox[1].p,
                          c->cursors.p, c->leaves.p, c->sel_flags.p, c->sel_data.p, c->scan_states.p, (void*)st};
    put(ptrs, sizeof ptrs);
    const int64_t vals[] = {w.Dmax, w.i64, c->pass_shape, events, c->num_sms, c->inject_tile,
                            (int64_t)(c->leaves.bytes / sizeof(DevLeaf)), (int64_t)cap.tiles,
                            (int64_t)cap.vox[0], (int64_t)cap.vox[1], (int64_t)cap.rec[0], (int64_t)cap.rec[1]};
    put(vals, sizeof vals);
    const std::vector<int> grids = graph_grids(c, w, cap);
    auto release = [&](hht_ctx::CachedGraph& cg) {
        for (auto& ev : cg.events) {
            c->ev_pool.push_back(ev.a);
            c->ev_pool.push_back(ev.b);
        }
        cg.events.clear();
        if (cg.exec) cudaGraphExecDestroy(cg.exec);
        cg.exec = nullptr;
    };

    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool can_capture = st != nullptr && !c->graph_capture_failed &&
                             cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    const hht_ctx::CachedGraph* use = nullptr;
    if (can_capture) {
        // of the graphs of these arguments whose grids cover the job's, the
        // one with the smallest grids (the most recently used among equals)
        size_t hit = c->graphs.size();
        long long best = -1;
        for (size_t k = 0; k < c->graphs.size(); ++k) {
            if (c->graphs[k].key != key || !grids_cover(c->graphs[k].grids, grids)) continue;
            long long sum = 0;
            for (int g : c->graphs[k].grids) sum += g;
            if (best < 0 || sum < best) {
                best = sum;
                hit = k;
            }
        }
        if (hit < c->graphs.size()) {
            std::rotate(c->graphs.begin(), c->graphs.begin() + hit, c->graphs.begin() + hit + 1);
        } else {
            hht_ctx::CachedGraph cg;
            cg.key = key;
            cg.grids = grids;
            cudaGraph_t g = nullptr;
            bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                const int lr = launch_graph_kernels(c, w, cap, grids, st, true, events ? &cg.events : nullptr);
                ok = cudaStreamEndCapture(st, &g) == cudaSuccess && lr == HHT_OK && g != nullptr;
            }
            if (ok) ok = cudaGraphInstantiate(&cg.exec, g, 0) == cudaSuccess;
            if (g) cudaGraphDestroy(g);
            if (ok) {
                c->prof.graph_captures += 1;
                if (c->graphs.size() >= hht_ctx::kGraphCache) {
                    release(c->graphs.back());
                    c->graphs.pop_back();
                }
                c->graphs.insert(c->graphs.begin(), std::move(cg));
            } else {
                cudaGetLastError();
                release(cg);
                c->graph_capture_failed = true;  // launch directly from now on
            }
        }
        if (!c->graphs.empty() && c->graphs.front().key == key && grids_cover(c->graphs.front().grids, grids))
            use = &c->graphs.front();
    }
    std::vector<hht_ctx::GraphEvent> direct;
    const bool graph = use != nullptr;
    if (graph) {
        TraceRange tr_k("level loop (graph)");
        CK(cudaGraphLaunch(use->exec, st));
    } else {
        TraceRange tr_k("level loop (direct launches)");
        RK(launch_graph_kernels(c, w, cap, grids, st, false, events ? &direct : nullptr));
    }
    // one read-back of the level totals, the statistics, the image errors,
    // the leaf count and the status (on the graph's stream), through the
    // page-locked staging buffer when it could be had
    DeviceStatus hs{};
    c->h_img_err.assign(w.count, 0);
    const size_t b_inf = (w.Dmax + 1) * sizeof(LevelInfo), b_st = w.stats_words * sizeof(uint64_t),
                 b_err = w.count * sizeof(uint32_t);
    const size_t o_st = (b_inf + 15) & ~size_t(15), o_err = (o_st + b_st + 15) & ~size_t(15),
                 o_tot = (o_err + b_err + 15) & ~size_t(15), o_hs = o_tot + 16, need = o_hs + sizeof(DeviceStatus);
    if (need > c->h_stage_bytes) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        const size_t want = std::max<size_t>(need + need / 2, 64 << 10);
        if (cudaHostAlloc(&c->h_stage, want, cudaHostAllocDefault) == cudaSuccess) {
            c->h_stage_bytes = want;
        } else {
            cudaGetLastError();
            c->h_stage = nullptr;
        }
    }
    char* hb = (char*)c->h_stage;
    struct Copy {
        void* dst;
        const void* src;
        size_t off, bytes;
    } copies[] = {{c->h_infos.data(), c->infos.p, 0, b_inf},
                  {c->h_stats.data(), c->stats.p, o_st, b_st},
                  {c->h_img_err.data(), c->img_err.p, o_err, b_err},
                  {leaf_total, c->leaf_total.p, o_tot, sizeof(uint64_t)},
                  {&hs, c->status.p, o_hs, sizeof hs}};
    for (const Copy& k : copies)
        CK(cudaMemcpyAsync(hb ? (void*)(hb + k.off) : k.dst, k.src, k.bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hb)
        for (const Copy& k : copies) std::memcpy(k.dst, hb + k.off, k.bytes);
    *err = hs.err;
    if (events) {
        for (const auto& ev : graph ? use->events : direct) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev.a, ev.b) != cudaSuccess) {
                cudaGetLastError();
                ms = 0.f;
            }
            switch (ev.kind) {
                case 0: c->prof.stage_ms += ms; break;
                case 1: c->prof.select_ms += ms; break;
                default: c->prof.pass_ms += ms; break;
            }
        }
        for (auto& ev : direct) {
            c->ev_pool.push_back(ev.a);
            c->ev_pool.push_back(ev.b);
        }
    }
    c->prof.graph_launches += graph ? 1 : 0;
    c->prof.launches += (uint64_t)(2 * w.Dmax);  // stage, Dmax selections, Dmax - 1 passes
    c->prof.select_launches += (uint64_t)w.Dmax;
    for (int s = 1; s < w.Dmax; ++s) {
        const uint64_t nin = c->h_infos[s - 1].n_voters, nout = c->h_infos[s].n_voters;
        c->prof.pass_launches += 1;
        c->prof.voters_read += nin;
        c->prof.voters_written += nout;
        c->prof.pass_bytes += 8 * (nin + nout);
    }
    if (c->debug)
        for (int s = 1; s <= w.Dmax; ++s)
            fprintf(stderr, "[hht]   graph step %d: regions %llu, voters %llu, leaves %llu\n", s,
                    (unsigned long long)c->h_infos[s].n_regions, (unsigned long long)c->h_infos[s].n_voters,
                    (unsigned long long)c->h_infos[s].n_leaves);
    return HHT_OK;
}

// Statistics, per-image leaf offsets and the copy of each image's leaves into
// its result (both forms).  `synced`: the statistics, image errors and status
// have been read back already (the graph form reads them with its totals).
int finish_wave(hht_ctx* c, const hht_image* im, const Wave& w, hht_result* outs, int job_first,
                uint64_t leaf_total, uint32_t err, bool synced) {
    cudaStream_t st = c->stream;
    const int count = w.count;
    if (!synced) {
        CK(cudaMemcpyAsync(c->h_stats.data(), c->stats.p, w.stats_words * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                           st));
        c->h_img_err.assign(count, 0);
        CK(cudaMemcpyAsync(c->h_img_err.data(), c->img_err.p, count * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        DeviceStatus hs{};
        CK(cudaMemcpyAsync(&hs, c->status.p, sizeof hs, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        err |= hs.err;
    }
    if (err & kErrTimeout) return HHT_E_TIMEOUT;
    if (err & kErrOverflow) return HHT_E_NOMEM;
    if (err & kErrInvariant) return HHT_E_CUDA;
    if (err & kErrBounds) {
        if (c->debug) fprintf(stderr, "[hht] a kernel met an out-of-range index (checked build)\n");
        return HHT_E_CUDA;
    }

    // Leaves need no sort: a step emits the leaves of the units whose depth it
    // reaches, in record order, and records stay in depth-first order (children
    // in quadrant order NE, NW, SW, SE under their parent, parents in order), so
    // every unit's leaves form one block in the order of the paper's
    // depth-first traversal, and blocks follow (depth, unit).  The selection
    // writes each leaf's half directly, so the leaves are final as written.
    std::vector<uint64_t> img_leaves(count, 0), img_off(count, 0);
    for (int g = 0; g < count; ++g)
        for (int h = 0; h < 2; ++h)
            img_leaves[g] += c->h_stats[((size_t)(2 * g + h) * (kMaxDepth + 1) + im[g].depth) * 4 + 1];
    {
        std::vector<int> order(count);
        for (int g = 0; g < count; ++g) order[g] = g;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return im[x].depth < im[y].depth; });
        uint64_t acc = w.leaf_base;
        for (int g : order) {
            img_off[g] = acc;
            acc += img_leaves[g];
        }
        if (acc != leaf_total) return HHT_E_CUDA;
    }
    c->job_leaves = leaf_total;
    for (int g = 0; g < count; ++g) {
        const uint64_t off = img_off[g];
        hht_result& r = outs[g];
        const int D = im[g].depth;
        r.depth = D;
        r.L = 1 << ceil_log2_i(std::max(im[g].W, im[g].H));
        std::memset(r.stats, 0, sizeof r.stats);
        uint64_t nl = 0;
        for (int h = 0; h < 2; ++h) {
            const uint64_t* su = &c->h_stats[(size_t)(2 * g + h) * (kMaxDepth + 1) * 4];
            for (int l = 0; l <= D; ++l) {
                r.stats[h][l].tested = su[4 * l + 0];
                r.stats[h][l].passed = su[4 * l + 1];
                r.stats[h][l].votes = su[4 * l + 2];
                r.stats[h][l].tests = su[4 * l + 3];
            }
            nl += su[4 * D + 1];
        }
        r.n_leaves = nl;
        c->job_off[job_first + g] = off;
        c->job_n[job_first + g] = c->h_img_err[g] ? 0 : nl;
        if (c->h_img_err[g]) {
            r.status = HHT_E_RANGE;
        } else if (nl > r.leaf_capacity || (nl > 0 && !r.leaves)) {
            r.status = HHT_E_CAPACITY;
        } else {
            r.status = HHT_OK;
            if (nl > 0) {
                RK(copy_out(c, r.leaves, (const char*)c->leaves.p + off * sizeof(DevLeaf), nl * sizeof(hht_leaf)));
            }
        }
    }
    CK(cudaStreamSynchronize(st));
    if (c->profile) resolve_profile(c);
    return HHT_OK;
}

// Run one wave of images through the level loop; fills outs[k] for k in
// [0, count).  Returns HHT_OK or a job-level error (per-image errors are in
// outs[k].status).  The graph form runs when the context asks for it, the
// wave's upper bounds fit the memory budget and the job is of the exact
// test without a subtree keep mask; the level form otherwise.
int run_wave(hht_ctx* c, const hht_image* im, int count, hht_result* outs, int job_first) {
    Wave w;
    describe_wave(c, im, count, job_first, w);
    if (w.fht && w.i64) return HHT_E_ARG;  // checked by the entry points before any device work
    GraphCaps cap;
    const bool graph = c->batch_mode == HHT_BATCH_GRAPH && !w.fht && !c->job_keep && size_graph_buffers(c, w, cap);
    if (graph && c->inject_graph_cap >= 0) {
        // hht_inject_fault: the kernels are told of less room than the buffer has
        cap.vox[1] = std::min<uint64_t>(cap.vox[1], (uint64_t)c->inject_graph_cap);
        c->inject_graph_cap = -1;
    }
    RK(upload_wave(c, im, w));
    uint64_t leaf_total = w.leaf_base;
    uint32_t err = 0;
    if (graph) {
        RK(run_graph(c, w, cap, &leaf_total, &err));
        if (!(err & kErrOverflow)) return finish_wave(c, im, w, outs, job_first, leaf_total, err, true);
        // the bounds hold for every input, so this is a defect; the wave is
        // still answered, level by level with exact sizes
        c->prof.graph_fallbacks += 1;
        if (c->debug) fprintf(stderr, "[hht] graph form ran out of room; rerun level by level\n");
        c->job_leaves = w.leaf_base;
        RK(upload_wave(c, im, w));
        err = 0;
    }
    RK(run_levels(c, w, &leaf_total, &err));
    return finish_wave(c, im, w, outs, job_first, leaf_total, err, false);
}


// Upper estimate of a wave member's peak device bytes (two voter streams of
// the two deepest written levels, both halves, dense regime).
uint64_t estimate_bytes(const hht_image& im, bool fht) {
    const double n = (double)im.n;
    const int D = im.depth;
    if (D < 3) return (uint64_t)(64.0 * n + 4096);
    const double dense = 1.25 * n * (std::ldexp(1.0, D - 2) + std::ldexp(1.0, D - 3));
    // the circle test's wider voter lists (the paper reports 2-8 times the votes)
    const double widen = fht ? 4.0 : 1.0;
    return (uint64_t)(2.0 * 8.0 * dense * 1.2 * widen + 64.0 * n + 4096);
}

int run_waves(hht_ctx* c, const hht_image* im, int count, hht_result* outs, int job_first) {
    // wave split by the memory budget (or 80% of the free device memory)
    uint64_t budget = c->budget;
    if (!budget) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        budget = (uint64_t)((double)(fr + c->held) * 0.8);
    }
    if (c->wave_cap && c->wave_cap < budget) budget = c->wave_cap;
    int first = 0;
    int rc_all = HHT_OK;
    while (first < count) {
        int last = first;
        uint64_t acc = 0;
        while (last < count) {
            const uint64_t e = estimate_bytes(im[last], c->predicate == HHT_PREDICATE_FHT);
            if (last > first && acc + e > budget) break;
            acc += e;
            ++last;
        }
        if (c->debug)
            fprintf(stderr, "[hht] wave of images [%d, %d): estimate %.2f GB, budget %.2f GB\n", first, last, acc / 1e9,
                    budget / 1e9);
        const uint64_t leaves_before = c->job_leaves;
        int rc = run_wave(c, im + first, last - first, outs + first, job_first + first);
        if (rc == HHT_E_NOMEM && last - first > 1) {
            // remember that this much did not fit, split the wave and retry each half
            c->wave_cap = acc / 2 > 0 ? acc / 2 : 1;
            if (c->debug) fprintf(stderr, "[hht] wave did not fit; wave estimate cap now %.2f GB\n", c->wave_cap / 1e9);
            c->job_leaves = leaves_before;
            const int mid = first + (last - first) / 2;
            rc = run_waves(c, im + first, mid - first, outs + first, job_first + first);
            if (rc == HHT_OK) rc = run_waves(c, im + mid, last - mid, outs + mid, job_first + mid);
        }
        if (rc != HHT_OK) {
            for (int g = first; g < last; ++g) outs[g].status = rc;
            return rc;
        }
        for (int g = first; g < last; ++g)
            if (outs[g].status != HHT_OK && rc_all == HHT_OK) rc_all = outs[g].status;
        first = last;
    }
    return rc_all;
}

int run_job(hht_ctx* c, const hht_image* im, int count, hht_result* outs, const uint8_t* halves = nullptr) {
    TraceRange tr("hht detection job");
    c->job_halves = halves;
    c->job_serial += 1;
    c->job_off.assign(count, 0);
    c->job_n.assign(count, 0);
    c->job_leaves = 0;
    const int rc = run_waves(c, im, count, outs, 0);
    c->inject_tile = -1;  // an injected fault lasts one job
    c->job_halves = nullptr;
    return rc;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

int hht_create(hht_ctx** out, int device, void* cuda_stream, uint64_t mem_budget_bytes) {
    return hht_create_with_allocator(out, device, cuda_stream, mem_budget_bytes, nullptr);
}

int hht_create_with_allocator(hht_ctx** out, int device, void* cuda_stream, uint64_t mem_budget_bytes,
                              const hht_allocator* allocator) {
    if (!out) return HHT_E_ARG;
    if (allocator && (!allocator->alloc || !allocator->free)) return HHT_E_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return HHT_E_CUDA;
    }
    if (device < 0 || device >= ndev) return HHT_E_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return HHT_E_CUDA;
    hht_ctx* c = new (std::nothrow) hht_ctx();
    if (!c) return HHT_E_NOMEM;
    c->device = device;
    if (allocator) {
        c->allocator = *allocator;
        c->has_allocator = true;
    }
    c->debug = getenv("HHT_DEBUG") && getenv("HHT_DEBUG")[0] == '1';
    c->stream = (cudaStream_t)cuda_stream;
    c->budget = mem_budget_bytes;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    c->occ_select = occupancy_select();
    c->occ_pass32 = occupancy_pass(false);
    c->occ_pass64 = occupancy_pass(true);
    for (int k = 0; k < kPassShapeCount; ++k) c->occ_shape[k] = occupancy_pass(false, k);
    c->occ_pass_fht = occupancy_pass_fht();
    if (const char* e = getenv("HHT_BATCH_MODE")) c->batch_mode = atoi(e) == 0 ? HHT_BATCH_LEVELS : HHT_BATCH_GRAPH;
    c->copy_engine_only = getenv("HHT_COPY_ENGINE") && getenv("HHT_COPY_ENGINE")[0] == '1';
    if (const char* e = getenv("HHT_PASS_SHAPE")) {
        const int k = atoi(e);
        if (k >= 0 && k < kPassShapeCount) c->pass_shape = k;
    }
    int rc = ensure(c, c->scan_states, 8 * sizeof(ScanState), true);
    if (rc == HHT_OK) {
        std::vector<ScanState> init(8, ScanState{0u, 0u, 1u, 0u});
        if (cudaMemcpyAsync(c->scan_states.p, init.data(), 8 * sizeof(ScanState), cudaMemcpyHostToDevice, c->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            rc = HHT_E_CUDA;
    }
    if (rc != HHT_OK) {
        hht_destroy(c);
        return rc;
    }
    *out = c;
    return HHT_OK;
}

void hht_destroy(hht_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    hht::serve_destroy(c->serve);
    resolve_profile(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (auto& cg : c->graphs) {
        if (cg.exec) cudaGraphExecDestroy(cg.exec);
        for (auto& ev : cg.events) {
            cudaEventDestroy(ev.a);
            cudaEventDestroy(ev.b);
        }
    }
    if (c->own_stream) {
        cudaStreamSynchronize(c->own_stream);
        cudaStreamDestroy(c->own_stream);
    }
    if (c->h_stage) cudaFreeHost(c->h_stage);
    DevBuf* all[] = {&c->pts,       &c->img_start,  &c->img_unit, &c->units,        &c->stats,     &c->infos,      &c->status,
                     &c->leaf_total, &c->img_err,   &c->scan_states,  &c->rec[0],    &c->rec[1],     &c->preg[0],
                     &c->preg[1],   &c->cnt[0],     &c->cnt[1],       &c->vox[0],    &c->vox[1],     &c->leaves,
                     &c->sel_flags, &c->sel_data,   &c->cursors,      &c->img_buf,   &c->edge_pts[0],
                     &c->edge_pts[1], &c->edge_tot,   &c->line_keys,    &c->line_vals, &c->line_parent,
                     &c->line_cells, &c->line_sums,  &c->line_out,     &c->keep_buf,  &c->rem_pts,
                     &c->rem_lists,  &c->rem_bitmap, &c->rem_leaves,   &c->rem_stats, &c->rem_tasks,
                     &c->dims, &c->rem_flags, &c->rem_raster};
    for (DevBuf* b : all) release(c, *b);
    delete c;
}

int hht_detect(hht_ctx* c, const hht_point* points, int64_t n, int32_t W, int32_t H, int32_t depth, int32_t T,
               hht_result* out) {
    if (!c || !out) return HHT_E_ARG;
    hht_image im{points, n, W, H, depth, T};
    int rc = check_image(im);
    if (rc != HHT_OK) return rc;
    std::lock_guard<std::mutex> lk(c->mu);
    rc = check_predicate(c, im);
    if (rc != HHT_OK) return rc;
    cudaSetDevice(c->device);
    rc = run_job(c, &im, 1, out);
    if (rc != HHT_OK) return rc;
    return out->status;
}

int hht_detect_batch(hht_ctx* c, const hht_image* images, int32_t count, hht_result* outs) {
    if (!c || !outs || count < 0 || (count > 0 && !images)) return HHT_E_ARG;
    if (count == 0) return HHT_OK;
    if (count > (1 << 20)) return HHT_E_ARG;
    for (int g = 0; g < count; ++g) {
        const int rc = check_image(images[g]);
        if (rc != HHT_OK) return rc;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    for (int g = 0; g < count; ++g) {
        const int rc = check_predicate(c, images[g]);
        if (rc != HHT_OK) return rc;
    }
    cudaSetDevice(c->device);
    return run_job(c, images, count, outs);
}

int hht_fetch_leaves(hht_ctx* c, int32_t index, hht_leaf* leaves, uint64_t capacity) {
    if (!c) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (index < 0 || (size_t)index >= c->job_n.size()) return HHT_E_ARG;
    const uint64_t n = c->job_n[index];
    if (n == 0) return HHT_OK;
    if (!leaves) return HHT_E_ARG;
    if (capacity < n) return HHT_E_CAPACITY;
    cudaSetDevice(c->device);
    RK(copy_out(c, leaves, (const char*)c->leaves.p + c->job_off[index] * sizeof(DevLeaf), n * sizeof(hht_leaf)));
    CK(cudaStreamSynchronize(c->stream));
    return HHT_OK;
}

int hht_fetch_all_leaves(hht_ctx* c, hht_leaf* leaves, uint64_t capacity, uint64_t* offsets, uint64_t* counts,
                         uint64_t* total) {
    if (!c || !total) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    *total = c->job_leaves;
    if (capacity < c->job_leaves) return HHT_E_CAPACITY;
    if (c->job_leaves > 0 && !leaves) return HHT_E_ARG;
    for (size_t k = 0; k < c->job_n.size(); ++k) {
        if (offsets) offsets[k] = c->job_off[k];
        if (counts) counts[k] = c->job_n[k];
    }
    if (c->job_leaves == 0) return HHT_OK;
    cudaSetDevice(c->device);
    RK(copy_out(c, leaves, c->leaves.p, c->job_leaves * sizeof(hht_leaf)));
    CK(cudaStreamSynchronize(c->stream));
    return HHT_OK;
}

int hht_set_batch_mode(hht_ctx* c, int32_t mode) {
    if (!c || (mode != HHT_BATCH_LEVELS && mode != HHT_BATCH_GRAPH)) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    c->batch_mode = mode;
    return HHT_OK;
}

int hht_set_tuning(hht_ctx* c, int32_t shape) {
    if (!c || shape < 0 || shape >= kPassShapeCount) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    c->pass_shape = shape;
    return HHT_OK;
}

int hht_autotune(hht_ctx* c, const hht_image* images, int32_t count, int32_t* best, double* ms_per_shape) {
    if (!c || !best || count < 1 || !images) return HHT_E_ARG;
    for (int g = 0; g < count; ++g) {
        const int rc = check_image(images[g]);
        if (rc != HHT_OK) return rc;
    }
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    std::vector<hht_result> outs((size_t)count);
    // the tile shapes are those of the exact test's level kernel
    const int saved_predicate = c->predicate;
    c->predicate = HHT_PREDICATE_EXACT;
    const bool was_profiling = c->profile;
    const hht_profile_counters saved = c->prof;
    double best_ms = 1e300;
    int best_shape = c->pass_shape;
    int rc = HHT_OK;
    // warm-up with the current shape (allocations), then every shape timed by
    // its pass launches; no leaves are copied out (HHT_E_CAPACITY is expected)
    rc = run_job(c, images, count, outs.data());
    if (rc == HHT_E_CAPACITY) rc = HHT_OK;
    for (int k = 0; k < kPassShapeCount && rc == HHT_OK; ++k) {
        c->pass_shape = k;
        c->profile = true;
        c->prof = hht_profile_counters{};
        rc = run_job(c, images, count, outs.data());
        if (rc == HHT_E_CAPACITY) rc = HHT_OK;
        resolve_profile(c);
        const double ms = c->prof.pass_ms;
        if (ms_per_shape) ms_per_shape[k] = ms;
        if (rc == HHT_OK && ms < best_ms) {
            best_ms = ms;
            best_shape = k;
        }
    }
    c->pass_shape = best_shape;
    c->profile = was_profiling;
    c->prof = saved;
    c->predicate = saved_predicate;
    if (rc != HHT_OK) return rc;
    *best = best_shape;
    return HHT_OK;
}

int hht_detect_subtrees(hht_ctx* c, const hht_point* points, int64_t n, int32_t W, int32_t H, int32_t depth,
                        int32_t T, int32_t split_level, const uint8_t* keep, hht_result* out) {
    if (!c || !out || !keep) return HHT_E_ARG;
    hht_image im{points, n, W, H, depth, T};
    int rc = check_image(im);
    if (rc != HHT_OK) return rc;
    if (split_level < 1 || split_level > depth || split_level > HHT_MAX_SPLIT_LEVEL) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    rc = check_predicate(c, im);
    if (rc != HHT_OK) return rc;
    cudaSetDevice(c->device);
    const size_t bytes = (size_t)2 << (2 * split_level);  // 2 * 4^k
    RK(ensure(c, c->keep_buf, bytes));
    CK(cudaMemcpyAsync(c->keep_buf.p, keep, bytes, cudaMemcpyDefault, c->stream));
    c->job_keep = (const uint8_t*)c->keep_buf.p;
    c->job_keep_level = split_level;
    rc = run_job(c, &im, 1, out);
    c->job_keep = nullptr;
    c->job_keep_level = 0;
    if (rc != HHT_OK) return rc;
    return out->status;
}

int hht_set_predicate(hht_ctx* c, int32_t predicate) {
    if (!c || (predicate != HHT_PREDICATE_EXACT && predicate != HHT_PREDICATE_FHT)) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    c->predicate = predicate;
    return HHT_OK;
}

int hht_inject_fault(hht_ctx* c, int32_t kind, int64_t arg) {
    if (!c) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    switch (kind) {
        case HHT_FAULT_NONE:
            c->inject_tile = -1;
            c->inject_graph_cap = -1;
            return HHT_OK;
        case HHT_FAULT_GRAPH_CAPACITY:
            if (arg < 0 || arg >= (int64_t)UINT32_MAX) return HHT_E_ARG;
            c->inject_graph_cap = arg;
            return HHT_OK;
        case HHT_FAULT_WITHHOLD_SCAN_TILE:
            if (arg < 0 || arg >= (int64_t)UINT32_MAX) return HHT_E_ARG;
            c->inject_tile = arg;
            return HHT_OK;
        default:
            return HHT_E_ARG;
    }
}

int hht_profile_enable(hht_ctx* c, int on) {
    if (!c) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStreamSynchronize(c->stream);
    resolve_profile(c);
    c->profile = on != 0;
    c->prof = hht_profile_counters{};
    return HHT_OK;
}

int hht_profile_read(hht_ctx* c, hht_profile_counters* out) {
    if (!c || !out) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaStreamSynchronize(c->stream);
    resolve_profile(c);
    *out = c->prof;
    return HHT_OK;
}

const char* hht_strerror(int code) {
    switch (code) {
        case HHT_OK: return "ok";
        case HHT_E_ARG: return "invalid argument";
        case HHT_E_RANGE: return "point outside the image";
        case HHT_E_CAPACITY: return "leaf buffer too small";
        case HHT_E_NOMEM: return "out of device memory or budget";
        case HHT_E_TIMEOUT: return "bounded device wait expired";
        case HHT_E_CUDA: return "CUDA runtime error";
        case HHT_E_PENDING: return "request pending";
        case HHT_E_UNKNOWN_TICKET: return "unknown ticket";
        default: return "unknown error";
    }
}

const char* hht_version(void) {
#ifdef HHT_CHECKED
    return "hht 0.5 checked (sm_103a; every data-derived index of the level kernel bounds-checked)";
#endif
    return "hht 0.5 (sm_103a, device-driven level loop in one CUDA graph; pass tile shapes 4x256/3 4x128/6 3x256/4 "
           "4x384/2 4x192/4 3x256/3)";
}

}  // extern "C"

// Internal entry used by the serving loop.
int hht_internal_run_job(hht_ctx* c, const hht_image* im, int count, hht_result* outs) {
    return run_job(c, im, count, outs);
}

// Internal entry used by the front end: halves[k] bit h set when half h of
// image k takes its points (the caller holds the context's lock).
int hht_internal_run_job_halves(hht_ctx* c, const hht_image* im, int count, hht_result* outs, const uint8_t* halves) {
    return run_job(c, im, count, outs, halves);
}

hht::ServeState** hht_internal_serve_slot(hht_ctx* c) { return &c->serve; }
