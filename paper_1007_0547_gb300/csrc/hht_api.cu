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
constexpr int kPersistentRetry = 1;  // run_wave: persistent capacities too small, run again level by level

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

int hht::copy_out(hht_ctx* c, void* dst, const void* src, size_t bytes) {
    constexpr size_t kKernelMin = 1u << 20;
    if (bytes >= kKernelMin && !c->copy_engine_only && ((uintptr_t)dst % 16) == 0 && ((uintptr_t)src % 16) == 0 &&
        bytes % 16 == 0) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer) {
            if (launch_copy16(src, at.devicePointer, bytes / 16, c->num_sms * 4, c->stream) != 0) return HHT_E_CUDA;
            c->prof.launches += 1;
            return HHT_OK;
        }
        cudaGetLastError();
    }
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream));
    return HHT_OK;
}

namespace {

// The persistent launch, through a CUDA graph captured once per argument set
// (replayed while the buffers and sizes are unchanged).  Capture is not
// possible on the legacy default stream or inside another capture; then the
// kernel is launched directly.
int launch_persistent_graph(hht_ctx* c, const PersistentArgs& f, bool i64, int grid) {
    cudaStream_t st = c->stream;
    const unsigned char* fb = reinterpret_cast<const unsigned char*>(&f);
    std::vector<unsigned char> key(fb, fb + sizeof f);
    key.push_back(i64 ? 1 : 0);
    if (c->graph_exec && c->graph_grid == grid && key == c->graph_args) {
        CK(cudaGraphLaunch(c->graph_exec, st));
        return HHT_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool can_capture = st != nullptr && !c->graph_capture_failed &&
                             cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    if (can_capture) {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        bool ok = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            const int lr = launch_persistent(f, i64, grid, st);
            ok = cudaStreamEndCapture(st, &g) == cudaSuccess && lr == 0 && g != nullptr;
        }
        if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        if (ok) {
            if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = ge;
            c->graph_args = key;
            c->graph_grid = grid;
            CK(cudaGraphLaunch(c->graph_exec, st));
            return HHT_OK;
        }
        cudaGetLastError();
        c->graph_capture_failed = true;  // launch directly from now on
    }
    return launch_persistent(f, i64, grid, st) == 0 ? HHT_OK : HHT_E_CUDA;
}

// Run one wave of images through the level loop; fills outs[k] for k in
// [0, count).  Returns HHT_OK or a job-level error (per-image errors are in
// outs[k].status).
int run_wave(hht_ctx* c, const hht_image* im, int count, hht_result* outs, int job_first) {
    cudaStream_t st = c->stream;
    const int n_units = 2 * count;
    int Dmax = 0;
    bool i64 = false;
    uint64_t total = 0, v0_len = 0;
    std::vector<Unit> units(n_units);
    std::vector<uint64_t> img_start(count + 1);
    for (int g = 0; g < count; ++g) {
        const int lL = ceil_log2_i(std::max(im[g].W, im[g].H));
        Dmax = std::max(Dmax, im[g].depth);
        // int32 corner arithmetic is exact while lL + depth <= 27: then
        // |G| <= 4LK = 2^29 at every vertex of the parameter space, and the
        // level kernel's partial sums (u0 = dJ - 1 - G(SW) built as
        // W0 - x*A + (x + y)*K, with |x*A|, (x + y)*K < 2^28, and its column
        // steps of at most 4x*S/4 < 2^28) stay within 1.5 * 2^30; the FHT's
        // 2G values stay within 8LK = 2^30.  Both sides of the switch (27 and
        // 28, on 32767^2 and 16^2 frames, points at the far corners and on
        // lines through one vertex) are checked against the oracle on the GPU.
        if (lL + im[g].depth > 27) i64 = true;
        img_start[g] = total;
        for (int h = 0; h < 2; ++h) {
            Unit& U = units[2 * g + h];
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
            U.v0_off = v0_len;
            if (U.D >= 2 && on) v0_len += (uint64_t)im[g].n;
        }
        total += (uint64_t)im[g].n;
    }
    img_start[count] = total;

    // ---- inputs and job state
    RK(ensure(c, c->pts, std::max<uint64_t>(total, 1) * sizeof(hht_point)));
    for (int g = 0; g < count; ++g)
        if (im[g].n > 0)
            CK(cudaMemcpyAsync((char*)c->pts.p + img_start[g] * sizeof(hht_point), im[g].points,
                               (size_t)im[g].n * sizeof(hht_point), cudaMemcpyDefault, st));
    RK(ensure(c, c->units, n_units * sizeof(Unit)));
    RK(ensure(c, c->img_start, (count + 1) * sizeof(uint64_t)));
    RK(ensure(c, c->img_unit, count * sizeof(uint32_t)));
    std::vector<uint32_t> img_unit(count);
    for (int g = 0; g < count; ++g) img_unit[g] = (uint32_t)(2 * g);
    RK(ensure(c, c->img_err, count * sizeof(uint32_t)));
    const size_t stats_words = (size_t)n_units * (kMaxDepth + 1) * 4;
    RK(ensure(c, c->stats, stats_words * sizeof(uint64_t)));
    RK(ensure(c, c->infos, (kMaxDepth + 1) * sizeof(LevelInfo)));
    RK(ensure(c, c->status, sizeof(DeviceStatus)));
    RK(ensure(c, c->leaf_total, sizeof(uint64_t)));

    c->h_stats.assign(stats_words, 0);
    for (int u = 0; u < n_units; ++u) {
        uint64_t* s0 = &c->h_stats[(size_t)u * (kMaxDepth + 1) * 4];
        s0[0] = 1;                       // level 0: one region tested
        s0[1] = 1;                       // ... and always split
        s0[3] = (uint64_t)units[u].n;    // one code per point
    }
    c->h_infos.assign(kMaxDepth + 1, LevelInfo{});
    c->h_infos[0].n_regions = (uint64_t)n_units;
    c->h_infos[0].n_voters = v0_len;
    std::vector<Region> roots(n_units);
    for (int u = 0; u < n_units; ++u) roots[u] = Region{(uint32_t)u, 0u, 0u, (uint32_t)units[u].n};

    // job signature for the persistent form's size plan
    uint64_t sig = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { sig = (sig ^ v) * 1099511628211ull; };
    mix((uint64_t)count);
    for (int g = 0; g < count; ++g) {
        mix((uint64_t)im[g].n);
        mix(((uint64_t)im[g].W << 32) | (uint64_t)im[g].H);
        mix(((uint64_t)im[g].depth << 32) | (uint64_t)im[g].T);
    }
    const bool fht = c->predicate == HHT_PREDICATE_FHT;
    if (fht && i64) return HHT_E_ARG;  // checked by the entry points before any device work
    const int occ_p = i64 ? c->occ_persistent64 : c->occ_persistent32;
    const bool persistent = !fht && !c->job_halves && !c->job_keep && c->batch_mode == 1 && c->plan.valid &&
                            c->plan.sig == sig && occ_p > 0;
    uint64_t cap_rec = 0, cap_vox = 0, cap_tiles = 0;
    if (persistent) {
        cap_rec = std::max<uint64_t>(c->plan.cap_rec, (uint64_t)n_units);
        cap_vox = std::max<uint64_t>(c->plan.cap_vox, v0_len);
        cap_tiles = (cap_rec + kSelTile - 1) / kSelTile + 1;
        for (int k = 0; k < 2; ++k) {
            RK(ensure(c, c->rec[k], cap_rec * sizeof(Region)));
            RK(ensure(c, c->preg[k], cap_rec * sizeof(PassRegion)));
            RK(ensure(c, c->cnt[k], cap_rec * 4 * sizeof(uint32_t)));
            RK(ensure(c, c->vox[k], std::max<uint64_t>(cap_vox, 1) * sizeof(Voter)));
        }
        RK(ensure(c, c->cursors, cap_rec * sizeof(unsigned long long)));
        RK(ensure_keep(c, c->leaves, (c->job_leaves + c->plan.cap_leaves + 1) * sizeof(DevLeaf),
                       c->job_leaves * sizeof(DevLeaf)));
        if (cap_tiles * 4 > c->sel_flags.bytes) RK(ensure(c, c->sel_flags, cap_tiles * 4, true));
        RK(ensure(c, c->sel_data, cap_tiles * 2 * 3 * sizeof(uint64_t)));
    }
    RK(ensure(c, c->rec[0], n_units * sizeof(Region)));
    RK(ensure(c, c->cnt[0], n_units * 4 * sizeof(uint32_t)));
    RK(ensure(c, c->vox[0], std::max<uint64_t>(v0_len, 1) * sizeof(Voter)));
    CK(cudaMemcpyAsync(c->units.p, units.data(), n_units * sizeof(Unit), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->img_start.p, img_start.data(), (count + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->img_unit.p, img_unit.data(), count * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->stats.p, c->h_stats.data(), stats_words * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->infos.p, c->h_infos.data(), (kMaxDepth + 1) * sizeof(LevelInfo), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(c->rec[0].p, roots.data(), n_units * sizeof(Region), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(c->cnt[0].p, 0, n_units * 4 * sizeof(uint32_t), st));
    CK(cudaMemsetAsync(c->status.p, 0, sizeof(DeviceStatus), st));
    // this wave's leaves follow those of the job's earlier waves
    const uint64_t wave_leaf_base = c->job_leaves;
    CK(cudaMemcpyAsync(c->leaf_total.p, &c->job_leaves, sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(c->img_err.p, 0, count * sizeof(uint32_t), st));

    LevelInfo* d_infos = (LevelInfo*)c->infos.p;
    DeviceStatus* d_status = (DeviceStatus*)c->status.p;
    ScanState* d_scan = (ScanState*)c->scan_states.p;

    uint64_t leaf_total = wave_leaf_base;
    uint32_t err = 0;
    if (persistent) {
        PersistentArgs f{};
        f.base.units = (const Unit*)c->units.p;
        f.base.cursor = (unsigned long long*)c->cursors.p;
        f.base.leaves = (DevLeaf*)c->leaves.p;
        f.base.stats = (uint64_t*)c->stats.p;
        f.base.leaf_total = (uint64_t*)c->leaf_total.p;
        f.base.scan = d_scan + 0;
        f.base.tile_flags = (uint32_t*)c->sel_flags.p;
        f.base.tile_data = (uint64_t*)c->sel_data.p;
        f.base.status = d_status;
        f.base.cap_children = cap_rec;
        f.base.cap_voters = cap_vox;
        f.base.cap_leaves = c->leaves.bytes / sizeof(DevLeaf);
        f.base.cap_tiles = cap_tiles;
        f.base.num_sms = c->num_sms;
        f.base.withhold_tile_plus1 = c->inject_tile >= 0 ? (uint32_t)(c->inject_tile + 1) : 0u;
        for (int k = 0; k < 2; ++k) {
            f.rec[k] = (Region*)c->rec[k].p;
            f.preg[k] = (PassRegion*)c->preg[k].p;
            f.cnt[k] = (uint32_t*)c->cnt[k].p;
            f.vox[k] = (Voter*)c->vox[k].p;
        }
        f.infos = d_infos;
        f.pts = (const int16_t*)c->pts.p;
        f.total_pts = total;
        f.img_start = (const uint64_t*)c->img_start.p;
        f.img_unit = (const uint32_t*)c->img_unit.p;
        f.img_err = (uint32_t*)c->img_err.p;
        f.n_images = count;
        f.Dmax = Dmax;
        {
            TraceRange tr_k("persistent level loop");
            ProfScope ps(c, 2);
            RK(launch_persistent_graph(c, f, i64, c->num_sms * occ_p));
        }
        c->prof.launches += 1;
        CK(cudaMemcpyAsync(&leaf_total, c->leaf_total.p, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(c->h_infos.data(), d_infos, (Dmax + 1) * sizeof(LevelInfo), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        c->persistent_runs += 1;
        c->prof.persistent_launches += 1;
        // algorithmic bytes of the level passes inside the launch (as if launched one by one)
        for (int s = 1; s < Dmax; ++s) {
            const uint64_t nin = c->h_infos[s - 1].n_voters, nout = c->h_infos[s].n_voters;
            if (nin == 0) continue;
            c->prof.pass_launches += 1;
            c->prof.voters_read += nin;
            c->prof.voters_written += nout;
            c->prof.pass_bytes += 8 * (nin + nout);
        }
    }
    if (!persistent) {
        TraceRange tr_k("stage");
        ProfScope ps(c, 0);
        if (launch_stage((const int16_t*)c->pts.p, total, (const Unit*)c->units.p, count,
                         (const uint64_t*)c->img_start.p, (const uint32_t*)c->img_unit.p, (Voter*)c->vox[0].p,
                         (uint32_t*)c->cnt[0].p, (uint64_t*)c->stats.p, (uint32_t*)c->img_err.p, d_status, i64,
                         st, fht) != 0)
            return HHT_E_CUDA;
        if (total > 0) c->prof.launches += 1;
    }

    // ---- level loop (sizes recorded as the plan of the persistent form)
    uint64_t plan_rec = (uint64_t)n_units, plan_vox = v0_len;
    for (int s = 1; s <= Dmax && !persistent; ++s) {
        TraceRange tr_level(level_name(s));
        const int pi = (s - 1) & 1, ci = s & 1;
        const uint64_t P = c->h_infos[s - 1].n_regions;
        if (P == 0) break;
        if (4 * P > kMaxLevelRecords) return HHT_E_NOMEM;
        RK(ensure(c, c->preg[pi], P * sizeof(PassRegion)));
        RK(ensure(c, c->rec[ci], 4 * P * sizeof(Region)));
        RK(ensure(c, c->cnt[ci], 4 * P * 4 * sizeof(uint32_t)));
        const uint64_t cap_leaves = leaf_total + 4 * P;
        RK(ensure_keep(c, c->leaves, cap_leaves * sizeof(DevLeaf), leaf_total * sizeof(DevLeaf)));
        const uint64_t sel_tiles = (P + kSelTile - 1) / kSelTile;
        if ((sel_tiles + 1) * 4 > c->sel_flags.bytes) {
            RK(ensure(c, c->sel_flags, (sel_tiles + 1) * 4, true));
        }
        RK(ensure(c, c->sel_data, (sel_tiles + 1) * 2 * 3 * sizeof(uint64_t)));
        RK(ensure(c, c->cursors, 4 * P * sizeof(unsigned long long)));

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
        a.info_prev = d_infos + (s - 1);
        a.info = d_infos + s;
        a.leaf_total = (uint64_t*)c->leaf_total.p;
        a.status = d_status;
        a.cap_children = 4 * P;
        a.cap_leaves = cap_leaves;
        a.cap_voters = c->vox[ci].bytes / sizeof(Voter);
        a.level = s;
        a.num_sms = c->num_sms;
        a.scan = d_scan + 0;
        a.tile_flags = (uint32_t*)c->sel_flags.p;
        a.tile_data = (uint64_t*)c->sel_data.p;
        a.cap_tiles = sel_tiles;
        a.withhold_tile_plus1 = c->inject_tile >= 0 ? (uint32_t)(c->inject_tile + 1) : 0u;
        a.keep = c->job_keep;
        a.keep_level = c->job_keep_level;
        const int sel_grid = (int)std::min<uint64_t>(sel_tiles, (uint64_t)c->num_sms * c->occ_select);
        // select's capacity test on the voter stream is re-done below with the exact size
        a.cap_voters = UINT64_MAX;
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
        err = hs.err;
        if (c->debug)
            fprintf(stderr, "[hht]   step %d: parents %llu, regions %llu, voters in %llu, out %llu, leaves %llu, held %.2f GB\n",
                    s, (unsigned long long)P, (unsigned long long)c->h_infos[s].n_regions,
                    (unsigned long long)c->h_infos[s - 1].n_voters, (unsigned long long)c->h_infos[s].n_voters,
                    (unsigned long long)c->h_infos[s].n_leaves, c->held / 1e9);
        if (err) break;
        leaf_total += c->h_infos[s].n_leaves;
        plan_rec = std::max<uint64_t>(plan_rec, c->h_infos[s].n_regions);
        plan_vox = std::max<uint64_t>(plan_vox, c->h_infos[s].n_voters);
        if (s == Dmax) break;

        const uint64_t nin = c->h_infos[s - 1].n_voters;
        if (nin == 0) continue;  // no unit needs level s+1 counts
        const uint64_t nout = c->h_infos[s].n_voters;
        RK(ensure(c, c->vox[ci], std::max<uint64_t>(nout, 1) * sizeof(Voter)));
        a.vin = (const Voter*)c->vox[pi].p;
        a.vout = (Voter*)c->vox[ci].p;
        a.cap_voters = nout;
        const int shape = (i64 || fht) ? 0 : c->pass_shape;
        const int occ = fht ? c->occ_pass_fht : (i64 ? c->occ_pass64 : c->occ_shape[shape]);
        // enough warp slices to fill the device, no more than the stream needs
        const uint64_t tile = 8ull * (uint64_t)(fht ? 256 : pass_threads(i64, shape));
        const uint64_t want_blocks = (nin + tile - 1) / tile;
        const int pass_grid = (int)std::min<uint64_t>(want_blocks, (uint64_t)c->num_sms * occ);
        {
            TraceRange tr_k("pass");
            ProfScope ps(c, 2);
            if (launch_pass(a, i64, std::max(pass_grid, 1), st, shape, fht) != 0) return HHT_E_CUDA;
        }
        c->prof.launches += 1;
        c->prof.pass_launches += 1;
        c->prof.voters_read += nin;
        c->prof.voters_written += nout;
        c->prof.pass_bytes += 8 * (nin + nout);
    }

    // ---- outputs
    CK(cudaMemcpyAsync(c->h_stats.data(), c->stats.p, stats_words * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    c->h_img_err.assign(count, 0);
    CK(cudaMemcpyAsync(c->h_img_err.data(), c->img_err.p, count * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    DeviceStatus hs{};
    CK(cudaMemcpyAsync(&hs, d_status, sizeof hs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    err |= hs.err;
    if (persistent && (err & kErrOverflow)) {
        // the plan's capacities were too small for this data: level by level instead
        c->plan.valid = false;
        c->persistent_fallbacks += 1;
        c->prof.persistent_fallbacks += 1;
        return kPersistentRetry;
    }
    if (err & kErrTimeout) return HHT_E_TIMEOUT;
    if (err & kErrOverflow) return HHT_E_NOMEM;
    if (err & kErrInvariant) return HHT_E_CUDA;
    if (err & kErrBounds) {
        if (c->debug) fprintf(stderr, "[hht] a kernel met an out-of-range index (checked build)\n");
        return HHT_E_CUDA;
    }
    if (!persistent) {
        // capacities for the persistent form of the same job, with a margin
        c->plan.sig = sig;
        c->plan.cap_rec = plan_rec + plan_rec / 8 + 64;
        c->plan.cap_vox = plan_vox + plan_vox / 8 + 64;
        const uint64_t wl = leaf_total - wave_leaf_base;
        c->plan.cap_leaves = wl + wl / 8 + 64;
        c->plan.valid = true;
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
        uint64_t acc = wave_leaf_base;
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
        if (rc == kPersistentRetry) {
            c->job_leaves = leaves_before;
            rc = run_wave(c, im + first, last - first, outs + first, job_first + first);
        }
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
    c->occ_persistent32 = occupancy_persistent(false);
    c->occ_persistent64 = occupancy_persistent(true);
    if (const char* e = getenv("HHT_BATCH_MODE")) c->batch_mode = atoi(e) == 1 ? 1 : 0;
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
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    DevBuf* all[] = {&c->pts,       &c->img_start,  &c->img_unit, &c->units,        &c->stats,     &c->infos,      &c->status,
                     &c->leaf_total, &c->img_err,   &c->scan_states,  &c->rec[0],    &c->rec[1],     &c->preg[0],
                     &c->preg[1],   &c->cnt[0],     &c->cnt[1],       &c->vox[0],    &c->vox[1],     &c->leaves,
                     &c->sel_flags, &c->sel_data,   &c->cursors,      &c->img_buf,   &c->edge_pts[0],
                     &c->edge_pts[1], &c->edge_tot,   &c->line_keys,    &c->line_vals, &c->line_parent,
                     &c->line_cells, &c->line_sums,  &c->line_out,     &c->keep_buf,  &c->rem_pts,
                     &c->rem_lists,  &c->rem_bitmap, &c->rem_leaves,   &c->rem_stats, &c->rem_tasks};
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
    if (!c || (mode != HHT_BATCH_LEVELS && mode != HHT_BATCH_PERSISTENT)) return HHT_E_ARG;
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
    if (predicate != c->predicate) c->plan.valid = false;  // the persistent form's size plan was for the other test
    c->predicate = predicate;
    return HHT_OK;
}

int hht_inject_fault(hht_ctx* c, int32_t kind, int64_t arg) {
    if (!c) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    switch (kind) {
        case HHT_FAULT_NONE:
            c->inject_tile = -1;
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
    return "hht 0.4 checked (sm_103a; every data-derived index of the level kernel bounds-checked)";
#endif
    return "hht 0.4 (sm_103a, level-synchronous stage/select/pass; pass tile shapes 4x256/3 2x256/4 3x256/4 4x128/6 "
           "4x256/4 4x512/2)";
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
