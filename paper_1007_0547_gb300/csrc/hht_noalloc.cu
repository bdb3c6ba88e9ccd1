// hht_detect_noalloc: single-image detection that allocates nothing.
//
// Some callers cannot let a library allocate device memory: code running where
// another framework owns the device memory, so that a stray cudaMalloc could
// fail or fragment its pool, and loops where the implicit device-wide
// synchronisation of an allocation or free is not acceptable.  For them this
// entry point runs the same stage / select / pass kernels as hht_detect, with
// every piece of scratch carved from one file-scope device array of
// kScratchBytes.  It synchronises its stream once per level, to read the
// level's totals that size the next level.
//
// That array exists on every GPU that loads the library, from load until
// the process exits.  Its device address is looked up once per device, by
// the first call on that device, with cudaGetSymbolAddress, and kept for the
// process's life: a cudaDeviceReset between calls is not supported.  Every call shares
// the array and it keeps the last call's contents, so everything a call needs
// at zero is cleared by that call, and calls that overlap on the GPU
// (different streams, or different host threads on the same device) race on
// it and must not be issued.  Every return after the call's first device work
// synchronises the stream first, so no kernel of a failed call is still
// writing the array when it returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/hht.h"
#include "hht_internal.h"

using namespace hht;

namespace {

constexpr size_t kScratchBytes = HHT_NOALLOC_SCRATCH_BYTES;  // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return HHT_E_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return HHT_E_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = (unsigned char*)g_scratch_ptr[dev];
    return HHT_OK;
}

int frame_log2(int v) {
    int e = 0;
    while ((1 << e) < v) ++e;
    return e;
}

// Bump allocation from both ends of the level area: buffers of even steps
// from the bottom, of odd steps from the top, so a step only reuses the space
// of the step two before it.
struct TwoSided {
    size_t lo, hi, bottom, top;  // [lo, hi) is the area; bottom / top are the free ends
    void reset_side(int side) {
        if (side == 0) bottom = lo; else top = hi;
    }
    // returns offset or SIZE_MAX when the two sides would meet
    size_t take(int side, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        if (side == 0) {
            if (bottom + bytes > top) return SIZE_MAX;
            const size_t o = bottom;
            bottom += bytes;
            return o;
        }
        if (top < bottom + bytes) return SIZE_MAX;
        top -= bytes;
        return top;
    }
};

// The detection proper.  *touched is set once the call has queued device work
// on `st` (the caller then synchronises before any error return).
int noalloc_body(const hht_point* points, int64_t n, int32_t W, int32_t H, int32_t depth, int32_t T,
                 hht_leaf* leaves, uint64_t leaf_capacity, hht_result* out, cudaStream_t st, bool* touched) {
    unsigned char* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc != HHT_OK) return rc;
    int nsm = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);

    // ---- fixed part of the scratch
    size_t off = 0;
    auto fixed = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return base + o;
    };
    const int n_units = 2;
    const size_t stats_words = (size_t)n_units * (kMaxDepth + 1) * 4;
    int16_t* d_pts = (int16_t*)fixed((size_t)std::max<int64_t>(n, 1) * sizeof(hht_point));
    Unit* d_units = (Unit*)fixed(n_units * sizeof(Unit));
    uint64_t* d_img_start = (uint64_t*)fixed(2 * sizeof(uint64_t));
    uint32_t* d_img_unit = (uint32_t*)fixed(sizeof(uint32_t));
    uint32_t* d_img_err = (uint32_t*)fixed(sizeof(uint32_t));
    uint64_t* d_stats = (uint64_t*)fixed(stats_words * sizeof(uint64_t));
    LevelInfo* d_infos = (LevelInfo*)fixed((kMaxDepth + 1) * sizeof(LevelInfo));
    DeviceStatus* d_status = (DeviceStatus*)fixed(sizeof(DeviceStatus));
    uint64_t* d_leaf_total = (uint64_t*)fixed(sizeof(uint64_t));
    ScanState* d_scan = (ScanState*)fixed(sizeof(ScanState));
    DevLeaf* d_leaves = (DevLeaf*)fixed((size_t)HHT_NOALLOC_MAX_LEAVES * sizeof(DevLeaf));
    if (off >= kScratchBytes) return HHT_E_NOMEM;
    TwoSided area{off, kScratchBytes, off, kScratchBytes};

    // ---- host-side job description
    const int lL = frame_log2(std::max(W, H));
    const bool i64 = lL + depth > 27;
    Unit units[2];
    uint64_t h_stats[2 * (kMaxDepth + 1) * 4];
    std::memset(units, 0, sizeof units);
    std::memset(h_stats, 0, sizeof h_stats);
    for (int h = 0; h < 2; ++h) {
        Unit& U = units[h];
        U.lL = lL; U.D = depth; U.T = T; U.image = 0; U.n = n; U.W = W; U.H = H; U.half = h; U.t0 = 0;
        U.root_rec = (uint32_t)h;
        U.v0_off = depth >= 2 ? (uint64_t)h * (uint64_t)n : 0;
        uint64_t* s0 = &h_stats[(size_t)h * (kMaxDepth + 1) * 4];
        s0[0] = 1; s0[1] = 1; s0[3] = (uint64_t)n;
    }
    const uint64_t img_start[2] = {0, (uint64_t)n};
    const uint32_t img_unit = 0;
    LevelInfo h_info[kMaxDepth + 1];
    std::memset(h_info, 0, sizeof h_info);
    h_info[0].n_regions = 2;
    h_info[0].n_voters = depth >= 2 ? 2 * (uint64_t)n : 0;
    const Region roots[2] = {{0u, 0u, 0u, (uint32_t)n}, {1u, 0u, 0u, (uint32_t)n}};

    // level-0 records, counters and voter stream: side 0 of the level area
    const size_t o_rec0 = area.take(0, 2 * sizeof(Region));
    const size_t o_cnt0 = area.take(0, 2 * 4 * sizeof(uint32_t));
    const size_t o_v0 = area.take(0, std::max<uint64_t>(h_info[0].n_voters, 1) * sizeof(Voter));
    if (o_rec0 == SIZE_MAX || o_cnt0 == SIZE_MAX || o_v0 == SIZE_MAX) return HHT_E_NOMEM;

#define NA_CK(call)                                 \
    do {                                            \
        if ((call) != cudaSuccess) {                \
            cudaGetLastError();                     \
            return HHT_E_CUDA;                      \
        }                                           \
    } while (0)
    // everything a call relies on being zero or freshly written is set here
    *touched = true;
    if (n > 0) NA_CK(cudaMemcpyAsync(d_pts, points, (size_t)n * sizeof(hht_point), cudaMemcpyDefault, st));
    NA_CK(cudaMemcpyAsync(d_units, units, sizeof units, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_img_start, img_start, sizeof img_start, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_img_unit, &img_unit, sizeof img_unit, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(d_img_err, 0, sizeof(uint32_t), st));
    NA_CK(cudaMemcpyAsync(d_stats, h_stats, stats_words * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(d_infos, h_info, sizeof h_info, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(d_status, 0, sizeof(DeviceStatus), st));
    NA_CK(cudaMemsetAsync(d_leaf_total, 0, sizeof(uint64_t), st));
    NA_CK(cudaMemsetAsync(d_scan, 0, sizeof(ScanState), st));
    NA_CK(cudaMemcpyAsync(base + o_rec0, roots, sizeof roots, cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(base + o_cnt0, 0, 2 * 4 * sizeof(uint32_t), st));
    // host copies above read stack memory: make sure they are done before it goes
    NA_CK(cudaStreamSynchronize(st));

    if (launch_stage(d_pts, (uint64_t)n, d_units, 1, d_img_start, d_img_unit,
                     (Voter*)(base + o_v0), (uint32_t*)(base + o_cnt0), d_stats, d_img_err, d_status, i64, st) != 0)
        return HHT_E_CUDA;

    // ---- level loop (same kernels as hht_detect; buffers from the two-sided area)
    size_t rec_off[2] = {o_rec0, 0}, cnt_off[2] = {o_cnt0, 0}, vox_off[2] = {o_v0, 0}, preg_off[2] = {0, 0};
    uint64_t leaf_total = 0;
    for (int s = 1; s <= depth; ++s) {
        const int pi = (s - 1) & 1, ci = s & 1;
        const uint64_t P = h_info[s - 1].n_regions;
        if (P == 0) break;
        // the children's side was used by step s-2, which is no longer needed
        area.reset_side(ci);
        const size_t sel_tiles = (P + 1023) / 1024 + 1;
        preg_off[pi] = area.take(pi, P * sizeof(PassRegion));
        rec_off[ci] = area.take(ci, 4 * P * sizeof(Region));
        cnt_off[ci] = area.take(ci, 4 * P * 4 * sizeof(uint32_t));
        const size_t cur_off = area.take(ci, 4 * P * sizeof(unsigned long long));
        const size_t flag_off = area.take(ci, sel_tiles * 4);
        const size_t data_off = area.take(ci, sel_tiles * 2 * 3 * sizeof(uint64_t));
        if (preg_off[pi] == SIZE_MAX || rec_off[ci] == SIZE_MAX || cnt_off[ci] == SIZE_MAX || cur_off == SIZE_MAX ||
            flag_off == SIZE_MAX || data_off == SIZE_MAX)
            return HHT_E_NOMEM;
        // select flags carry an epoch; cleared each time they are placed anew
        NA_CK(cudaMemsetAsync(base + flag_off, 0, sel_tiles * 4, st));
        NA_CK(cudaMemsetAsync(d_scan, 0, sizeof(ScanState), st));

        LevelArgs a{};
        a.units = d_units;
        a.parents = (const Region*)(base + rec_off[pi]);
        a.pregions = (PassRegion*)(base + preg_off[pi]);
        a.parent_cnt = (const uint32_t*)(base + cnt_off[pi]);
        a.children = (Region*)(base + rec_off[ci]);
        a.child_cnt = (uint32_t*)(base + cnt_off[ci]);
        a.cursor = (unsigned long long*)(base + cur_off);
        a.leaves = d_leaves;
        a.stats = d_stats;
        a.info_prev = d_infos + (s - 1);
        a.info = d_infos + s;
        a.leaf_total = d_leaf_total;
        a.scan = d_scan;
        a.tile_flags = (uint32_t*)(base + flag_off);
        a.tile_data = (uint64_t*)(base + data_off);
        a.status = d_status;
        a.img_err = d_img_err;
        a.cap_children = 4 * P;
        a.cap_leaves = HHT_NOALLOC_MAX_LEAVES;
        a.cap_voters = UINT64_MAX;
        a.level = s;
        a.num_sms = nsm;
        const int sel_grid = (int)std::min<uint64_t>(sel_tiles, (uint64_t)nsm * occupancy_select());
        if (launch_select(a, 256, std::max(sel_grid, 1), st) != 0) return HHT_E_CUDA;
        DeviceStatus hs{};
        NA_CK(cudaMemcpyAsync(&h_info[s], d_infos + s, sizeof(LevelInfo), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaMemcpyAsync(&hs, d_status, sizeof hs, cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        if (hs.err & kErrOverflow) return HHT_E_NOMEM;
        if (hs.err & kErrTimeout) return HHT_E_TIMEOUT;
        if (hs.err) return HHT_E_CUDA;
        leaf_total += h_info[s].n_leaves;
        if (s == depth) break;
        const uint64_t nin = h_info[s - 1].n_voters, nout = h_info[s].n_voters;
        if (nin == 0) continue;
        vox_off[ci] = area.take(ci, std::max<uint64_t>(nout, 1) * sizeof(Voter));
        if (vox_off[ci] == SIZE_MAX) return HHT_E_NOMEM;
        a.vin = (const Voter*)(base + vox_off[pi]);
        a.vout = (Voter*)(base + vox_off[ci]);
        a.cap_voters = nout;
        const uint64_t want = (nin + 2047) / 2048;
        const int grid = (int)std::min<uint64_t>(want, (uint64_t)nsm * occupancy_pass(i64));
        if (launch_pass(a, i64, std::max(grid, 1), st) != 0) return HHT_E_CUDA;
    }

    // ---- outputs: statistics to the caller's result, leaves to the caller's buffer
    uint32_t img_err = 0;
    NA_CK(cudaMemcpyAsync(h_stats, d_stats, stats_words * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaMemcpyAsync(&img_err, d_img_err, sizeof img_err, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    std::memset(out->stats, 0, sizeof out->stats);
    out->depth = depth;
    out->L = 1 << lL;
    out->leaves = leaves;
    out->leaf_capacity = leaf_capacity;
    uint64_t nl = 0;
    for (int h = 0; h < 2; ++h) {
        const uint64_t* su = &h_stats[(size_t)h * (kMaxDepth + 1) * 4];
        for (int l = 0; l <= depth; ++l) {
            out->stats[h][l].tested = su[4 * l + 0];
            out->stats[h][l].passed = su[4 * l + 1];
            out->stats[h][l].votes = su[4 * l + 2];
            out->stats[h][l].tests = su[4 * l + 3];
        }
        nl += su[4 * depth + 1];
    }
    out->n_leaves = nl;
    if (img_err) return HHT_E_RANGE;
    if (nl != leaf_total) return HHT_E_CUDA;
    if (nl > leaf_capacity || (nl > 0 && !leaves)) return HHT_E_CAPACITY;
    if (nl > 0) {
        NA_CK(cudaMemcpyAsync(leaves, d_leaves, nl * sizeof(hht_leaf), cudaMemcpyDefault, st));
        NA_CK(cudaStreamSynchronize(st));
    }
#undef NA_CK
    return HHT_OK;
}

}  // namespace

extern "C" int hht_detect_noalloc(const hht_point* points, int64_t n, int32_t W, int32_t H, int32_t depth,
                                  int32_t T, hht_leaf* leaves, uint64_t leaf_capacity, hht_result* out,
                                  void* cuda_stream) {
    if (!out || n < 0 || (n > 0 && !points) || W < 1 || H < 1 || W > HHT_MAX_SIDE || H > HHT_MAX_SIDE ||
        depth < 1 || depth > HHT_MAX_DEPTH || T < 1)
        return HHT_E_ARG;
    if (n > HHT_NOALLOC_MAX_POINTS || depth > HHT_NOALLOC_MAX_DEPTH) return HHT_E_NOMEM;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    out->n_leaves = 0;
    bool touched = false;
    const int rc = noalloc_body(points, n, W, H, depth, T, leaves, leaf_capacity, out, st, &touched);
    if (rc != HHT_OK && touched) {
        // a failed call may still have kernels writing the shared array: wait
        // for them (this wait's own error is not the one to report)
        cudaStreamSynchronize(st);
        cudaGetLastError();
    }
    out->status = rc;
    return rc;
}
