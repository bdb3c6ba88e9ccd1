// Context of libhht.so (hht_ctx) and the device-buffer helpers shared by the
// batch path (hht_api.cu) and the serving engine (hht_serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/hht.h"
#include "hht_internal.h"

namespace hht {
struct ServeState;

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

inline int ceil_log2_i(int v) {
    int e = 0;
    while ((1 << e) < v) ++e;
    return e;
}
}  // namespace hht

struct hht_ctx {
    using DevBuf = hht::DevBuf;
    int device = 0;
    hht_allocator allocator{};   // the caller's device allocator (hht_create_with_allocator)
    bool has_allocator = false;
    bool debug = false;          // HHT_DEBUG=1: wave and allocation trace on stderr
    bool copy_engine_only = false;  // HHT_COPY_ENGINE=1: leaves to host memory by cudaMemcpyAsync only
    uint64_t wave_cap = 0;       // largest wave estimate known to fit (0 = none failed yet)
    cudaStream_t stream = nullptr;
    uint64_t budget = 0;
    uint64_t held = 0;
    int num_sms = 0;
    int occ_select = 1, occ_pass32 = 1, occ_pass64 = 1;
    int pass_shape = 0;                                   // pass-kernel tile shape (autotuned)
    int batch_mode = HHT_BATCH_GRAPH;                     // HHT_BATCH_GRAPH or HHT_BATCH_LEVELS
    // CUDA graphs of the device-driven level loop (stage, then select and pass
    // per level, sizes read on the device), each replayed while its arguments
    // are unchanged; with profiling on, event records around its kernels.
    // The most recently used come first; at most kGraphCache are kept.
    struct GraphEvent {
        cudaEvent_t a, b;
        int kind;  // as Pending::kind
    };
    struct CachedGraph {
        std::vector<unsigned char> key;
        std::vector<int> grids;  // stage, then the selection and pass grids by step
        cudaGraphExec_t exec = nullptr;
        std::vector<GraphEvent> events;
    };
    static constexpr size_t kGraphCache = 8;
    std::vector<CachedGraph> graphs;
    bool graph_capture_failed = false;
    cudaStream_t own_stream = nullptr;  // the graph's stream when the context's stream is the legacy default
    DevBuf dims;  // JobDims of the job in flight (read by the graph's stage kernel)
    int occ_shape[hht::kPassShapeCount] = {1, 1, 1, 1, 1, 1};  // resident blocks per SM of each shape
    int64_t inject_tile = -1;  // hht_inject_fault: selection tile withheld in the next job (-1 = none)
    int64_t inject_graph_cap = -1;  // hht_inject_fault: level-1 stream capacity told to the next graph job
    int predicate = 0;         // HHT_PREDICATE_EXACT or HHT_PREDICATE_FHT (hht_detect / hht_detect_batch)
    const uint8_t* job_halves = nullptr;  // during a job: per image, bit h set when half h takes its points
    const uint8_t* job_keep = nullptr;    // during a job: device keep mask of subtree sharding (or NULL)
    int32_t job_keep_level = 0;
    DevBuf keep_buf;
    // solution() traversal (hht_detect_removal): points, per-level lists, removed bitmaps, leaves, stats, tasks
    DevBuf rem_pts, rem_lists, rem_bitmap, rem_leaves, rem_stats, rem_tasks, rem_flags, rem_raster;
    // the last removal job, per image: points offset, n, bitmap offsets of
    // half 0 and half 1, W, H (hht_removal_raster)
    std::vector<uint64_t> rem_last;
    // front end (hht_edges, hht_detect_image): staged image, ALPHA and BETA point lists, their counts
    DevBuf img_buf, edge_pts[2], edge_tot;
    // leaves -> lines (hht_lines): hash table, union-find parents, per-root sums, output
    DevBuf line_keys, line_vals, line_parent, line_cells, line_sums, line_out;
    uint64_t job_serial = 0;    // detection jobs run on the context (results of hht_lines refer to one)
    uint64_t lines_serial = ~0ull;  // job and image whose lines line_out holds
    int32_t lines_index = -1;
    uint64_t lines_count = 0;
    int occ_pass_fht = 1;

    // job buffers
    DevBuf pts, img_start, img_unit, units, stats, infos, status, leaf_total, img_err, scan_states;
    DevBuf rec[2], preg[2], cnt[2], vox[2];
    DevBuf leaves;
    DevBuf sel_flags, sel_data, cursors;
    // host staging
    std::vector<uint64_t> h_stats;
    std::vector<hht::LevelInfo> h_infos;
    std::vector<hht::Region> h_roots;
    hht::JobDims h_dims{};
    std::vector<uint32_t> h_img_err;
    // page-locked staging of the graph form's read-back (one wait for all of
    // its copies instead of a staged round trip per pageable copy)
    void* h_stage = nullptr;
    size_t h_stage_bytes = 0;

    hht::ServeState* serve = nullptr;
    std::mutex mu;

    // leaves of the last job stay in `leaves` until the next job
    // (hht_fetch_leaves): per image offset and count
    std::vector<uint64_t> job_off, job_n;
    uint64_t job_leaves = 0;

    // kernel timing (hht_profile_enable)
    bool profile = false;
    hht_profile_counters prof{};
    std::vector<cudaEvent_t> ev_pool;
    struct Pending {
        cudaEvent_t a, b;
        int kind;  // 0 stage, 1 select, 2 pass, 3 front end
    };
    std::vector<Pending> pending;
};


namespace hht {
int cuda_fail(cudaError_t e);
// Copy leaves (or any 16-byte-aligned device data) to a caller's buffer on
// the context's stream (hht_api.cu).
int copy_out(hht_ctx* c, void* dst, const void* src, size_t bytes);
// The same on `stream`, without touching the context's counters (callers
// that do not hold the context's lock, such as hht_poll).
int copy_out_on(hht_ctx* c, void* dst, const void* src, size_t bytes, cudaStream_t stream);
// Grow a device buffer to at least `bytes` (contents are not kept; zeroed when asked).
int ensure(hht_ctx* c, DevBuf& b, size_t bytes, bool zero = false);
// Grow a device buffer keeping its first `keep` bytes.
int ensure_keep(hht_ctx* c, DevBuf& b, size_t bytes, size_t keep);
// Grow a device buffer that holds fewer than `bytes` to exactly
// max(bytes, target) (no growth margin: a caller that knows what the buffer
// will need passes that as `target`), keeping its first `keep` bytes.
int ensure_sized(hht_ctx* c, DevBuf& b, size_t bytes, size_t keep, size_t target);
void release(hht_ctx* c, DevBuf& b);
}  // namespace hht
