// Leaves -> lines.  The paper stops at the peak cells (Section 3: the
// solution() step plots the voters of every accepted cell); turning cells into
// image lines is a reading of its own:
//   - leaves of the same half whose cells touch (|di| <= 1 and |dj| <= 1) form
//     one cluster (connected components of that adjacency);
//   - a cluster's peak is its leaf with the most votes, ties to the leaf that
//     comes first in the depth-first leaf order;
//   - a cluster also gives its vote-weighted centre as exact integer sums
//     V = sum of votes, S_i = sum of votes * (2i + 1), S_j = sum of
//     votes * (2j + 1): m = (S_i / V - K) / K, b = 2L (S_j / V - K) / K;
//   - lines are reported in the order of each cluster's first leaf.
//
// Device steps, for the n leaves of one image of the last job:
//   1. an open-addressing hash table (key (half, i, j) -> leaf index, linear
//      probing, at least twice as many slots as leaves, so every probe
//      sequence ends);
//   2. lock-free union-find over the four forward neighbours of every leaf,
//      always hooking the larger root under the smaller one, so parent chains
//      strictly decrease and the root of a cluster is its first leaf;
//   3. per root: cells, votes, centre sums (atomic adds) and the peak (one
//      64-bit atomic max of votes and the complemented leaf index), after a
//      warp-level reduction of runs of leaves with the same root;
//   4. roots compacted in index order (block scan and the look-back scan).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/hht.h"
#include "hht_ctx.h"
#include "hht_device.cuh"
#include "hht_internal.h"
#include "hht_trace.h"

namespace hht {
namespace {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr uint32_t kUnionLimit = 1u << 22;  // retries of one union (never reached: each retry follows a new hook)

__device__ __forceinline__ uint64_t cell_key(const DevLeaf& f) {
    return ((uint64_t)f.half << 48) | ((uint64_t)f.i << 24) | (uint64_t)f.j;
}
__device__ __forceinline__ uint64_t key_hash(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    return k ^ (k >> 33);
}

__global__ void lines_insert_kernel(const DevLeaf* __restrict__ lv, uint32_t n, unsigned long long* keys,
                                    uint32_t* vals, uint64_t mask, uint32_t* parent, DeviceStatus* status) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        parent[k] = k;
        const uint64_t key = cell_key(lv[k]);
        uint64_t h = key_hash(key) & mask;
        bool done = false;
        for (uint64_t probe = 0; probe <= mask; ++probe) {
            const unsigned long long old = atomicCAS(&keys[h], (unsigned long long)kEmptyKey, (unsigned long long)key);
            if (old == kEmptyKey || old == key) {
                vals[h] = k;
                done = true;
                break;
            }
            h = (h + 1) & mask;
        }
        if (!done) atomicOr(&status->err, kErrOverflow);  // cannot happen: the table has at least 2n slots
    }
}

__device__ __forceinline__ int64_t lines_lookup(const unsigned long long* keys, const uint32_t* vals, uint64_t mask,
                                                uint64_t key) {
    uint64_t h = key_hash(key) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long k = keys[h];
        if (k == key) return vals[h];
        if (k == kEmptyKey) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

// Root of x; parent chains strictly decrease, so the walk ends.  Path
// halving writes only smaller values, which other threads may see or not.
__device__ __forceinline__ uint32_t uf_find(uint32_t* parent, uint32_t x) {
    volatile uint32_t* p = parent;
    while (true) {
        const uint32_t px = p[x];
        if (px == x) return x;
        const uint32_t gp = p[px];
        if (gp != px) p[x] = gp;
        x = px;
    }
}

__global__ void lines_union_kernel(const DevLeaf* __restrict__ lv, uint32_t n, const unsigned long long* keys,
                                   const uint32_t* vals, uint64_t mask, uint32_t* parent, DeviceStatus* status) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const DevLeaf f = lv[k];
        // forward neighbours: every touching pair is met once
        const int di[4] = {1, 1, 1, 0}, dj[4] = {-1, 0, 1, 1};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t ni = (int64_t)f.i + di[e], nj = (int64_t)f.j + dj[e];
            if (nj < 0 || ni >= (1ll << 24) || nj >= (1ll << 24)) continue;
            DevLeaf g;
            g.half = f.half;
            g.i = (uint32_t)ni;
            g.j = (uint32_t)nj;
            const int64_t m = lines_lookup(keys, vals, mask, cell_key(g));
            if (m < 0) continue;
            uint32_t a = k, b = (uint32_t)m;
            bool joined = false;
            for (uint32_t tries = 0; tries < kUnionLimit; ++tries) {
                uint32_t ra = uf_find(parent, a), rb = uf_find(parent, b);
                if (ra == rb) {
                    joined = true;
                    break;
                }
                if (ra > rb) {
                    const uint32_t t = ra;
                    ra = rb;
                    rb = t;
                }
                if (atomicCAS(&parent[rb], rb, ra) == rb) {  // hook the larger root under the smaller
                    joined = true;
                    break;
                }
                a = ra;
                b = rb;
            }
            if (!joined) atomicOr(&status->err, kErrTimeout);
        }
    }
}

// Final roots, then every leaf's contribution to its root's line.  Leaves
// of one cluster often sit next to each other in the depth-first order, so
// the lanes of a warp first reduce runs of equal roots (a segmented scan that
// never crosses a run boundary) and one lane per run does the atomics.
__global__ void lines_gather_kernel(const DevLeaf* __restrict__ lv, uint32_t n, uint32_t* parent, uint32_t* cells,
                                    unsigned long long* sums /* [n][3] */, unsigned long long* peak) {
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t kb = blockIdx.x * blockDim.x; kb < n; kb += stride) {
        const uint32_t k = kb + threadIdx.x;
        const bool live = k < n;
        uint32_t r = 0xffffffffu - (uint32_t)lane;  // a distinct key for every idle lane
        unsigned long long v = 0, vi = 0, vj = 0, pk = 0;
        uint32_t cnt = 0;
        if (live) {
            r = uf_find(parent, k);
            const DevLeaf f = lv[k];
            v = f.votes;
            vi = (unsigned long long)f.votes * (2ull * f.i + 1ull);
            vj = (unsigned long long)f.votes * (2ull * f.j + 1ull);
            pk = ((unsigned long long)f.votes << 32) | (unsigned long long)(0xffffffffu - k);  // ties: smaller k
            cnt = 1;
        }
        const uint32_t nxt = __shfl_down_sync(0xffffffffu, r, 1);
        const uint32_t prv = __shfl_up_sync(0xffffffffu, r, 1);
        const uint32_t ends = __ballot_sync(0xffffffffu, lane == 31 || nxt != r);
        const int run_end = __ffs(ends & (0xffffffffu << lane)) - 1;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned long long ov = __shfl_down_sync(0xffffffffu, v, off);
            const unsigned long long oi = __shfl_down_sync(0xffffffffu, vi, off);
            const unsigned long long oj = __shfl_down_sync(0xffffffffu, vj, off);
            const unsigned long long op = __shfl_down_sync(0xffffffffu, pk, off);
            const uint32_t oc = __shfl_down_sync(0xffffffffu, cnt, off);
            if (lane + off <= run_end) {
                v += ov;
                vi += oi;
                vj += oj;
                pk = op > pk ? op : pk;
                cnt += oc;
            }
        }
        if (live && (lane == 0 || prv != r)) {  // the first lane of each run
            atomicAdd(&cells[r], cnt);
            atomicAdd(&sums[3 * (uint64_t)r + 0], v);
            atomicAdd(&sums[3 * (uint64_t)r + 1], vi);
            atomicAdd(&sums[3 * (uint64_t)r + 2], vj);
            atomicMax(&peak[r], pk);
        }
    }
}

constexpr int kEmitTPB = 256;
constexpr int kEmitPPT = 4;
constexpr int kEmitTile = kEmitTPB * kEmitPPT;

// Roots in index order -> lines.
__global__ void __launch_bounds__(kEmitTPB) lines_emit_kernel(const DevLeaf* __restrict__ lv, uint32_t n,
                                                              const uint32_t* __restrict__ parent,
                                                              const uint32_t* __restrict__ cells,
                                                              const unsigned long long* __restrict__ sums,
                                                              const unsigned long long* __restrict__ peak,
                                                              hht_line* __restrict__ out,
                                                              unsigned long long* total, ScanState* scan,
                                                              uint32_t* flags, uint64_t* data, DeviceStatus* status,
                                                              uint32_t ntiles) {
    __shared__ uint32_t s_slot;
    __shared__ uint32_t s_w[kEmitTPB / 32];
    __shared__ uint64_t s_pre;
    __shared__ unsigned long long s_n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_n = 0;
    const uint32_t epoch = scan->epoch;
    while (true) {
        const uint32_t t = claim_tile(scan, &s_slot);
        if (t >= ntiles) break;
        const uint64_t k0 = (uint64_t)t * kEmitTile + (uint64_t)tid * kEmitPPT;
        uint32_t is_root = 0;
#pragma unroll
        for (int j = 0; j < kEmitPPT; ++j)
            if (k0 + j < n && parent[k0 + j] == (uint32_t)(k0 + j)) is_root |= 1u << j;
        const uint32_t c = __popc(is_root);
        uint32_t inc = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += u;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            constexpr int NW = kEmitTPB / 32;
            const uint32_t w = lane < NW ? s_w[lane] : 0u;
            uint32_t jw = w;
#pragma unroll
            for (int off = 1; off < NW; off <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, jw, off);
                if (lane >= off) jw += u;
            }
            const uint64_t agg[1] = {__shfl_sync(0xffffffffu, jw, NW - 1)};
            __syncwarp();
            if (lane < NW) s_w[lane] = jw - w;
            uint64_t pre[1];
            tile_lookback<1>(flags, data, t, epoch, agg, pre, status);
            if (lane == 0) {
                s_pre = pre[0];
                s_n += agg[0];
            }
        }
        __syncthreads();
        uint64_t o = s_pre + s_w[warp] + (inc - c);
#pragma unroll
        for (int j = 0; j < kEmitPPT; ++j) {
            if (!((is_root >> j) & 1u)) continue;
            const uint64_t r = k0 + j;
            const uint32_t pk = 0xffffffffu - (uint32_t)(peak[r] & 0xffffffffull);
            const DevLeaf f = lv[pk];
            hht_line line;
            line.half = f.half;
            line.i = f.i;
            line.j = f.j;
            line.votes = f.votes;
            line.cells = cells[r];
            line.reserved = 0;
            line.total_votes = sums[3 * r + 0];
            line.sum_i2 = sums[3 * r + 1];
            line.sum_j2 = sums[3 * r + 2];
            out[o++] = line;
        }
    }
    __syncthreads();
    if (tid == 0 && s_n) atomicAdd(total, s_n);
    scan_finish(scan);
}

#define CKL(call)                                    \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)
#define RKL(call)                    \
    do {                             \
        int r_ = (call);             \
        if (r_ != HHT_OK) return r_; \
    } while (0)

}  // namespace
}  // namespace hht

using namespace hht;

extern "C" int hht_lines(hht_ctx* c, int32_t index, hht_line* lines, uint64_t capacity, uint64_t* n_lines) {
    hht::TraceRange tr("leaves to lines");
    if (!c || !n_lines) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (index < 0 || (size_t)index >= c->job_n.size()) return HHT_E_ARG;
    const uint64_t n = c->job_n[index];
    *n_lines = 0;
    if (n == 0) return HHT_OK;
    if (n >= 0xffffffe0ull) return HHT_E_ARG;  // leaf indices and the idle-lane keys of the gather stay distinct
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    // the second call of the two-call protocol copies the lines the first one kept
    if (c->lines_serial == c->job_serial && c->lines_index == index) {
        const uint64_t nl = c->lines_count;
        *n_lines = nl;
        if (nl > capacity) return HHT_E_CAPACITY;
        if (!lines) return HHT_E_ARG;
        RKL(copy_out(c, lines, c->line_out.p, nl * sizeof(hht_line)));
        CKL(cudaStreamSynchronize(st));
        return HHT_OK;
    }
    const DevLeaf* lv = (const DevLeaf*)c->leaves.p + c->job_off[index];
    uint64_t slots = 1024;
    while (slots < 2 * n) slots <<= 1;
    RKL(ensure(c, c->line_keys, slots * sizeof(unsigned long long)));
    RKL(ensure(c, c->line_vals, slots * sizeof(uint32_t)));
    RKL(ensure(c, c->line_parent, n * sizeof(uint32_t)));
    RKL(ensure(c, c->line_cells, n * sizeof(uint32_t)));
    RKL(ensure(c, c->line_sums, n * 4 * sizeof(unsigned long long)));  // [n][3] sums, then [n] peaks
    RKL(ensure(c, c->line_out, n * sizeof(hht_line) + 16));
    RKL(ensure(c, c->status, sizeof(DeviceStatus)));
    const uint64_t ntiles = (n + kEmitTile - 1) / kEmitTile;
    if ((ntiles + 1) * 4 > c->sel_flags.bytes) RKL(ensure(c, c->sel_flags, (ntiles + 1) * 4, true));
    RKL(ensure(c, c->sel_data, (ntiles + 1) * 2 * sizeof(uint64_t)));
    unsigned long long* keys = (unsigned long long*)c->line_keys.p;
    uint32_t* vals = (uint32_t*)c->line_vals.p;
    uint32_t* parent = (uint32_t*)c->line_parent.p;
    uint32_t* cells = (uint32_t*)c->line_cells.p;
    unsigned long long* sums = (unsigned long long*)c->line_sums.p;
    unsigned long long* peak = sums + 3 * n;
    unsigned long long* total = (unsigned long long*)((char*)c->line_out.p + n * sizeof(hht_line));
    CKL(cudaMemsetAsync(keys, 0xff, slots * sizeof(unsigned long long), st));
    CKL(cudaMemsetAsync(cells, 0, n * sizeof(uint32_t), st));
    CKL(cudaMemsetAsync(sums, 0, n * 4 * sizeof(unsigned long long), st));
    CKL(cudaMemsetAsync(total, 0, sizeof(unsigned long long), st));
    CKL(cudaMemsetAsync(c->status.p, 0, sizeof(DeviceStatus), st));
    DeviceStatus* status = (DeviceStatus*)c->status.p;
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)c->num_sms * 8);
    lines_insert_kernel<<<grid, 256, 0, st>>>(lv, (uint32_t)n, keys, vals, slots - 1, parent, status);
    lines_union_kernel<<<grid, 256, 0, st>>>(lv, (uint32_t)n, keys, vals, slots - 1, parent, status);
    lines_gather_kernel<<<grid, 256, 0, st>>>(lv, (uint32_t)n, parent, cells, sums, peak);
    const int egrid = (int)std::min<uint64_t>(ntiles, (uint64_t)c->num_sms * 4);
    lines_emit_kernel<<<std::max(egrid, 1), kEmitTPB, 0, st>>>(
        lv, (uint32_t)n, parent, cells, sums, peak, (hht_line*)c->line_out.p, total, (ScanState*)c->scan_states.p,
        (uint32_t*)c->sel_flags.p, (uint64_t*)c->sel_data.p, status, (uint32_t)ntiles);
    CKL(cudaGetLastError());
    c->prof.launches += 4;
    unsigned long long nl = 0;
    DeviceStatus hs{};
    CKL(cudaMemcpyAsync(&nl, total, sizeof nl, cudaMemcpyDeviceToHost, st));
    CKL(cudaMemcpyAsync(&hs, status, sizeof hs, cudaMemcpyDeviceToHost, st));
    CKL(cudaStreamSynchronize(st));
    if (hs.err & kErrTimeout) return HHT_E_TIMEOUT;
    if (hs.err) return HHT_E_CUDA;
    *n_lines = nl;
    c->lines_serial = c->job_serial;
    c->lines_index = index;
    c->lines_count = nl;
    if (nl > capacity) return HHT_E_CAPACITY;
    if (!lines) return HHT_E_ARG;
    RKL(copy_out(c, lines, c->line_out.p, nl * sizeof(hht_line)));
    CKL(cudaStreamSynchronize(st));
    return HHT_OK;
}
