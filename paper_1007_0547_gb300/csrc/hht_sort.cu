// Leaf output order: a stable LSD radix sort (8-bit digits) of the leaf
// records by the key (unit, i, j), so that every image's leaves come out
// grouped by half and sorted by cell, independent of the order in which the
// level kernels emitted them.  Per pass: a per-tile digit histogram, one
// single-pass look-back scan over the digit-major histogram, and a stable
// scatter that ranks equal digits within a tile with warp match masks.
#include <cuda_runtime.h>

#include <cstdint>

#include "hht_device.cuh"
#include "hht_internal.h"

namespace hht {

namespace {
constexpr int kTPB = 256;
constexpr int kIPT = 8;  // items per thread
constexpr int kTile = kTPB * kIPT;
constexpr int kRadix = 256;

__device__ __forceinline__ uint64_t leaf_key(const DevLeaf& l, int depth_bits) {
    return ((uint64_t)l.unit << (2 * depth_bits)) | ((uint64_t)l.i << depth_bits) | (uint64_t)l.j;
}

__global__ void __launch_bounds__(kTPB) hist_kernel(const DevLeaf* __restrict__ in, uint64_t n, int shift, int depth_bits,
                                                    uint32_t* __restrict__ hist, uint32_t ntiles) {
    __shared__ uint32_t h[kRadix];
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        h[threadIdx.x] = 0;
        __syncthreads();
        const uint64_t base = (uint64_t)t * kTile;
#pragma unroll
        for (int r = 0; r < kIPT; ++r) {
            const uint64_t idx = base + (uint64_t)r * kTPB + threadIdx.x;
            if (idx < n) atomicAdd(&h[(leaf_key(in[idx], depth_bits) >> shift) & 0xffu], 1u);
        }
        __syncthreads();
        hist[(size_t)threadIdx.x * ntiles + t] = h[threadIdx.x];
        __syncthreads();
    }
}

// Exclusive scan of m uint32 values in place (single pass, decoupled look-back).
__global__ void __launch_bounds__(kTPB) scan_kernel(uint32_t* __restrict__ v, uint64_t m, ScanState* st,
                                                    uint32_t* flags, uint64_t* data, DeviceStatus* status) {
    __shared__ uint32_t s_slot;
    __shared__ uint32_t s_w[8];
    __shared__ uint64_t s_pre;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ntiles = (uint32_t)((m + kTile - 1) / kTile);
    const uint32_t epoch = st->epoch;
    while (true) {
        const uint32_t t = claim_tile(st, &s_slot);
        if (t >= ntiles) break;
        const uint64_t base = (uint64_t)t * kTile + (uint64_t)threadIdx.x * kIPT;
        uint32_t x[kIPT];
        uint32_t sum = 0;
#pragma unroll
        for (int k = 0; k < kIPT; ++k) {
            x[k] = (base + k < m) ? v[base + k] : 0u;
            sum += x[k];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += o;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < 8 ? s_w[lane] : 0u;
            uint32_t iw = w;
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
                const uint32_t o = __shfl_up_sync(0xffffffffu, iw, off);
                if (lane >= off) iw += o;
            }
            const uint64_t agg[1] = {__shfl_sync(0xffffffffu, iw, 7)};
            if (lane < 8) s_w[lane] = iw - w;
            uint64_t pre[1];
            tile_lookback<1>(flags, data, t, epoch, agg, pre, status);
            if (lane == 0) s_pre = pre[0];
        }
        __syncthreads();
        uint64_t run = s_pre + s_w[warp] + (inc - sum);
#pragma unroll
        for (int k = 0; k < kIPT; ++k) {
            if (base + k < m) v[base + k] = (uint32_t)run;
            run += x[k];
        }
    }
    scan_finish(st);
}

__global__ void __launch_bounds__(kTPB) scatter_kernel(const DevLeaf* __restrict__ in, DevLeaf* __restrict__ out,
                                                       uint64_t n, int shift, int depth_bits,
                                                       const uint32_t* __restrict__ offs, uint32_t ntiles) {
    __shared__ uint32_t s_warp_cnt[8][kRadix];
    __shared__ uint32_t s_run[kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        s_run[threadIdx.x] = offs[(size_t)threadIdx.x * ntiles + t];
        const uint64_t base = (uint64_t)t * kTile;
        for (int r = 0; r < kIPT; ++r) {
#pragma unroll
            for (int w = 0; w < 8; ++w) s_warp_cnt[w][threadIdx.x] = 0;
            __syncthreads();
            const uint64_t idx = base + (uint64_t)r * kTPB + threadIdx.x;
            const bool ok = idx < n;
            DevLeaf it{};
            uint32_t d = 0xffffffffu;  // sentinel never equal to a digit
            if (ok) {
                it = in[idx];
                d = (uint32_t)((leaf_key(it, depth_bits) >> shift) & 0xffu);
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t rank = __popc(peers & lt);
            if (ok && rank == 0) s_warp_cnt[warp][d] = __popc(peers);
            __syncthreads();
            // per digit: exclusive prefix over warps, then advance the running offset
            {
                const int dd = threadIdx.x;
                uint32_t acc = 0;
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    const uint32_t c = s_warp_cnt[w][dd];
                    s_warp_cnt[w][dd] = acc;
                    acc += c;
                }
                __syncthreads();
                if (ok) out[s_run[d] + s_warp_cnt[warp][d] + rank] = it;
                __syncthreads();
                s_run[dd] += acc;
            }
            __syncthreads();
        }
    }
}
}  // namespace

namespace {
constexpr uint64_t align256(uint64_t v) { return (v + 255) & ~uint64_t(255); }
struct SortLayout {
    uint64_t ntiles, m, stiles, hist_off, flags_off, data_off, bytes;
};
SortLayout sort_layout(uint64_t n) {
    SortLayout L;
    L.ntiles = (n + kTile - 1) / kTile;
    L.m = L.ntiles * kRadix;
    L.stiles = (L.m + kTile - 1) / kTile + 1;
    L.hist_off = 256;  // [0, 256): ScanState
    L.flags_off = L.hist_off + align256(L.m * 4);
    L.data_off = L.flags_off + align256(L.stiles * 4);
    L.bytes = L.data_off + align256(L.stiles * 16);
    return L;
}
}  // namespace

size_t sort_scratch_bytes(uint64_t n) { return (size_t)sort_layout(n).bytes; }

int launch_leaf_sort(DevLeaf* leaves, DevLeaf* tmp, uint64_t n, int unit_bits, int depth_bits, void* scratch,
                     size_t scratch_bytes, DeviceStatus* status, int num_sms, void* stream, int* kernels_launched) {
    *kernels_launched = 0;
    if (n <= 1) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    const SortLayout L = sort_layout(n);
    const uint64_t ntiles = L.ntiles, m = L.m, stiles = L.stiles;
    if (L.bytes > scratch_bytes) return -1;
    char* p = (char*)scratch;
    ScanState* ss = (ScanState*)p;
    uint32_t* hist = (uint32_t*)(p + L.hist_off);
    uint32_t* flags = (uint32_t*)(p + L.flags_off);
    uint64_t* data = (uint64_t*)(p + L.data_off);
    // flags of an earlier sort may carry any epoch: clear them and the scan
    // state (epoch 0 with state 0 never reads as published)
    cudaMemsetAsync(flags, 0, stiles * 4, st);
    cudaMemsetAsync(ss, 0, sizeof(ScanState), st);
    const int total_bits = unit_bits + 2 * depth_bits;
    const int grid = (int)(ntiles < (uint64_t)num_sms * 8 ? ntiles : (uint64_t)num_sms * 8);
    int scan_grid = num_sms * 4;
    if ((uint64_t)scan_grid > stiles) scan_grid = (int)stiles;
    DevLeaf* src = leaves;
    DevLeaf* dst = tmp;
    int passes = 0;
    for (int shift = 0; shift < total_bits; shift += 8, ++passes) {
        hist_kernel<<<grid, kTPB, 0, st>>>(src, n, shift, depth_bits, hist, (uint32_t)ntiles);
        scan_kernel<<<scan_grid, kTPB, 0, st>>>(hist, m, ss, flags, data, status);
        scatter_kernel<<<grid, kTPB, 0, st>>>(src, dst, n, shift, depth_bits, hist, (uint32_t)ntiles);
        DevLeaf* sw = src; src = dst; dst = sw;
        *kernels_launched += 3;
    }
    if (src != leaves) cudaMemcpyAsync(leaves, src, n * sizeof(DevLeaf), cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hht
