// Device helpers: exact corner-sign grids, bit-sliced 4-bit codes, single-pass
// scan state (decoupled look-back) with bounded waits, warp reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hht_internal.h"

namespace hht {

// ----------------------------------------------------------------- memory-model helpers
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// ----------------------------------------------------------------- corner signs and codes
//
// For one line and one region, the corner vertices of an N x N sub-grid
// (N = 3: the region's four children; N = 5: also its sixteen grandchildren)
// are classified exactly.  Along a column of the sub-grid, G grows by the
// positive power of two dJ = 2^k per step, so the number of vertices with
// G < 0 in that column is t = ceil(-G_column_base / dJ) clamped to [0, N],
// an exact shift.  The result is an N*N-bit mask M with bit (alpha*N + beta)
// set when vertex (column alpha, row beta) lies strictly below the line.
// Column alpha contributes bits [N*alpha, N*alpha + t): summed as
// 2^(N*alpha + t) - 2^(N*alpha) over the columns.
template <int N>
__device__ __forceinline__ constexpr uint32_t column_bases() {
    uint32_t b = 0;
    for (int alpha = 0; alpha < N; ++alpha) b += 1u << (N * alpha);
    return b;
}

template <typename I, int N>
__device__ __forceinline__ uint32_t below_mask(I G0, I dI, int k) {
    const I dJm1 = (I(1) << k) - I(1);
    uint32_t M = 0;
    I G = G0;
#pragma unroll
    for (int alpha = 0; alpha < N; ++alpha) {
        I t = (dJm1 - G) >> k;  // floor((-G + dJ - 1) / dJ) = ceil(-G / dJ)
        int ti;
        if constexpr (sizeof(I) == 4) {
            ti = __vimin_s32_relu((int)t, N);  // clamp to [0, N]
        } else {
            t = t < I(0) ? I(0) : (t > I(N) ? I(N) : t);
            ti = (int)t;
        }
        M += 1u << (N * alpha + ti);
        G += dI;
    }
    return M - column_bases<N>();
}

// Bit-sliced 4-bit codes: for cells of side `sz` sub-grid steps, the word
// `M >> (sz*N + sz)` holds at bit (alpha*N + beta) the NE-corner bit of the
// cell whose SW corner is vertex (alpha, beta); likewise NW (>> sz),
// SW (>> 0) and SE (>> sz*N).  A line votes for a cell when the cell's code
// is neither 0000 nor 1111: some corner bit set and not all four.
template <int N, int sz>
__device__ __forceinline__ uint32_t crossing_cells(uint32_t M) {
    const uint32_t ne = M >> (sz * N + sz), nw = M >> sz, sw = M, se = M >> (sz * N);
    const uint32_t any = ne | nw | sw | se;
    const uint32_t all = ne & nw & sw & se;
    return any & ~all;
}

// Quadrant index of (east, north) halves: NE = 0, NW = 1, SW = 2, SE = 3.
__device__ __forceinline__ int quad_of(int east, int north) {
    return north ? (east ? NE : NW) : (east ? SE : SW);
}

// Child votes (bit q = quadrant q) from a 3 x 3 below-mask: children are the
// 1 x 1 step cells with SW corners NE (1,1), NW (0,1), SW (0,0), SE (1,0).
__device__ __forceinline__ uint32_t child_votes3(uint32_t M) {
    const uint32_t v = crossing_cells<3, 1>(M);
    return ((v >> 4) & 1u) | (((v >> 1) & 1u) << 1) | ((v & 1u) << 2) | (((v >> 3) & 1u) << 3);
}
// Code of the whole region from a 3 x 3 mask: NE, NW, SW, SE corners are the
// vertices (2,2), (0,2), (0,0), (2,0), i.e. bits 8, 2, 0, 6 (NE is the code's
// leftmost bit).
__device__ __forceinline__ uint32_t region_code3(uint32_t M) {
    return (((M >> 8) & 1u) << 3) | (((M >> 2) & 1u) << 2) | (((M >> 0) & 1u) << 1) | ((M >> 6) & 1u);
}

// ---------------------------------------------------------------- pass-kernel bit layouts
// The corner-sign mask M of the 5 x 5 quarter-step grid holds vertex
// (alpha, beta) at bit 5*alpha + beta.  Every column of M is a prefix (the
// vertices below the line are the lowest t of the column).  G grows with i
// (x >= 0) and with j, so a cell's SW corner is its lowest and its NE corner
// its highest: the cell's 4-bit code is neither 0000 nor 1111 exactly when SW
// is below the line and NE is not.  The pass kernel forms that test for all
// cells of side sz at once as (M << 6*sz) & ~M, which leaves the result of the
// cell whose SW vertex is p at bit p + 6*sz, its NE vertex.
// Children (2 x 2 steps, sz = 2) of quadrant q = NE, NW, SW, SE have SW
// vertices 12, 2, 0, 10 and so vote at bits 24, 14, 12, 22.
__host__ __device__ __forceinline__ constexpr int quad_bit(int q) { return q == 0 ? 24 : q == 1 ? 14 : q == 2 ? 12 : 22; }
// Grandchild (alpha, beta), alpha, beta < 4 (sz = 1), votes at bit kGrandBase + 5*alpha + beta.
constexpr int kGrandBase = 6;

// The four quadrant bits of `q4` (bit q = quadrant q) at quad_bit positions.
__device__ __forceinline__ uint32_t spread_quads(uint32_t q4) {
    return ((q4 & 1u) << 24) | ((q4 & 2u) << 13) | ((q4 & 4u) << 10) | ((q4 & 8u) << 19);
}

// Grandchild cells of the children whose vote bits (quad_bit positions) are
// set in `kids`: child q's 2 x 2 grandchildren sit at its bit - 6 + {0, 1, 5, 6}
// (one multiply; the four children's cells are disjoint, so nothing carries).
__device__ __forceinline__ uint32_t grand_cells(uint32_t kids) { return (kids >> 6) * 0x63u; }

// Bits pos .. pos + t - 1 set (0 <= pos, t and pos + t <= 32).
template <int pos>
__device__ __forceinline__ uint32_t prefix_bits(int t) {
    uint32_t r;
    asm("bmsk.clamp.b32 %0, %1, %2;" : "=r"(r) : "n"(pos), "r"(t));
    return r;
}

// The children's vote bits (quad_bit positions) of `kw` as byte counters:
// ((kw >> 12) * 0x1041) moves bits 12, 14, 22, 24 to bits 0, 8, 16, 24 and
// every other product lands off those bits without a carry into them.
// Quadrant q counts in byte quad_byte(q).
__device__ __forceinline__ uint32_t quad_counts(uint32_t kw) { return ((kw >> 12) * 0x1041u) & 0x01010101u; }
__host__ __device__ __forceinline__ constexpr int quad_byte(int q) { return q == 0 ? 3 : q == 1 ? 1 : q == 2 ? 0 : 2; }
// quad_byte for a quadrant known only at run time (a nibble table, no local array).
__host__ __device__ __forceinline__ constexpr uint32_t quad_byte_rt(uint32_t q) { return (0x2013u >> (4 * q)) & 0xfu; }
static_assert(quad_byte_rt(0) == 3 && quad_byte_rt(1) == 1 && quad_byte_rt(2) == 0 && quad_byte_rt(3) == 2,
              "run-time quadrant byte table");

// An 8-byte store made only when `pred` is non-zero, as one predicated
// instruction (a plain `if` around a store may become a branch).
__device__ __forceinline__ void st_pred_v2(void* p, uint32_t pred, uint32_t x, uint32_t y) {
    asm volatile("{ .reg .pred q; setp.ne.u32 q, %0, 0; @q st.global.v2.u32 [%1], {%2, %3}; }"
                 :: "r"(pred), "l"(p), "r"(x), "r"(y));
}

// Spread 4 bits into the low bit of 4 bytes (bit b -> byte b).
__device__ __forceinline__ uint32_t spread4(uint32_t r) { return (r * 0x204081u) & 0x01010101u; }

// ----------------------------------------------------------------- bounded spin
constexpr uint32_t kSpinLimit = 1u << 22;  // ~0.5-1 s with the back-off below

// ----------------------------------------------------------------- look-back scan
// Per tile: flag word (epoch << 2 | state), state 1 = aggregate published,
// 2 = inclusive prefix published; data[tile * 2C + c] = aggregate,
// data[tile * 2C + C + c] = inclusive.
//
// The scan is split in two so that a tile can publish its aggregate as soon
// as it is known and do other work before it needs its prefix:
// publish_aggregate() (one lane) and resolve_prefix() (all 32 lanes of one
// warp; returns the exclusive prefix of tile t and publishes its inclusive
// value).
template <int C>
__device__ __forceinline__ void publish_aggregate(uint32_t* flags, uint64_t* data, uint32_t t, uint32_t epoch,
                                                  const uint64_t (&agg)[C]) {
    // tile 0's aggregate is already its inclusive prefix
    const int slot = (t == 0) ? C : 0;
#pragma unroll
    for (int c = 0; c < C; ++c) st_relaxed_u64(&data[(size_t)t * 2 * C + slot + c], agg[c]);
    st_release_u32(&flags[t], (epoch << 2) | (t == 0 ? 2u : 1u));
}

// `publish` is false only for a tile withheld by host-side fault injection
// (hht_inject_fault): it then publishes nothing, and the tiles after it wait
// until their bounded wait expires.
template <int C>
__device__ void resolve_prefix(uint32_t* flags, uint64_t* data, uint32_t t, uint32_t epoch, const uint64_t (&agg)[C],
                               uint64_t (&prefix)[C], DeviceStatus* status, bool publish = true) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < C; ++c) prefix[c] = 0;
    if (t == 0) return;
    int64_t top = (int64_t)t - 1;
    // once any wait of this job has expired, no further wait is started
    bool timed_out = (*reinterpret_cast<volatile uint32_t*>(&status->err) & kErrTimeout) != 0u;
    while (true) {
        const int64_t idx = top - lane;
        uint32_t state = 2;  // before tile 0: an inclusive prefix of zero
        if (idx >= 0) {
            uint32_t f = 0;
            uint32_t spins = 0;
            while (true) {
                f = ld_acquire_u32(&flags[idx]);
                if ((f >> 2) == epoch && (f & 3u) != 0) break;
                if (timed_out || ++spins > kSpinLimit) {
                    timed_out = true;
                    f = (epoch << 2) | 1u;  // treat as an empty aggregate; the job is reported failed
                    break;
                }
                if (spins > 64) __nanosleep(spins > 4096 ? 256 : 32);
            }
            state = f & 3u;
        }
        timed_out = __any_sync(0xffffffffu, timed_out);
        const uint32_t inc = __ballot_sync(0xffffffffu, state == 2u);
        const int first = inc ? (__ffs(inc) - 1) : 32;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            uint64_t v = 0;
            if (idx >= 0 && lane <= first && !timed_out)
                v = ld_relaxed_u64(&data[(size_t)idx * 2 * C + (lane == first ? C : 0) + c]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            prefix[c] += v;
        }
        if (inc) break;
        top -= 32;
    }
    if (timed_out && lane == 0) atomicOr(&status->err, kErrTimeout);
    if (lane == 0 && publish) {
#pragma unroll
        for (int c = 0; c < C; ++c) st_relaxed_u64(&data[(size_t)t * 2 * C + C + c], prefix[c] + agg[c]);
        st_release_u32(&flags[t], (epoch << 2) | 2u);
    }
}

// Both halves back to back (for kernels with nothing to overlap).
template <int C>
__device__ __forceinline__ void tile_lookback(uint32_t* flags, uint64_t* data, uint32_t t, uint32_t epoch,
                                              const uint64_t (&agg)[C], uint64_t (&prefix)[C], DeviceStatus* status,
                                              bool publish = true) {
    if ((threadIdx.x & 31) == 0 && publish) publish_aggregate<C>(flags, data, t, epoch, agg);
    __syncwarp();
    resolve_prefix<C>(flags, data, t, epoch, agg, prefix, status, publish);
}

// End-of-launch protocol for a scan: the last block to finish resets the tile
// counter and advances the epoch.  Returns true in thread 0 of the last block.
__device__ __forceinline__ bool scan_finish(ScanState* st) {
    __syncthreads();
    bool last = false;
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t d = atomicAdd(&st->done_counter, 1u);
        if (d == gridDim.x - 1) {
            st->tile_counter = 0;
            st->done_counter = 0;
            st->epoch = st->epoch + 1u;
            __threadfence();
            last = true;
        }
    }
    return last;
}

__device__ __forceinline__ uint32_t claim_tile(ScanState* st, uint32_t* s_slot) {
    __syncthreads();
    if (threadIdx.x == 0) *s_slot = atomicAdd(&st->tile_counter, 1u);
    __syncthreads();
    return *s_slot;
}

}  // namespace hht
