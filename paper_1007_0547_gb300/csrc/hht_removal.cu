// The paper's solution() step (Section 3): the traversal is depth-first
// (quad1..quad4 = NE, NW, SW, SE at every level), and when a cell at the leaf
// level gets enough votes its voters are plotted and their codes zeroed at
// every level, so they take no part in any region reached later.  A region's
// count therefore depends on every cell accepted before it, which makes the
// traversal order part of the result.
//
// GPU form: one block of four warps per (image, half) walks that half's
// quadtree in the paper's order, with
//   - an explicit stack in shared memory (per level: next quadrant, region,
//     its children's list lengths, its votes when entered and the number of
//     points plotted by then), one copy per warp: every warp takes the same
//     decisions, and every pass over a list is shared out among the warps;
//   - the voters of a region split into its four children's lists once,
//     when it is entered (exact integer corner signs on the region's 3 x 3
//     grid decide all four children's votes at once, in int32 when
//     log2 L + depth <= 27; a ballot per quadrant, positions from popc), so
//     that a child's list only has to lose the points plotted since, and
//     while none were, its votes are its length and no pass is needed;
//   - the split of a region two levels above the leaves also counting its 16
//     grandchildren, and that of a region three levels above them its 64
//     great-grandchildren too, so that a child one or two levels above the
//     leaves is split (and entered) only when one of its leaves can pass;
//   - a removed-point bitmap (one bit per point) read through L2, so that the
//     block sees its own atomic updates.
// Many images and both halves run as independent blocks.  Readings (see the
// oracle): removal is per half; the `tests` statistic counts the codes
// actually evaluated (parent voters not removed by then); a region passes
// when its votes reach T.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/hht.h"
#include "hht_ctx.h"
#include "hht_device.cuh"
#include "hht_internal.h"
#include "hht_trace.h"

namespace hht {
namespace {

// One (image, half) of a removal job.
struct alignas(16) RemovalTask {
    uint64_t pts;        // offset of the image's points (int16 x, y pairs)
    uint64_t lists;      // offset of 4 D voter lists of n entries (four children per level)
    uint64_t bitmap;     // offset (in 32-bit words) of the removed-point bitmap
    uint64_t leaves;     // offset of the leaf output, `cap` entries
    uint64_t stats;      // offset of [D + 1][4] statistics
    uint64_t cap;        // leaf capacity: at most n / T + 1 cells can be accepted
    uint64_t max_steps;  // steps of the walk can never exceed this (see step_bound)
    int32_t n, lL, D, T;
    int32_t half, W, H;
    int32_t pad[3];
};

// Upper bound on the steps of one walk: every step either evaluates a child
// (four per region entered) or leaves a region, and at most
// min(4^l, n * (3 * 2^l + 1)) regions of level l can be entered (a line
// votes for at most 3 * 2^l + 1 cells of a level).  The walk ends on its own;
// the bound only turns a corrupted stack into an error instead of a hang.
uint64_t step_bound(uint64_t n, int D) {
    double regions = 1.0;
    for (int l = 1; l < D; ++l) regions += std::min(std::ldexp(1.0, 2 * l), (double)n * (3.0 * std::ldexp(1.0, l) + 1.0));
    const double steps = 5.0 * regions + 16.0;
    return steps > 1.8e19 ? ~0ull : (uint64_t)steps;
}

constexpr int kRemWarps = 4;  // warps per (image, half): one block walks one half

__device__ __forceinline__ int64_t scaled_g(int64_t x, int64_t y, int64_t i, int64_t j, int64_t L2, int64_t K) {
    // K * F at grid vertex (i, j): 4L j + 2x i - 2LK - Kx - Ky (L2 = 2L)
    return 2 * L2 * j + 2 * x * i - L2 * K - K * x - K * y;
}

// The children of region (i0, j0) of side 2h that the line of point (x, y)
// crosses, bit q = quadrant q.  G grows with i (x >= 0) and with j, so a
// cell's code is neither 0000 nor 1111 exactly when its SW corner is below the
// line and its NE corner is not; the children's SW and NE corners are 7
// vertices of the region's 3 x 3 grid (in steps of h from its SW corner):
// NE child (1,1)-(2,2), NW (0,1)-(1,2), SW (0,0)-(1,1), SE (1,0)-(2,1).
// I = int32_t when log2 L + depth <= 27 (every vertex value then lies within
// 2^29).
template <typename I>
__device__ __forceinline__ uint32_t child_crossings(int64_t x, int64_t y, int64_t i0, int64_t j0, int64_t h,
                                                    int64_t L2, int64_t K) {
    const I g00 = (I)scaled_g(x, y, i0, j0, L2, K);
    const I di = (I)(2 * x * h), dj = (I)(2 * L2 * h);
    const I g01 = g00 + dj, g10 = g00 + di, g11 = g10 + dj;
    const I g12 = g11 + dj, g21 = g11 + di, g22 = g21 + dj;
    return ((g11 < 0 && g22 >= 0) ? 1u : 0u) | ((g01 < 0 && g12 >= 0) ? 2u : 0u) |
           ((g00 < 0 && g11 >= 0) ? 4u : 0u) | ((g10 < 0 && g21 >= 0) ? 8u : 0u);
}

// The 16 grandchildren of region (i0, j0) of side 4g (cells of side g) that
// the line of point (x, y) crosses: bit 4a + b for the cell a steps of g east
// and b north of the region's SW corner, by the same SW / NE corner test on
// the region's 5 x 5 grid.
template <typename I>
__device__ __forceinline__ uint32_t grand_crossings(int64_t x, int64_t y, int64_t i0, int64_t j0, int64_t g,
                                                    int64_t L2, int64_t K) {
    const I g00 = (I)scaled_g(x, y, i0, j0, L2, K);
    const I di = (I)(2 * x * g), dj = (I)(2 * L2 * g);
    uint32_t bits = 0u;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const I sw = g00 + (I)a * di + (I)b * dj;
            if (sw < 0 && sw + di + dj >= 0) bits |= 1u << (4 * a + b);
        }
    }
    return bits;
}

// Grandchild cell (bit of grand_crossings) of leaf quadrant q2 of child quadrant q.
__device__ __forceinline__ int grand_cell(int q, int q2) {
    const int e = (q == NE || q == SE) ? 2 : 0, nn = (q == NE || q == NW) ? 2 : 0;
    const int e2 = (q2 == NE || q2 == SE) ? 1 : 0, n2 = (q2 == NE || q2 == NW) ? 1 : 0;
    return 4 * (e + e2) + (nn + n2);
}

// The 64 great-grandchildren of region (i0, j0) of side 8e (cells of side e)
// that the line of point (x, y) crosses: in w[a >> 2], bit 8 (a & 3) + b for
// the cell a steps east and b north of the region's SW corner.  Column a of
// the region's 9 x 9 grid has t_a vertices below the line (a prefix, as G
// grows with j; dj = 2 L2 e is a power of two, 2^ldj), and a cell is crossed
// exactly when its SW vertex is below and its NE vertex is not:
// t_{a+1} - 1 <= b < t_a.
template <typename I>
__device__ __forceinline__ void great_crossings(int64_t x, int64_t y, int64_t i0, int64_t j0, int64_t e, int64_t L2,
                                                int64_t K, int ldj, uint32_t (&w)[2]) {
    const I g00 = (I)scaled_g(x, y, i0, j0, L2, K);
    const I di = (I)(2 * x * e), dj1 = (I)((int64_t)1 << ldj) - 1;
    uint32_t below[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        const I v = (dj1 - (g00 + (I)a * di)) >> ldj;  // vertices of column a below the line, unclamped
        const int t = v < (I)0 ? 0 : (v > (I)9 ? 9 : (int)v);
        below[a] = (1u << t) - 1u;
    }
    w[0] = w[1] = 0u;
#pragma unroll
    for (int a = 0; a < 8; ++a) w[a >> 2] |= ((below[a] & ~(below[a + 1] >> 1)) & 0xffu) << (8 * (a & 3));
}

// Leaf (bit of great_crossings, as 8a + b) under leaf quadrant q3 of
// grandchild quadrant q2 of child quadrant q.
__device__ __forceinline__ int great_cell(int q, int q2, int q3) {
    auto e = [](int k) { return (k == NE || k == SE) ? 1 : 0; };
    auto nn = [](int k) { return (k == NE || k == NW) ? 1 : 0; };
    return 8 * (4 * e(q) + 2 * e(q2) + e(q3)) + (4 * nn(q) + 2 * nn(q2) + nn(q3));
}

// The walk of one (image, half) by a block of WARPS warps.  Every warp keeps
// its own copy of the stack and takes the same decisions from the same
// values, so the walk's control runs in step in all of them; every pass over
// a list (a split, a count of a leaf's voters not removed, the marking of an
// accepted leaf's voters) is shared out among the warps in groups of 128
// entries and ends with a block barrier.  Every read of a list or of the
// bitmap happens inside such a pass, so no warp rewrites a list (or marks a
// point) while another still reads it.  Lists are sets: the warps append to
// a child's list through shared cursors, so the order of its entries varies
// from run to run but no count does.
template <typename I, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) removal_kernel(const RemovalTask* __restrict__ tasks, int ntasks,
                                                          const int16_t* __restrict__ pts_all,
                                                          uint32_t* __restrict__ lists_all,
                                                          uint32_t* __restrict__ bitmap_all,
                                                          DevLeaf* __restrict__ leaves_all,
                                                          uint64_t* __restrict__ stats_all,
                                                          uint64_t* __restrict__ leaf_counts,
                                                          DeviceStatus* status) {
    // the walk's stack (one copy per warp), per level: next quadrant, the
    // region's SW corner, the lengths of its children's lists, its votes when
    // entered and the removed-point count at that time
    __shared__ int32_t s_quad[WARPS][kMaxDepth + 1];
    __shared__ uint32_t s_i0[WARPS][kMaxDepth + 1], s_j0[WARPS][kMaxDepth + 1];
    __shared__ uint32_t s_len[WARPS][kMaxDepth + 1][4];
    __shared__ uint32_t s_m[WARPS][kMaxDepth + 1], s_rem[WARPS][kMaxDepth + 1];
    // votes of the 16 grandchildren (the leaves) of the region last split at
    // level depth - 2, counted in its split
    __shared__ uint32_t s_g[WARPS][16];
    // votes of the 16 grandchildren and the 64 great-grandchildren (the
    // leaves) of the region last split at level depth - 3, counted in its split
    __shared__ uint32_t s_gd16[WARPS][16], s_gd64[WARPS][64];
    // each warp's share of a pass, two sets used in turn: [0, 16) grandchild
    // votes, [16, 80) great-grandchild votes, 80 the entries not removed,
    // [81, 85) the entries appended to each child's list
    constexpr int kPart = 85;
    __shared__ uint32_t s_part[2][WARPS][kPart];
    // the children's list cursors; they count on across passes (mod 2^32),
    // and each warp knows their value at the start of a pass
    __shared__ uint32_t s_cur[4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool lead = threadIdx.x == 0;
    const uint32_t lt = (1u << lane) - 1u;
    const int task = blockIdx.x;
    if (task >= ntasks) return;  // the same for the whole block
    const RemovalTask tk = tasks[task];
    const int16_t* pts = pts_all + 2 * tk.pts;
    uint32_t* lists = lists_all + tk.lists;
    uint32_t* bitmap = bitmap_all + tk.bitmap;
    DevLeaf* leaves = leaves_all + tk.leaves;
    uint64_t* stats = stats_all + tk.stats;
    const int64_t n = tk.n, D = tk.D, T = tk.T;
    const int64_t L2 = int64_t(2) << tk.lL, K = int64_t(1) << tk.D;
    const int half = tk.half;
    // the four children's lists of the region entered at level l
    auto child_list = [&](int l, int q) { return lists + (uint64_t)(4 * l + q) * (uint64_t)n; };
    uint32_t cur0[4] = {0u, 0u, 0u, 0u};  // the cursors at the start of the next pass
    int epoch = 0;                        // passes ended so far (selects the set of shares)

    // End of a pass: wait for every warp's share, then lane k of every warp
    // sums entries k, k + 32 and k + 64 of the shares.
    auto gather = [&](uint32_t (&t)[3]) {
        __syncthreads();
        const uint32_t(*p)[kPart] = s_part[epoch & 1];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int k = lane + 32 * r;
            uint32_t s = 0u;
            if (k < kPart)
#pragma unroll
                for (int v = 0; v < WARPS; ++v) s += p[v][k];
            t[r] = s;
        }
        ++epoch;
    };

    // Split the voters of `src` (len entries, or the points 0 .. len - 1 when
    // src is null) that are not removed into the lists of the four children
    // of region (i0, j0) of side 2h, kept at level l; lens[q] receive their
    // lengths.  Returns the number of voters not removed.  `check`: some
    // entry may have been removed since the list was built (else the bitmap
    // is not read).  `mode` 1: the votes of the region's 16 grandchildren
    // are counted too, into s_g; 2: into s_gd16, and those of its 64
    // great-grandchildren into s_gd64.  Warp w takes the groups of 128
    // entries w, w + WARPS, ...; in a group, each lane's four entries are
    // loaded as independent requests (list entries, then their bitmap words,
    // then their points).
    auto split = [&](const uint32_t* src, uint32_t len, bool check, int l, int64_t i0, int64_t j0, int64_t h,
                     uint32_t (&lens)[4], int mode) -> uint32_t {
        constexpr int U = 4;
        const bool grand = mode != 0, deep = mode == 2;
        uint32_t alive = 0, mine[4] = {0u, 0u, 0u, 0u};
        uint32_t gc[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) gc[k] = 0u;
        // great-grandchildren: lane L < 16 sums the 4 cells of nibble L (word
        // L >> 3, nibble L & 7) of the masks
        uint32_t acc64[4] = {0u, 0u, 0u, 0u};
        const int ldj = deep ? 1 + (tk.lL + 1) + (31 - __clz((unsigned)(h >> 2))) : 0;
        uint32_t* dst[4] = {child_list(l, 0), child_list(l, 1), child_list(l, 2), child_list(l, 3)};
        bool bad = false;
        for (uint32_t base = 32 * U * w; base < len; base += 32 * U * WARPS) {
            uint32_t v[U], bw[U], xm[U];
            bool in[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t idx = base + 32 * u + lane;
                in[u] = idx < len;
                v[u] = in[u] ? (src ? __ldcg(&src[idx]) : idx) : 0u;
                if (v[u] >= (uint32_t)n) {  // an entry that names no point (cannot happen)
                    bad = bad || in[u];
                    in[u] = false;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) bw[u] = (in[u] && check) ? __ldcg(&bitmap[v[u] >> 5]) : 0u;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                in[u] = in[u] && ((bw[u] >> (v[u] & 31u)) & 1u) == 0u;  // not removed
                xm[u] = in[u] ? __ldg(reinterpret_cast<const uint32_t*>(pts) + v[u]) : 0u;
            }
            uint32_t gw[U][2], cross[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint32_t gbits = 0u;
                cross[u] = 0u;
                gw[u][0] = gw[u][1] = 0u;
                if (in[u]) {
                    const int64_t px = (int16_t)(xm[u] & 0xffffu), py = (int16_t)(xm[u] >> 16);
                    const int64_t x = half ? py : px, y = half ? px : py;
                    cross[u] = child_crossings<I>(x, y, i0, j0, h, L2, K);
                    if (grand) gbits = grand_crossings<I>(x, y, i0, j0, h >> 1, L2, K);
                    if (deep) great_crossings<I>(x, y, i0, j0, h >> 2, L2, K, ldj, gw[u]);
                }
                if (grand) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) gc[k] += __popc(__ballot_sync(0xffffffffu, (gbits >> k) & 1u));
                }
                alive += __popc(__ballot_sync(0xffffffffu, in[u]));
            }
            // this group's entries per child, one cursor reservation per child
            // (lanes 0-3), then every entry at its reserved position
            uint32_t c[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int q = 0; q < 4; ++q) c[q] += __popc(__ballot_sync(0xffffffffu, (cross[u] >> q) & 1u));
            const uint32_t cq = lane == 0 ? c[0] : (lane == 1 ? c[1] : (lane == 2 ? c[2] : c[3]));
            uint32_t at = 0u;
            if (lane < 4 && cq != 0u) at = atomicAdd(&s_cur[lane], cq);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t pos = __shfl_sync(0xffffffffu, at, q) - cur0[q];  // offset in the child's list
                if (c[q] == 0u) continue;
                mine[q] += c[q];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool x = (cross[u] >> q) & 1u;
                    const uint32_t m = __ballot_sync(0xffffffffu, x);
                    const uint32_t at_q = pos + __popc(m & lt);
                    if (x) {
                        if (at_q < (uint32_t)n) dst[q][at_q] = v[u];
                        else bad = true;
                    }
                    pos += __popc(m);
                }
            }
            if (deep) {
                // the four groups' great-grandchild crossings as carry-save bit
                // planes (ones, twos, fours), spread into byte fields four cells
                // at a time and summed over the warp (at most 4 x 32 a byte)
                uint32_t red[16];
#pragma unroll
                for (int wd = 0; wd < 2; ++wd) {
                    const uint32_t s01 = gw[0][wd] ^ gw[1][wd], c01 = gw[0][wd] & gw[1][wd];
                    const uint32_t s23 = gw[2][wd] ^ gw[3][wd], c23 = gw[2][wd] & gw[3][wd];
                    const uint32_t ones = s01 ^ s23, c_ = s01 & s23;
                    const uint32_t twos = c01 ^ c23 ^ c_, fours = (c01 & c23) | (c_ & (c01 | c23));
#pragma unroll
                    for (int nb = 0; nb < 8; ++nb) {
                        const uint32_t packed = ((((ones >> (4 * nb)) & 0xfu) * 0x204081u) & 0x01010101u) +
                                                ((((twos >> (4 * nb)) & 0xfu) * 0x408102u) & 0x02020202u) +
                                                ((((fours >> (4 * nb)) & 0xfu) * 0x810204u) & 0x04040404u);
                        red[8 * wd + nb] = __reduce_add_sync(0xffffffffu, packed);
                    }
                }
                uint32_t r = red[0];
#pragma unroll
                for (int k = 1; k < 16; ++k) r = lane == k ? red[k] : r;
#pragma unroll
                for (int i = 0; i < 4; ++i) acc64[i] += (r >> (8 * i)) & 0xffu;
            }
        }
        if (bad) atomicOr(&status->err, kErrInvariant);  // a cursor ran past the list (cannot happen)
        uint32_t* part = s_part[epoch & 1][w];
        if (lane == 0) {
            if (grand)
#pragma unroll
                for (int k = 0; k < 16; ++k) part[k] = gc[k];
            part[80] = alive;
#pragma unroll
            for (int q = 0; q < 4; ++q) part[81 + q] = mine[q];
        }
        if (deep && lane < 16) {
            // nibble lane: cells a = 4 (lane >> 3) + ((lane & 7) >> 1), b = 4 (lane & 1) + i
            const int a = 4 * (lane >> 3) + ((lane & 7) >> 1), b0 = 4 * (lane & 1);
#pragma unroll
            for (int i = 0; i < 4; ++i) part[16 + 8 * a + b0 + i] = acc64[i];
        }
        uint32_t t[3];
        gather(t);
        if (grand && lane < 16) (deep ? s_gd16[w] : s_g[w])[lane] = t[0];
        if (deep) {
            if (lane >= 16) s_gd64[w][lane - 16] = t[0];
            s_gd64[w][16 + lane] = t[1];
            if (lane < 16) s_gd64[w][48 + lane] = t[2];
        }
        const uint32_t total = __shfl_sync(0xffffffffu, t[2], 16);  // entry 80
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            lens[q] = __shfl_sync(0xffffffffu, t[2], 17 + q);  // entries 81-84
            cur0[q] += lens[q];
        }
        __syncwarp();
        return total;
    };

    // level 0: every line crosses the whole parameter space (points outside
    // the image fail the image); the root's voters are split at once
    for (int64_t k = threadIdx.x; k < n; k += 32 * WARPS) {
        const int32_t px = pts[2 * k], py = pts[2 * k + 1];
        if (px < 0 || px >= tk.W || py < 0 || py >= tk.H) atomicOr(&status->err, kErrRange);
    }
    for (int64_t k = threadIdx.x; k < (n + 31) / 32; k += 32 * WARPS) bitmap[k] = 0u;
    if (threadIdx.x < 4) s_cur[threadIdx.x] = 0u;
    __syncthreads();
    {
        uint32_t lens[4];
        split(nullptr, (uint32_t)n, false, 0, 0, 0, K >> 1, lens, D == 2 ? 1 : (D == 3 ? 2 : 0));
        if (lead) {
            stats[0] = 1;
            stats[1] = 1;
            stats[2] = (uint64_t)n;
            stats[3] = (uint64_t)n;
        }
        if (lane == 0) {
            s_quad[w][0] = 0;
            s_i0[w][0] = 0;
            s_j0[w][0] = 0;
            s_m[w][0] = (uint32_t)n;
            s_rem[w][0] = 0u;
#pragma unroll
            for (int q = 0; q < 4; ++q) s_len[w][0][q] = lens[q];
        }
    }
    __syncwarp();
    uint64_t nleaves = 0;
    uint32_t removed = 0;  // points plotted so far in this half
    int level = 0;
    // every region is entered once and left after its fourth child, so the
    // walk ends (within tk.max_steps steps)
    bool finished = false;
    for (uint64_t step = 0; step < tk.max_steps; ++step) {
        const int q = s_quad[w][level];
        if (q == 4) {
            if (level == 0) {
                finished = true;
                break;
            }
            --level;
            continue;
        }
        __syncwarp();
        if (lane == 0) s_quad[w][level] = q + 1;
        const int64_t S = K >> level, h = S >> 1;
        const int64_t i0 = (int64_t)s_i0[w][level], j0 = (int64_t)s_j0[w][level];
        const int64_t ci = i0 + ((q == NE || q == SE) ? h : 0);
        const int64_t cj = j0 + ((q == NE || q == NW) ? h : 0);
        const int cl = level + 1;
        const uint32_t* src = child_list(level, q);
        const uint32_t len = s_len[w][level][q];
        // codes evaluated for this child: the parent's voters not removed by
        // now, i.e. its votes when entered less the points plotted since
        // (every one of them was a voter of this parent)
        const uint32_t evaluated = s_m[w][level] - (removed - s_rem[w][level]);
        // the child's list was split off when the parent was entered; when
        // nothing has been plotted since, every entry still votes
        const bool stale = removed != s_rem[w][level];
        uint32_t cnt = len;
        uint32_t lens[4] = {0u, 0u, 0u, 0u};
        bool accounted = false;  // the child's subtree was accounted from counts
        if (cl == D) {
            // a leaf: its voters not removed are counted
            if (stale) {
                uint32_t c = 0u;
                for (uint32_t base = 128 * w; base < len; base += 128 * WARPS) {
                    uint32_t v[4];
                    bool in[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        in[u] = base + 32 * u + lane < len;
                        v[u] = in[u] ? __ldcg(&src[base + 32 * u + lane]) : 0u;
                        in[u] = in[u] && v[u] < (uint32_t)n;  // an entry names a point (always)
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (in[u]) in[u] = ((__ldcg(&bitmap[v[u] >> 5]) >> (v[u] & 31u)) & 1u) == 0u;
                        c += __popc(__ballot_sync(0xffffffffu, in[u]));
                    }
                }
                if (lane == 0) s_part[epoch & 1][w][80] = c;
                uint32_t t[3];
                gather(t);
                cnt = __shfl_sync(0xffffffffu, t[2], 16);
            }
        } else if (cl == D - 2 && !stale) {
            // its children's and grandchildren's votes (levels D - 1 and D)
            // were counted when its parent was split, and nothing was plotted
            // since: unless one of its leaves can pass, its subtree follows
            // from those counts (none of it is accepted, so nothing is plotted
            // while it is tested) and it is not entered
            bool leaf_can_pass = false;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t ck = s_gd16[w][grand_cell(q, k)];
                if (ck >= (uint32_t)T)
#pragma unroll
                    for (int m = 0; m < 4; ++m) leaf_can_pass |= s_gd64[w][great_cell(q, k, m)] >= (uint32_t)T;
            }
            if (leaf_can_pass && len >= (uint32_t)T) {
                cnt = split(src, len, false, cl, ci, cj, h >> 1, lens, 1);
            } else {
                accounted = true;
                if (lead && len >= (uint32_t)T) {
                    // the region passes: its four children are tested (each
                    // evaluating its votes), and the four leaves of each child
                    // that passes (each evaluating that child's votes)
                    uint64_t cv = 0, cp = 0;
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t ck = s_gd16[w][grand_cell(q, k)];
                        cv += ck;
                        if (ck < (uint32_t)T) continue;
                        ++cp;
                        uint64_t lv = 0;
                        for (int m = 0; m < 4; ++m) lv += s_gd64[w][great_cell(q, k, m)];
                        stats[4 * D + 0] += 4;
                        stats[4 * D + 2] += lv;
                        stats[4 * D + 3] += 4ull * ck;
                    }
                    stats[4 * (D - 1) + 0] += 4;
                    stats[4 * (D - 1) + 1] += cp;
                    stats[4 * (D - 1) + 2] += cv;
                    stats[4 * (D - 1) + 3] += 4ull * len;
                }
            }
        } else if (cl == D - 1 && !stale) {
            // its leaves' votes were counted when its parent was split, and
            // nothing was plotted since: its own split is needed only when one
            // of them can pass (it is then entered)
#pragma unroll
            for (int k = 0; k < 4; ++k) lens[k] = s_g[w][grand_cell(q, k)];
            if (max(max(lens[0], lens[1]), max(lens[2], lens[3])) >= (uint32_t)T && len >= (uint32_t)T)
                split(src, len, false, cl, ci, cj, h >> 1, lens, 0);
        } else {
            cnt = split(src, len, stale, cl, ci, cj, h >> 1, lens, cl == D - 2 ? 1 : (cl == D - 3 ? 2 : 0));
        }
        __syncwarp();
        if (lead) {
            stats[4 * cl + 0] += 1;
            stats[4 * cl + 2] += cnt;
            stats[4 * cl + 3] += evaluated;
        }
        if ((int64_t)cnt >= T) {
            if (lead) stats[4 * cl + 1] += 1;
            if (cl == D) {
                // solution(): plot the voters and remove them from later regions
                if (lead) {
                    if (nleaves < tk.cap) {
                        DevLeaf f;
                        f.half = (uint32_t)half;
                        f.i = (uint32_t)ci;
                        f.j = (uint32_t)cj;
                        f.votes = cnt;
                        leaves[nleaves] = f;
                    } else {
                        atomicOr(&status->err, kErrOverflow);
                    }
                }
                ++nleaves;
                // the same voters as counted (nothing was removed in between);
                // an entry removed earlier keeps its bit, so every entry's bit
                // is set
                for (uint32_t k = threadIdx.x; k < len; k += 32 * WARPS) {
                    const uint32_t v = __ldcg(&src[k]);
                    if (v < (uint32_t)n) atomicOr(&bitmap[v >> 5], 1u << (v & 31u));
                }
                removed += cnt;
                __threadfence();
                __syncthreads();
            } else if (accounted) {
                // its subtree's statistics were added above
            } else if (cl == D - 1 && max(max(lens[0], lens[1]), max(lens[2], lens[3])) < (uint32_t)T) {
                // no leaf under this region can reach T, so none is accepted and
                // nothing is plotted while its four leaves are tested: each one's
                // votes are its list's length and its evaluated codes are this
                // region's votes, so the region is not entered
                if (lead) {
                    stats[4 * D + 0] += 4;
                    stats[4 * D + 2] += (uint64_t)lens[0] + lens[1] + lens[2] + lens[3];
                    stats[4 * D + 3] += 4ull * cnt;
                }
            } else {
                if (lane == 0) {
                    s_quad[w][cl] = 0;
                    s_i0[w][cl] = (uint32_t)ci;
                    s_j0[w][cl] = (uint32_t)cj;
                    s_m[w][cl] = cnt;
                    s_rem[w][cl] = removed;
#pragma unroll
                    for (int k = 0; k < 4; ++k) s_len[w][cl][k] = lens[k];
                }
                __syncwarp();
                level = cl;
            }
        }
    }
    if (!finished && lead) atomicOr(&status->err, kErrInvariant);
    if (lead) leaf_counts[task] = nleaves;
}

// One byte per point and half (half-major) from the removed-point bitmaps of
// one (image) task pair: 1 where the point was plotted.
__global__ void __launch_bounds__(256) flags_kernel(const uint32_t* __restrict__ bitmap, uint64_t b0, uint64_t b1,
                                                    int64_t n, uint8_t* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < 2 * n; k += stride) {
        const bool h1 = k >= n;
        const int64_t p = h1 ? k - n : k;
        out[k] = (uint8_t)((bitmap[(h1 ? b1 : b0) + (uint64_t)(p >> 5)] >> (p & 31)) & 1u);
    }
}

// The plotted points of one half scattered into a W-wide raster: `bit` is
// set in the byte of every pixel where a plotted point lies.  One launch per
// half, so that within a launch every thread that writes a pixel writes the
// same value (points may repeat).
__global__ void __launch_bounds__(256) raster_kernel(const int16_t* __restrict__ pts, int64_t n,
                                                     const uint32_t* __restrict__ bits, uint8_t* __restrict__ raster,
                                                     int32_t W, uint32_t bit) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
        if (((bits[k >> 5] >> (k & 31)) & 1u) == 0u) continue;
        uint8_t* px = raster + (size_t)pts[2 * k + 1] * (size_t)W + (size_t)pts[2 * k];
        *px = (uint8_t)(*px | bit);
    }
}

#define CKR(call)                                    \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)
#define RKR(call)                    \
    do {                             \
        int r_ = (call);             \
        if (r_ != HHT_OK) return r_; \
    } while (0)

int check_removal_image(const hht_image& im) {
    if (im.n < 0 || im.n > INT32_MAX || (im.n > 0 && !im.points)) return HHT_E_ARG;
    if (im.W < 1 || im.H < 1 || im.W > HHT_MAX_SIDE || im.H > HHT_MAX_SIDE) return HHT_E_ARG;
    if (im.depth < 1 || im.depth > HHT_MAX_DEPTH || im.T < 1) return HHT_E_ARG;
    return HHT_OK;
}

// Run the solution() traversal of `count` images; outs[k] as hht_detect
// (leaves: accepted cells, half 0's then half 1's, each in traversal order);
// plotted[k] (may be NULL) receives 2 * n flags (half-major).
int run_removal(hht_ctx* c, const hht_image* im, int count, hht_result* outs, uint8_t* const* plotted) {
    TraceRange tr("solution() walk");
    cudaStream_t st = c->stream;
    std::vector<RemovalTask> tasks((size_t)2 * count);
    uint64_t pts_len = 0, lists_len = 0, bitmap_len = 0, leaves_len = 0, stats_len = 0;
    std::vector<uint64_t> pts_off(count);
    for (int g = 0; g < count; ++g) {
        const int lL = ceil_log2_i(std::max(im[g].W, im[g].H));
        pts_off[g] = pts_len;
        const uint64_t n = (uint64_t)im[g].n;
        for (int h = 0; h < 2; ++h) {
            RemovalTask& t = tasks[(size_t)2 * g + h];
            std::memset(&t, 0, sizeof t);
            t.pts = pts_len;
            t.lists = lists_len;
            t.bitmap = bitmap_len;
            t.leaves = leaves_len;
            t.stats = stats_len;
            t.cap = n / (uint64_t)im[g].T + 1;
            t.max_steps = step_bound(n, im[g].depth);
            t.n = (int32_t)n;
            t.W = im[g].W;
            t.H = im[g].H;
            t.lL = lL;
            t.D = im[g].depth;
            t.T = im[g].T;
            t.half = h;
            lists_len += (uint64_t)4 * im[g].depth * std::max<uint64_t>(n, 1);  // four children's lists per level
            bitmap_len += (n + 31) / 32 + 1;
            leaves_len += t.cap;
            stats_len += (uint64_t)(im[g].depth + 1) * 4;
        }
        pts_len += n;
    }
    RKR(ensure(c, c->rem_pts, std::max<uint64_t>(pts_len, 1) * sizeof(hht_point)));
    RKR(ensure(c, c->rem_lists, std::max<uint64_t>(lists_len, 1) * sizeof(uint32_t)));
    RKR(ensure(c, c->rem_bitmap, std::max<uint64_t>(bitmap_len, 1) * sizeof(uint32_t)));
    RKR(ensure(c, c->rem_leaves, std::max<uint64_t>(leaves_len, 1) * sizeof(DevLeaf)));
    RKR(ensure(c, c->rem_stats, std::max<uint64_t>(stats_len, 1) * sizeof(uint64_t)));
    RKR(ensure(c, c->rem_tasks, tasks.size() * sizeof(RemovalTask) + (size_t)2 * count * sizeof(uint64_t)));
    RKR(ensure(c, c->status, sizeof(DeviceStatus)));
    for (int g = 0; g < count; ++g)
        if (im[g].n > 0)
            CKR(cudaMemcpyAsync((hht_point*)c->rem_pts.p + pts_off[g], im[g].points, (size_t)im[g].n * sizeof(hht_point),
                                cudaMemcpyDefault, st));
    CKR(cudaMemcpyAsync(c->rem_tasks.p, tasks.data(), tasks.size() * sizeof(RemovalTask), cudaMemcpyHostToDevice, st));
    CKR(cudaMemsetAsync(c->rem_stats.p, 0, std::max<uint64_t>(stats_len, 1) * sizeof(uint64_t), st));
    CKR(cudaMemsetAsync(c->status.p, 0, sizeof(DeviceStatus), st));
    uint64_t* d_counts = (uint64_t*)((char*)c->rem_tasks.p + tasks.size() * sizeof(RemovalTask));
    const int ntasks = 2 * count;
    const int grid = ntasks;  // one block per (image, half)
    // int32 corner arithmetic is exact while log2 L + depth <= 27 (every
    // vertex value then lies within 2^29), as in the level kernel
    bool i64 = false;
    for (int g = 0; g < count; ++g)
        if (ceil_log2_i(std::max(im[g].W, im[g].H)) + im[g].depth > 27) i64 = true;
    if (i64)
        removal_kernel<int64_t, kRemWarps><<<grid, 32 * kRemWarps, 0, st>>>(
            (const RemovalTask*)c->rem_tasks.p, ntasks, (const int16_t*)c->rem_pts.p, (uint32_t*)c->rem_lists.p,
            (uint32_t*)c->rem_bitmap.p, (DevLeaf*)c->rem_leaves.p, (uint64_t*)c->rem_stats.p,
            d_counts, (DeviceStatus*)c->status.p);
    else
        removal_kernel<int32_t, kRemWarps><<<grid, 32 * kRemWarps, 0, st>>>(
            (const RemovalTask*)c->rem_tasks.p, ntasks, (const int16_t*)c->rem_pts.p, (uint32_t*)c->rem_lists.p,
            (uint32_t*)c->rem_bitmap.p, (DevLeaf*)c->rem_leaves.p, (uint64_t*)c->rem_stats.p,
            d_counts, (DeviceStatus*)c->status.p);
    CKR(cudaGetLastError());
    c->prof.launches += 1;
    std::vector<uint64_t> counts((size_t)ntasks), h_stats(stats_len);
    DeviceStatus hs{};
    CKR(cudaMemcpyAsync(counts.data(), d_counts, counts.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CKR(cudaMemcpyAsync(h_stats.data(), c->rem_stats.p, stats_len * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    CKR(cudaMemcpyAsync(&hs, c->status.p, sizeof hs, cudaMemcpyDeviceToHost, st));
    CKR(cudaStreamSynchronize(st));
    c->rem_last.clear();
    if (hs.err & kErrRange) return HHT_E_RANGE;
    if (hs.err) return HHT_E_CUDA;
    for (int g = 0; g < count; ++g) {
        const RemovalTask& t0 = tasks[(size_t)2 * g], &t1 = tasks[(size_t)2 * g + 1];
        const uint64_t rec[6] = {pts_off[g], (uint64_t)im[g].n, t0.bitmap, t1.bitmap, (uint64_t)im[g].W,
                                 (uint64_t)im[g].H};
        c->rem_last.insert(c->rem_last.end(), rec, rec + 6);
    }
    int rc_all = HHT_OK;
    for (int g = 0; g < count; ++g) {
        hht_result& r = outs[g];
        const int D = im[g].depth;
        r.depth = D;
        r.L = 1 << ceil_log2_i(std::max(im[g].W, im[g].H));
        std::memset(r.stats, 0, sizeof r.stats);
        uint64_t nl = 0;
        for (int h = 0; h < 2; ++h) {
            const RemovalTask& t = tasks[(size_t)2 * g + h];
            for (int l = 0; l <= D; ++l) {
                const uint64_t* s = &h_stats[t.stats + 4 * (uint64_t)l];
                r.stats[h][l].tested = s[0];
                r.stats[h][l].passed = s[1];
                r.stats[h][l].votes = s[2];
                r.stats[h][l].tests = s[3];
            }
            nl += counts[(size_t)2 * g + h];
        }
        r.n_leaves = nl;
        if (nl > r.leaf_capacity || (nl > 0 && !r.leaves)) {
            r.status = HHT_E_CAPACITY;
        } else {
            r.status = HHT_OK;
            uint64_t at = 0;
            for (int h = 0; h < 2; ++h) {
                const RemovalTask& t = tasks[(size_t)2 * g + h];
                const uint64_t k = counts[(size_t)2 * g + h];
                if (k > 0)
                    RKR(copy_out(c, r.leaves + at, (const DevLeaf*)c->rem_leaves.p + t.leaves, k * sizeof(hht_leaf)));
                at += k;
            }
        }
        if (plotted && plotted[g] && im[g].n > 0) {
            // one byte per point and half, expanded on the device
            const RemovalTask& t0 = tasks[(size_t)2 * g], &t1 = tasks[(size_t)2 * g + 1];
            const uint64_t bytes = 2 * (uint64_t)im[g].n;
            cudaPointerAttributes at{};
            const bool dev = cudaPointerGetAttributes(&at, plotted[g]) == cudaSuccess && at.type == cudaMemoryTypeDevice;
            cudaGetLastError();
            uint8_t* dst = plotted[g];
            if (!dev) {
                RKR(ensure(c, c->rem_flags, bytes));
                dst = (uint8_t*)c->rem_flags.p;
            }
            const int fgrid = (int)std::min<uint64_t>((bytes + 255) / 256, (uint64_t)c->num_sms * 8);
            flags_kernel<<<fgrid, 256, 0, st>>>((const uint32_t*)c->rem_bitmap.p, t0.bitmap, t1.bitmap, im[g].n, dst);
            CKR(cudaGetLastError());
            c->prof.launches += 1;
            if (!dev) CKR(cudaMemcpyAsync(plotted[g], dst, bytes, cudaMemcpyDefault, st));
        }
        if (r.status != HHT_OK && rc_all == HHT_OK) rc_all = r.status;
    }
    CKR(cudaStreamSynchronize(st));
    return rc_all;
}

}  // namespace
}  // namespace hht

using namespace hht;

extern "C" {

int hht_detect_removal(hht_ctx* c, const hht_point* points, int64_t n, int32_t W, int32_t H, int32_t depth, int32_t T,
                       hht_result* out, uint8_t* plotted) {
    if (!c || !out) return HHT_E_ARG;
    hht_image im{points, n, W, H, depth, T};
    RKR(check_removal_image(im));
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    uint8_t* pl[1] = {plotted};
    return run_removal(c, &im, 1, out, pl);
}

int hht_removal_raster(hht_ctx* c, int32_t index, uint8_t* raster, uint64_t capacity) {
    if (!c || !raster || index < 0) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if ((uint64_t)index >= c->rem_last.size() / 6) return HHT_E_ARG;
    const uint64_t* rec = &c->rem_last[(size_t)6 * index];
    const uint64_t n = rec[1], W = rec[4], H = rec[5];
    if (capacity < W * H) return HHT_E_ARG;
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    cudaPointerAttributes at{};
    const bool dev = cudaPointerGetAttributes(&at, raster) == cudaSuccess && at.type == cudaMemoryTypeDevice;
    cudaGetLastError();
    uint8_t* dst = raster;
    if (!dev) {
        RKR(ensure(c, c->rem_raster, W * H));
        dst = (uint8_t*)c->rem_raster.p;
    }
    CKR(cudaMemsetAsync(dst, 0, W * H, st));
    if (n > 0) {
        const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)c->num_sms * 8);
        const int16_t* pts = (const int16_t*)c->rem_pts.p + 2 * rec[0];
        for (int h = 0; h < 2; ++h) {
            raster_kernel<<<grid, 256, 0, st>>>(pts, (int64_t)n, (const uint32_t*)c->rem_bitmap.p + rec[2 + h], dst,
                                                (int32_t)W, 1u << h);
            CKR(cudaGetLastError());
            c->prof.launches += 1;
        }
    }
    if (!dev) CKR(cudaMemcpyAsync(raster, dst, W * H, cudaMemcpyDefault, st));
    CKR(cudaStreamSynchronize(st));
    return HHT_OK;
}

int hht_detect_removal_batch(hht_ctx* c, const hht_image* images, int32_t count, hht_result* outs) {
    if (!c || !outs || count < 0 || (count > 0 && !images) || count > (1 << 20)) return HHT_E_ARG;
    for (int g = 0; g < count; ++g) RKR(check_removal_image(images[g]));
    if (count == 0) return HHT_OK;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    return run_removal(c, images, count, outs, nullptr);
}

}  // extern "C"
