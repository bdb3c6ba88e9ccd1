// Level kernels of the hierarchical Hough transform (sm_103a).
//
//   stage   level 0: range-check the points, write the level-0 voter streams of
//           both halves and count the votes of the four level-1 quadrants.
//   select  level s: a level-(s-1) region's child passes when its votes >= T
//           (Section 3).  Passed children become the level-s region
//           records (or leaves at the unit's depth); a look-back scan gives
//           every child its record index.  Also writes the level statistics.
//   pass    level s: one read of the level-(s-1) voter stream.  Per voter the
//           exact 5 x 5 corner-sign grid of its parent region gives the 4-bit
//           codes of the four children (level s) and of the sixteen
//           grandchildren (level s+1).  Voters of passed children are copied
//           (stable, decoupled look-back scan with a 4-vector of per-quadrant
//           counts) into the level-s stream, and grandchild votes are counted
//           for the next selection.  The copy is skipped where the next level
//           is the unit's last one, so the largest list is never written.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "hht_device.cuh"
#include "hht_internal.h"

namespace hht {

namespace {

constexpr uint32_t kNoRegion = 0xffffffffu;
constexpr uint32_t kAbortMask = kErrTimeout | kErrOverflow | kErrInvariant;

__device__ __forceinline__ bool job_aborted(const DeviceStatus* st) {
    return (*reinterpret_cast<const volatile uint32_t*>(&st->err) & kAbortMask) != 0u;
}

// Segmented suffix sum over the lanes of a warp for keys that are sorted
// across lanes (equal keys are contiguous): afterwards the first lane of each
// key run holds the run's total.
template <int W>
__device__ __forceinline__ void warp_segmented_total(uint32_t key, uint32_t (&v)[W]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t ko = __shfl_down_sync(0xffffffffu, key, off);
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t o = __shfl_down_sync(0xffffffffu, v[w], off);
            if (lane + off < 32 && ko == key) v[w] += o;
        }
    }
}

__device__ __forceinline__ bool run_head(uint32_t key) {
    const int lane = threadIdx.x & 31;
    const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
    return key != kNoRegion && (lane == 0 || prev != key);
}

}  // namespace

// ============================================================================ stage
// FHT circle test of the four level-1 quadrants (side K/2) of the level-0
// region: with 2G at a child's centre = -2LK + 4LK*n - K*x + 2K*x*e - 2K*y
// (e, n: east and north halves), the child gets the vote when
// (2G)^2 <= 2 K^2 (x^2 + 4L^2).  Bit q = quadrant q.
__device__ __forceinline__ uint32_t fht_root_children(int32_t x, int32_t y, int lL, int D) {
    const int64_t L = int64_t(1) << lL, K = int64_t(1) << D;
    const int64_t X = (int64_t)x * x + 4 * L * L;
    const int64_t r = X << (2 * D + 1);
    uint32_t bits = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int64_t e = (q == NE || q == SE) ? 1 : 0, n = (q == NE || q == NW) ? 1 : 0;
        const int64_t g2 = -2 * L * K + 4 * L * K * n - K * x + 2 * K * x * e - 2 * K * y;
        bits |= (g2 * g2 <= r ? 1u : 0u) << q;
    }
    return bits;
}

template <typename I, bool FHT = false>
__device__ __forceinline__ void stage_body(const int16_t* __restrict__ pts, uint64_t total,
                                           const Unit* __restrict__ units, int n_images,
                                           const uint64_t* __restrict__ img_start,
                                           const uint32_t* __restrict__ img_unit, Voter* __restrict__ v0,
                                           uint32_t* __restrict__ root_cnt, uint64_t* __restrict__ stats,
                                           uint32_t* __restrict__ img_err, DeviceStatus* status,
                                           const JobDims* __restrict__ dims) {
    if (dims) {
        total = dims->total_points;
        n_images = dims->n_images;
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t kb = (uint64_t)blockIdx.x * blockDim.x; kb < total; kb += stride) {
        const uint64_t k = kb + threadIdx.x;
        const bool active = k < total;
        int img = 0;
        if (active) {  // image of point k: last img with img_start[img] <= k
            int lo = 0, hi = n_images - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (img_start[mid] <= k) lo = mid; else hi = mid - 1;
            }
            img = lo;
        }
        int32_t px = 0, py = 0;
        bool ok = false;
        if (active) {
            const Unit& U = units[img_unit[img]];
            px = pts[2 * k];
            py = pts[2 * k + 1];
            ok = px >= 0 && px < U.W && py >= 0 && py < U.H;
            // the image fails; the others are unaffected.  Flags are indexed by
            // unit pair (img_unit / 2): the image's index in a batch, its
            // request slot in serving
            if (!ok) atomicOr(&img_err[img_unit[img] >> 1], kErrRange);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t u0 = active ? img_unit[img] + (uint32_t)h : 0u;
            // a half that takes none of the image's points (its unit has no
            // level-0 voters) behaves as past the end
            const bool on = active && units[u0].inactive == 0u;
            const uint32_t u = on ? u0 : 0u;
            uint32_t key = (on && ok) ? u : kNoRegion;
            if (on && !ok) {
                // a point outside its image fails the image; its level-0 slot
                // still gets a record, marked as belonging to no region, so
                // that the stream holds no uninitialised entries
                const Unit& U = units[u];
                if (U.D >= 2) {
                    Voter dead;
                    dead.x = 0;
                    dead.y = 0;
                    dead.region = kNoRegion;
                    v0[U.v0_off + (k - img_start[img])] = dead;
                }
            }
            uint32_t vals[2] = {0u, 0u};  // [0]: child votes as 4 bytes, [1]: level-0 votes
            if (on && ok) {
                const Unit& U = units[u];
                const int32_t x = h ? py : px, y = h ? px : py;
                const int D = U.D, lL = U.lL;
                // 3 x 3 grid over the level-0 region: vertices (alpha*K/2, beta*K/2)
                const I G0 = -(I(1) << (lL + D + 1)) - (I(x + y) << D);  // G(0, 0) = -2LK - K(x + y)
                const I dI = I(x) << D;                                    // 2x * K/2
                const uint32_t M = below_mask<I, 3>(G0, dI, lL + D + 1);   // dJ = 4L * K/2
                const uint32_t code = region_code3(M);
                const bool votes_root = code != 0u && code != 15u;
                if (!votes_root) atomicOr(&status->err, kErrInvariant);
                vals[0] = spread4(FHT ? fht_root_children(x, y, lL, D) : child_votes3(M));
                vals[1] = votes_root ? 1u : 0u;
                if (D >= 2) {
                    Voter vr;
                    vr.x = (int16_t)x;
                    vr.y = (int16_t)y;
                    vr.region = U.root_rec;
                    v0[U.v0_off + (k - img_start[img])] = vr;
                }
            }
            warp_segmented_total<2>(key, vals);
            if (run_head(key)) {
                const uint32_t rr = units[key].root_rec;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t c = (vals[0] >> (8 * q)) & 0xffu;
                    if (c) atomicAdd(&root_cnt[4 * (size_t)rr + q], c);
                }
                if (vals[1]) atomicAdd((unsigned long long*)&stats[((size_t)key * (kMaxDepth + 1) + 0) * 4 + 2],
                                       (unsigned long long)vals[1]);
            }
        }
    }
}

template <typename I, bool FHT = false>
__global__ void __launch_bounds__(256) stage_kernel(const int16_t* __restrict__ pts, uint64_t total,
                                                    const Unit* __restrict__ units, int n_images,
                                                    const uint64_t* __restrict__ img_start,
                                                    const uint32_t* __restrict__ img_unit, Voter* __restrict__ v0,
                                                    uint32_t* __restrict__ root_cnt, uint64_t* __restrict__ stats,
                                                    uint32_t* __restrict__ img_err, DeviceStatus* status,
                                                    const JobDims* __restrict__ dims) {
    stage_body<I, FHT>(pts, total, units, n_images, img_start, img_unit, v0, root_cnt, stats, img_err, status,
                       dims);
}

// ============================================================================ select
namespace {
constexpr int kSelTPB = 256;
constexpr int kSelPPT = 4;
constexpr int kSelTile = kSelTPB * kSelPPT;
}  // namespace

// Level totals once every block is done: leaf count, capacity checks.
__device__ __forceinline__ void select_totals(const LevelArgs& a) {
    volatile LevelInfo* info = a.info;
    volatile uint64_t* lt = a.leaf_total;
    const uint64_t q0 = info->n_voters;
    const uint64_t nl = info->n_leaves;
    const uint64_t total_leaves = *lt + nl;
    if (info->n_regions > a.cap_children || q0 > a.cap_voters || total_leaves > a.cap_leaves)
        atomicOr(&a.status->err, kErrOverflow);
    *lt = total_leaves;
    __threadfence();
}

// standalone: the last block to finish writes the totals; otherwise the
// caller does after a grid-wide barrier.
__device__ __forceinline__ void select_body(const LevelArgs& a, bool standalone) {
    __shared__ uint32_t s_slot;
    __shared__ uint32_t s_wrec[8], s_wleaf[8];
    __shared__ uint64_t s_wvox[8];
    __shared__ uint64_t s_prefix[3];
    __shared__ unsigned long long s_nrec, s_nleaf, s_nvox;

    const int s = a.level;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) { s_nrec = 0; s_nleaf = 0; s_nvox = 0; }
    const uint64_t np = a.info_prev->n_regions;
    const bool aborted = job_aborted(a.status);
    const uint32_t ntiles = aborted ? 0u : (uint32_t)((np + kSelTile - 1) / kSelTile);
    const uint32_t epoch = a.scan->epoch;
    const uint64_t leaf_base = *a.leaf_total;

    while (true) {
        const uint32_t t = claim_tile(a.scan, &s_slot);
        if (t >= ntiles) break;
        const uint64_t base = (uint64_t)t * kSelTile + (uint64_t)tid * kSelPPT;

        uint32_t cnt[kSelPPT][4];
        uint32_t pass[kSelPPT], wmask[kSelPPT], geo[kSelPPT];
        bool leafy[kSelPPT];
        // voters to copy are summed in 64 bits at every stage: a tile's
        // parents can hand their children more than 2^32 voters
        uint32_t my_rec = 0, my_leaf = 0;
        uint64_t my_vox = 0;
        // statistics run (records are sorted by unit)
        uint32_t run_unit = kNoRegion;
        int run_lev = 0;
        unsigned long long run_stat[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < kSelPPT; ++j) {
            const uint64_t p = base + j;
            pass[j] = 0; wmask[j] = 0; leafy[j] = false; geo[j] = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) cnt[j][q] = 0;
            if (p >= np) continue;
            const Region R = a.parents[p];
            const Unit U = a.units[R.unit];
            const int lev = s - U.t0;  // the children's level in this unit
            const uint4 c4 = reinterpret_cast<const uint4*>(a.parent_cnt)[p];
            cnt[j][0] = c4.x; cnt[j][1] = c4.y; cnt[j][2] = c4.z; cnt[j][3] = c4.w;
            uint32_t pm = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) pm |= (cnt[j][q] >= (uint32_t)U.T ? 1u : 0u) << q;
            // an image with a point outside it fails: its root passes nothing
            if (lev == 1 && a.img_err && a.img_err[R.unit >> 1]) pm = 0u;
            if (a.keep && lev == a.keep_level) {
                // subtrees that another shard runs: tested and counted, not split
                const uint64_t side = 1ull << lev;
                const uint64_t base = (uint64_t)(R.unit & 1u) * side * side;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint64_t ca = 2ull * R.a + ((q == NE || q == SE) ? 1u : 0u);
                    const uint64_t cb = 2ull * R.b + ((q == NE || q == NW) ? 1u : 0u);
                    if (!a.keep[base + ca * side + cb]) pm &= ~(1u << q);
                }
            }
            pass[j] = pm;
            leafy[j] = (lev == U.D);
            // voters of a level-lev child are read by the next pass only when
            // that pass still has a level below lev + 1 to count
            wmask[j] = (!leafy[j] && lev <= U.D - 2) ? pm : 0u;
            // geometry of this parent for the pass: side S = 2^(D - lev + 1) cells
            geo[j] = pack_region(0u, 0u, (uint32_t)(U.D - lev + 1), (uint32_t)U.lL, (uint32_t)U.D);
            const uint32_t np_c = __popc(pm);
            if (leafy[j]) my_leaf += np_c; else my_rec += np_c;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (wmask[j] & (1u << q)) my_vox += cnt[j][q];
            const unsigned long long votes = (unsigned long long)cnt[j][0] + cnt[j][1] + cnt[j][2] + cnt[j][3];
            if (R.unit != run_unit) {
                if (run_unit != kNoRegion) {
                    unsigned long long* st = (unsigned long long*)&a.stats[((size_t)run_unit * (kMaxDepth + 1) + run_lev) * 4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) if (run_stat[k]) atomicAdd(&st[k], run_stat[k]);
                }
                run_unit = R.unit;
                run_lev = lev;
                run_stat[0] = run_stat[1] = run_stat[2] = run_stat[3] = 0;
            }
            run_stat[0] += 4;                                  // regions tested
            run_stat[1] += np_c;                               // regions passed
            run_stat[2] += votes;                              // votes
            run_stat[3] += 4ull * (unsigned long long)R.count; // four codes per parent voter
        }
        // statistics: merge the per-thread tail runs across the warp
        {
            // a thread's run values are < 2^36 (at most 16 children of n <= 2^31 votes):
            // sum their low 16 bits and their bits 16..47 in separate 32-bit lanes
            uint32_t packed[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                packed[k] = (uint32_t)(run_stat[k] & 0xffffu);
                packed[4 + k] = (uint32_t)(run_stat[k] >> 16);
            }
            warp_segmented_total<8>(run_unit, packed);
            if (run_head(run_unit)) {
                unsigned long long* st = (unsigned long long*)&a.stats[((size_t)run_unit * (kMaxDepth + 1) + run_lev) * 4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const unsigned long long tot = (unsigned long long)packed[k] + ((unsigned long long)packed[4 + k] << 16);
                    if (tot) atomicAdd(&st[k], tot);
                }
            }
        }
        // scan of (records, leaves, copied voters) over the tile
        uint32_t inc_rec = my_rec, inc_leaf = my_leaf;
        uint64_t inc_vox = my_vox;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t r = __shfl_up_sync(0xffffffffu, inc_rec, off);
            const uint32_t l = __shfl_up_sync(0xffffffffu, inc_leaf, off);
            const uint64_t v = __shfl_up_sync(0xffffffffu, inc_vox, off);
            if (lane >= off) { inc_rec += r; inc_leaf += l; inc_vox += v; }
        }
        if (lane == 31) { s_wrec[warp] = inc_rec; s_wleaf[warp] = inc_leaf; s_wvox[warp] = inc_vox; }
        __syncthreads();
        if (warp == 0) {
            const uint32_t wr = lane < 8 ? s_wrec[lane] : 0u, wl = lane < 8 ? s_wleaf[lane] : 0u;
            const uint64_t wv = lane < 8 ? s_wvox[lane] : 0ull;
            uint32_t ir = wr, il = wl;
            uint64_t iv = wv;
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
                const uint32_t r = __shfl_up_sync(0xffffffffu, ir, off);
                const uint32_t l = __shfl_up_sync(0xffffffffu, il, off);
                const uint64_t v = __shfl_up_sync(0xffffffffu, iv, off);
                if (lane >= off) { ir += r; il += l; iv += v; }
            }
            const uint64_t agg[3] = {__shfl_sync(0xffffffffu, ir, 7), __shfl_sync(0xffffffffu, il, 7),
                                     __shfl_sync(0xffffffffu, iv, 7)};
            __syncwarp();
            if (lane < 8) { s_wrec[lane] = ir - wr; s_wleaf[lane] = il - wl; s_wvox[lane] = iv - wv; }
            uint64_t pre[3];
            tile_lookback<3>(a.tile_flags, a.tile_data, t, epoch, agg, pre, a.status, t + 1u != a.withhold_tile_plus1);
            if (lane == 0) {
                s_prefix[0] = pre[0];
                s_prefix[1] = pre[1];
                s_prefix[2] = pre[2];
                s_nrec += agg[0];
                s_nleaf += agg[1];
                s_nvox += agg[2];
            }
        }
        __syncthreads();
        uint64_t rec = s_prefix[0] + s_wrec[warp] + (inc_rec - my_rec);
        uint64_t leaf = leaf_base + s_prefix[1] + s_wleaf[warp] + (inc_leaf - my_leaf);
        uint64_t vox = s_prefix[2] + s_wvox[warp] + (inc_vox - my_vox);
#pragma unroll
        for (int j = 0; j < kSelPPT; ++j) {
            const uint64_t p = base + j;
            if (p >= np) continue;
            const Region R = a.parents[p];
            if (!leafy[j]) {
                // the pass record (a parent whose children are leaves has no
                // voters in the stream the pass reads, so it needs none)
                PassRegion pr;
                pr.a = R.a;
                pr.b = R.b;
                pr.child_base = (uint32_t)rec;
                pr.packed = geo[j] | pass[j] | (wmask[j] << 4);
                a.pregions[p] = pr;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!(pass[j] & (1u << q))) continue;
                const uint32_t east = (q == NE || q == SE) ? 1u : 0u;
                const uint32_t north = (q == NE || q == NW) ? 1u : 0u;
                const uint32_t ca = 2u * R.a + east, cb = 2u * R.b + north;
                if (leafy[j]) {
                    if (leaf < a.cap_leaves) {
                        DevLeaf lf;
                        lf.half = R.unit & 1u;  // units are numbered 2 * image (or request slot) + half
                        lf.i = ca; lf.j = cb; lf.votes = cnt[j][q];
                        a.leaves[leaf] = lf;
                    }
                    ++leaf;
                } else {
                    if (rec < a.cap_children) {
                        Region c;
                        c.unit = R.unit; c.a = ca; c.b = cb; c.count = cnt[j][q];
                        a.children[rec] = c;
                        reinterpret_cast<uint4*>(a.child_cnt)[rec] = make_uint4(0, 0, 0, 0);
                        // the child's voters fill [vox, vox + count) of the next
                        // stream (only a child whose list is written has a cursor)
                        if (wmask[j] & (1u << q)) a.cursor[rec] = vox;
                    }
                    if (wmask[j] & (1u << q)) vox += cnt[j][q];
                    ++rec;
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_nrec) atomicAdd((unsigned long long*)&a.info->n_regions, s_nrec);
        if (s_nleaf) atomicAdd((unsigned long long*)&a.info->n_leaves, s_nleaf);
        if (s_nvox) atomicAdd((unsigned long long*)&a.info->n_voters, s_nvox);
    }
    if (standalone && scan_finish(a.scan)) select_totals(a);
}

__global__ void __launch_bounds__(kSelTPB) select_kernel(LevelArgs a) { select_body(a, true); }

// ============================================================================ pass
namespace {

// Child record index of quadrant q of a parent (its passed children are
// stored consecutively in quadrant order).
__device__ __forceinline__ uint32_t child_index(const PassRegion& pr, int q) {
    return pr.child_base + __popc(pr.packed & 0xfu & ((1u << q) - 1u));
}

// Add the grandchild counts of one parent to the level-(s+1) counters of its
// passed children.  c16[2*alpha + (beta & 1)] holds the counts of cells
// (alpha, beta) and (alpha, beta + 2) in its low and high 16 bits, the same
// values in every lane.  The lanes add them in parallel: lane l < 16 adds the
// count of grandchild cell (alpha, beta) = (l >> 2, l & 3) of the parent whose
// passed children start at record child_base (pass mask in the low bits of
// `packed`), so one atomic instruction covers all sixteen cells.  Every lane
// must call this.
__device__ __forceinline__ void add_counts_lanes(uint32_t* __restrict__ cnt, uint32_t child_base, uint32_t packed,
                                                 const uint32_t (&c16)[8], uint64_t n_children, DeviceStatus* st) {
    const int lane = threadIdx.x & 31;
    const int al = (lane >> 2) & 3, be = lane & 3;
    const int sel = 2 * al + (be & 1);
    uint32_t w = c16[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) w = sel == k ? c16[k] : w;
    const uint32_t c = (be & 2) ? (w >> 16) : (w & 0xffffu);
    const int q = quad_of(al >> 1, be >> 1), g = quad_of(al & 1, be & 1);
    const uint32_t ci = child_base + __popc(packed & 0xfu & ((1u << q) - 1u));
    if (lane < 16 && c && HHT_CHECK_INDEX(ci, n_children, st)) atomicAdd(&cnt[4 * (size_t)ci + g], c);
}

// Per-lane byte counters rows[alpha] (byte beta) -> 16-bit pairs summed over
// the lanes of `mask` (every lane of the mask must call this).
__device__ __forceinline__ void reduce_rows(const uint32_t (&rows)[4], uint32_t mask, uint32_t (&c16)[8]) {
#pragma unroll
    for (int al = 0; al < 4; ++al) {
        c16[2 * al] = __reduce_add_sync(mask, rows[al] & 0x00ff00ffu);             // beta 0 and 2
        c16[2 * al + 1] = __reduce_add_sync(mask, (rows[al] >> 8) & 0x00ff00ffu);  // beta 1 and 3
    }
}

// Grandchild votes of a lane's voters of one chunk (up to four) added to its
// byte counters: row alpha of the 4 x 4 cells, byte beta.  Per cell the number
// of the voters that cross it is first formed as three bit planes (carry-save
// adds: ones, twos, fours) and then spread into the bytes once per chunk
// instead of once per voter (the spreading is most of the cost).
__device__ __forceinline__ void add_rows4(uint32_t (&rows)[4], uint32_t g0, uint32_t g1, uint32_t g2, uint32_t g3) {
    const uint32_t s01 = g0 ^ g1, c01 = g0 & g1, s23 = g2 ^ g3, c23 = g2 & g3;
    const uint32_t ones = s01 ^ s23, c_ = s01 & s23;
    const uint32_t twos = c01 ^ c23 ^ c_;
    const uint32_t fours = (c01 & c23) | (c_ & (c01 | c23));
#pragma unroll
    for (int al = 0; al < 4; ++al) {
        const int sh = kGrandBase + 5 * al;
        rows[al] += ((((ones >> sh) & 0xfu) * 0x204081u) & 0x01010101u) +
                    ((((twos >> sh) & 0xfu) * 0x408102u) & 0x02020202u) +
                    ((((fours >> sh) & 0xfu) * 0x810204u) & 0x04040404u);
    }
}

template <int S>
__device__ __forceinline__ void add_rows_chunk(uint32_t (&rows)[4], const uint32_t (&g)[S]) {
    static_assert(S >= 1 && S <= 4, "a chunk has one to four warp steps");
    add_rows4(rows, g[0], S > 1 ? g[S > 1 ? 1 : 0] : 0u, S > 2 ? g[S > 2 ? 2 : 0] : 0u, S > 3 ? g[S > 3 ? 3 : 0] : 0u);
}

// Constants of one parent region for the corner grid of its voters.  With
// u0 = dJ - 1 - G(SW vertex) = W0 - x*A + (x + y)*Kc and column step
// d = x*dmul, the number of below-the-line vertices in column alpha of the
// 5 x 5 quarter-step grid is t = clamp((u0 - alpha*d) >> k, 0, 5).
template <typename I>
struct ParentGeo {
    PassRegion pr;
    I W0, A, Kc, dmul;
    int k;
    uint32_t pspread, wspread;  // pass / write masks at the children's vote bits
    uint32_t gmask;             // grandchild cells of the passed children (kGrandBase layout)
    // int32 form on the packed point word xy = x + 2^16 y, in arithmetic mod
    // 2^32 (exact, because every true value fits in int32):
    // u0 = xy*cxy + W0 + y*cy and d = xy*dmul + y*d16
    uint32_t cxy, cy, d16;
    __device__ __forceinline__ void load(const PassRegion* p, uint32_t r) {
        pr = p[r];
        const int sS = (pr.packed >> 8) & 31, lL = (pr.packed >> 13) & 31, D = (pr.packed >> 18) & 31;
        k = lL + sS;                                                    // dJ = 4L * S/4 = 2^(lL + sS)
        const I Gr = (I(pr.b) << (sS + lL + 2)) - (I(1) << (lL + D + 1));  // 4L*bS - 2LK
        W0 = ((I(1) << k) - I(1)) - Gr;
        A = I(pr.a) << (sS + 1);                                        // 2*aS: G gains 2x*aS
        Kc = I(1) << D;                                                 // G loses K(x + y)
        dmul = I(1) << (sS - 1);                                        // 2x * S/4
        pspread = spread_quads(pr.packed & 0xfu);
        wspread = spread_quads((pr.packed >> 4) & 0xfu);
        gmask = grand_cells(pspread);
        cxy = (uint32_t)Kc - (uint32_t)A;
        cy = (uint32_t)Kc - 65536u * cxy;
        d16 = 0u - ((uint32_t)dmul << 16);
    }
};
}  // namespace

// One step of the level loop over the voter stream of the parents.  Every
// warp owns a contiguous slice of the stream and walks it in chunks of four
// steps of 32 voters (one coalesced 8-byte record per lane and step):
//   - the exact 5 x 5 corner-sign grid of the voter's parent gives the 4-bit
//     codes of the four children and of the sixteen grandchildren;
//   - a voter of a passed child whose list is kept is appended to that
//     child's segment of the next stream (segments were sized by the
//     selection; one atomic per child and chunk reserves the slots);
//   - grandchild votes of passed children are accumulated in per-lane byte
//     counters while the parent stays the same, then summed across the warp
//     (redux.sync) and added to the next level's counters.
// A chunk whose voters do not all share one parent goes step by step with
// per-parent lane groups.  Within a child's segment the voter order depends
// on scheduling; no result depends on it (counts, leaves and statistics are
// order-free).
namespace {

template <typename I>
struct Classified {
    uint32_t kw;  // children whose list keeps this voter, at the children's vote bits (quad_bit)
    uint32_t gv;  // grandchild cells of passed children the voter crosses, at kGrandBase + 5*alpha + beta
};

// Classify one voter against its parent: the exact 5 x 5 corner-sign grid,
// then the 4-bit codes of the four children and the sixteen grandchildren
// (vote when the code is neither 0000 nor 1111).
template <typename I>
__device__ __forceinline__ Classified<I> classify(const ParentGeo<I>& g, uint32_t xy, uint32_t live) {
    int t[5];
    if constexpr (sizeof(I) == 4) {
        // the integer (ALU) pipe limits this kernel: the point's coordinates
        // enter as multiply-adds on the packed word (y = xy >> 16 as a high
        // product), which run on the otherwise idle FMA pipe
        const uint32_t y = __umulhi(xy, 65536u);
        const int32_t u0 = (int32_t)(xy * g.cxy + (uint32_t)g.W0 + y * g.cy);
        const int32_t d = (int32_t)(xy * (uint32_t)g.dmul + y * g.d16);
#pragma unroll
        for (int alpha = 0; alpha < 5; ++alpha) t[alpha] = __vimin_s32_relu((u0 - alpha * d) >> g.k, 5);
    } else {
        const I x = I(xy & 0xffffu), y = I(xy >> 16);
        const I u0 = g.W0 - x * g.A + (x + y) * g.Kc;
        const I d = x * g.dmul;
#pragma unroll
        for (int alpha = 0; alpha < 5; ++alpha) {
            I tt = (u0 - I(alpha) * d) >> g.k;
            tt = tt < I(0) ? I(0) : (tt > I(5) ? I(5) : tt);
            t[alpha] = (int)tt;
        }
    }
    const uint32_t M = prefix_bits<0>(t[0]) | prefix_bits<5>(t[1]) | prefix_bits<10>(t[2]) |
                       prefix_bits<15>(t[3]) | prefix_bits<20>(t[4]);
    // G grows with i (x >= 0) and with j, so a cell's SW corner is its lowest
    // and its NE corner its highest: its code is neither 0000 nor 1111 exactly
    // when SW is below the line and NE is not.  Results at the NE vertex bit
    // (SW bit + 6 * side): children at quad_bit(q), grandchildren at
    // kGrandBase + 5*alpha + beta.
    const uint32_t v2 = (M << 12) & ~M;
    const uint32_t v1 = (M << 6) & ~M;
    Classified<I> c;
    c.kw = v2 & g.wspread & live;
    // a line that crosses a grandchild cell crosses its child, so the cells of
    // the passed children need no test of the child's own vote
    c.gv = v1 & g.gmask & live;
    return c;
}

// ---- the prior-art FHT circle test (Sections 1-3: the paper's comparison)
// A line votes for a region when its distance from the region's centre is at
// most the radius of the circle through the region's corners, distances in
// cell units (regions are squares).  In those units the line is G(i, j) = 0
// with |grad G| = 2 sqrt(x^2 + 4L^2), and a region of side s has radius
// s / sqrt(2), so the test is G(centre)^2 <= 2 s^2 (x^2 + 4L^2), decided
// exactly on integers.  Centres of the parent's 4 x 4 grandchildren (side
// S/4) are half-integer vertices, so 2 G is used:
//   2G(alpha, beta) = C0 + x*Cx - 2K*y + alpha * (x*S) + beta * 2LS,
//   C0 = 8L*bS + L*S - 4LK, Cx = 4*aS + S/2 - 2K,
// and a grandchild votes when (2G)^2 <= S^2 (x^2 + 4L^2) / 2.  A child's
// centre is the midpoint of the centres of its SW and NE grandchildren, so
// with h = the sum of those two 2G values it votes when
// h^2 <= 8 S^2 (x^2 + 4L^2).  A grandchild's circle lies inside its child's
// (centre offset and radius both half the child's radius), so, as for the
// exact test, every grandchild voter is a voter of its child.  int32 holds
// every 2G when lL + D <= 27 (|2G| <= 8LK at points of the parameter space);
// the squares and bounds are int64.
struct ParentGeoF {
    PassRegion pr;
    int32_t C0, Cx, dB, yK;  // yK = 2K
    int64_t L4;              // 4L^2
    int sS;
    uint32_t pspread, wspread;
    __device__ __forceinline__ void load(const PassRegion* p, uint32_t r) {
        pr = p[r];
        sS = (pr.packed >> 8) & 31;
        const int lL = (pr.packed >> 13) & 31, D = (pr.packed >> 18) & 31;
        const int64_t S = int64_t(1) << sS, K = int64_t(1) << D, L = int64_t(1) << lL;
        C0 = (int32_t)(8 * L * (int64_t)pr.b * S + L * S - 4 * L * K);
        Cx = (int32_t)(4 * (int64_t)pr.a * S + S / 2 - 2 * K);
        dB = (int32_t)(2 * L * S);
        yK = (int32_t)(2 * K);
        L4 = 4 * L * L;
        pspread = spread_quads(pr.packed & 0xfu);
        wspread = spread_quads((pr.packed >> 4) & 0xfu);
    }
};

template <typename I>
__device__ __forceinline__ Classified<I> classify(const ParentGeoF& g, uint32_t xy, uint32_t live) {
    const int32_t x = (int32_t)(xy & 0xffffu), y = (int32_t)(xy >> 16);
    const int32_t h00 = g.C0 + x * g.Cx - g.yK * y;
    const int32_t hx = x << g.sS;
    const int64_t X = (int64_t)x * x + g.L4;
    const int64_t rg = X << (2 * g.sS - 1);  // grandchildren: (2G)^2 <= S^2 X / 2
    const int64_t rc = X << (2 * g.sS + 3);  // children: h^2 <= 8 S^2 X
    int32_t h[4][4];
    uint32_t v1 = 0;
#pragma unroll
    for (int al = 0; al < 4; ++al) {
#pragma unroll
        for (int be = 0; be < 4; ++be) {
            h[al][be] = h00 + al * hx + be * g.dB;
            v1 |= ((int64_t)h[al][be] * h[al][be] <= rg ? 1u : 0u) << (kGrandBase + 5 * al + be);
        }
    }
    uint32_t v2 = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int e = (q == NE || q == SE) ? 1 : 0, n = (q == NE || q == NW) ? 1 : 0;
        const int64_t sum = (int64_t)h[2 * e][2 * n] + h[2 * e + 1][2 * n + 1];
        v2 |= (sum * sum <= rc ? 1u : 0u) << quad_bit(q);
    }
    Classified<I> c;
    c.kw = v2 & g.wspread & live;
    c.gv = v1 & grand_cells(v2 & g.pspread) & live;
    return c;
}
}  // namespace

// Pass-kernel work distribution: grabs of about 1/kGrabShare of a warp's
// even share of the stream, within [kMinGrab, kMaxGrab] records.
constexpr uint32_t kGrabShare = 4;
constexpr int kMinGrab = kPassMinGrab;
constexpr int kMaxGrab = 4096;

// Tile shape (autotuned): STEPS warp steps of 32 voters per chunk (one
// cursor reservation per child and chunk), TPB threads per block, at least
// MINB resident blocks per SM (register budget).
template <typename I, int STEPS, int TPB, bool FHT = false>
__device__ __forceinline__ void pass_body(const LevelArgs& a) {
    using Geo = typename std::conditional<FHT, ParentGeoF, ParentGeo<I>>::type;
    constexpr int kChunkSteps = STEPS;
    constexpr int kPassTPB = TPB;
    static_assert(32 * STEPS <= 255, "a chunk's per-quadrant counts are summed in byte fields");
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t nin = a.info_prev->n_voters;
    if (job_aborted(a.status)) return;
#ifdef HHT_CHECKED
    const uint64_t n_par = a.info_prev->n_regions, n_chi = a.info->n_regions;
#else
    const uint64_t n_chi = 0;  // only read by the checks of HHT_CHECKED builds
#endif
    // Work distribution: the stream is cut into grabs of G consecutive
    // records, G = a quarter of a warp's even share rounded to whole chunks
    // and kept within [kMinGrab, kMaxGrab].  Warp w takes grab w first and
    // then claims the next free grab from the level's counter (one atomic,
    // issued a grab ahead of its use).  All warps thus sweep the stream
    // together, which keeps the child segments being written (laid out in
    // parent order) in a narrow window of L2, and warps that meet many short
    // parents do not hold up the launch.
    constexpr int kChunk = 32 * kChunkSteps;
    static_assert(kMinGrab >= kChunk, "a grab holds whole chunks");
    const uint32_t nwarps = gridDim.x * (kPassTPB / 32);
    const uint32_t wid = blockIdx.x * (kPassTPB / 32) + (threadIdx.x >> 5);
    uint32_t G;
    {
        const int lg = 32 - __clz(kGrabShare * nwarps - 1);  // kGrabShare * nwarps <= 2^lg
        const uint64_t g = nin >> lg;
        G = g < (uint64_t)kMinGrab ? (uint32_t)kMinGrab : (g > (uint64_t)kMaxGrab ? (uint32_t)kMaxGrab : (uint32_t)g);
        G = G / kChunk * kChunk;
    }
    uint64_t c = (uint64_t)wid * G;  // start of this warp's first grab
    if (c >= nin) return;
    unsigned long long* const claim_ctr = &a.info_prev->pass_next;
    uint64_t claim_at = 0;  // lane 0: start of the warp's claimed next grab
    if (lane == 0) claim_at = (uint64_t)nwarps * G + atomicAdd(claim_ctr, (unsigned long long)G);
    const uint2* __restrict__ vin = reinterpret_cast<const uint2*>(a.vin);
    uint2* __restrict__ vout = reinterpret_cast<uint2*>(a.vout);

    // the run being counted: warp-uniform parent and per-lane byte counters
    uint32_t cur = kNoRegion;
    Geo cg;
    uint32_t ci[4] = {0u, 0u, 0u, 0u};  // child record index per quadrant of cur
    uint32_t rows[4] = {0u, 0u, 0u, 0u};
    uint32_t steps = 0;

    auto settle = [&]() {
        if (cur != kNoRegion) {
            uint32_t c16[8];
            reduce_rows(rows, 0xffffffffu, c16);
            add_counts_lanes(a.child_cnt, cg.pr.child_base, cg.pr.packed, c16, n_chi, a.status);
        }
        rows[0] = rows[1] = rows[2] = rows[3] = 0u;
        steps = 0;
    };
    auto start_run = [&](uint32_t r) {
        if (!HHT_CHECK_INDEX(r, n_par, a.status)) r = 0u;
        cur = r;
        cg.load(a.pregions, r);
#pragma unroll
        for (int q = 0; q < 4; ++q) ci[q] = child_index(cg.pr, q);
    };

    // The voters of one chunk that belong to the run's parent `cur`: every
    // record when `all` (a constant at each call), else those whose parent
    // is P.  They are classified against it, the kept ones appended to their
    // children's segments and the grandchild votes counted.
    auto run_chunk = [&](const uint2* rec, bool all, uint32_t P) {
        auto live = [&](int k) { return (all || rec[k].y == P) ? 0xffffffffu : 0u; };
        if (cg.wspread == 0u) {
            // no child keeps a list (the children's level is the unit's last
            // but one): the voters are only counted for the grandchildren
            uint32_t gc[kChunkSteps];
#pragma unroll
            for (int k = 0; k < kChunkSteps; ++k) gc[k] = classify<I>(cg, rec[k].x, live(k)).gv;
            add_rows_chunk<kChunkSteps>(rows, gc);
            steps += kChunkSteps;
            if (steps >= 255 - kChunkSteps) settle();  // byte counters nearly full
            return;
        }
        uint32_t kw[kChunkSteps], gv[kChunkSteps];
        uint32_t cnt = 0;
#pragma unroll
        for (int k = 0; k < kChunkSteps; ++k) {
            const Classified<I> cl = classify<I>(cg, rec[k].x, live(k));
            kw[k] = cl.kw;
            gv[k] = cl.gv;
            cnt += quad_counts(kw[k]);
        }
        // reserve each kept child's slots for the whole chunk (one atomic per
        // child): per-lane counts per quadrant as byte fields, one warp scan
        // for all four quadrants, then every lane writes its kept voters of a
        // quadrant to consecutive slots
        uint32_t inc = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, inc, off);
            if (lane >= off) inc += o;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, inc, 31);
        // lanes 0..3 reserve the slots of quadrant `lane` in parallel; the
        // grandchild counts are added while the reservations are in flight
        unsigned long long mybase = 0;
        const uint32_t tq_mine = lane < 4 ? (tot >> (8 * quad_byte_rt(lane))) & 0xffu : 0u;
        if (tq_mine) {
            const uint32_t cq = lane == 0 ? ci[0] : lane == 1 ? ci[1] : lane == 2 ? ci[2] : ci[3];
            if (HHT_CHECK_INDEX(cq, n_chi, a.status)) mybase = atomicAdd(&a.cursor[cq], (unsigned long long)tq_mine);
        }
        add_rows_chunk<kChunkSteps>(rows, gv);
        const bool over = tq_mine && mybase + tq_mine > a.cap_voters;
        const bool any_over = __any_sync(0xffffffffu, over);
        steps += kChunkSteps;
        if (steps >= 255 - kChunkSteps) settle();  // byte counters nearly full
        const uint32_t excl = inc - cnt;
        if (!any_over) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int sh = 8 * quad_byte(q);
                const uint32_t tq = (tot >> sh) & 0xffu;
                if (!tq) continue;
                uint2* dst = vout + __shfl_sync(0xffffffffu, mybase, q) + ((excl >> sh) & 0xffu);
                const uint32_t bit = 1u << quad_bit(q);
                uint32_t j = 0;
#pragma unroll
                for (int k = 0; k < kChunkSteps; ++k) {
                    const uint32_t keep = (kw[k] & bit) ? 1u : 0u;
                    st_pred_v2(dst + j, keep, rec[k].x, ci[q]);
                    j += keep;
                }
            }
        } else {
            // the stream overflows its capacity (the host reruns with more room)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int sh = 8 * quad_byte(q);
                const uint32_t tq = (tot >> sh) & 0xffu;
                if (!tq) continue;
                uint64_t p = __shfl_sync(0xffffffffu, mybase, q) + ((excl >> sh) & 0xffu);
                const uint32_t bit = 1u << quad_bit(q);
#pragma unroll
                for (int k = 0; k < kChunkSteps; ++k) {
                    if (kw[k] & bit) {
                        if (p < a.cap_voters) vout[p] = make_uint2(rec[k].x, ci[q]);
                        ++p;
                    }
                }
            }
        }
    };

    // chunks are loaded one ahead through a lane pointer with constant
    // offsets; `rem` counts the records of the loaded chunk's grab from the
    // chunk on (at most G; grabs hold whole chunks, so only the stream's last
    // chunk is partial)
    const uint2* pin = vin + c + lane;
    int rem = (int)(c + G < nin ? G : nin - c);
    uint2 nxt[kChunkSteps];
#pragma unroll
    for (int k = 0; k < kChunkSteps; ++k) nxt[k] = 32 * k + lane < rem ? pin[32 * k] : make_uint2(0u, kNoRegion);
    while (rem > 0) {
        uint2 rec[kChunkSteps];
#pragma unroll
        for (int k = 0; k < kChunkSteps; ++k) rec[k] = nxt[k];
        const bool full = rem >= kChunk;
        // the chunk after this one: the rest of this grab, else the claimed grab
        rem -= kChunk;
        pin += kChunk;
        if (rem <= 0) {
            c = __shfl_sync(0xffffffffu, claim_at, 0);
            rem = c < nin ? (int)(c + G < nin ? G : nin - c) : 0;
            pin = vin + c + lane;
            if (lane == 0 && rem > 0) claim_at = (uint64_t)nwarps * G + atomicAdd(claim_ctr, (unsigned long long)G);
        }
        if (rem >= kChunk) {
#pragma unroll
            for (int k = 0; k < kChunkSteps; ++k) nxt[k] = pin[32 * k];
        } else {
#pragma unroll
            for (int k = 0; k < kChunkSteps; ++k)
                nxt[k] = 32 * k + lane < rem ? pin[32 * k] : make_uint2(0u, kNoRegion);
        }
        const uint32_t r_first = __shfl_sync(0xffffffffu, rec[0].y, 0);
        const uint32_t r_last = __shfl_sync(0xffffffffu, rec[kChunkSteps - 1].y, 31);

        if (full && r_first == r_last && r_first != kNoRegion) {
            // ---- a whole chunk of one parent: the stream is grouped by parent,
            // so every record between the first and the last is the parent's
            // (records without a parent, of points outside their image, lie
            // only within their own image's level-0 run, whose root passes
            // nothing, so they count nowhere)
            if (r_first != cur) {
                settle();
                start_run(r_first);
            }
            run_chunk(rec, true, r_first);
            continue;
        }

        // ---- more than one parent in the chunk (a run ends inside it), the
        // stream's partial last chunk, or records without a parent: the same
        // body once per parent, a record taking part when its parent is the
        // run's.  Parent indices never decrease along the stream (segments
        // are laid out in region order; records without a parent carry the
        // largest value), so the runs are taken in order by a warp minimum
        // over the larger parents.
        uint32_t m = rec[0].y;
#pragma unroll
        for (int k = 1; k < kChunkSteps; ++k) m = min(m, rec[k].y);
        uint32_t P = __reduce_min_sync(0xffffffffu, m);
#pragma unroll 1
        while (P != kNoRegion) {
            if (P != cur) {
                settle();
                start_run(P);
            }
            run_chunk(rec, false, P);
            m = kNoRegion;
#pragma unroll
            for (int k = 0; k < kChunkSteps; ++k) m = min(m, rec[k].y > P ? rec[k].y : kNoRegion);
            P = __reduce_min_sync(0xffffffffu, m);
        }
    }
    settle();
}

template <typename I, int STEPS, int TPB, int MINB, bool FHT = false>
__global__ void __launch_bounds__(TPB, MINB) pass_kernel(LevelArgs a) {
    pass_body<I, STEPS, TPB, FHT>(a);
}


// ============================================================================ launchers
int occupancy_select() {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel, kSelTPB, 0);
    return per_sm < 1 ? 1 : per_sm;
}

int launch_stage(const int16_t* pts, uint64_t total_points, const Unit* units, int n_images,
                 const uint64_t* img_start, const uint32_t* img_unit, Voter* v0, uint32_t* root_cnt,
                 uint64_t* stats, uint32_t* img_err, DeviceStatus* status, bool int64_path, void* stream,
                 bool fht, const JobDims* dims, int grid) {
    if (total_points == 0 && !dims) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (grid <= 0) {
        const uint64_t want = (total_points + 255) / 256;
        grid = (int)(want < 4096 ? want : 4096);
    }
    if (fht) {
        if (int64_path) return -1;  // the circle test is built for int32 corner arithmetic only
        stage_kernel<int32_t, true><<<grid, 256, 0, st>>>(pts, total_points, units, n_images, img_start, img_unit,
                                                          v0, root_cnt, stats, img_err, status, dims);
    } else if (int64_path)
        stage_kernel<int64_t><<<grid, 256, 0, st>>>(pts, total_points, units, n_images, img_start, img_unit, v0,
                                                     root_cnt, stats, img_err, status, dims);
    else
        stage_kernel<int32_t><<<grid, 256, 0, st>>>(pts, total_points, units, n_images, img_start, img_unit, v0,
                                                     root_cnt, stats, img_err, status, dims);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_select(const LevelArgs& a, int tpb_unused, int grid, void* stream) {
    (void)tpb_unused;
    select_kernel<<<grid, kSelTPB, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ============================================================================ copy out
// Leaves to a caller's pinned host buffer, written by the SMs through its
// device mapping (over the CPU-GPU link) instead of by a copy engine.  16-byte
// words, four per thread and iteration, grid-stride.
__global__ void __launch_bounds__(256) copy16_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                     uint64_t n16) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; k + 3 * stride < n16; k += 4 * stride) {
        const uint4 a = src[k], b = src[k + stride], c = src[k + 2 * stride], d = src[k + 3 * stride];
        dst[k] = a;
        dst[k + stride] = b;
        dst[k + 2 * stride] = c;
        dst[k + 3 * stride] = d;
    }
    for (; k < n16; k += stride) dst[k] = src[k];
}

int launch_copy16(const void* src, void* dst, uint64_t n16, int grid, void* stream) {
    if (n16 == 0) return 0;
    copy16_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>((const uint4*)src, (uint4*)dst, n16);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Pass-kernel tile shapes: {steps per chunk, threads per block, min blocks per SM}.
struct PassShape {
    int steps, tpb, minb;
};
constexpr PassShape kPassShapes[kPassShapeCount] = {{4, 256, 3}, {4, 128, 6}, {3, 256, 4},
                                                    {4, 384, 2}, {4, 192, 4}, {3, 256, 3}};

namespace {
template <int S>
const void* pass_fn32() {
    constexpr PassShape p = kPassShapes[S];
    return (const void*)pass_kernel<int32_t, p.steps, p.tpb, p.minb>;
}
const void* pass_fn(bool int64_path, int shape, bool fht = false) {
    if (fht) return (const void*)pass_kernel<int32_t, 4, 256, 2, true>;
    if (int64_path) return (const void*)pass_kernel<int64_t, 4, 256, 3>;
    switch (shape) {
        case 1: return pass_fn32<1>();
        case 2: return pass_fn32<2>();
        case 3: return pass_fn32<3>();
        case 4: return pass_fn32<4>();
        case 5: return pass_fn32<5>();
        default: return pass_fn32<0>();
    }
}
}  // namespace

int pass_threads(bool int64_path, int shape) {
    return int64_path ? 256 : kPassShapes[(shape >= 0 && shape < kPassShapeCount) ? shape : 0].tpb;
}

int occupancy_pass(bool int64_path, int shape) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_fn(int64_path, shape), pass_threads(int64_path, shape),
                                                  0);
    return per_sm < 1 ? 1 : per_sm;
}

int launch_pass(const LevelArgs& a, bool int64_path, int grid, void* stream, int shape, bool fht) {
    if (fht && int64_path) return -1;
    void* args[] = {(void*)&a};
    const int tpb = fht ? 256 : pass_threads(int64_path, shape);
    const cudaError_t e = cudaLaunchKernel(pass_fn(int64_path, shape, fht), dim3(grid), dim3(tpb), args, 0,
                                           (cudaStream_t)stream);
    return e == cudaSuccess ? 0 : -1;
}

int occupancy_pass_fht() {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_fn(false, 0, true), 256, 0);
    return per_sm < 1 ? 1 : per_sm;
}

}  // namespace hht
