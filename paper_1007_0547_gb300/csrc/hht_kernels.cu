// Level kernels of the hierarchical Hough transform (sm_103a).
//
//   stage   level 0: range-check the points, write the level-0 voter streams of
//           both halves and count the votes of the four level-1 quadrants.
//   select  level s: a level-(s-1) region's child passes when its votes >= T
//           (Section 3, step 13).  Passed children become the level-s region
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
template <typename I>
__global__ void __launch_bounds__(256) stage_kernel(const int16_t* __restrict__ pts, uint64_t total,
                                                    const Unit* __restrict__ units, int n_images,
                                                    const uint64_t* __restrict__ img_start,
                                                    const uint32_t* __restrict__ img_unit, Voter* __restrict__ v0,
                                                    uint32_t* __restrict__ root_cnt, uint64_t* __restrict__ stats,
                                                    uint32_t* __restrict__ img_err, DeviceStatus* status) {
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
            if (!ok) atomicOr(&img_err[img], kErrRange);  // the image fails; the others are unaffected
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t u = active ? img_unit[img] + (uint32_t)h : 0u;
            uint32_t key = (active && ok) ? u : kNoRegion;
            uint32_t vals[2] = {0u, 0u};  // [0]: child votes as 4 bytes, [1]: level-0 votes
            if (active && ok) {
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
                vals[0] = spread4(child_votes3(M));
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

// ============================================================================ select
namespace {
constexpr int kSelTPB = 256;
constexpr int kSelPPT = 4;
constexpr int kSelTile = kSelTPB * kSelPPT;
}  // namespace

__global__ void __launch_bounds__(kSelTPB) select_kernel(LevelArgs a) {
    __shared__ uint32_t s_slot;
    __shared__ uint32_t s_wrec[8], s_wleaf[8];
    __shared__ uint64_t s_prefix[2];
    __shared__ unsigned long long s_kept[4];
    __shared__ unsigned long long s_nrec, s_nleaf;

    const int s = a.level;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 4) s_kept[tid] = 0;
    if (tid == 0) { s_nrec = 0; s_nleaf = 0; }
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
        uint32_t pass[kSelPPT], wmask[kSelPPT];
        bool leafy[kSelPPT];
        uint32_t my_rec = 0, my_leaf = 0;
        unsigned long long kept[4] = {0, 0, 0, 0};
        // statistics run (records are sorted by unit)
        uint32_t run_unit = kNoRegion;
        int run_lev = 0;
        unsigned long long run_stat[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < kSelPPT; ++j) {
            const uint64_t p = base + j;
            pass[j] = 0; wmask[j] = 0; leafy[j] = false;
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
            pass[j] = pm;
            leafy[j] = (lev == U.D);
            // voters of a level-lev child are read by the next pass only when
            // that pass still has a level below lev + 1 to count
            wmask[j] = (!leafy[j] && lev <= U.D - 2) ? pm : 0u;
            const uint32_t np_c = __popc(pm);
            if (leafy[j]) my_leaf += np_c; else my_rec += np_c;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (wmask[j] & (1u << q)) kept[q] += cnt[j][q];
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
        // block-wide kept totals
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (kept[q]) atomicAdd(&s_kept[q], kept[q]);

        // scan of (records, leaves) over the tile
        uint32_t inc_rec = my_rec, inc_leaf = my_leaf;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t r = __shfl_up_sync(0xffffffffu, inc_rec, off);
            const uint32_t l = __shfl_up_sync(0xffffffffu, inc_leaf, off);
            if (lane >= off) { inc_rec += r; inc_leaf += l; }
        }
        if (lane == 31) { s_wrec[warp] = inc_rec; s_wleaf[warp] = inc_leaf; }
        __syncthreads();
        if (warp == 0) {
            uint32_t wr = lane < 8 ? s_wrec[lane] : 0u, wl = lane < 8 ? s_wleaf[lane] : 0u;
            uint32_t ir = wr, il = wl;
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
                const uint32_t r = __shfl_up_sync(0xffffffffu, ir, off);
                const uint32_t l = __shfl_up_sync(0xffffffffu, il, off);
                if (lane >= off) { ir += r; il += l; }
            }
            const uint64_t agg[2] = {__shfl_sync(0xffffffffu, ir, 7), __shfl_sync(0xffffffffu, il, 7)};
            if (lane < 8) { s_wrec[lane] = ir - wr; s_wleaf[lane] = il - wl; }
            uint64_t pre[2];
            tile_lookback<2>(a.tile_flags, a.tile_data, t, epoch, agg, pre, a.status);
            if (lane == 0) {
                s_prefix[0] = pre[0];
                s_prefix[1] = pre[1];
                s_nrec += agg[0];
                s_nleaf += agg[1];
            }
        }
        __syncthreads();
        uint64_t rec = s_prefix[0] + s_wrec[warp] + (inc_rec - my_rec);
        uint64_t leaf = leaf_base + s_prefix[1] + s_wleaf[warp] + (inc_leaf - my_leaf);
#pragma unroll
        for (int j = 0; j < kSelPPT; ++j) {
            const uint64_t p = base + j;
            if (p >= np) continue;
            const Region R = a.parents[p];
            RegionLink lk;
            lk.child_base = (uint32_t)rec;
            lk.pass_mask = leafy[j] ? 0 : (uint8_t)pass[j];
            lk.write_mask = (uint8_t)wmask[j];
            lk.pad = 0;
            a.links[p] = lk;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!(pass[j] & (1u << q))) continue;
                const uint32_t east = (q == NE || q == SE) ? 1u : 0u;
                const uint32_t north = (q == NE || q == NW) ? 1u : 0u;
                const uint32_t ca = 2u * R.a + east, cb = 2u * R.b + north;
                if (leafy[j]) {
                    if (leaf < a.cap_leaves) {
                        DevLeaf lf;
                        lf.unit = R.unit; lf.i = ca; lf.j = cb; lf.votes = cnt[j][q];
                        a.leaves[leaf] = lf;
                    }
                    ++leaf;
                } else {
                    if (rec < a.cap_children) {
                        Region c;
                        c.unit = R.unit; c.a = ca; c.b = cb; c.count = cnt[j][q];
                        a.children[rec] = c;
                        reinterpret_cast<uint4*>(a.child_cnt)[rec] = make_uint4(0, 0, 0, 0);
                    }
                    ++rec;
                }
            }
        }
    }
    __syncthreads();
    if (tid < 4 && s_kept[tid]) atomicAdd((unsigned long long*)&a.info->kept[tid], s_kept[tid]);
    if (tid == 0) {
        if (s_nrec) atomicAdd((unsigned long long*)&a.info->n_regions, s_nrec);
        if (s_nleaf) atomicAdd((unsigned long long*)&a.info->n_leaves, s_nleaf);
    }
    if (scan_finish(a.scan)) {
        volatile LevelInfo* info = a.info;
        uint64_t q0 = 0;
        for (int q = 0; q < 4; ++q) {
            info->Q[q] = q0;
            q0 += info->kept[q];
        }
        info->n_voters = q0;
        const uint64_t nl = info->n_leaves;
        const uint64_t total_leaves = leaf_base + nl;
        if (info->n_regions > a.cap_children || q0 > a.cap_voters || total_leaves > a.cap_leaves)
            atomicOr(&a.status->err, kErrOverflow);
        *a.leaf_total = total_leaves;
        __threadfence();
    }
}

// ============================================================================ pass
namespace {
constexpr int kPassTPB = 256;
constexpr int kPassVPT = 8;
constexpr int kPassTile = kPassTPB * kPassVPT;

// Add a run's grandchild counts (byte counters acc[alpha] >> 8*beta) to the
// level-(s+1) counters of the parent's passed children.
__device__ __forceinline__ void flush_rows(uint32_t* __restrict__ cnt, const RegionLink lk, const uint32_t (&acc)[4]) {
#pragma unroll
    for (int al = 0; al < 4; ++al) {
        if (!acc[al]) continue;
#pragma unroll
        for (int be = 0; be < 4; ++be) {
            const uint32_t c = (acc[al] >> (8 * be)) & 0xffu;
            if (!c) continue;
            const int q = quad_of(al >> 1, be >> 1), g = quad_of(al & 1, be & 1);
            const uint32_t child = lk.child_base + __popc((uint32_t)lk.pass_mask & ((1u << q) - 1u));
            atomicAdd(&cnt[4 * (size_t)child + g], c);
        }
    }
}
}  // namespace

template <typename I>
__global__ void __launch_bounds__(kPassTPB) pass_kernel(LevelArgs a) {
    __shared__ uint32_t s_slot;
    __shared__ uint32_t s_wlo[8], s_whi[8];
    __shared__ uint64_t s_prefix[4];

    const int s = a.level;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t nin = a.info_prev->n_voters;
    const bool aborted = job_aborted(a.status);
    const uint32_t ntiles = aborted ? 0u : (uint32_t)((nin + kPassTile - 1) / kPassTile);
    const uint32_t epoch = a.scan->epoch;
    uint64_t Q[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) Q[q] = a.info->Q[q];

    while (true) {
        const uint32_t t = claim_tile(a.scan, &s_slot);
        if (t >= ntiles) break;
        const uint64_t base = (uint64_t)t * kPassTile + (uint64_t)tid * kPassVPT;

        Voter v[kPassVPT];
        if (base + kPassVPT <= nin) {
            const uint4* src = reinterpret_cast<const uint4*>(a.vin + base);
#pragma unroll
            for (int k = 0; k < kPassVPT / 2; ++k) {
                const uint4 w = src[k];
                v[2 * k].x = (int16_t)(w.x & 0xffffu); v[2 * k].y = (int16_t)(w.x >> 16); v[2 * k].region = w.y;
                v[2 * k + 1].x = (int16_t)(w.z & 0xffffu); v[2 * k + 1].y = (int16_t)(w.z >> 16); v[2 * k + 1].region = w.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kPassVPT; ++j) {
                if (base + j < nin) v[j] = a.vin[base + j];
                else { v[j].x = 0; v[j].y = 0; v[j].region = kNoRegion; }
            }
        }

        // ---- codes, grandchild counts (run-length by region), copy masks
        uint32_t cur = kNoRegion;
        RegionLink lk{};
        I Gr = 0;
        uint32_t ra = 0;
        int sh_xa = 0, D = 0, sh_dI = 0, k_dJ = 0;
        uint32_t acc[4] = {0u, 0u, 0u, 0u};
        uint32_t kw_all = 0, tsum = 0;
#pragma unroll
        for (int j = 0; j < kPassVPT; ++j) {
            const uint32_t r = v[j].region;
            if (r == kNoRegion) continue;
            if (r != cur) {
                if (cur != kNoRegion) {
                    flush_rows(a.child_cnt, lk, acc);
                    acc[0] = acc[1] = acc[2] = acc[3] = 0u;
                }
                cur = r;
                const Region R = a.parents[r];
                lk = a.links[r];
                const Unit U = a.units[R.unit];
                D = U.D;
                const int lL = U.lL;
                const int sS = D - (s - U.t0) + 1;  // parent region side S = 2^sS cells
                // G at the parent's SW vertex (aS, bS): 4L*bS + 2x*aS - 2LK - K(x+y)
                Gr = (I(R.b) << (sS + lL + 2)) - (I(1) << (lL + D + 1));
                ra = R.a;
                sh_xa = sS + 1;
                sh_dI = sS - 1;   // quarter step h = S/4: 2x*h = x << (sS - 1)
                k_dJ = lL + sS;   // 4L*h = 2^(lL + sS)
            }
            const int32_t x = v[j].x, y = v[j].y;
            const I G0 = Gr + (I(x) * I(ra) << sh_xa) - (I(x + y) << D);
            const uint32_t M = below_mask<I, 5>(G0, I(x) << sh_dI, k_dJ);
            const uint32_t cv = child_votes5(M);
            const uint32_t kc = cv & lk.pass_mask;
            const uint32_t kw = cv & lk.write_mask;
            const uint32_t gv = crossing_cells<5, 1>(M) & grandchild_mask(kc);
#pragma unroll
            for (int al = 0; al < 4; ++al) acc[al] += spread4((gv >> (5 * al)) & 0xfu);
            kw_all |= kw << (4 * j);
            tsum += spread4(kw);
        }
        // tail run: merge equal regions across the warp, first lane adds
        {
            uint32_t w[8];
#pragma unroll
            for (int al = 0; al < 4; ++al) {
                w[2 * al] = acc[al] & 0x00ff00ffu;             // beta 0 and 2
                w[2 * al + 1] = (acc[al] >> 8) & 0x00ff00ffu;  // beta 1 and 3
            }
            warp_segmented_total<8>(cur, w);
            if (run_head(cur)) {
                const RegionLink hl = a.links[cur];
                // 16-bit sums per (alpha, beta): a warp total may exceed 255
#pragma unroll
                for (int al = 0; al < 4; ++al) {
#pragma unroll
                    for (int be = 0; be < 4; ++be) {
                        const uint32_t word = w[2 * al + (be & 1)];
                        const uint32_t c = (be >> 1) ? (word >> 16) : (word & 0xffffu);
                        if (!c) continue;
                        const int q = quad_of(al >> 1, be >> 1), g = quad_of(al & 1, be & 1);
                        const uint32_t child = hl.child_base + __popc((uint32_t)hl.pass_mask & ((1u << q) - 1u));
                        atomicAdd(&a.child_cnt[4 * (size_t)child + g], c);
                    }
                }
            }
        }

        // ---- stable copy: scan of per-quadrant copy counts over the tile
        uint32_t lo = (tsum & 0xffu) | ((tsum & 0xff00u) << 8);          // quadrants 0, 1
        uint32_t hi = ((tsum >> 16) & 0xffu) | ((tsum >> 8) & 0xff0000u); // quadrants 2, 3
        const uint32_t own_lo = lo, own_hi = hi;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t l2 = __shfl_up_sync(0xffffffffu, lo, off);
            const uint32_t h2 = __shfl_up_sync(0xffffffffu, hi, off);
            if (lane >= off) { lo += l2; hi += h2; }
        }
        if (lane == 31) { s_wlo[warp] = lo; s_whi[warp] = hi; }
        __syncthreads();
        if (warp == 0) {
            const uint32_t wl = lane < 8 ? s_wlo[lane] : 0u, wh = lane < 8 ? s_whi[lane] : 0u;
            uint32_t il = wl, ih = wh;
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
                const uint32_t l2 = __shfl_up_sync(0xffffffffu, il, off);
                const uint32_t h2 = __shfl_up_sync(0xffffffffu, ih, off);
                if (lane >= off) { il += l2; ih += h2; }
            }
            const uint32_t tl = __shfl_sync(0xffffffffu, il, 7), th = __shfl_sync(0xffffffffu, ih, 7);
            if (lane < 8) { s_wlo[lane] = il - wl; s_whi[lane] = ih - wh; }
            const uint64_t agg[4] = {tl & 0xffffu, tl >> 16, th & 0xffffu, th >> 16};
            uint64_t pre[4];
            tile_lookback<4>(a.tile_flags, a.tile_data, t, epoch, agg, pre, a.status);
            if (lane < 4) s_prefix[lane] = pre[lane == 0 ? 0 : lane == 1 ? 1 : lane == 2 ? 2 : 3];
        }
        __syncthreads();
        if (kw_all) {
            const uint32_t el = lo - own_lo + s_wlo[warp], eh = hi - own_hi + s_whi[warp];
            uint64_t pos[4] = {Q[0] + s_prefix[0] + (el & 0xffffu), Q[1] + s_prefix[1] + (el >> 16),
                               Q[2] + s_prefix[2] + (eh & 0xffffu), Q[3] + s_prefix[3] + (eh >> 16)};
            uint32_t lr = kNoRegion;
            RegionLink ll{};
#pragma unroll
            for (int j = 0; j < kPassVPT; ++j) {
                const uint32_t kw = (kw_all >> (4 * j)) & 0xfu;
                if (!kw) continue;
                if (v[j].region != lr) { lr = v[j].region; ll = a.links[lr]; }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!(kw & (1u << q))) continue;
                    const uint64_t p = pos[q]++;
                    if (p < a.cap_voters) {
                        Voter o;
                        o.x = v[j].x; o.y = v[j].y;
                        o.region = ll.child_base + __popc((uint32_t)ll.pass_mask & ((1u << q) - 1u));
                        a.vout[p] = o;
                    }
                }
            }
        }
    }
    scan_finish(a.scan);
}

// ============================================================================ output fix-up
__global__ void unit_to_half_kernel(DevLeaf* __restrict__ l, uint64_t n) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
        l[k].unit &= 1u;
}

int launch_unit_to_half(void* leaves, uint64_t n, void* stream) {
    if (n == 0) return 0;
    const uint64_t want = (n + 255) / 256;
    unit_to_half_kernel<<<(int)(want < 2048 ? want : 2048), 256, 0, (cudaStream_t)stream>>>((DevLeaf*)leaves, n);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ============================================================================ launchers
namespace {
int grid_for(const void* fn, int tpb, int num_sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tpb, 0) != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * num_sms;
}
}  // namespace

int occupancy_select() {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_kernel, kSelTPB, 0);
    return per_sm < 1 ? 1 : per_sm;
}

int occupancy_pass(bool int64_path) {
    int per_sm = 0;
    if (int64_path)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_kernel<int64_t>, kPassTPB, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_kernel<int32_t>, kPassTPB, 0);
    return per_sm < 1 ? 1 : per_sm;
}

int launch_stage(const int16_t* pts, uint64_t total_points, const Unit* units, int n_images,
                 const uint64_t* img_start, const uint32_t* img_unit, Voter* v0, uint32_t* root_cnt,
                 uint64_t* stats, uint32_t* img_err, DeviceStatus* status, bool int64_path, void* stream) {
    if (total_points == 0) return 0;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t want = (total_points + 255) / 256;
    const int grid = (int)(want < 4096 ? want : 4096);
    if (int64_path)
        stage_kernel<int64_t><<<grid, 256, 0, st>>>(pts, total_points, units, n_images, img_start, img_unit, v0,
                                                     root_cnt, stats, img_err, status);
    else
        stage_kernel<int32_t><<<grid, 256, 0, st>>>(pts, total_points, units, n_images, img_start, img_unit, v0,
                                                     root_cnt, stats, img_err, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_select(const LevelArgs& a, int tpb_unused, int grid, void* stream) {
    (void)tpb_unused;
    select_kernel<<<grid, kSelTPB, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_pass(const LevelArgs& a, bool int64_path, int grid, void* stream) {
    if (int64_path)
        pass_kernel<int64_t><<<grid, kPassTPB, 0, (cudaStream_t)stream>>>(a);
    else
        pass_kernel<int32_t><<<grid, kPassTPB, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace hht
