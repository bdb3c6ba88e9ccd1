// Front end of the hierarchical Hough transform (Section 3): Sobel's gradient
// operator on a grey-level image and the split of the edge points into ALPHA
// (lines of absolute slope <= 1) and BETA (the rest), then detection with
// ALPHA as half 0 and BETA as half 1.
//
// Readings where the paper is silent:
//   - only interior pixels (1 <= x <= W-2, 1 <= y <= H-2) have a full 3 x 3
//     neighbourhood; border pixels are never edge points;
//   - a pixel is an edge point when gx^2 + gy^2 >= threshold^2;
//   - the line through an edge point runs across its gradient (slope
//     -gx / gy), so it is an ALPHA point when |gx| <= |gy|.
// Points come out in row-major order (y, then x) in each list.
//
// One kernel pass: tiles of 8192 consecutive pixels (row-major), claimed in
// order; a tile stages its pixels and the rows above and below into shared
// memory (three 8194-byte segments, coalesced word loads), each warp walks
// its 1024 pixels in steps of 32 (one pixel per lane), and a single-pass
// decoupled look-back scan of the two counts gives every tile its offsets in
// the two lists; only steps with edge pixels are visited to write them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/hht.h"
#include "hht_ctx.h"
#include "hht_device.cuh"
#include "hht_internal.h"
#include "hht_trace.h"

int hht_internal_run_job_halves(hht_ctx* c, const hht_image* im, int count, hht_result* outs, const uint8_t* halves);

namespace hht {
namespace {

constexpr int kEdgeTPB = 256;
constexpr int kEdgeWarps = kEdgeTPB / 32;
constexpr int kEdgeSteps = 32;                       // warp steps of 32 pixels per warp and tile
constexpr int kEdgeTile = kEdgeTPB * kEdgeSteps;     // pixels per tile (row-major, consecutive)
constexpr int kEdgeSeg = kEdgeTile + 2;              // a row segment with one halo pixel on each side
constexpr int kEdgeSegWords = (kEdgeSeg + 3 + 3) / 4;  // 4-byte words covering a segment at any byte shift

// Byte q of the image, 0 outside [0, npix).
__device__ __forceinline__ uint32_t pixel_or_zero(const uint8_t* __restrict__ img, int64_t q, int64_t npix) {
    return (q >= 0 && q < npix) ? (uint32_t)__ldg(img + q) : 0u;
}

// Warp w of a tile owns its pixels [w * 1024, (w + 1) * 1024): step s covers
// 32 consecutive pixels, one per lane, so the lanes read consecutive bytes of
// shared memory (no bank conflicts).  A step's edge pixels come out of two
// ballots; lane s keeps step s's masks, so one warp scan orders the steps.
__global__ void __launch_bounds__(kEdgeTPB) edges_kernel(const uint8_t* __restrict__ img, int32_t W, int32_t H,
                                                         int32_t thr2, uint32_t* __restrict__ out_a,
                                                         uint32_t* __restrict__ out_b, uint64_t cap,
                                                         unsigned long long* __restrict__ tot, ScanState* scan,
                                                         uint32_t* flags, uint64_t* data, DeviceStatus* status,
                                                         uint32_t ntiles) {
    // segw[r] holds the image bytes from (p0 + (r - 1) * W - 1) rounded down
    // to a 4-byte boundary; byte k of segment r is segb[r][shift[r] + k]
    __shared__ uint32_t segw[3][kEdgeSegWords];
    __shared__ uint32_t s_slot;
    __shared__ uint32_t s_wa[kEdgeWarps], s_wb[kEdgeWarps];
    __shared__ uint64_t s_pre[2];
    __shared__ unsigned long long s_na, s_nb;
    const uint8_t(*segb)[kEdgeSegWords * 4] = reinterpret_cast<const uint8_t(*)[kEdgeSegWords * 4]>(segw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t npix = (int64_t)W * H;
    const bool aligned = ((uintptr_t)img & 3u) == 0u;
    if (tid == 0) {
        s_na = 0;
        s_nb = 0;
    }
    const uint32_t epoch = scan->epoch;
    while (true) {
        const uint32_t t = claim_tile(scan, &s_slot);
        if (t >= ntiles) break;
        const int64_t p0 = (int64_t)t * kEdgeTile;
        int shift[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int64_t g0 = p0 + (int64_t)(r - 1) * W - 1;
            const int64_t ga = g0 >= 0 ? (g0 & ~int64_t(3)) : -((-g0 + 3) & ~int64_t(3));
            shift[r] = (int)(g0 - ga);
            for (int m = tid; m < kEdgeSegWords; m += kEdgeTPB) {
                const int64_t q = ga + 4 * (int64_t)m;
                uint32_t w;
                if (aligned && q >= 0 && q + 4 <= npix) {
                    w = __ldg(reinterpret_cast<const uint32_t*>(img + q));
                } else {
                    w = pixel_or_zero(img, q, npix) | (pixel_or_zero(img, q + 1, npix) << 8) |
                        (pixel_or_zero(img, q + 2, npix) << 16) | (pixel_or_zero(img, q + 3, npix) << 24);
                }
                segw[r][m] = w;
            }
        }
        __syncthreads();

        // classify: pixel i = base + 32 s + lane of the tile; its neighbours
        // at linear positions i - 1 and i + 1 are its left and right pixels
        // whenever it is an interior pixel
        const int base = warp * (32 * kEdgeSteps);
        const int64_t qw = p0 + base + lane;  // this lane's pixel at step 0
        int32_t y = (int32_t)(qw / W), x = (int32_t)(qw - (int64_t)y * W);
        const int32_t step_y = 32 / W, step_x = 32 - step_y * W;  // (x, y) advance of 32 pixels
        uint32_t my_a = 0, my_b = 0;  // lane s: step s's ALPHA and BETA masks
#pragma unroll 4
        for (int s = 0; s < kEdgeSteps; ++s) {
            const int i = base + 32 * s + lane;
            const int32_t a0 = segb[0][shift[0] + i], a1 = segb[0][shift[0] + i + 1], a2 = segb[0][shift[0] + i + 2];
            const int32_t m0 = segb[1][shift[1] + i], m2 = segb[1][shift[1] + i + 2];
            const int32_t b0 = segb[2][shift[2] + i], b1 = segb[2][shift[2] + i + 1], b2 = segb[2][shift[2] + i + 2];
            const int32_t gx = (a2 + 2 * m2 + b2) - (a0 + 2 * m0 + b0);
            const int32_t gy = (b0 + 2 * b1 + b2) - (a0 + 2 * a1 + a2);
            const bool inside = qw + 32 * s < npix && x >= 1 && x <= W - 2 && y >= 1 && y <= H - 2;
            const bool edge = inside && gx * gx + gy * gy >= thr2;
            const bool alpha = edge && abs(gx) <= abs(gy);
            const uint32_t ma = __ballot_sync(0xffffffffu, alpha);
            const uint32_t mb = __ballot_sync(0xffffffffu, edge && !alpha);
            if (lane == s) {
                my_a = ma;
                my_b = mb;
            }
            x += step_x;
            y += step_y;
            if (x >= W) {
                x -= W;
                ++y;
            }
        }

        // offsets: scan of the steps within the warp, block scan, then the look-back
        const uint32_t ca = __popc(my_a), cb = __popc(my_b);
        uint32_t ia = ca, ib = cb;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t ua = __shfl_up_sync(0xffffffffu, ia, off), ub = __shfl_up_sync(0xffffffffu, ib, off);
            if (lane >= off) {
                ia += ua;
                ib += ub;
            }
        }
        if (lane == 31) {
            s_wa[warp] = ia;
            s_wb[warp] = ib;
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t wa = lane < kEdgeWarps ? s_wa[lane] : 0u, wb = lane < kEdgeWarps ? s_wb[lane] : 0u;
            uint32_t ja = wa, jb = wb;
#pragma unroll
            for (int off = 1; off < kEdgeWarps; off <<= 1) {
                const uint32_t ua = __shfl_up_sync(0xffffffffu, ja, off), ub = __shfl_up_sync(0xffffffffu, jb, off);
                if (lane >= off) {
                    ja += ua;
                    jb += ub;
                }
            }
            const uint64_t agg[2] = {__shfl_sync(0xffffffffu, ja, kEdgeWarps - 1),
                                     __shfl_sync(0xffffffffu, jb, kEdgeWarps - 1)};
            __syncwarp();
            if (lane < kEdgeWarps) {
                s_wa[lane] = ja - wa;
                s_wb[lane] = jb - wb;
            }
            uint64_t pre[2];
            tile_lookback<2>(flags, data, t, epoch, agg, pre, status);
            if (lane == 0) {
                s_pre[0] = pre[0];
                s_pre[1] = pre[1];
                s_na += agg[0];
                s_nb += agg[1];
            }
        }
        __syncthreads();
        // write: step s's edge pixels follow the earlier steps' (exclusive scan
        // ia - ca), lanes in order within the step
        const uint64_t oa0 = s_pre[0] + s_wa[warp], ob0 = s_pre[1] + s_wb[warp];
        uint32_t steps_with_edges = __ballot_sync(0xffffffffu, (my_a | my_b) != 0u);
        while (steps_with_edges) {
            const int s = __ffs(steps_with_edges) - 1;
            steps_with_edges &= steps_with_edges - 1u;
            const uint32_t ma = __shfl_sync(0xffffffffu, my_a, s), mb = __shfl_sync(0xffffffffu, my_b, s);
            const uint32_t ea = __shfl_sync(0xffffffffu, ia - ca, s), eb = __shfl_sync(0xffffffffu, ib - cb, s);
            const bool wa = (ma >> lane) & 1u, wb = (mb >> lane) & 1u;
            if (wa || wb) {
                const int64_t q = p0 + base + 32 * s + lane;
                const int32_t yy = (int32_t)(q / W), xx = (int32_t)(q - (int64_t)yy * W);
                const uint32_t pt = ((uint32_t)xx & 0xffffu) | ((uint32_t)yy << 16);  // hht_point {x, y}
                if (wa) {
                    const uint64_t o = oa0 + ea + __popc(ma & lt);
                    if (o < cap) out_a[o] = pt;
                } else {
                    const uint64_t o = ob0 + eb + __popc(mb & lt);
                    if (o < cap) out_b[o] = pt;
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_na) atomicAdd(&tot[0], s_na);
        if (s_nb) atomicAdd(&tot[1], s_nb);
    }
    scan_finish(scan);
}

int edges_occupancy() {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, edges_kernel, kEdgeTPB, 0);
    return per_sm < 1 ? 1 : per_sm;
}

#define CKE(call)                                  \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)
#define RKE(call)                    \
    do {                             \
        int r_ = (call);             \
        if (r_ != HHT_OK) return r_; \
    } while (0)

bool args_ok(const uint8_t* image, int32_t W, int32_t H, int32_t threshold) {
    return image && W >= 1 && H >= 1 && W <= HHT_MAX_SIDE && H <= HHT_MAX_SIDE && threshold >= 0;
}

// Sobel + split of one image into c->edge_pts[0] (ALPHA) and [1] (BETA);
// *na and *nb receive the counts.  The image is host or device memory.
int run_edges(hht_ctx* c, const uint8_t* image, int32_t W, int32_t H, int32_t threshold, uint64_t* na,
              uint64_t* nb) {
    TraceRange tr("front end");
    cudaStream_t st = c->stream;
    const uint64_t npix = (uint64_t)W * (uint64_t)H;
    const uint8_t* d_img = image;
    cudaPointerAttributes at{};
    const bool on_device = cudaPointerGetAttributes(&at, image) == cudaSuccess &&
                           (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (!on_device) {
        RKE(ensure(c, c->img_buf, npix));
        CKE(cudaMemcpyAsync(c->img_buf.p, image, npix, cudaMemcpyDefault, st));
        d_img = (const uint8_t*)c->img_buf.p;
    }
    const uint64_t interior = (W >= 3 && H >= 3) ? (uint64_t)(W - 2) * (uint64_t)(H - 2) : 0;
    for (int k = 0; k < 2; ++k) RKE(ensure(c, c->edge_pts[k], std::max<uint64_t>(interior, 1) * sizeof(hht_point)));
    RKE(ensure(c, c->edge_tot, 2 * sizeof(unsigned long long)));
    RKE(ensure(c, c->status, sizeof(DeviceStatus)));
    const uint64_t ntiles = (npix + kEdgeTile - 1) / kEdgeTile;
    if ((ntiles + 1) * 4 > c->sel_flags.bytes) RKE(ensure(c, c->sel_flags, (ntiles + 1) * 4, true));
    RKE(ensure(c, c->sel_data, (ntiles + 1) * 2 * 2 * sizeof(uint64_t)));
    CKE(cudaMemsetAsync(c->edge_tot.p, 0, 2 * sizeof(unsigned long long), st));
    CKE(cudaMemsetAsync(c->status.p, 0, sizeof(DeviceStatus), st));
    const int grid = (int)std::min<uint64_t>(ntiles, (uint64_t)c->num_sms * edges_occupancy());
    // no Sobel response exceeds 2 * 1020^2 in gx^2 + gy^2, so larger thresholds clamp
    const int32_t thr2 = (int32_t)std::min<int64_t>((int64_t)threshold * threshold, int64_t(1) << 24);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (c->profile) {  // device time of the launch, resolved with the context's other timings
        for (cudaEvent_t* e : {&ev0, &ev1}) {
            if (!c->ev_pool.empty()) {
                *e = c->ev_pool.back();
                c->ev_pool.pop_back();
            } else {
                cudaEventCreate(e);
            }
        }
        cudaEventRecord(ev0, st);
    }
    edges_kernel<<<std::max(grid, 1), kEdgeTPB, 0, st>>>(
        d_img, W, H, thr2, (uint32_t*)c->edge_pts[0].p, (uint32_t*)c->edge_pts[1].p, std::max<uint64_t>(interior, 1),
        (unsigned long long*)c->edge_tot.p, (ScanState*)c->scan_states.p, (uint32_t*)c->sel_flags.p,
        (uint64_t*)c->sel_data.p, (DeviceStatus*)c->status.p, (uint32_t)ntiles);
    CKE(cudaGetLastError());
    if (c->profile) {
        cudaEventRecord(ev1, st);
        c->pending.push_back({ev0, ev1, 3});
    }
    c->prof.launches += 1;
    c->prof.edges_launches += 1;
    c->prof.edges_pixels += npix;
    unsigned long long tot[2] = {0, 0};
    DeviceStatus hs{};
    CKE(cudaMemcpyAsync(tot, c->edge_tot.p, sizeof tot, cudaMemcpyDeviceToHost, st));
    CKE(cudaMemcpyAsync(&hs, c->status.p, sizeof hs, cudaMemcpyDeviceToHost, st));
    CKE(cudaStreamSynchronize(st));
    if (hs.err & kErrTimeout) return HHT_E_TIMEOUT;
    *na = tot[0];
    *nb = tot[1];
    c->prof.edges_points += tot[0] + tot[1];
    return HHT_OK;
}

}  // namespace
}  // namespace hht

using namespace hht;

extern "C" {

int hht_edges(hht_ctx* c, const uint8_t* image, int32_t W, int32_t H, int32_t threshold, hht_point* alpha,
              uint64_t alpha_capacity, uint64_t* n_alpha, hht_point* beta, uint64_t beta_capacity, uint64_t* n_beta) {
    if (!c || !n_alpha || !n_beta || !args_ok(image, W, H, threshold)) return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    cudaSetDevice(c->device);
    uint64_t na = 0, nb = 0;
    RKE(run_edges(c, image, W, H, threshold, &na, &nb));
    *n_alpha = na;
    *n_beta = nb;
    if (na > alpha_capacity || nb > beta_capacity) return HHT_E_CAPACITY;
    if ((na > 0 && !alpha) || (nb > 0 && !beta)) return HHT_E_ARG;
    if (na > 0) RKE(copy_out(c, alpha, c->edge_pts[0].p, na * sizeof(hht_point)));
    if (nb > 0) RKE(copy_out(c, beta, c->edge_pts[1].p, nb * sizeof(hht_point)));
    CKE(cudaStreamSynchronize(c->stream));
    return HHT_OK;
}

int hht_detect_image(hht_ctx* c, const uint8_t* image, int32_t W, int32_t H, int32_t threshold, int32_t depth,
                     int32_t T, hht_result* out) {
    if (!c || !out || !args_ok(image, W, H, threshold) || depth < 1 || depth > HHT_MAX_DEPTH || T < 1)
        return HHT_E_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->predicate == HHT_PREDICATE_FHT && ceil_log2_i(std::max(W, H)) + depth > 27) return HHT_E_ARG;
    cudaSetDevice(c->device);
    uint64_t na = 0, nb = 0;
    RKE(run_edges(c, image, W, H, threshold, &na, &nb));
    // ALPHA as an image whose points enter half 0 only, BETA half 1 only
    hht_image ims[2] = {{(const hht_point*)c->edge_pts[0].p, (int64_t)na, W, H, depth, T},
                        {(const hht_point*)c->edge_pts[1].p, (int64_t)nb, W, H, depth, T}};
    hht_result outs[2];
    std::memset(outs, 0, sizeof outs);
    const uint8_t halves[2] = {1u, 2u};
    int rc = hht_internal_run_job_halves(c, ims, 2, outs, halves);
    if (rc == HHT_E_CAPACITY) rc = HHT_OK;  // the leaves stay in the context; copied below
    if (rc != HHT_OK) return rc;
    for (int k = 0; k < 2; ++k)
        if (outs[k].status != HHT_OK && outs[k].status != HHT_E_CAPACITY) return outs[k].status;
    out->depth = depth;
    out->L = 1 << ceil_log2_i(std::max(W, H));
    std::memset(out->stats, 0, sizeof out->stats);
    for (int l = 0; l <= depth; ++l) {
        out->stats[0][l] = outs[0].stats[0][l];
        out->stats[1][l] = outs[1].stats[1][l];
    }
    const uint64_t n = outs[0].n_leaves + outs[1].n_leaves;
    out->n_leaves = n;
    // both images have the same depth, so ALPHA's leaves are followed directly
    // by BETA's in the context's leaf store: one block, fetched as image 0
    if (c->job_off.size() != 2 || c->job_off[1] != c->job_off[0] + outs[0].n_leaves) return HHT_E_CUDA;
    const uint64_t off = c->job_off[0];
    c->job_off.assign(1, off);
    c->job_n.assign(1, n);
    if (n > out->leaf_capacity || (n > 0 && !out->leaves)) {
        out->status = HHT_E_CAPACITY;
        return HHT_E_CAPACITY;
    }
    if (n > 0) RKE(copy_out(c, out->leaves, (const char*)c->leaves.p + off * sizeof(hht_leaf), n * sizeof(hht_leaf)));
    CKE(cudaStreamSynchronize(c->stream));
    out->status = HHT_OK;
    return HHT_OK;
}

}  // extern "C"
