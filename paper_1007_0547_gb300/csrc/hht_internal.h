// Internal layouts shared by the kernels (hht_kernels.cu, hht_sort.cu) and the
// host orchestration (hht_api.cu).  Nothing here is part of the public ABI.
//
// Geometry (the paper's Sections 2-3, on a dyadic grid).  A unit is one half
// (0 = points as given, 1 = x/y swapped) of one image.  With L = 2^lL the
// smallest power of two >= max(W, H) and K = 2^D the number of leaf cells per
// side, grid vertex (i, j) is the parameter point m_i = -1 + 2i/K,
// b_j = -2L + 4Lj/K.  For edge point (x, y) of the unit,
//     G(i, j) = K * (b_j + x*m_i - y) = 4L*j + 2x*i - 2LK - K*x - K*y
// is K times F = y0 - m*x0 - b of Section 2 evaluated at that vertex for the
// parameter-space line of slope -x and intercept y; a vertex is "below" the
// line exactly when G < 0.  A region at level l is the square of side
// S = K >> l cells with lower-left vertex (a*S, b*S), (a, b) in [0, 2^l)^2.
#pragma once

#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace hht {

constexpr int kMaxDepth = 24;

// The region records of one level are addressed by 32-bit indices (a voter
// record's parent word; 0xffffffff marks no region), so a level holds at most
// this many.  The host refuses a level whose parents could give more children
// (4 per parent) with HHT_E_NOMEM, which splits a batch into smaller waves.
constexpr uint64_t kMaxLevelRecords = 0xfffffffeull;

// The pass kernel cuts its voter stream into grabs of at least this many
// records (one warp's unit of work; one chunk of 4 x 32), so a level's stream
// of v records can keep at most ceil(v / kPassMinGrab) warps busy.  Large
// streams get larger grabs (a quarter of a warp's share, up to 4096); the
// minimum matters for small streams, whose latency it sets (1024 made each
// warp of a 128^2 image's passes walk eight chunks in a row: 0.297 against
// 0.222 ms per image).
constexpr int kPassMinGrab = 128;

// Quadrant order of the paper's quad1..quad4.
enum Quad : int { NE = 0, NW = 1, SW = 2, SE = 3 };

// One (image, half) of a job.  Units advance one level per step of the level
// loop; a unit that joined at step t0 is at level (step - t0), so requests can
// join a running loop (continuous batching) without changing the kernels.
struct alignas(16) Unit {
    int32_t lL;        // log2 of the frame side L
    int32_t D;         // depth (leaf level)
    int32_t T;         // threshold: a region passes when votes >= T
    int32_t image;     // caller's image index
    int64_t n;         // points of the image
    uint64_t v0_off;   // offset of this unit's level-0 voters in the stream of step t0 (if D >= 2)
    int32_t W, H;      // image size (range check)
    int32_t half;      // 0: (x, y); 1: (y, x)
    int32_t t0;        // loop step at which the unit's level 0 is current
    uint32_t root_rec; // record index of the unit's level-0 region at step t0
    uint32_t inactive; // 1: this half takes none of the image's points (front-end split images)
    uint64_t pad2;
};
static_assert(sizeof(Unit) == 64, "unit record is 64 bytes");

// Voter record: the (half-swapped) point and the index of the region whose
// voter list it belongs to.  Two records form one 16-byte vector load.
struct alignas(8) Voter {
    int16_t x, y;
    uint32_t region;
};
static_assert(sizeof(Voter) == 8, "voter record is 8 bytes");

// A region that passed (level-0 regions always do).
struct alignas(16) Region {
    uint32_t unit;
    uint32_t a, b;     // cell indices at the region's level
    uint32_t count;    // votes = length of its voter list
};
static_assert(sizeof(Region) == 16, "region record is 16 bytes");

// Everything the pass kernel needs about a parent region, in one 16-byte
// record written by the selection of the next level: the parent's cell, its
// geometry and where its passed children are.
struct alignas(16) PassRegion {
    uint32_t a, b;        // parent cell indices at its level
    uint32_t child_base;  // record index of its first passed child at the next level
    uint32_t packed;      // see pack_region()
};
static_assert(sizeof(PassRegion) == 16, "pass region record is 16 bytes");

// packed: bits 0-3 pass mask (child q reached T and is a region of the next
// level), 4-7 write mask (child q's voters are copied to the next stream),
// 8-12 log2 of the parent side S in cells, 13-17 lL, 18-22 depth D.
__host__ __device__ inline uint32_t pack_region(uint32_t pass, uint32_t write, uint32_t sS, uint32_t lL, uint32_t D) {
    return pass | (write << 4) | (sS << 8) | (lL << 13) | (D << 18);
}

// Leaf as produced on the device (the layout of hht_leaf): half, cell, votes.
struct alignas(16) DevLeaf {
    uint32_t half, i, j, votes;
};

// Per-level totals written by the selection kernel's last block.
struct LevelInfo {
    uint64_t n_regions;      // passed regions of this level (records)
    uint64_t n_voters;       // length of this level's voter stream
    uint64_t n_leaves;       // leaves emitted at this level
    unsigned long long pass_next;  // voters of this level's stream claimed by the pass reading it (starts at 0)
    uint64_t pad[11];
};

// State of one single-pass (decoupled look-back) scan: tile ids are claimed in
// order with an atomic counter, and tile flags carry an epoch that the last
// block of each launch advances, so no memset is needed between launches.
struct ScanState {
    uint32_t tile_counter;
    uint32_t done_counter;
    uint32_t epoch;
    uint32_t pad;
};

// Status bits set on the device (checked by the host after a job).
enum : uint32_t {
    kErrRange = 1u,        // a point outside the image
    kErrTimeout = 2u,      // a bounded wait expired
    kErrOverflow = 4u,     // a capacity was exceeded (host re-runs with more memory)
    kErrInvariant = 8u,    // a line did not cross the level-0 region (cannot happen)
    kErrBounds = 16u       // HHT_CHECKED builds: an index read from the data was out of range
};

// HHT_CHECKED builds check every index that a kernel takes from its data
// (parent and child record indices) against the current sizes; a bad index
// sets kErrBounds and the access is skipped.  Normal builds compile the check
// away.
#ifdef HHT_CHECKED
#define HHT_CHECK_INDEX(i, n, st) (((uint64_t)(i) < (uint64_t)(n)) ? true : (atomicOr(&(st)->err, kErrBounds), false))
#else
#define HHT_CHECK_INDEX(i, n, st) true
#endif

struct DeviceStatus {
    uint32_t err;
    uint32_t pad[3];
};

// Launch parameters of one step of the level loop (host -> kernels).  For
// a unit that joined at step t0, the parents are its level (step - t0 - 1)
// regions and the children its level (step - t0) regions.
struct LevelArgs {
    const Unit* units;
    const Region* parents;     // records of level s-1
    PassRegion* pregions;      // pass records of level s-1 (written by select, read by pass)
    const uint32_t* parent_cnt;// [n_parents][4] vote counters of level-s children
    Region* children;          // records of level s (written by select)
    uint32_t* child_cnt;       // [n_children][4] counters of level s+1 (zeroed by select, filled by pass)
    unsigned long long* cursor;// [n_children] next free slot of each child's voter segment
    const Voter* vin;          // voter stream of level s-1
    Voter* vout;               // voter stream of level s
    DevLeaf* leaves;
    uint64_t* stats;           // [n_units][kMaxDepth + 1][4]
    LevelInfo* info_prev;      // level s-1
    LevelInfo* info;           // level s
    uint64_t* leaf_total;      // running leaf count
    ScanState* scan;
    uint32_t* tile_flags;
    uint64_t* tile_data;       // per tile: aggregate[C], inclusive[C]
    DeviceStatus* status;
    uint64_t cap_children, cap_voters, cap_leaves, cap_tiles;
    int32_t level;             // step of the level loop
    int32_t num_sms;
    uint32_t withhold_tile_plus1;  // fault injection: 1 + the selection tile that publishes nothing (0 = none)
    // subtree sharding: a region (a, b) of level keep_level passes only when
    // keep[half * 4^k + a * 2^k + b] != 0 (NULL = every region may pass)
    const uint8_t* keep;
    int32_t keep_level;
    // range flags per unit pair (unit / 2), written by the stage kernel: the
    // root of an image with a point outside it passes no children, so the
    // dead records of those points in the level-0 stream vote for nothing
    // (NULL = no flags)
    const uint32_t* img_err;
};

// Sizes of a job that the stage kernel reads from device memory when it is
// launched from a CUDA graph replayed for many jobs (the graph's arguments
// stay fixed; the host writes these before each launch).
struct alignas(16) JobDims {
    uint64_t total_points;  // points of all images
    int32_t n_images;
    int32_t pad;
};

// Kernel launchers (hht_kernels.cu).  All are asynchronous on `stream`.
// Level 0 of the images [0, n_images) of `pts` (image g owns points
// [img_start[g], img_start[g+1]) and the units img_unit[g], img_unit[g] + 1;
// a point outside its image sets kErrRange in img_err[img_unit[g] / 2]).
// With `dims` the kernel reads total_points and n_images from device memory
// instead, and `grid` (> 0) fixes the grid (for a CUDA graph reused across jobs).
int launch_stage(const int16_t* pts, uint64_t total_points, const Unit* units, int n_images,
                 const uint64_t* img_start, const uint32_t* img_unit, Voter* vstream, uint32_t* cnt,
                 uint64_t* stats, uint32_t* img_err, DeviceStatus* status, bool int64_path, void* stream,
                 bool fht = false, const JobDims* dims = nullptr, int grid = 0);
int launch_select(const LevelArgs& a, int threads_per_block, int grid, void* stream);
// Copy n16 16-byte words from device memory to `dst` (device memory, or the
// device mapping of pinned host memory).
int launch_copy16(const void* src, void* dst, uint64_t n16, int grid, void* stream);
// Pass-kernel tile shapes for the autotuner; shape 0 is the default.
constexpr int kPassShapeCount = 6;
// fht: the prior-art circumscribed-circle test instead of the 4-bit code
// (int32 corner arithmetic and tile shape 0 only).
int launch_pass(const LevelArgs& a, bool int64_path, int grid, void* stream, int shape = 0, bool fht = false);
int occupancy_pass_fht();
int pass_threads(bool int64_path, int shape = 0);
int occupancy_select();
int occupancy_pass(bool int64_path, int shape = 0);

// Rewrite each leaf's unit (2 * image + half) to its half.


}  // namespace hht
