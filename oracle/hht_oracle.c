/*
 * CPU oracle for the hierarchical Hough transform of Singh & Bhatia,
 * "A Fast Decision Technique for Hierarchical Hough Transform for Line
 * Detection" (arXiv:1007.0547).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product library never calls it and shares no code with it.
 *
 * What it computes (Section 3):
 *   - Every edge point (x, y) is the parameter-space line b = y - m*x.  Points
 *     are processed in two halves: ALPHA as given and BETA with x and y
 *     swapped (Section 3, first paragraph).  Here every point enters both
 *     halves; the Sobel-gradient split is not part of this path.
 *   - The parameter space m in [-1, 1], b in [-2L, 2L] (L = smallest power of
 *     two >= max(W, H)) is the level-0 region.  A region is split into four
 *     quadrants NE, NW, SW, SE (quad1..quad4, Section 3).
 *   - A line gets a 4-bit code per region: one bit per corner in the order
 *     NE, NW, SW, SE (NE is the leftmost bit); a bit is 1 when the corner is
 *     below the line, i.e. F = y0 - m*x0 - b < 0 for the corner (x0, y0) and
 *     the line's slope m and intercept b (Section 2, getcode() in Section 3).
 *   - A line votes for a region when its code is neither 0000 nor 1111
 *     (Section 3).
 *   - A region whose votes reach the threshold T is split further, down to
 *     level `depth`, where it is reported as a peak cell (Section 3).
 *
 * Readings where the paper is silent or ambiguous:
 *   - The grid is dyadic: at depth D there are K = 2^D cells per side, with
 *     m_i = -1 + 2i/K and b_j = -2L + 4Lj/K.  All arithmetic is done on
 *     K * F, which is an exact integer (int64 here; int128 for the squared
 *     circle test).
 *   - Threshold: a region passes when votes >= T (the paper's algorithm
 *     compares the votes strictly with its threshold, which is the same rule
 *     with T one larger).
 *   - The level-0 region is always split (the paper's algorithm subdivides it
 *     without a threshold test).
 *   - The solution() removal of plotted voters is not applied, so the result
 *     is independent of traversal order.
 *   - The shortcut that skips children from the parent's code is not
 *     applied: every child code is computed, which cannot change any result.
 *
 * The traversal visits regions in the paper's depth-first order (NE, NW, SW,
 * SE) with one voter list per level instead of one code array per level: a
 * point is tested for a child only when it voted for the parent, the same
 * condition under which the paper's algorithm computes a child's code.
 * Leaves are reported in the order this traversal reaches them (half 0
 * first), which is the order in which solution() would be called.
 *
 * The FHT mode replaces the code test by the circumscribed-circle test of the
 * prior-art Fast Hough Transform that the paper compares with (Sections 1-2):
 * a line votes when its distance from the region centre is at most the radius
 * of the circle through the region's corners.  Distances are measured in cell
 * units, where regions are squares, and decided exactly with int128.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_E_ARG (-1)
#define ORACLE_E_RANGE (-2)
#define ORACLE_E_INVARIANT (-3)
#define ORACLE_E_CAPACITY (-4)
#define ORACLE_E_NOMEM (-5)

#define ORACLE_MODE_EXACT 0
#define ORACLE_MODE_FHT 1

typedef struct {
    uint32_t half, i, j, votes;
} oracle_leaf;

typedef struct {
    uint32_t half, level, i0, j0, size, votes;
} oracle_region;

/* Side L of the square image frame: smallest power of two >= max(W, H). */
int64_t oracle_frame_side(int32_t W, int32_t H)
{
    int64_t m = W > H ? W : H, L = 1;
    while (L < m) L <<= 1;
    return L;
}

/*
 * K * F for edge point (x, y) at grid corner (i, j) of a depth-D grid.
 * The parameter-space line of the point has slope -x and intercept y; the
 * corner is the parameter point (m_i, b_j).  F = b_j - (-x) * m_i - y
 * (Section 2), multiplied by K so that it is an integer.
 */
int64_t oracle_scaled_F(int32_t x, int32_t y, int64_t i, int64_t j, int64_t L, int32_t D)
{
    const int64_t K = (int64_t)1 << D;
    const int64_t K_b = -2 * L * K + 4 * L * j; /* K * b_j */
    const int64_t K_m = -K + 2 * i;             /* K * m_i */
    const int64_t slope = -(int64_t)x, intercept = y;
    return K_b - slope * K_m - K * intercept;
}

/* getcode() of Section 3 for region (i0, j0) of side S cells. */
uint32_t oracle_getcode(int32_t x, int32_t y, int64_t i0, int64_t j0, int64_t S, int64_t L, int32_t D)
{
    uint32_t code = 0;
    if (oracle_scaled_F(x, y, i0 + S, j0 + S, L, D) < 0) code |= 8u; /* bit 1: NorthEast */
    if (oracle_scaled_F(x, y, i0, j0 + S, L, D) < 0) code |= 4u;     /* bit 2: NorthWest */
    if (oracle_scaled_F(x, y, i0, j0, L, D) < 0) code |= 2u;         /* bit 3: SouthWest */
    if (oracle_scaled_F(x, y, i0 + S, j0, L, D) < 0) code |= 1u;     /* bit 4: SouthEast */
    return code;
}

/*
 * Circumscribed-circle test of the FHT for region (i0, j0, S).
 * In cell units the line is G(i, j) = K*F = 4L*j + 2x*i - 2LK - Kx - Ky = 0;
 * its distance from the centre c = (i0 + S/2, j0 + S/2) is |G(c)| / |(2x, 4L)|
 * and the circle radius is S / sqrt(2).  G(c) is an integer, so the test
 * G(c)^2 <= 2 S^2 (x^2 + 4 L^2) is exact in int128.
 */
int oracle_fht_votes(int32_t x, int32_t y, int64_t i0, int64_t j0, int64_t S, int64_t L, int32_t D)
{
    const int64_t K = (int64_t)1 << D;
    const __int128 Gc = (__int128)(2 * L) * (2 * j0 + S - K) + (__int128)x * (2 * i0 + S - K) - (__int128)K * y;
    const __int128 lhs = Gc * Gc;
    const __int128 rhs = (__int128)2 * S * S * ((__int128)x * x + (__int128)4 * L * L);
    return lhs <= rhs;
}

typedef struct {
    const int32_t *px, *py; /* current half's coordinates */
    int64_t L;
    int32_t D, T, mode, half;
    uint32_t **lists;       /* lists[l]: voter ids of the region being visited at level l */
    uint64_t *stats;        /* [2][D+1][4]: tested, passed, votes, tests */
    oracle_leaf *leaves;
    int64_t leaf_cap, n_leaves;
    oracle_region *regions;
    int64_t region_cap, n_regions;
    const uint8_t *keep;    /* subtree split: keep[half * 4^k + a * 2^k + b] for regions (a, b) of level k */
    int32_t keep_level;     /* k (used when keep is not NULL) */
} walk_t;

static uint64_t *stat_at(walk_t *w, int level, int k)
{
    return &w->stats[((int64_t)w->half * (w->D + 1) + level) * 4 + k];
}

static int line_votes(const walk_t *w, uint32_t v, int64_t i0, int64_t j0, int64_t S)
{
    if (w->mode == ORACLE_MODE_FHT) return oracle_fht_votes(w->px[v], w->py[v], i0, j0, S, w->L, w->D);
    const uint32_t code = oracle_getcode(w->px[v], w->py[v], i0, j0, S, w->L, w->D);
    return code != 0u && code != 15u;
}

static void record_region(walk_t *w, int level, int64_t i0, int64_t j0, int64_t S, int64_t votes)
{
    if (w->regions && w->n_regions < w->region_cap) {
        oracle_region *r = &w->regions[w->n_regions];
        r->half = (uint32_t)w->half; r->level = (uint32_t)level;
        r->i0 = (uint32_t)i0; r->j0 = (uint32_t)j0; r->size = (uint32_t)S; r->votes = (uint32_t)votes;
    }
    w->n_regions++;
}

/* Split a region of level `level` that reached the threshold (or is the root). */
static void subdivide(walk_t *w, int level, int64_t i0, int64_t j0, int64_t S, const uint32_t *V, int64_t nV)
{
    const int64_t h = S / 2;
    /* quad1..quad4 = NE, NW, SW, SE: lower-left corners of the children. */
    const int64_t ci[4] = {i0 + h, i0, i0, i0 + h};
    const int64_t cj[4] = {j0 + h, j0 + h, j0, j0};
    const int child = level + 1;
    uint32_t *buf = w->lists[child];

    *stat_at(w, child, 3) += 4 * (uint64_t)nV; /* four child codes per voter */
    for (int q = 0; q < 4; ++q) {
        int64_t cnt = 0;
        for (int64_t k = 0; k < nV; ++k)
            if (line_votes(w, V[k], ci[q], cj[q], h)) buf[cnt++] = V[k];
        *stat_at(w, child, 0) += 1;
        *stat_at(w, child, 2) += (uint64_t)cnt;
        record_region(w, child, ci[q], cj[q], h, cnt);
        int kept = 1;
        if (w->keep && child == w->keep_level) {
            /* a subtree that another shard runs: tested and counted here, not split */
            const int64_t side = (int64_t)1 << child;
            kept = w->keep[(int64_t)w->half * side * side + (ci[q] / h) * side + cj[q] / h] != 0;
        }
        if (kept && cnt >= w->T) {
            *stat_at(w, child, 1) += 1;
            if (child == w->D) {
                if (w->n_leaves < w->leaf_cap) {
                    oracle_leaf *lf = &w->leaves[w->n_leaves];
                    lf->half = (uint32_t)w->half; lf->i = (uint32_t)ci[q]; lf->j = (uint32_t)cj[q];
                    lf->votes = (uint32_t)cnt;
                }
                w->n_leaves++;
            } else {
                subdivide(w, child, ci[q], cj[q], h, buf, cnt);
            }
        }
    }
}

/*
 * Run the hierarchy on n points (xy[2k] = x, xy[2k+1] = y) of a W x H image.
 *   stats: caller array of 2 * (depth + 1) * 4 uint64, per half and level:
 *          {regions tested, regions passed, votes, code evaluations}.
 *   leaves: caller array of leaf_cap entries; *n_leaves receives the count
 *          (also when it exceeds leaf_cap, which returns ORACLE_E_CAPACITY).
 *   regions: optional (may be NULL) dump of every tested region.
 * Leaves are in depth-first order (children NE, NW, SW, SE), half 0 first.
 */
static int detect_walk(const int16_t *xy, int64_t n, int32_t W, int32_t H, int32_t depth, int32_t T, int32_t mode,
                       oracle_leaf *leaves, int64_t leaf_cap, int64_t *n_leaves, uint64_t *stats,
                       oracle_region *regions, int64_t region_cap, int64_t *n_regions, const uint8_t *keep,
                       int32_t keep_level)
{
    if (n < 0 || W < 1 || H < 1 || W > 32767 || H > 32767 || depth < 1 || depth > 24 || T < 1 || !n_leaves ||
        !stats || (n > 0 && !xy) || (leaf_cap > 0 && !leaves) || (mode != ORACLE_MODE_EXACT && mode != ORACLE_MODE_FHT))
        return ORACLE_E_ARG;
    for (int64_t k = 0; k < n; ++k)
        if (xy[2 * k] < 0 || xy[2 * k] >= W || xy[2 * k + 1] < 0 || xy[2 * k + 1] >= H) return ORACLE_E_RANGE;

    walk_t w;
    memset(&w, 0, sizeof w);
    w.L = oracle_frame_side(W, H);
    w.D = depth; w.T = T; w.mode = mode;
    w.stats = stats; w.leaves = leaves; w.leaf_cap = leaf_cap;
    w.regions = regions; w.region_cap = regions ? region_cap : 0;
    w.keep = keep; w.keep_level = keep_level;
    memset(stats, 0, sizeof(uint64_t) * 2 * (size_t)(depth + 1) * 4);

    int rc = ORACLE_OK;
    const size_t cap = (size_t)(n > 0 ? n : 1);
    int32_t *px = (int32_t *)malloc(cap * sizeof(int32_t));
    int32_t *py = (int32_t *)malloc(cap * sizeof(int32_t));
    uint32_t *pool = (uint32_t *)malloc(cap * sizeof(uint32_t) * (size_t)(depth + 1));
    uint32_t **lists = (uint32_t **)malloc(sizeof(uint32_t *) * (size_t)(depth + 1));
    if (!px || !py || !pool || !lists) { rc = ORACLE_E_NOMEM; goto done; }
    for (int l = 0; l <= depth; ++l) lists[l] = pool + cap * (size_t)l;
    w.lists = lists; w.px = px; w.py = py;

    const int64_t K = (int64_t)1 << depth;
    for (int half = 0; half < 2; ++half) {
        w.half = half;
        for (int64_t k = 0; k < n; ++k) {
            /* ALPHA takes (x, y); BETA takes (y, x) (Section 3). */
            px[k] = half == 0 ? xy[2 * k] : xy[2 * k + 1];
            py[k] = half == 0 ? xy[2 * k + 1] : xy[2 * k];
        }
        /* Level 0: every line is tested against the whole parameter space. */
        int64_t nv = 0;
        for (int64_t k = 0; k < n; ++k)
            if (line_votes(&w, (uint32_t)k, 0, 0, K)) lists[0][nv++] = (uint32_t)k;
        if (nv != n) { rc = ORACLE_E_INVARIANT; goto done; } /* every line crosses the root */
        *stat_at(&w, 0, 0) = 1;
        *stat_at(&w, 0, 1) = 1; /* the root is always split */
        *stat_at(&w, 0, 2) = (uint64_t)nv;
        *stat_at(&w, 0, 3) = (uint64_t)n;
        record_region(&w, 0, 0, 0, K, nv);
        subdivide(&w, 0, 0, 0, K, lists[0], nv);
    }
    *n_leaves = w.n_leaves;
    if (n_regions) *n_regions = w.n_regions;
    if (w.n_leaves > leaf_cap) { rc = ORACLE_E_CAPACITY; goto done; }

done:
    free(px); free(py); free(pool); free(lists);
    return rc;
}

int oracle_detect(const int16_t *xy, int64_t n, int32_t W, int32_t H, int32_t depth, int32_t T, int32_t mode,
                  oracle_leaf *leaves, int64_t leaf_cap, int64_t *n_leaves, uint64_t *stats,
                  oracle_region *regions, int64_t region_cap, int64_t *n_regions)
{
    return detect_walk(xy, n, W, H, depth, T, mode, leaves, leaf_cap, n_leaves, stats, regions, region_cap,
                       n_regions, NULL, 0);
}

/*
 * One shard of a detection split by subtrees: the level-k regions (a, b) of
 * half h with keep[h * 4^k + a * 2^k + b] == 0 are tested and counted (so the
 * statistics of levels <= k, apart from the level-k pass count, are those of
 * the whole detection) but never split; everything below them belongs to
 * another shard.
 */
int oracle_detect_subtrees(const int16_t *xy, int64_t n, int32_t W, int32_t H, int32_t depth, int32_t T,
                           int32_t split_level, const uint8_t *keep, oracle_leaf *leaves, int64_t leaf_cap,
                           int64_t *n_leaves, uint64_t *stats)
{
    if (!keep || split_level < 1 || split_level > depth) return ORACLE_E_ARG;
    return detect_walk(xy, n, W, H, depth, T, ORACLE_MODE_EXACT, leaves, leaf_cap, n_leaves, stats, NULL, 0, NULL,
                       keep, split_level);
}

/*
 * Direct vote count of one region: the number of points whose line has a code
 * other than 0000 and 1111 for region (i0, j0, S) of the given half, counted
 * over all n points with no hierarchy.  Used to check single cells of
 * full-size results.
 */
int64_t oracle_count_region(const int16_t *xy, int64_t n, int32_t W, int32_t H, int32_t depth, int32_t half,
                            int64_t i0, int64_t j0, int64_t S)
{
    const int64_t L = oracle_frame_side(W, H);
    int64_t cnt = 0;
    for (int64_t k = 0; k < n; ++k) {
        const int32_t x = half == 0 ? xy[2 * k] : xy[2 * k + 1];
        const int32_t y = half == 0 ? xy[2 * k + 1] : xy[2 * k];
        const uint32_t code = oracle_getcode(x, y, i0, j0, S, L, depth);
        if (code != 0u && code != 15u) ++cnt;
    }
    return cnt;
}

/*
 * Front end (Section 3): Sobel's gradient operator on a grey-level image and
 * the split of the edge points into ALPHA and BETA.
 *
 * gx and gy are Sobel's 3 x 3 responses at (x, y) (x to the right, y down):
 *   gx = [p(x+1, y-1) + 2 p(x+1, y) + p(x+1, y+1)] - [p(x-1, y-1) + 2 p(x-1, y) + p(x-1, y+1)]
 *   gy = [p(x-1, y+1) + 2 p(x, y+1) + p(x+1, y+1)] - [p(x-1, y-1) + 2 p(x, y-1) + p(x+1, y-1)]
 * for interior pixels (1 <= x <= W-2, 1 <= y <= H-2); border pixels have no
 * full neighbourhood and are never edge points.
 *
 * Readings where the paper is silent:
 *   - a pixel is an edge point when gx^2 + gy^2 >= threshold^2 (the gradient
 *     magnitude reaches `threshold`, compared exactly in integers);
 *   - the line through an edge point runs across its gradient, so its slope
 *     is -gx / gy; the point belongs to ALPHA (|slope| <= 1) when
 *     |gx| <= |gy| and to BETA otherwise.
 * Points are emitted in row-major order (y, then x).
 */
void oracle_sobel(const uint8_t *img, int32_t W, int32_t H, int32_t x, int32_t y, int32_t *gx, int32_t *gy)
{
    (void)H; /* the caller passes an interior pixel */
#define P(dx, dy) ((int32_t)img[(int64_t)(y + (dy)) * W + (x + (dx))])
    *gx = (P(1, -1) + 2 * P(1, 0) + P(1, 1)) - (P(-1, -1) + 2 * P(-1, 0) + P(-1, 1));
    *gy = (P(-1, 1) + 2 * P(0, 1) + P(1, 1)) - (P(-1, -1) + 2 * P(0, -1) + P(1, -1));
#undef P
}

int oracle_edges(const uint8_t *img, int32_t W, int32_t H, int32_t threshold, int16_t *alpha, int64_t alpha_cap,
                 int64_t *n_alpha, int16_t *beta, int64_t beta_cap, int64_t *n_beta)
{
    if (!img || W < 1 || H < 1 || W > 32767 || H > 32767 || threshold < 0 || !n_alpha || !n_beta)
        return ORACLE_E_ARG;
    int64_t na = 0, nb = 0;
    const int64_t t2 = (int64_t)threshold * threshold;
    for (int32_t y = 1; y + 1 < H; ++y) {
        for (int32_t x = 1; x + 1 < W; ++x) {
            int32_t gx, gy;
            oracle_sobel(img, W, H, x, y, &gx, &gy);
            if ((int64_t)gx * gx + (int64_t)gy * gy < t2) continue;
            const int32_t ax = gx < 0 ? -gx : gx, ay = gy < 0 ? -gy : gy;
            if (ax <= ay) {
                if (na < alpha_cap) { alpha[2 * na] = (int16_t)x; alpha[2 * na + 1] = (int16_t)y; }
                ++na;
            } else {
                if (nb < beta_cap) { beta[2 * nb] = (int16_t)x; beta[2 * nb + 1] = (int16_t)y; }
                ++nb;
            }
        }
    }
    *n_alpha = na;
    *n_beta = nb;
    return (na > alpha_cap || nb > beta_cap) ? ORACLE_E_CAPACITY : ORACLE_OK;
}

/*
 * Leaves -> lines (the paper stops at the peak cells; this step is a reading
 * of its own).  Leaves of the same half whose cells touch (|di| <= 1 and
 * |dj| <= 1) belong to one cluster (connected components of that adjacency).
 * Each cluster is one line: its peak is the leaf with the most votes, ties
 * going to the leaf that comes first in the input (depth-first) order.  The
 * line of peak cell (i, j) is the cell's centre in parameter space,
 *   m = (2i + 1 - K) / K,   b = 2L (2j + 1 - K) / K,
 * read as y = m x + b for half 0 and as x = m y + b for half 1 (Section 3:
 * BETA points were processed with x and y swapped).  A cluster also gives
 * its vote-weighted centre, kept exact as integer sums: with V the total
 * votes, S_i = sum of votes * (2i + 1) and S_j = sum of votes * (2j + 1),
 *   m = (S_i / V - K) / K,   b = 2L (S_j / V - K) / K,
 * which lands between cells when several share the peak.  Lines are reported
 * in the order of each cluster's first leaf.
 */
typedef struct {
    uint32_t half, i, j, votes, cells, pad;
    uint64_t total_votes, sum_i2, sum_j2;
} oracle_line;

static int64_t uf_find(int64_t *parent, int64_t a)
{
    while (parent[a] != a) a = parent[a];
    return a;
}

int oracle_lines(const oracle_leaf *leaves, int64_t n, oracle_line *out, int64_t cap, int64_t *n_lines)
{
    if (n < 0 || (n > 0 && !leaves) || !n_lines) return ORACLE_E_ARG;
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *line_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!parent || !line_of) { free(parent); free(line_of); return ORACLE_E_NOMEM; }
    for (int64_t k = 0; k < n; ++k) parent[k] = k;
    /* every pair of touching leaves (quadratic: the oracle runs on small sets) */
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = a + 1; b < n; ++b) {
            if (leaves[a].half != leaves[b].half) continue;
            const int64_t di = (int64_t)leaves[a].i - (int64_t)leaves[b].i;
            const int64_t dj = (int64_t)leaves[a].j - (int64_t)leaves[b].j;
            if (di < -1 || di > 1 || dj < -1 || dj > 1) continue;
            const int64_t ra = uf_find(parent, a), rb = uf_find(parent, b);
            if (ra != rb) parent[ra > rb ? ra : rb] = ra < rb ? ra : rb;
        }
    int64_t nl = 0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t r = uf_find(parent, k);
        if (r == k) {
            line_of[k] = nl;
            if (nl < cap) {
                oracle_line *L = &out[nl];
                L->half = leaves[k].half; L->i = leaves[k].i; L->j = leaves[k].j; L->votes = leaves[k].votes;
                L->cells = 0; L->pad = 0; L->total_votes = 0; L->sum_i2 = 0; L->sum_j2 = 0;
            }
            ++nl;
        }
        const int64_t id = line_of[r];
        if (id < cap) {
            oracle_line *L = &out[id];
            L->cells += 1;
            L->total_votes += leaves[k].votes;
            L->sum_i2 += (uint64_t)leaves[k].votes * (2u * (uint64_t)leaves[k].i + 1u);
            L->sum_j2 += (uint64_t)leaves[k].votes * (2u * (uint64_t)leaves[k].j + 1u);
            if (leaves[k].votes > L->votes) { /* strictly more: ties keep the earlier leaf */
                L->i = leaves[k].i; L->j = leaves[k].j; L->votes = leaves[k].votes;
            }
        }
    }
    *n_lines = nl;
    free(parent); free(line_of);
    return nl > cap ? ORACLE_E_CAPACITY : ORACLE_OK;
}

/*
 * The paper's solution() step (Section 3): when a region at the leaf level
 * gets enough votes, its voters are plotted and their codes are zeroed at
 * every level, so they take no part in any region the depth-first traversal
 * reaches later.  Readings where the paper is silent:
 *   - removal is per half: the two halves are two runs of the algorithm
 *     (ALPHA, then BETA), so a point plotted in one half still takes part in
 *     the other (every point enters both halves here);
 *   - the `tests` statistic of a level counts the codes actually evaluated:
 *     for each tested region, the voters of its parent not removed by then;
 *   - a region passes when its votes reach T, as in the order-free detection.
 * Leaves are the accepted cells in traversal order with their votes at the
 * time they were reached; plotted[h * n + k] is set for every point plotted
 * in half h.
 */
typedef struct {
    walk_t *w;
    uint8_t *removed;  /* current half: 1 once plotted */
} removal_t;

static void subdivide_removal(removal_t *r, int level, int64_t i0, int64_t j0, int64_t S, const uint32_t *V,
                              int64_t nV)
{
    walk_t *w = r->w;
    const int64_t h = S / 2;
    const int64_t ci[4] = {i0 + h, i0, i0, i0 + h};
    const int64_t cj[4] = {j0 + h, j0 + h, j0, j0};
    const int child = level + 1;
    uint32_t *buf = w->lists[child];
    for (int q = 0; q < 4; ++q) {
        int64_t cnt = 0, evaluated = 0;
        for (int64_t k = 0; k < nV; ++k) {
            if (r->removed[V[k]]) continue; /* its codes were zeroed by an earlier solution() */
            ++evaluated;
            if (line_votes(w, V[k], ci[q], cj[q], h)) buf[cnt++] = V[k];
        }
        *stat_at(w, child, 0) += 1;
        *stat_at(w, child, 2) += (uint64_t)cnt;
        *stat_at(w, child, 3) += (uint64_t)evaluated;
        if (cnt >= w->T) {
            *stat_at(w, child, 1) += 1;
            if (child == w->D) {
                if (w->n_leaves < w->leaf_cap) {
                    oracle_leaf *lf = &w->leaves[w->n_leaves];
                    lf->half = (uint32_t)w->half; lf->i = (uint32_t)ci[q]; lf->j = (uint32_t)cj[q];
                    lf->votes = (uint32_t)cnt;
                }
                w->n_leaves++;
                for (int64_t k = 0; k < cnt; ++k) r->removed[buf[k]] = 1; /* solution(): plot and remove */
            } else {
                subdivide_removal(r, child, ci[q], cj[q], h, buf, cnt);
            }
        }
    }
}

int oracle_detect_removal(const int16_t *xy, int64_t n, int32_t W, int32_t H, int32_t depth, int32_t T,
                          oracle_leaf *leaves, int64_t leaf_cap, int64_t *n_leaves, uint64_t *stats, uint8_t *plotted)
{
    if (n < 0 || W < 1 || H < 1 || W > 32767 || H > 32767 || depth < 1 || depth > 24 || T < 1 || !n_leaves ||
        !stats || (n > 0 && !xy) || (leaf_cap > 0 && !leaves))
        return ORACLE_E_ARG;
    for (int64_t k = 0; k < n; ++k)
        if (xy[2 * k] < 0 || xy[2 * k] >= W || xy[2 * k + 1] < 0 || xy[2 * k + 1] >= H) return ORACLE_E_RANGE;
    walk_t w;
    memset(&w, 0, sizeof w);
    w.L = oracle_frame_side(W, H);
    w.D = depth; w.T = T; w.mode = ORACLE_MODE_EXACT;
    w.stats = stats; w.leaves = leaves; w.leaf_cap = leaf_cap;
    memset(stats, 0, sizeof(uint64_t) * 2 * (size_t)(depth + 1) * 4);
    int rc = ORACLE_OK;
    const size_t cap = (size_t)(n > 0 ? n : 1);
    int32_t *px = (int32_t *)malloc(cap * sizeof(int32_t));
    int32_t *py = (int32_t *)malloc(cap * sizeof(int32_t));
    uint32_t *pool = (uint32_t *)malloc(cap * sizeof(uint32_t) * (size_t)(depth + 1));
    uint32_t **lists = (uint32_t **)malloc(sizeof(uint32_t *) * (size_t)(depth + 1));
    uint8_t *removed = (uint8_t *)malloc(cap);
    if (!px || !py || !pool || !lists || !removed) { rc = ORACLE_E_NOMEM; goto done; }
    for (int l = 0; l <= depth; ++l) lists[l] = pool + cap * (size_t)l;
    w.lists = lists; w.px = px; w.py = py;
    const int64_t K = (int64_t)1 << depth;
    removal_t r;
    r.w = &w;
    r.removed = removed;
    for (int half = 0; half < 2; ++half) {
        w.half = half;
        memset(removed, 0, cap);
        for (int64_t k = 0; k < n; ++k) {
            px[k] = half == 0 ? xy[2 * k] : xy[2 * k + 1];
            py[k] = half == 0 ? xy[2 * k + 1] : xy[2 * k];
        }
        int64_t nv = 0;
        for (int64_t k = 0; k < n; ++k)
            if (line_votes(&w, (uint32_t)k, 0, 0, K)) lists[0][nv++] = (uint32_t)k;
        if (nv != n) { rc = ORACLE_E_INVARIANT; goto done; }
        *stat_at(&w, 0, 0) = 1;
        *stat_at(&w, 0, 1) = 1;
        *stat_at(&w, 0, 2) = (uint64_t)nv;
        *stat_at(&w, 0, 3) = (uint64_t)n;
        subdivide_removal(&r, 0, 0, 0, K, lists[0], nv);
        if (plotted) memcpy(plotted + (size_t)half * cap, removed, (size_t)n);
    }
    *n_leaves = w.n_leaves;
    if (w.n_leaves > leaf_cap) rc = ORACLE_E_CAPACITY;
done:
    free(px); free(py); free(pool); free(lists); free(removed);
    return rc;
}
