// Internal types and device helpers of the lcc CUDA library (sm_103a).
//
// Arithmetic contract shared with any independent implementation of the
// method: every per-point fp32 expression below is written with explicit
// IEEE-rounded intrinsics (__fmul_rn, __fadd_rn, __fdiv_rn, fmaf, sqrtf) and
// the library is compiled with -fmad=false, so no multiply-add is fused
// behind our back.  Binning, residual tests and quantised codes are therefore
// bit-reproducible given the same fp32 plane.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "lcc.h"

namespace lcc {

// Pixel-boundary directions of the grid of Sec. III-B, fp64 libm rounded to fp32 (host).
// Row boundary k in 0..rows (k = 0 is the top edge); column boundary j in 0..cols-1 (j = 0
// is azimuth -pi).
inline void row_boundary(const lcc_sensor &s, int k, float *c, float *sn) {
    const double d_el = (s.elev_max_deg - s.elev_min_deg) / s.rows;
    const double e = (s.elev_max_deg - k * d_el) * (M_PI / 180.0);
    *c = (float)cos(e);
    *sn = (float)sin(e);
}
inline void col_boundary(const lcc_sensor &s, int j, float *c, float *sn) {
    const double b = -M_PI + j * (2.0 * M_PI / s.cols);
    *c = (float)cos(b);
    *sn = (float)sin(b);
}

constexpr int kMaxBatch = 64;          // frames per batched launch
constexpr uint32_t kEmptyBits = 0xFFFFFFFFu;  // range-image pixel with no point
constexpr int kHeaderBytes = 64;
constexpr uint32_t kMagic = 0x3143434Cu;     // "LCC1"
constexpr int kVersion = 1;
constexpr int kMaxTilePx = 128;

// tile codes in the stream
enum : uint8_t { T_EMPTY = 0, T_RAW = 1, T_RUN_START = 2, T_RUN_CONT = 3, T_TEMPORAL = 4, T_TEMPORAL_CONT = 5,
                 T_RUN_START3 = 6 /* .. 8: a three-coefficient run start, dominant axis x, y, z */ };
// own-fit status of a tile
enum : uint8_t { S_EMPTY = 0, S_FAIL = 1, S_FIT = 2, S_TEMPORAL = 3 };
// latched device error bits
enum : uint32_t { E_CAPACITY = 1u, E_CORRUPT = 2u, E_TIMEOUT = 4u, E_INTERNAL = 8u };

// Per-tile fit record; layout identical to lcc_tile_info.
struct alignas(16) TileRec {
    float4 plane;        // own spatial plane (n, d) or (n', c') if temporal
    float4 tplane;       // temporal test plane
    uint32_t kref;       // K tile of the anchor, ~0u if none
    uint32_t ahead_mask; // bit j: this tile passes the plane of tile t-1-j (run pre-test, j < 32)
    uint8_t status, rounds, flags, n_valid;
    uint8_t n_inlier, t_rounds, t_inlier, t_status;
    uint8_t ahead_cnt[16];  // inlier counts of the first 16 of those tests
};
static_assert(sizeof(TileRec) == 64, "TileRec layout");
static_assert(sizeof(TileRec) == sizeof(lcc_tile_info), "TileRec matches lcc_tile_info");

// Output of the run merge: how the tile is coded, its stream counts and everything the
// packer needs about its plane, so that the packer's loads do not depend on one another.
struct alignas(16) TileCode {
    uint8_t mode, cand, fitted, raw;
    uint32_t plane_tile;  // tile whose plane codes this one (run start)
    uint32_t kref;        // key-frame tile of a temporal tile
    uint32_t pad;
    float4 plane;         // coding plane: the run's plane, or (n', c') of a temporal tile
};
static_assert(sizeof(TileCode) == 32, "TileCode layout");

// Exclusive stream offsets of a tile (in codes) within its tile row.
struct TileOff {
    uint32_t cand, fitted, raw, run, temporal, pad0, pad1, pad2;
};

// Word offsets of the stream sections of one frame (written by the scan).
struct FrameLayout {
    uint32_t sec[8];     // word offsets after the header: bitmap, tiles, runs, temporal, fitted, res, raw, end
    uint32_t total_bytes;
    uint32_t ok;         // 1 if the stream fits the output buffer
    uint32_t n_valid, pad;
};

// Per-frame device counters (atomics).
struct DevStats {
    unsigned long long points_in, invalid, fov, binned, valid;
    unsigned long long empty, raw_tiles, run_start, run_cont, temporal, temporal_cont;
    unsigned long long rounds[8];
    unsigned long long borderline, cand, fitted, raw;
    unsigned long long bytes;
    unsigned long long net_tiles;   // tiles the proposal net must cover (3 valid pixels)
};

// Decoder per-tile state.
struct alignas(16) DecTile {
    float4 plane;
    uint32_t off_cand, off_fit, off_raw;
    uint8_t mode, n_valid, pad0, pad1;
};

// Sensor geometry and parameters, passed by value to every kernel.
struct Geometry {
    int H, W;            // image rows, cols
    int th, tw, tpx;     // tile shape and pixels per tile
    int TR, TC, NT;      // tile rows, tile cols, tiles per frame
    float thr, q, rmax, fmin;
    int R;               // refit rounds after the first fit
    int merge, lookahead;
    int solver;          // 0 float-float plane solve, 1 FP64
    int schedule;        // 0 per-thread fit rounds; 1, 2: that many rounds per thread, the rest queued;
                         // 3: one round per thread, the rest in one dense launch; 4: as 3, and batched
                         // P frames fit spatially first and run the temporal test after; 5: as 4 with
                         // every round on a lane group per tile (the first pass only queues); 6: as 4
                         // with the queued rounds on a thread per tile
    int first_rounds;    // fit rounds of the first pass under a queued schedule (0 under schedule 5)
    int no_delta;        // 1: plane-coded points carry no residual code (no residual section)
    int raw_exact;       // 1: raw pixels carry their fp32 range bits (32-bit raw codes)
    int tcand;           // K tiles a P tile's relaxed-plane test may try (1..4)
    int truns;           // 1: temporal tiles of P frames grow runs (TEMPORAL_CONT tiles)
    int plane3;          // 1: planes in Eq. 3's three-coefficient form (dominant axis)
    int k_max, w_res, w_raw;
    float elev_max_rad, inv_d_el, inv_d_az;   // first guesses only (1/row and 1/column pitch, rad); the tables decide
    const float *ce, *se, *ct, *st;       // beam tables
    const float *rbc, *rbs, *cbc, *cbs;   // boundary tables
};

// Per-slot scratch pointers (slot = batch position's scratch area).
struct Scratch {
    uint32_t *rimg;      // [slots][H*W]
    TileRec *tiles;      // [slots][NT]
    TileCode *codes;     // [slots][NT]
    TileOff *offs;       // [slots][NT]
    FrameLayout *layout; // [slots]
    DevStats *stats;     // [slots]
    unsigned long long *bytes;  // [slots] stream size (or needed size)
    uint32_t *err;       // latched error bits
    uint8_t *lbcnt;      // [slots][NT][32] run pre-test inlier counts (byte j: vs the plane of tile t-1-j)
    uint32_t *rowtot;    // [slots][TR][8] per tile-row totals: cand, fitted, raw, run, temporal, valid
    uint32_t *rowbase;   // [slots][TR][8] exclusive prefix of rowtot over the frame's rows
    uint32_t *queue;     // [2 sets][2][qcap] fit work queues (frame << 26 | tile)
    uint32_t *qcount;    // [2 sets][8] items pushed per fit round
    uint32_t *rowdone;   // [slots] tile rows of the frame merged so far (0 between launches)
    uint32_t qcap;       // entries per queue (slots * tiles)
    float4 *coef;        // [slots][NT] plane3: a tile's plane coefficients (a, b, c, axis) of its last fit
};

// One batched launch over up to kMaxBatch frames of the same sensor.
struct Batch {
    int nframes;
    int kind;                      // 0 key frames, 1 P frames
    int slot[kMaxBatch];
    const float4 *pts[kMaxBatch];
    long long n[kMaxBatch];
    uint8_t *out[kMaxBatch];
    unsigned long long cap[kMaxBatch];
    long long blk_prefix[kMaxBatch + 1];  // binning blocks before each frame
    const float4 *kf[kMaxBatch];   // per frame: key-frame planes (P frames) or NULL
    float4 *kf_out[kMaxBatch];     // per frame: key-frame plane table to fill (K frames) or NULL
    unsigned long long *nbytes_out[kMaxBatch];  // per frame: extra copy of the stream size, or NULL
    const float *prop[kMaxBatch];  // per frame: fit proposals [NT][5] (logit, v, d_rel), or NULL
    int qset;                      // queue set of the queued fit schedule (batches that overlap use different sets)
    float skip_logit;              // tiles whose proposal logit is below this are not fitted
};

struct Poses {
    double m[kMaxBatch][16];
};

// ------------------------------------------------------------------------
// device helpers
// ------------------------------------------------------------------------

__device__ __forceinline__ bool bits_valid(uint32_t b) { return b < 0x7F800000u && b != 0u; }

// Beam of pixel (i, j): fp32 products of the row and column tables.
__device__ __forceinline__ void beam(const Geometry &g, int i, int j, float &ux, float &uy, float &uz) {
    const float ce = __ldg(g.ce + i), se = __ldg(g.se + i);
    ux = __fmul_rn(ce, __ldg(g.ct + j));
    uy = __fmul_rn(ce, __ldg(g.st + j));
    uz = se;
}

// Along-ray residual against an fp32 plane; true if |e| <= thr.
__device__ __forceinline__ bool residual(const float4 &pl, float ux, float uy, float uz, float r, float thr,
                                         float &e) {
    const float dot = fmaf(pl.x, ux, fmaf(pl.y, uy, __fmul_rn(pl.z, uz)));
    if (!(dot > 1e-3f)) {
        e = __int_as_float(0x7f800000);
        return false;
    }
    const float rhat = __fdiv_rn(pl.w, dot);
    e = __fsub_rn(r, rhat);
    return fabsf(e) <= thr;
}

// The same decision as residual() (|r - d/(n.u)| <= thr with an IEEE
// division), reached without the division for all but the pixels near the
// threshold: the quotient from the fast reciprocal is within 2 ulp of the
// exact one, so when the approximate residual is farther than a safe margin
// from thr the exact test cannot decide differently.  Pixels inside the margin
// (which always includes |e| within 1e-6 m of thr) take the exact path.
__device__ __forceinline__ bool inlier_screened(const float4 &pl, float ux, float uy, float uz, float r, float thr,
                                                bool &border) {
    const float dot = fmaf(pl.x, ux, fmaf(pl.y, uy, __fmul_rn(pl.z, uz)));
    if (!(dot > 1e-3f)) return false;
    const float rh = __fdividef(pl.w, dot);
    const float ea = fabsf(__fsub_rn(r, rh));
    const float margin = fmaxf(3.0e-6f * (fabsf(rh) + fabsf(r)), 2.0e-6f);
    if (ea < thr - margin) return true;
    if (ea > thr + margin) return false;
    float e;
    const bool in = residual(pl, ux, uy, uz, r, thr, e);
    if (isfinite(e) && fabsf(fabsf(e) - thr) <= 1e-6f) border = true;
    return in;
}

__device__ __forceinline__ int quant_res(float e, float q) {
    const float k = floorf(__fadd_rn(__fdiv_rn(fabsf(e), q), 0.5f));
    return e < 0.0f ? -(int)k : (int)k;
}

__device__ __forceinline__ uint32_t quant_raw(float r, float q) {
    return (uint32_t)floorf(__fadd_rn(__fdiv_rn(r, q), 0.5f));
}

__device__ __forceinline__ int need_inliers(float fmin, int nv) {
    const int need = (int)ceilf(__fmul_rn(fmin, (float)nv));
    return need < 3 ? 3 : need;
}

// Sign tests against the boundary tables.
__device__ __forceinline__ float row_side(const Geometry &g, int k, float z, float rho) {
    return fmaf(z, __ldg(g.rbc + k), -__fmul_rn(rho, __ldg(g.rbs + k)));
}
__device__ __forceinline__ float col_side(const Geometry &g, int j, float x, float y) {
    return fmaf(y, __ldg(g.cbc + j), -__fmul_rn(x, __ldg(g.cbs + j)));
}

// Starting guess of atan(a) for a in [0, 1]: an odd polynomial of degree 7 whose
// coefficients were fitted to atan on [0, 1] by iteratively reweighted least squares
// (maximum error 8.2e-5 rad).  It only picks where the boundary walks below start.
__device__ __forceinline__ float atan01_guess(float a) {
    const float a2 = __fmul_rn(a, a);
    return __fmul_rn(a, fmaf(fmaf(fmaf(-0.03898929f, a2, 0.14626859f), a2, -0.32117667f), a2, 0.99921398f));
}

// Starting guess of atan2(y, x) in [-pi, pi] (octant reduction of atan01_guess).
__device__ __forceinline__ float atan2_guess(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    float t = mx > 0.0f ? atan01_guess(__fdividef(mn, mx)) : 0.0f;
    if (ay > ax) t = 1.5707963f - t;
    if (x < 0.0f) t = 3.1415927f - t;
    return y < 0.0f ? -t : t;
}

// Eq. 1-2 for one point: 0 binned (r, pix set), 1 invalid, 2 out of FOV.
// The pixel is the unique one whose boundary sign tests hold (the signs are
// monotone along the rows and around the columns, so the result does not
// depend on the starting guess, which only sets how many steps the walks take).
__device__ __forceinline__ int bin_point(const Geometry &g, float x, float y, float z, float &r, int &pix) {
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) return 1;
    r = sqrtf(fmaf(x, x, fmaf(y, y, __fmul_rn(z, z))));
    if (!(r > 0.0f) || !(r <= g.rmax)) return 1;
    const float rho = sqrtf(fmaf(x, x, __fmul_rn(y, y)));
    if (row_side(g, 0, z, rho) > 0.0f) return 2;
    if (!(row_side(g, g.H, z, rho) > 0.0f)) return 2;
    int i = (int)floorf(__fmul_rn(g.elev_max_rad - atan2_guess(z, rho), g.inv_d_el));
    i = min(max(i, 0), g.H - 1);
    // row i: !(side(i) > 0) and side(i + 1) > 0
    float lo = row_side(g, i, z, rho), hi = row_side(g, i + 1, z, rho);
    for (int it = 0; it < g.H && i > 0 && lo > 0.0f; it++) {
        i--;
        hi = lo;
        lo = row_side(g, i, z, rho);
    }
    for (int it = 0; it < g.H && i < g.H - 1 && !(hi > 0.0f); it++) {
        i++;
        lo = hi;
        hi = row_side(g, i + 1, z, rho);
    }
    if (lo > 0.0f || !(hi > 0.0f)) return 2;
    int j = (int)floorf(__fmul_rn(atan2_guess(y, x) + 3.1415927f, g.inv_d_az));
    j = j < 0 ? j + g.W : (j >= g.W ? j - g.W : j);
    j = min(max(j, 0), g.W - 1);
    // column j: side(j) >= 0 and !(side(j + 1) >= 0), indices modulo W
    float cl = col_side(g, j, x, y), ch = col_side(g, (j + 1 == g.W) ? 0 : j + 1, x, y);
    for (int it = 0; it < g.W && !(cl >= 0.0f); it++) {
        j = (j == 0) ? g.W - 1 : j - 1;
        ch = cl;
        cl = col_side(g, j, x, y);
    }
    for (int it = 0; it < g.W && ch >= 0.0f; it++) {
        j = (j + 1 == g.W) ? 0 : j + 1;
        cl = ch;
        ch = col_side(g, (j + 1 == g.W) ? 0 : j + 1, x, y);
    }
    if (!(cl >= 0.0f) || ch >= 0.0f) return 2;
    pix = i * g.W + j;
    return 0;
}

// Eq. 3 generalised to the dominant axis k of a unit-normal plane (largest |n_k|, lowest index on
// ties; i, j the next axes in cyclic order): a = n_i / n_k, b = n_j / n_k, c = d / n_k, and back:
// n_k = 1 / sqrt(a^2 + b^2 + 1), n_i = a n_k, n_j = b n_k, d = c n_k, negated when d < 0 (|d| <
// 1e-9 keeps n_k > 0).  IEEE fp32 operations in a fixed order, so encoder and decoder agree.
__device__ __forceinline__ float4 plane_to3(float4 pl) {
    const float n[3] = {pl.x, pl.y, pl.z};
    int k = 0;
    float m = fabsf(n[0]);
    if (fabsf(n[1]) > m) { k = 1; m = fabsf(n[1]); }
    if (fabsf(n[2]) > m) k = 2;
    const float nk = n[k];
    return make_float4(__fdiv_rn(n[(k + 1) % 3], nk), __fdiv_rn(n[(k + 2) % 3], nk), __fdiv_rn(pl.w, nk), (float)k);
}

__device__ __forceinline__ float4 plane_from3(float4 c) {
    const int k = (int)c.w;
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(fmaf(c.x, c.x, fmaf(c.y, c.y, 1.0f))));
    float n[3];
    n[k] = inv;
    n[(k + 1) % 3] = __fmul_rn(c.x, inv);
    n[(k + 2) % 3] = __fmul_rn(c.y, inv);
    float d = __fmul_rn(c.z, inv);
    if (!(fabsf(d) < 1e-9f) && d < 0.0f) {
        n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2]; d = -d;
    }
    return make_float4(n[0], n[1], n[2], d);
}

// n' = R^T n in fp64 with a fixed operation order, rounded to fp32.
__device__ __forceinline__ void rotate_normal(const double *M, float nx, float ny, float nz, float *o) {
#pragma unroll
    for (int j = 0; j < 3; j++) {
        double t = __dmul_rn(M[0 * 4 + j], (double)nx);
        t = fma(M[1 * 4 + j], (double)ny, t);
        t = fma(M[2 * 4 + j], (double)nz, t);
        o[j] = (float)t;
    }
}

// Eq. 6: p' = R p + T in fp64, rounded to fp32.
__device__ __forceinline__ void transform_point(const double *M, float px, float py, float pz, float *o) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
        double t = __dmul_rn(M[i * 4 + 0], (double)px);
        t = fma(M[i * 4 + 1], (double)py, t);
        t = fma(M[i * 4 + 2], (double)pz, t);
        o[i] = (float)__dadd_rn(t, M[i * 4 + 3]);
    }
}

// ---- float-float (double-single) arithmetic for compensated moments ----

struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, lo);
}

// Exact product of two floats as an unevaluated sum.
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}

// (a.hi + a.lo) * (b.hi + b.lo) ~ exact product of the hi parts plus cross terms.
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = fmaf(a.hi, b.hi, -p);
    const float c = fmaf(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    return fast_two_sum(p, __fadd_rn(e, c));
}

__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ ff shfl_xor_ff(ff v, int off) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
}

__device__ __forceinline__ ff shfl_xor_ff_m(unsigned mask, ff v, int off) {
    return {__shfl_xor_sync(mask, v.hi, off), __shfl_xor_sync(mask, v.lo, off)};
}

// Read `width` bits (<= 25) at bit position pos from little-endian words.
__device__ __forceinline__ uint32_t get_bits(const uint32_t *w, uint64_t pos, int width) {
    const uint64_t wi = pos >> 5;
    const int sh = (int)(pos & 31);
    uint64_t v = w[wi];
    if (sh + width > 32) v |= (uint64_t)w[wi + 1] << 32;
    return (uint32_t)((v >> sh) & ((1ull << width) - 1));
}

// ------------------------------------------------------------------------
// host-side launchers (one per kernel file)
// ------------------------------------------------------------------------

// max_blocks > 0 caps the grid (a CTA then takes several chunks of points): for points read
// over the host link, whose reads are link-bound, so that the binning does not occupy every
// SM's thread slots while other kernels wait for them.
cudaError_t launch_bin(const Geometry &g, const Scratch &s, const Batch &b, long long total_blocks,
                       cudaStream_t st, long long max_blocks = 0);
cudaError_t launch_range_image(const Geometry &g, const uint32_t *rimg, float *range, uint32_t *valid,
                               cudaStream_t st);
cudaError_t launch_fit(const Geometry &g, const Scratch &s, const Batch &b, const Poses &p, cudaStream_t st);
cudaError_t launch_temporal(const Geometry &g, const Scratch &s, const Batch &b, const Poses &p, cudaStream_t st);
// temporal_only: after the temporal test of P frames whose full pre-test ran before it, rewrite the
// bits and counts of the candidates that became temporal (tested against their relaxed planes)
cudaError_t launch_lookbehind(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st,
                              bool temporal_only = false);
cudaError_t launch_queued_rounds(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st);

// Spatial rounds still to run after a batch's first fit pass under a queued schedule: all of
// them for P frames whose first pass was their temporal test, else those the pass left.
inline int queued_rounds_left(const Geometry &g, const Batch &b) {
    return (b.kind == 1 && b.kf[0]) ? g.R + 1 : g.R + 1 - g.first_rounds;
}

// Kernels launch_queued_rounds launches for a batch (one per round, or one under schedule 3).
inline int queued_round_kernels(const Geometry &g, const Batch &b) {
    if (g.schedule < 1 || b.nframes <= 0) return 0;
    return g.schedule >= 3 ? 1 : queued_rounds_left(g, b);
}
cudaError_t launch_merge(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st);
size_t merge_smem_bytes(int TC);
cudaError_t launch_pack(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st);
// Streams decoded by one launch (frame f = blockIdx.y): its bytes, its per-tile decoder state
// (NT DecTiles, then its DecState) and its outputs (range and xyz may be NULL).
struct DecBatch {
    const uint8_t *bits[kMaxBatch];
    unsigned long long nbytes[kMaxBatch];
    DecTile *dt[kMaxBatch];
    float *range[kMaxBatch];
    float4 *xyz[kMaxBatch];
};
cudaError_t launch_decode_prep(const Geometry &g, const DecBatch &db, int nframes, const float4 *kf,
                               const Poses &poses, float4 *kf_out, uint32_t *err, int expect_kind, cudaStream_t st);
cudaError_t launch_maxdiff(const float *a, const float *b, long long n, uint32_t *out, cudaStream_t st);
cudaError_t launch_decode_px(const Geometry &g, const DecBatch &db, int nframes, uint32_t *err, cudaStream_t st);

}  // namespace lcc
