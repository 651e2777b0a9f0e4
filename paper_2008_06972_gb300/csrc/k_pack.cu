// Point coding and stream compaction.
//
// Each valid pixel, in canonical order (tiles row-major, raster order inside
// a tile), is coded against its tile's plane: a fitted bit, then either a
// residual code k = round-half-away(e / q) or a raw range code
// m = round-half-away(r / q) (unfit points go to the residual map of
// Sec. III-C as raw ranges).  A tile's pixels are held by one lane segment;
// warp ballots + popcounts give each pixel's rank inside the tile, the scan's
// offsets give the tile's position in every section, and the tile's code bits
// are assembled in shared memory and written out as whole 32-bit words (plain
// stores inside the tile's range, atomicOr only for the two boundary words
// shared with neighbour tiles).  The range-image pixels are reset to empty
// for the next frame.
#include "lcc_internal.cuh"

namespace lcc {

constexpr int kPackWarps = 8;

// Lanes per tile: an eighth of the tile's pixels (at least 4 lanes and a tile row, at most a
// warp), so every lane codes several pixels whose loads are in flight together: the kernel waits
// on memory, and more pixels per warp keep more loads in flight per resident warp (measured on
// 128x4096 frames: 2, 4 and 8 pixels per lane gave 8.9, 11.0 and 11.7 Gpoints/s for the whole
// plan).  A tile row's pixels must lie in one lane segment (the occupancy-bitmap step takes a
// row from one ballot).  Each segment stages its codes in SW shared words: one section of the
// tile's codes at up to 32 bits each (raw_exact) plus the partial words at both ends.
template <int TH_, int TW_>
struct PShape {
    static constexpr int PX = TH_ * TW_;
    static constexpr int LPT0 = PX / 8 < 4 ? 4 : (PX / 8 < 32 ? PX / 8 : 32);
    static constexpr int LPT = LPT0 < TW_ ? TW_ : LPT0;
    static constexpr int PPL = PX / LPT;
    static constexpr int TPW = 32 / LPT;
    static constexpr int SW = (PX + 2 + 3) / 4 * 4;   // staging words per segment
    static_assert(LPT <= 32 && PX % LPT == 0 && LPT % TW_ == 0, "lane segments");
};

// Write `count` codes of `width` bits, code index base0 + rank, into `sec`.
template <int LPT, int PPL>
__device__ __forceinline__ void stage_codes(uint32_t *buf, int sw, uint32_t *sec, uint32_t sec_words,
                                            uint64_t base0, int count, int width, const bool (&has)[PPL], const int (&rank)[PPL],
                                            const uint32_t (&val)[PPL], int sl) {
    const uint64_t base_bit = base0 * (uint64_t)width;
    const uint64_t w0 = base_bit >> 5;
    const int sh = (int)(base_bit & 31);
    const int nwords = count ? (sh + count * width + 31) >> 5 : 0;
    for (int w = sl; w < nwords && w < sw; w += LPT) buf[w] = 0u;
    __syncwarp();
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        if (has[m]) {
            const int lb = sh + rank[m] * width;
            const int wi = lb >> 5, bo = lb & 31;
            atomicOr(buf + wi, val[m] << bo);
            if (bo + width > 32) atomicOr(buf + wi + 1, val[m] >> (32 - bo));
        }
    }
    __syncwarp();
    for (int w = sl; w < nwords && w < sw; w += LPT) {
        const uint32_t x = buf[w];
        if (w0 + w >= sec_words) break;
        if (w == 0 || w == nwords - 1) {
            if (x) atomicOr(sec + w0 + w, x);
        } else {
            sec[w0 + w] = x;
        }
    }
    __syncwarp();
}

// Four blocks per SM (at most 64 registers a thread): twice the resident warps of the
// unconstrained allocation (112 registers), which hides the tile loads' latency; measured about
// 30% faster on 128x4096 frames, with the same bytes.
template <int TH_, int TW_>
__global__ void __launch_bounds__(kPackWarps * 32, 4) k_pack(Geometry g, Scratch s, Batch b) {
    using S = PShape<TH_, TW_>;
    constexpr int LPT = S::LPT, PPL = S::PPL, TPW = S::TPW;
    __shared__ uint32_t s_stage[kPackWarps][TPW * S::SW];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = lane / LPT, sl = lane % LPT;
    const int f = blockIdx.y;
    const size_t slot = (size_t)b.slot[f];
    const int t = (blockIdx.x * kPackWarps + warp) * TPW + seg;
    const bool tile_ok = t < g.NT;
    const int tr = tile_ok ? t / g.TC : 0, tc = tile_ok ? t % g.TC : 0;
    uint32_t *rimg = s.rimg + slot * g.H * g.W;
    const uint32_t segmask = (LPT == 32) ? FULL : (((1u << LPT) - 1u) << (seg * LPT));
    const uint32_t below = segmask & ((1u << lane) - 1u);

    // every load of the tile is independent of the others: one round trip
    const FrameLayout L = s.layout[slot];
    uint8_t mode = T_EMPTY;
    TileOff off = {0, 0, 0, 0, 0, 0, 0, 0};
    float4 pl = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t kref = 0, want_cand = 0, want_fit = 0, want_raw = 0;
    if (tile_ok) {
        const uint4 *cp = reinterpret_cast<const uint4 *>(s.codes + slot * g.NT + t);
        const uint4 c = cp[0], cpl = cp[1];
        mode = (uint8_t)(c.x & 0xff);
        want_cand = (c.x >> 8) & 0xff;
        want_fit = (c.x >> 16) & 0xff;
        want_raw = c.x >> 24;
        kref = c.z;
        const uint4 o0 = *reinterpret_cast<const uint4 *>(s.offs + slot * g.NT + t);
        const uint4 o1 = *(reinterpret_cast<const uint4 *>(s.offs + slot * g.NT + t) + 1);
        const uint4 *rb = reinterpret_cast<const uint4 *>(s.rowbase + (slot * g.TR + tr) * 8);   // row base offsets
        const uint4 rb0 = rb[0], rb1 = rb[1];
        off.cand = o0.x + rb0.x; off.fitted = o0.y + rb0.y; off.raw = o0.z + rb0.z; off.run = o0.w + rb0.w;
        off.temporal = o1.x + rb1.x;
        if (mode >= T_RUN_START)
            pl = make_float4(__uint_as_float(cpl.x), __uint_as_float(cpl.y), __uint_as_float(cpl.z),
                             __uint_as_float(cpl.w));
    }
    const bool coded = mode >= T_RUN_START;

    bool v[PPL], fit[PPL];
    uint32_t kc[PPL], mc[PPL];
    // the pixels' ranges and rays: every load issued before any is used (one round trip)
    uint32_t bits[PPL];
    float ux[PPL], uy[PPL], uz[PPL];
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        const int k = sl + LPT * m;
        const int i = tr * TH_ + k / TW_, j = tc * TW_ + k % TW_;
        const bool in = tile_ok && i < g.H && j < g.W;
        bits[m] = in ? __ldcg(rimg + (size_t)i * g.W + j) : kEmptyBits;
        beam(g, in ? i : 0, in ? j : 0, ux[m], uy[m], uz[m]);
    }
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        const int k = sl + LPT * m;
        const int i = tr * TH_ + k / TW_, j = tc * TW_ + k % TW_;
        if (tile_ok && i < g.H && j < g.W) rimg[(size_t)i * g.W + j] = kEmptyBits;   // ready for the next frame
    }
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        v[m] = bits_valid(bits[m]);
        const float r = __uint_as_float(bits[m]);
        fit[m] = false;
        kc[m] = 0;
        mc[m] = 0;
        if (v[m]) {
            float e = 0.f;
            fit[m] = coded && residual(pl, ux[m], uy[m], uz[m], r, g.thr, e);
            if (fit[m]) kc[m] = (uint32_t)(quant_res(e, g.q) + g.k_max);
            else mc[m] = g.raw_exact ? __float_as_uint(r) : quant_raw(r, g.q);
        }
    }
    if (!L.ok) return;
    uint32_t *words = reinterpret_cast<uint32_t *>(b.out[f] + kHeaderBytes);

    // ranks within the tile (raster order k = sl + LPT*m)
    uint32_t vb[PPL], fb[PPL];
    int vrank[PPL], frank[PPL];
    int vacc = 0, facc = 0;
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        vb[m] = __ballot_sync(FULL, v[m]) & segmask;
        fb[m] = __ballot_sync(FULL, fit[m]) & segmask;
        vrank[m] = vacc + __popc(vb[m] & below);
        frank[m] = facc + __popc(fb[m] & below);
        vacc += __popc(vb[m]);
        facc += __popc(fb[m]);
    }
    // the counts the scan placed this tile with must be the ones it writes
    const bool consistent = !tile_ok || (coded ? (want_cand == (uint32_t)vacc && want_fit == (uint32_t)facc &&
                                                  want_raw == (uint32_t)(vacc - facc))
                                               : (want_cand == 0u && want_fit == 0u && want_raw == (uint32_t)vacc));
    const uint32_t bad = __ballot_sync(FULL, !consistent) & segmask;
    if (bad) {
        if (sl == 0) atomicOr(s.err, E_INTERNAL);
        vacc = facc = 0;
        mode = T_EMPTY;
#pragma unroll
        for (int m = 0; m < PPL; m++) v[m] = fit[m] = false;
    }

    if (tile_ok && sl == 0) {
        // occupancy bitmap: one row piece of the tile per image row
#pragma unroll
        for (int rr = 0; rr < TH_; rr++) {
            const int i = tr * TH_ + rr;
            if (i >= g.H) break;
            const int k0 = rr * TW_;
            const int m = k0 / LPT;
            const uint32_t piece = (vb[m] >> (seg * LPT + (k0 % LPT))) & ((TW_ == 32) ? FULL : ((1u << TW_) - 1u));
            if (!piece) continue;
            const uint64_t pos = (uint64_t)i * g.W + (uint64_t)tc * TW_;
            const uint32_t sh = (uint32_t)(pos & 31);
            atomicOr(words + L.sec[0] + (pos >> 5), piece << sh);
            if (sh + TW_ > 32) atomicOr(words + L.sec[0] + (pos >> 5) + 1, piece >> (32 - sh));
        }
        // three-coefficient planes: a run start's record is its fit's coefficients and its tile code
        // names the dominant axis
        const float4 cf = (g.plane3 && mode == T_RUN_START) ? s.coef[slot * g.NT + t] : make_float4(0.f, 0.f, 0.f, 0.f);
        const uint32_t code = (g.plane3 && mode == T_RUN_START) ? (uint32_t)T_RUN_START3 + (uint32_t)cf.w : mode;
        if (code) atomicOr(words + L.sec[1] + (t >> 3), code << (4 * (t & 7)));
        if (mode == T_RUN_START) {
            if (g.plane3) {
                uint32_t *d = words + L.sec[2] + 3u * off.run;
                d[0] = __float_as_uint(cf.x);
                d[1] = __float_as_uint(cf.y);
                d[2] = __float_as_uint(cf.z);
            } else {
                uint32_t *d = words + L.sec[2] + 4u * off.run;
                d[0] = __float_as_uint(pl.x);
                d[1] = __float_as_uint(pl.y);
                d[2] = __float_as_uint(pl.z);
                d[3] = __float_as_uint(pl.w);
            }
        }
        if (mode == T_TEMPORAL) {
            uint32_t *d = words + L.sec[3] + 2u * off.temporal;
            d[0] = kref;
            d[1] = __float_as_uint(pl.w);
        }
    }

    uint32_t *buf = &s_stage[warp][seg * S::SW];
    bool has[PPL];
    int rank[PPL];
    uint32_t val[PPL];
    // fitted bits of candidate pixels
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        has[m] = coded && v[m];
        rank[m] = vrank[m];
        val[m] = fit[m] ? 1u : 0u;
    }
    stage_codes<LPT, PPL>(buf, S::SW, words + L.sec[4], L.sec[5] - L.sec[4], off.cand, coded ? vacc : 0, 1, has, rank, val, sl);
    // residual codes of plane-coded pixels (none in the no-delta mode)
    if (!g.no_delta) {
#pragma unroll
        for (int m = 0; m < PPL; m++) {
            has[m] = fit[m];
            rank[m] = frank[m];
            val[m] = kc[m];
        }
        stage_codes<LPT, PPL>(buf, S::SW, words + L.sec[5], L.sec[6] - L.sec[5], off.fitted, facc, g.w_res, has, rank,
                              val, sl);
    }
    // raw codes of the remaining valid pixels
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        has[m] = v[m] && !fit[m];
        rank[m] = vrank[m] - frank[m];
        val[m] = mc[m];
    }
    stage_codes<LPT, PPL>(buf, S::SW, words + L.sec[6], L.sec[7] - L.sec[6], off.raw, vacc - facc, g.w_raw, has, rank, val, sl);
}

template <int TH_, int TW_>
static cudaError_t launch_pack_t(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st) {
    using S = PShape<TH_, TW_>;
    const int tiles_per_block = kPackWarps * S::TPW;
    dim3 grid((g.NT + tiles_per_block - 1) / tiles_per_block, b.nframes);
    k_pack<TH_, TW_><<<grid, kPackWarps * 32, 0, st>>>(g, s, b);
    return cudaGetLastError();
}

cudaError_t launch_pack(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st) {
    if (b.nframes <= 0) return cudaSuccess;
    if (g.th == 4 && g.tw == 4) return launch_pack_t<4, 4>(g, s, b, st);
    if (g.th == 4 && g.tw == 8) return launch_pack_t<4, 8>(g, s, b, st);
    if (g.th == 8 && g.tw == 8) return launch_pack_t<8, 8>(g, s, b, st);
    if (g.th == 8 && g.tw == 16) return launch_pack_t<8, 16>(g, s, b, st);
    return cudaErrorInvalidValue;
}

}  // namespace lcc
