// Greedy horizontal run growth (Sec. III-C) — one block per tile row.
//
// The paper grows a run of tiles to the right while the plane "fit so far"
// (the run's first plane) still codes the next tile under the threshold, and
// restarts at the first tile that fails.  The walk is inherently sequential
// along a row, so everything around it is parallel: the followers'
// look-behind bits (from the fit stage) decide the first `lookahead` joins of
// a run in one ballot, and the walk itself is a pointer chase in shared
// memory.  Temporal tiles of P frames are coded first (Sec. III-D): each ends
// the spatial run before it and starts a run of its own, which with temporal
// runs grows to the right by the same rule against its relaxed plane, over any
// tile that passes it (TEMPORAL_CONT); the walk treats both kinds of start alike.
//
// Output per tile: its stream mode, the tile whose plane codes it, its counts
// of candidate / plane-coded / raw-coded pixels and their offsets within the
// tile row; per row: the totals.
#include "lcc_internal.cuh"
#include "scan_frame.cuh"

namespace lcc {

// Per-tile fields of one tile row, staged in shared memory so that each walk
// step costs shared-memory latency instead of a dependent L2 round trip.
struct alignas(16) RowRec {
    float4 plane;
    uint32_t amask;          // look-behind bits: bit j = this tile passes the plane of tile c-1-j
    uint8_t status, n_valid, n_inlier, rounds;
    uint32_t acnt[4];        // look-behind inlier counts (byte j)
    uint8_t flags, pad0, pad1, pad2;
    uint32_t kref;           // key-frame tile (temporal tiles)
};
static_assert(sizeof(RowRec) == 48, "RowRec layout");

// Byte offset of the staged row in the merge kernel's dynamic shared memory (after the row
// records, the next-fitted / run-end / reach tables and the explicit-join counts).
__host__ __device__ __forceinline__ size_t merge_stage_offset(int TC) {
    const size_t raw = sizeof(RowRec) * (size_t)TC + 2 * (size_t)(TC + 1) + 6 * (size_t)TC + (size_t)TC + 16;
    return (raw + 15) & ~size_t(15);
}

constexpr size_t kMergeStageMaxSmem = 200 * 1024;

__device__ __forceinline__ void put_code(TileCode *codes, int t, uint8_t mode, int cand, int fitted, int raw,
                                         uint32_t plane_tile, uint32_t kref, float4 plane) {
    const uint32_t w0 = (uint32_t)mode | ((uint32_t)cand << 8) | ((uint32_t)fitted << 16) | ((uint32_t)raw << 24);
    uint4 *dst = reinterpret_cast<uint4 *>(codes + t);
    dst[0] = make_uint4(w0, plane_tile, kref, 0u);
    dst[1] = make_uint4(__float_as_uint(plane.x), __float_as_uint(plane.y), __float_as_uint(plane.z),
                        __float_as_uint(plane.w));
}

__device__ __forceinline__ uint32_t warp_incl_sum(uint32_t x, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    return x;
}

constexpr int kMergeThreads = 256;

// One block per tile row (the row lives in dynamic shared memory).  Stages:
// (A) all threads stage the row's fit records; (B) the next fitted tile at or after every position
// (suffix scan, warp 0), for every fitted tile how far its run would reach by
// the followers' look-behind bits (all threads, branch-free), and where the
// walk goes next from it when that run ends inside the look-behind horizon;
// (C) all threads walk the greedy chain together: one shared-memory load per
// run that ends inside the horizon; past it, block-wide steps test one tile
// per kEL lanes against the run's plane (the staged variant loads the row's
// ranges and ray directions into shared memory on the first such step); (D) all threads assign codes and
// counts, then a block scan gives the intra-row stream offsets and the row
// totals; (E) the last block of a frame to finish lays out the frame's
// stream from the row totals (scan_frame).
template <int TH_, int TW_, bool kStage>
__global__ void __launch_bounds__(kMergeThreads) k_merge(Geometry g, Scratch s, Batch b) {
    extern __shared__ __align__(16) uint8_t smem[];
    constexpr int PX = TH_ * TW_;
    constexpr int kEL = PX >= 64 ? 8 : 4;              // lanes per tile in an extension step
    constexpr int kStepTiles = kMergeThreads / kEL;    // tiles tested per extension step
    const int TC = g.TC;
    RowRec *row = reinterpret_cast<RowRec *>(smem);
    uint16_t *nextstart = reinterpret_cast<uint16_t *>(row + TC); // next run start (fitted or temporal tile), TC + 1 entries
    uint16_t *runend = nextstart + (TC + 1);                         // end of the run started at c, 0 if none
    uint16_t *reach = runend + TC;                                 // look-behind reach of a fitted tile
    uint16_t *jmp = reach + TC;                                    // walk successor of a fitted tile (below)
    uint8_t *extcnt = reinterpret_cast<uint8_t *>(jmp + TC);       // counts of explicitly tested joins
    // staged tile row for extension steps (kStage): range bits per tile (stride PX + 1), the
    // row's column directions and its TH_ row directions
    uint32_t *s_r = reinterpret_cast<uint32_t *>(smem + merge_stage_offset(TC));
    float *s_ct = reinterpret_cast<float *>(s_r + (size_t)TC * (PX + 1));
    float *s_st = s_ct + (size_t)TC * TW_;
    float *s_ce = s_st + (size_t)TC * TW_;
    float *s_se = s_ce + TH_;
    __shared__ uint32_t s_warp[kMergeThreads / 32][6];
    __shared__ uint32_t s_carry[6];
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int f = blockIdx.y;
    const int tr = blockIdx.x;
    const size_t slot = (size_t)b.slot[f];
    const TileRec *recs = s.tiles + slot * g.NT;
    TileCode *codes = s.codes + slot * g.NT;
    TileOff *offs = s.offs + slot * g.NT;
    const uint32_t *rimg = s.rimg + slot * g.H * g.W;
    float4 *kfo = (b.kind == 0) ? b.kf_out[f] : nullptr;
    const int row0 = tr * TC;
    const int hzmax = g.merge ? g.lookahead : 0;

    // (A) stage the row's records (coalesced 16-byte loads)
    for (int c = tid; c < TC; c += kMergeThreads) {
        const uint4 *src = reinterpret_cast<const uint4 *>(recs + row0 + c);
        const uint4 q0 = src[0], q2 = src[2], q3 = src[3];
        RowRec h;
        h.plane = make_float4(__uint_as_float(q0.x), __uint_as_float(q0.y), __uint_as_float(q0.z), __uint_as_float(q0.w));
        h.amask = q2.y;
        h.status = (uint8_t)(q2.z & 0xff);
        h.rounds = (uint8_t)((q2.z >> 8) & 0xff);
        h.flags = (uint8_t)((q2.z >> 16) & 0xff);
        h.n_valid = (uint8_t)(q2.z >> 24);
        h.n_inlier = (uint8_t)(q2.w & 0xff);
        h.pad0 = h.pad1 = h.pad2 = 0;
        h.kref = q2.x;
        h.acnt[0] = q3.x; h.acnt[1] = q3.y; h.acnt[2] = q3.z; h.acnt[3] = q3.w;
        row[c] = h;
        runend[c] = 0;
        extcnt[c] = 0;
    }
    if (tid < 6) s_carry[tid] = 0;
    __syncthreads();
    // (B) reach of every run start (a fitted tile, or a temporal one): 1 + the number of its
    // followers, from the next one on, whose look-behind bit for it is set (for a spatial start:
    // and that are not temporal; a temporal start without temporal runs keeps to itself); next
    // start at or after c
    for (int c = tid; c < TC; c += kMergeThreads) {
        int k = c + 1;
        const uint8_t sc = row[c].status;
        if (sc == S_FIT || (sc == S_TEMPORAL && g.truns)) {
            const bool temp = sc == S_TEMPORAL;
            const int hz = min(hzmax, TC - 1 - c);
            uint32_t m = 0u;
#pragma unroll 4
            for (int j = 0; j < hz; j++) {
                // amask and the status byte of follower c + 1 + j in one 8-byte load
                const uint2 w = *reinterpret_cast<const uint2 *>(&row[c + 1 + j].amask);
                if (((w.x >> j) & 1u) && (temp || (w.y & 0xffu) != S_TEMPORAL)) m |= 1u << j;
            }
            k += (m == 0xFFFFFFFFu) ? 32 : __ffs(~m) - 1;   // consecutive joins from j = 0
        }
        reach[c] = (uint16_t)k;
    }
    if (warp == 0) {
        uint32_t carry = (uint32_t)TC;
        if (lane == 0) nextstart[TC] = (uint16_t)TC;
        for (int base = ((TC - 1) / 32) * 32; base >= 0; base -= 32) {
            const int c = base + lane;
            uint32_t v = (c < TC && (row[c].status == S_FIT || row[c].status == S_TEMPORAL)) ? (uint32_t)c : 0xFFFFu;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_down_sync(FULL, v, off);
                if (lane + off < 32) v = min(v, y);
            }
            v = min(v, carry);
            if (c < TC) nextstart[c] = (uint16_t)v;
            carry = __shfl_sync(FULL, v, 0);
        }
    }
    __syncthreads();
    // walk successor of every fitted tile c: where the walk goes after a run started at c that
    // ends inside the look-behind horizon (the next fitted tile at or after its reach, TC at the
    // row end), or the reach itself with bit 15 set when the run reaches past the horizon and
    // must be extended by explicit tests (TC < 32768: the row records fit in shared memory)
    for (int c = tid; c < TC; c += kMergeThreads) {
        const uint8_t sc = row[c].status;
        if (sc != S_FIT && sc != S_TEMPORAL) continue;
        const int k = reach[c];
        const bool open = g.merge && k < TC && k - c - 1 >= hzmax && (sc == S_FIT || g.truns);
        jmp[c] = open ? (uint16_t)(0x8000 | k) : (uint16_t)(k < TC ? nextstart[k] : TC);
    }
    __syncthreads();
    // (C) the greedy walk.  Warp 0 follows the chain through the runs that end inside the
    // look-behind horizon (one shared-memory load per run) and hands the block the first run
    // that reaches past it; there the whole block tests the next kStepTiles tiles against the
    // run's plane in one step, kEL lanes per tile, and the walk resumes after the run.
    {
        __shared__ uint32_t s_fail[kMergeThreads / 32];
        __shared__ int s_walk;   // walk position handed from warp 0 to the block
        bool staged = false;
        int st = nextstart[0];
        for (;;) {
            if (warp == 0) {
                while (st < TC) {
                    const uint32_t jv = jmp[st];
                    if (jv & 0x8000u) break;
                    if (lane == 0) runend[st] = reach[st];
                    st = (int)jv;
                }
                if (lane == 0) s_walk = st;
            }
            __syncthreads();
            st = s_walk;
            if (st >= TC) break;
            int k = (int)(jmp[st] & 0x7FFFu);
            bool open = true;
            if (kStage && !staged) {
                // the tile row's ranges, per tile in raster order (stride PX + 1), and its ray directions;
                // 16-byte loads, eight in flight per thread, when image rows are whole 16-byte groups
                // (loaded once per row, by the first run that reaches past the look-behind horizon)
                const int rowpx = TC * TW_;   // TW_ is a multiple of 4
                if ((g.W & 3) == 0) {
                    const int q4 = rowpx / 4, nvec = TH_ * q4;
                    constexpr int U = 8;
                    for (int v0 = tid; v0 < nvec; v0 += kMergeThreads * U) {
                        uint4 q[U];
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            const int v = v0 + u * kMergeThreads;
                            q[u] = make_uint4(kEmptyBits, kEmptyBits, kEmptyBits, kEmptyBits);
                            if (v < nvec) {
                                const int i = tr * TH_ + v / q4, jj = (v % q4) * 4;
                                if (i < g.H && jj < g.W) q[u] = __ldg(reinterpret_cast<const uint4 *>(rimg + (size_t)i * g.W + jj));
                            }
                        }
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            const int v = v0 + u * kMergeThreads;
                            if (v < nvec) {
                                const int ii = v / q4, jj = (v % q4) * 4;
                                uint32_t *d = s_r + (jj / TW_) * (PX + 1) + ii * TW_ + jj % TW_;
                                d[0] = q[u].x; d[1] = q[u].y; d[2] = q[u].z; d[3] = q[u].w;
                            }
                        }
                    }
                } else {
                    for (int idx = tid; idx < TH_ * rowpx; idx += kMergeThreads) {
                        const int ii = idx / rowpx, jj = idx % rowpx;
                        const int i = tr * TH_ + ii;
                        s_r[(jj / TW_) * (PX + 1) + ii * TW_ + jj % TW_] =
                            (i < g.H && jj < g.W) ? __ldg(rimg + (size_t)i * g.W + jj) : kEmptyBits;
                    }
                }
                for (int jj = tid; jj < rowpx; jj += kMergeThreads) {
                    s_ct[jj] = jj < g.W ? __ldg(g.ct + jj) : 0.f;
                    s_st[jj] = jj < g.W ? __ldg(g.st + jj) : 0.f;
                }
                if (tid < TH_) {
                    const int i = tr * TH_ + tid;
                    s_ce[tid] = i < g.H ? __ldg(g.ce + i) : 0.f;
                    s_se[tid] = i < g.H ? __ldg(g.se + i) : 0.f;
                }
                __syncthreads();
                staged = true;
            }
            {
                const float4 pl = row[st].plane;
                const bool trun = row[st].status == S_TEMPORAL;   // a temporal run joins any tile
                while (open) {
                    const int c2 = k + tid / kEL, l = tid % kEL;
                    const bool cand = c2 < TC && (trun || row[c2].status != S_TEMPORAL);
                    int nin = 0;
                    if (cand) {
                        bool border = false;
#pragma unroll 4
                        for (int q = l; q < PX; q += kEL) {
                            const int ii = q / TW_, jj = c2 * TW_ + q % TW_;
                            uint32_t bits;
                            float ux, uy, uz;
                            if (kStage) {
                                bits = s_r[c2 * (PX + 1) + q];
                                const float ce = s_ce[ii];
                                ux = __fmul_rn(ce, s_ct[jj]);
                                uy = __fmul_rn(ce, s_st[jj]);
                                uz = s_se[ii];
                            } else {
                                const int i = tr * TH_ + ii;
                                bits = (i < g.H && jj < g.W) ? __ldg(rimg + (size_t)i * g.W + jj) : kEmptyBits;
                                if (bits_valid(bits)) beam(g, i, jj, ux, uy, uz);
                            }
                            if (bits_valid(bits))
                                nin += inlier_screened(pl, ux, uy, uz, __uint_as_float(bits), g.thr, border) ? 1 : 0;
                        }
                    }
#pragma unroll
                    for (int off = kEL / 2; off; off >>= 1) nin += __shfl_xor_sync(FULL, nin, off);
                    const int nvv = cand ? (int)row[c2].n_valid : 0;
                    const bool pass = cand && nvv >= 3 && nin >= need_inliers(g.fmin, nvv);
                    const uint32_t failb = __ballot_sync(FULL, !pass);
                    if (lane == 0) s_fail[warp] = failb;
                    __syncthreads();
                    int nj = kStepTiles;
#pragma unroll
                    for (int w = kMergeThreads / 32 - 1; w >= 0; w--)
                        if (s_fail[w]) nj = (w * 32 + __ffs(s_fail[w]) - 1) / kEL;
                    __syncthreads();   // s_fail is rewritten by the next step
                    if (l == 0 && tid / kEL < nj) extcnt[c2] = (uint8_t)nin;
                    k += nj;
                    open = nj == kStepTiles && k < TC;
                }
            }
            if (tid == 0) runend[st] = (uint16_t)k;
            st = k < TC ? nextstart[k] : TC;
            __syncthreads();   // every thread has read s_walk before warp 0 writes it again
        }
    }
    __syncthreads();
    // (D) codes, counts and intra-row offsets (block scan in chunks of the block size)
    uint32_t hist[6] = {0u, 0u, 0u, 0u, 0u, 0u}, rhist[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u}, border = 0;
    __shared__ int s_wmax[kMergeThreads / 32];
    __shared__ int s_last;
    if (tid == 0) s_last = -1;
    __syncthreads();
    for (int base = 0; base < TC; base += kMergeThreads) {
        const int c = base + tid;
        uint32_t v[6] = {0u, 0u, 0u, 0u, 0u, 0u};   // cand, fitted, raw, run, temporal, valid
        // the run covering c (if any) starts at the last run start at or before c:
        // block-wide inclusive max-scan of the start positions, carried across chunks
        const bool isstart = c < TC && runend[c] != 0;
        int stc = isstart ? c : -1;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(FULL, stc, off);
            if (lane >= off) stc = max(stc, y);
        }
        if (lane == 31) s_wmax[warp] = stc;
        __syncthreads();
        int pre = s_last;
        for (int w = 0; w < warp; w++) pre = max(pre, s_wmax[w]);
        stc = max(stc, pre);
        if (c < TC) {
            const RowRec &h = row[c];
            if (!isstart && (stc < 0 || c >= (int)runend[stc])) stc = -1;
            uint32_t cand = 0, fit = 0, raw = 0, ptile = (uint32_t)(row0 + c);
            uint8_t mode;
            if (isstart) {   // a run start: its own spatial plane, or its relaxed plane (temporal)
                mode = h.status == S_TEMPORAL ? T_TEMPORAL : T_RUN_START;
                cand = h.n_valid;
                fit = h.n_inlier;
            } else if (stc >= 0) {
                mode = row[stc].status == S_TEMPORAL ? T_TEMPORAL_CONT : T_RUN_CONT;
                const int j = c - stc - 1;
                cand = h.n_valid;
                fit = j < hzmax ? (uint32_t)s.lbcnt[(slot * g.NT + row0 + c) * 32 + j] : extcnt[c];
                ptile = (uint32_t)(row0 + stc);
            } else {
                mode = h.n_valid ? T_RAW : T_EMPTY;
                raw = h.n_valid;
            }
            if (mode >= T_RUN_START) raw = cand - fit;
            const float4 cpl = mode >= T_RUN_START ? row[stc].plane : make_float4(0.f, 0.f, 0.f, 0.f);
            put_code(codes, row0 + c, mode, (int)cand, (int)fit, (int)raw, ptile, h.kref, cpl);
            if (kfo) kfo[row0 + c] = (mode == T_RUN_START || mode == T_RUN_CONT) ? cpl : make_float4(0.f, 0.f, 0.f, 0.f);
            v[0] = cand; v[1] = fit; v[2] = raw; v[3] = mode == T_RUN_START; v[4] = mode == T_TEMPORAL;
            v[5] = h.n_valid;
            hist[mode]++;
            rhist[min((uint32_t)h.rounds, 7u)]++;
            border += h.flags & 1u;
        }
        uint32_t inc[6];
#pragma unroll
        for (int q = 0; q < 6; q++) inc[q] = warp_incl_sum(v[q], lane);
        if (lane == 31)
#pragma unroll
            for (int q = 0; q < 6; q++) s_warp[warp][q] = inc[q];
        __syncthreads();
        uint32_t wb[6] = {0u, 0u, 0u, 0u, 0u, 0u};
        for (int w = 0; w < warp; w++)
#pragma unroll
            for (int q = 0; q < 6; q++) wb[q] += s_warp[w][q];
        if (c < TC) {
            uint4 *dst = reinterpret_cast<uint4 *>(offs + row0 + c);
            dst[0] = make_uint4(s_carry[0] + wb[0] + inc[0] - v[0], s_carry[1] + wb[1] + inc[1] - v[1],
                                s_carry[2] + wb[2] + inc[2] - v[2], s_carry[3] + wb[3] + inc[3] - v[3]);
            dst[1] = make_uint4(s_carry[4] + wb[4] + inc[4] - v[4], 0u, 0u, 0u);
        }
        __syncthreads();
        if (tid < 6) {
            uint32_t t6 = 0;
            for (int w = 0; w < kMergeThreads / 32; w++) t6 += s_warp[w][tid];
            s_carry[tid] += t6;
        }
        if (tid == kMergeThreads - 1) {
            int m = s_last;
            for (int w = 0; w < kMergeThreads / 32; w++) m = max(m, s_wmax[w]);
            s_last = m;
        }
        __syncthreads();
    }
    uint32_t *tot = s.rowtot + (slot * g.TR + tr) * 8;
    if (tid < 6) tot[tid] = s_carry[tid];
    // tile statistics (A11): warp reductions, one atomic per counter and warp
#pragma unroll
    for (int off = 16; off; off >>= 1) {
#pragma unroll
        for (int q = 0; q < 6; q++) hist[q] += __shfl_xor_sync(FULL, hist[q], off);
#pragma unroll
        for (int q = 0; q < 8; q++) rhist[q] += __shfl_xor_sync(FULL, rhist[q], off);
        border += __shfl_xor_sync(FULL, border, off);
    }
    if (lane == 0) {
        DevStats *stt = s.stats + slot;
        for (int q = 0; q < 6; q++)   // empty, raw, run start, run continuation, temporal, temporal continuation
            if (hist[q]) atomicAdd(&(&stt->empty)[q], (unsigned long long)hist[q]);
        for (int q = 0; q < 8; q++)
            if (rhist[q]) atomicAdd(&stt->rounds[q], (unsigned long long)rhist[q]);
        if (border) atomicAdd(&stt->borderline, (unsigned long long)border);
    }
    // (E) the last tile row of the frame to finish (the classic fence + counter pattern)
    __shared__ int s_lastrow;
    __threadfence();
    __syncthreads();
    if (tid == 0) s_lastrow = atomicAdd(s.rowdone + slot, 1u) == (unsigned)g.TR - 1u;
    __syncthreads();
    if (s_lastrow) {
        __threadfence();
        scan_frame<kMergeThreads>(g, s, b, f);
        if (tid == 0) s.rowdone[slot] = 0u;   // ready for the next frame in this slot
    }
}

size_t merge_smem_bytes(int TC) { return merge_stage_offset(TC); }

size_t merge_stage_bytes(int TC, int th, int tw) {
    return 4 * ((size_t)TC * (th * tw + 1) + 2 * (size_t)TC * tw + 2 * (size_t)th);
}

template <int TH_, int TW_, bool kStage>
static cudaError_t launch_merge_v(const Geometry &g, const Scratch &s, const Batch &b, size_t smem, cudaStream_t st) {
    // above 48 KB of shared memory per block, counting the kernel's own static arrays (a few
    // hundred bytes) with the dynamic part, a launch needs the opt-in
    if (smem + 4096 > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_merge<TH_, TW_, kStage>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_merge<TH_, TW_, kStage><<<dim3(g.TR, b.nframes), kMergeThreads, smem, st>>>(g, s, b);
    return cudaGetLastError();
}

// The staged variant keeps the tile row's ranges and directions in shared memory for the
// extension steps; rows too wide for that read them from L2 instead.
template <int TH_, int TW_>
static cudaError_t launch_merge_t(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st) {
    const size_t base = merge_stage_offset(g.TC);
    const size_t staged = base + merge_stage_bytes(g.TC, TH_, TW_);
    if (staged <= kMergeStageMaxSmem) return launch_merge_v<TH_, TW_, true>(g, s, b, staged, st);
    return launch_merge_v<TH_, TW_, false>(g, s, b, base, st);
}

cudaError_t launch_merge(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st) {
    if (b.nframes <= 0) return cudaSuccess;
    if (g.th == 4 && g.tw == 4) return launch_merge_t<4, 4>(g, s, b, st);
    if (g.th == 4 && g.tw == 8) return launch_merge_t<4, 8>(g, s, b, st);
    if (g.th == 8 && g.tw == 8) return launch_merge_t<8, 8>(g, s, b, st);
    if (g.th == 8 && g.tw == 16) return launch_merge_t<8, 16>(g, s, b, st);
    return cudaErrorInvalidValue;
}

}  // namespace lcc
