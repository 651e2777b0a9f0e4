// Greedy horizontal run growth (Sec. III-C) — one warp per tile row.
//
// The paper grows a run of tiles to the right while the plane "fit so far"
// (the run's first plane) still codes the next tile under the threshold, and
// restarts at the first tile that fails.  The walk is sequential along a row,
// so each step is made warp-wide: the 32 lanes look at 32 consecutive tiles,
// a ballot finds the first candidate run start, the precomputed look-behind
// bits of the following tiles (from the fit stage) decide the first
// `lookahead` joins,
// and only runs longer than that test further tiles explicitly, 32 tiles per
// step with one lane per tile.  Temporal tiles of P frames are already coded
// (Sec. III-D) and end a run.
//
// Output per tile: its stream mode, the tile whose plane codes it, and its
// counts of candidate / plane-coded / raw-coded pixels.
#include "lcc_internal.cuh"

namespace lcc {

// Per-tile fields of one tile row, staged in shared memory so that each walk
// step costs shared-memory latency instead of a dependent L2 round trip.
struct alignas(16) RowRec {
    float4 plane;
    uint32_t amask;
    uint8_t status, n_valid, n_inlier, pad;
    uint32_t acnt[4];
};

__device__ __forceinline__ void put_code(TileCode *codes, int t, uint8_t mode, int cand, int fitted, int raw,
                                         uint32_t plane_tile) {
    const uint32_t w0 = (uint32_t)mode | ((uint32_t)cand << 8) | ((uint32_t)fitted << 16) | ((uint32_t)raw << 24);
    *reinterpret_cast<uint2 *>(codes + t) = make_uint2(w0, plane_tile);
}

// Code of a tile that is not part of a spatial run.
__device__ __forceinline__ void put_plain(TileCode *codes, float4 *kfo, int t, const RowRec &h) {
    if (h.status == S_TEMPORAL)
        put_code(codes, t, T_TEMPORAL, h.n_valid, h.n_inlier, h.n_valid - h.n_inlier, (uint32_t)t);
    else
        put_code(codes, t, h.n_valid ? T_RAW : T_EMPTY, 0, 0, h.n_valid, (uint32_t)t);
    if (kfo) kfo[t] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// One warp per tile row (one warp per block; the row lives in dynamic shared memory).
template <int TH_, int TW_>
__global__ void __launch_bounds__(32) k_merge(Geometry g, Scratch s, Batch b) {
    extern __shared__ RowRec row[];
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x;
    const int f = blockIdx.y;
    const int tr = blockIdx.x;
    const size_t slot = (size_t)b.slot[f];
    const TileRec *recs = s.tiles + slot * g.NT;
    TileCode *codes = s.codes + slot * g.NT;
    const uint32_t *rimg = s.rimg + slot * g.H * g.W;
    float4 *kfo = (b.kind == 0) ? b.kf_out : nullptr;
    const int row0 = tr * g.TC;

    // stage the row's records (coalesced 16-byte loads)
    for (int c = lane; c < g.TC; c += 32) {
        const uint4 *src = reinterpret_cast<const uint4 *>(recs + row0 + c);
        const uint4 q0 = src[0], q2 = src[2], q3 = src[3];
        RowRec h;
        h.plane = make_float4(__uint_as_float(q0.x), __uint_as_float(q0.y), __uint_as_float(q0.z), __uint_as_float(q0.w));
        h.amask = q2.y;
        h.status = (uint8_t)(q2.z & 0xff);
        h.n_valid = (uint8_t)(q2.z >> 24);
        h.n_inlier = (uint8_t)(q2.w & 0xff);
        h.pad = 0;
        h.acnt[0] = q3.x; h.acnt[1] = q3.y; h.acnt[2] = q3.z; h.acnt[3] = q3.w;
        row[c] = h;
    }
    __syncwarp();

    int j = 0;
    while (j < g.TC) {
        const int c = j + lane;
        const bool inrow = c < g.TC;
        const uint8_t st = inrow ? row[c].status : (uint8_t)S_EMPTY;
        const uint32_t fitb = __ballot_sync(FULL, inrow && st == S_FIT);
        const int first = fitb ? __ffs(fitb) - 1 : 32;
        if (inrow && lane < first) put_plain(codes, kfo, row0 + c, row[c]);
        if (!fitb) {
            j += 32;
            continue;
        }
        const int s0 = j + first;
        const RowRec &start = row[s0];
        const float4 pl = start.plane;
        if (lane == first) {
            put_code(codes, row0 + s0, T_RUN_START, start.n_valid, start.n_inlier, start.n_valid - start.n_inlier,
                     (uint32_t)(row0 + s0));
            if (kfo) kfo[row0 + s0] = pl;
        }
        int k = s0 + 1;
        bool open = g.merge && k < g.TC;
        // phase 1: joins decided by the precomputed look-behind bits
        const int hz = g.merge ? min(g.lookahead, g.TC - 1 - s0) : 0;
        if (hz > 0) {
            const int c1 = s0 + 1 + lane;
            bool pass = false;
            int cnt = 0, nv1 = 0;
            if (lane < hz) {
                // tile c1's look-behind bit `lane` refers to the plane of tile c1-1-lane = s0
                const RowRec &h1 = row[c1];
                pass = ((h1.amask >> lane) & 1u) && h1.status != S_TEMPORAL;
                cnt = (h1.acnt[lane >> 2] >> (8 * (lane & 3))) & 0xff;
                nv1 = h1.n_valid;
            }
            const uint32_t failb = __ballot_sync(FULL, lane < hz && !pass);
            const int nj = failb ? __ffs(failb) - 1 : hz;
            if (lane < nj) {
                put_code(codes, row0 + c1, T_RUN_CONT, nv1, cnt, nv1 - cnt, (uint32_t)(row0 + s0));
                if (kfo) kfo[row0 + c1] = pl;
            }
            k = s0 + 1 + nj;
            open = (failb == 0) && k < g.TC;
        }
        // phase 2: explicit tests, one tile per lane, 32 tiles per step
        while (open) {
            const int c2 = k + lane;
            bool pass = false;
            int nvv = 0, nin = 0;
            if (c2 < g.TC && row[c2].status != S_TEMPORAL) {
                for (int q = 0; q < TH_ * TW_; q++) {
                    const int i = tr * TH_ + q / TW_, jj = c2 * TW_ + q % TW_;
                    if (i >= g.H || jj >= g.W) continue;
                    const uint32_t bits = __ldg(rimg + (size_t)i * g.W + jj);
                    if (!bits_valid(bits)) continue;
                    nvv++;
                    float ux, uy, uz, e;
                    beam(g, i, jj, ux, uy, uz);
                    nin += residual(pl, ux, uy, uz, __uint_as_float(bits), g.thr, e) ? 1 : 0;
                }
                pass = nvv >= 3 && nin >= need_inliers(g.fmin, nvv);
            }
            const uint32_t failb = __ballot_sync(FULL, !pass);
            const int nj = failb ? __ffs(failb) - 1 : 32;
            if (lane < nj) {
                put_code(codes, row0 + c2, T_RUN_CONT, nvv, nin, nvv - nin, (uint32_t)(row0 + s0));
                if (kfo) kfo[row0 + c2] = pl;
            }
            k += nj;
            open = (failb == 0) && k < g.TC;
        }
        j = k;
    }
}

template <int TH_, int TW_>
static cudaError_t launch_merge_t(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st) {
    const size_t smem = sizeof(RowRec) * (size_t)g.TC;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_merge<TH_, TW_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(g.TR, b.nframes);
    k_merge<TH_, TW_><<<grid, 32, smem, st>>>(g, s, b);
    return cudaGetLastError();
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
