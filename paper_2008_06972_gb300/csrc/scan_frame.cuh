// Stream layout of one frame, run by the last block of the run merge to finish
// a frame (the rows' totals are final then).
#pragma once

#include "lcc_internal.cuh"

namespace lcc {

constexpr int kScanVals = 6;

__device__ __forceinline__ uint32_t words_for(uint64_t bits) { return (uint32_t)((bits + 31) >> 5); }

// Per frame: exclusive prefix of the tile-row totals (cand, fitted, raw, run
// starts, temporal tiles, valid pixels) gives every row its base offset in
// each section; the frame totals give the section layout, the header and the
// capacity check.  The block then zeroes the frame's output words so the packer
// can OR bits in.  Called by all kScanThreads threads of one block.
template <int kScanThreads>
__device__ __forceinline__ void scan_frame(const Geometry &g, const Scratch &s, const Batch &b, int f) {
    const size_t slot = (size_t)b.slot[f];
    const uint32_t *rowtot = s.rowtot + slot * g.TR * 8;
    uint32_t *rowbase = s.rowbase + slot * g.TR * 8;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kScanThreads / 32;

    __shared__ uint32_t s_warp[NW][kScanVals];
    __shared__ uint32_t s_carry[kScanVals];
    __shared__ uint32_t s_ok, s_total;
    if (tid < kScanVals) s_carry[tid] = 0;
    __syncthreads();

    for (int base = 0; base < g.TR; base += kScanThreads) {
        const int r = base + tid;
        uint32_t v[kScanVals] = {0, 0, 0, 0, 0, 0};
        if (r < g.TR)
#pragma unroll
            for (int q = 0; q < kScanVals; q++) v[q] = __ldcg(rowtot + r * 8 + q);   // written by other blocks
        uint32_t inc[kScanVals];
#pragma unroll
        for (int q = 0; q < kScanVals; q++) {
            uint32_t x = v[q];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += y;
            }
            inc[q] = x;
        }
        if (lane == 31)
#pragma unroll
            for (int q = 0; q < kScanVals; q++) s_warp[warp][q] = inc[q];
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < kScanVals; q++) {
                uint32_t x = lane < NW ? s_warp[lane][q] : 0u;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
                    if (lane >= off) x += y;
                }
                if (lane < NW) s_warp[lane][q] = x;   // inclusive over warps
            }
        }
        __syncthreads();
        if (r < g.TR)
#pragma unroll
            for (int q = 0; q < kScanVals; q++)
                rowbase[r * 8 + q] = s_carry[q] + (warp ? s_warp[warp - 1][q] : 0u) + inc[q] - v[q];
        __syncthreads();
        if (tid < kScanVals) s_carry[tid] += s_warp[NW - 1][tid];
        __syncthreads();
    }

    if (tid == 0) {
        const uint32_t cand = s_carry[0], fitted = s_carry[1], raw = s_carry[2], runs = s_carry[3],
                       temporal = s_carry[4], valid = s_carry[5];
        FrameLayout L;
        L.sec[0] = 0;
        L.sec[1] = L.sec[0] + words_for((uint64_t)g.H * g.W);
        L.sec[2] = L.sec[1] + words_for((uint64_t)g.NT * 4);
        L.sec[3] = L.sec[2] + (g.plane3 ? 3u : 4u) * runs;   // three-coefficient planes: 3 words a run
        L.sec[4] = L.sec[3] + 2u * temporal;
        L.sec[5] = L.sec[4] + words_for(cand);
        L.sec[6] = L.sec[5] + (g.no_delta ? 0u : words_for((uint64_t)fitted * g.w_res));   // no deltas: none
        L.sec[7] = L.sec[6] + words_for((uint64_t)raw * g.w_raw);
        const unsigned long long total = (unsigned long long)kHeaderBytes + 4ull * L.sec[7];
        L.total_bytes = (uint32_t)total;
        L.ok = total <= b.cap[f] ? 1u : 0u;
        L.n_valid = valid;
        L.pad = 0;
        s.layout[slot] = L;
        s.bytes[slot] = total;
        if (b.nbytes_out[f]) *b.nbytes_out[f] = total;
        if (!L.ok) atomicOr(s.err, E_CAPACITY);
        s_ok = L.ok;
        s_total = L.total_bytes;
        if (L.ok) {
            uint32_t hw[16];
            hw[0] = kMagic;
            hw[1] = (uint32_t)kVersion | ((uint32_t)b.kind << 16) | ((uint32_t)(g.merge ? 1 : 0) << 24) |
                    ((uint32_t)(g.no_delta ? 1 : 0) << 25) | ((uint32_t)(g.raw_exact ? 1 : 0) << 26) |
                    ((uint32_t)(g.truns && b.kind == 1 ? 1 : 0) << 27) | ((uint32_t)(g.plane3 ? 1 : 0) << 28);
            hw[2] = (uint32_t)g.H | ((uint32_t)g.W << 16);
            hw[3] = (uint32_t)g.th | ((uint32_t)g.tw << 8) | ((uint32_t)g.w_res << 16) | ((uint32_t)g.w_raw << 24);
            hw[4] = __float_as_uint(g.thr);
            hw[5] = __float_as_uint(g.q);
            hw[6] = (uint32_t)g.NT;
            hw[7] = valid;
            hw[8] = runs;
            hw[9] = temporal;
            hw[10] = cand;
            hw[11] = fitted;
            hw[12] = raw;
            hw[13] = (uint32_t)g.k_max;
            hw[14] = L.total_bytes;
            hw[15] = 0;
            uint4 *o = reinterpret_cast<uint4 *>(b.out[f]);
            for (int q = 0; q < 4; q++) o[q] = make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
        }
        DevStats *st = s.stats + slot;
        st->valid = valid;
        st->cand = cand;
        st->fitted = fitted;
        st->raw = raw;
        st->bytes = total;
    }
    __syncthreads();
    if (s_ok) {
        // zero everything after the header: 16-byte stores then the tail words
        const uint32_t nw = (s_total - kHeaderBytes) / 4;
        uint4 *o4 = reinterpret_cast<uint4 *>(b.out[f] + kHeaderBytes);
        for (uint32_t q = tid; q < nw / 4; q += kScanThreads) o4[q] = make_uint4(0u, 0u, 0u, 0u);
        uint32_t *o1 = reinterpret_cast<uint32_t *>(b.out[f] + kHeaderBytes);
        for (uint32_t q = (nw / 4) * 4 + tid; q < nw; q += kScanThreads) o1[q] = 0u;
    }
}

}  // namespace lcc
