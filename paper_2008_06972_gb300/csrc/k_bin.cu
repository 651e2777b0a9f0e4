// Range-image conversion (Sec. III-B, Eq. 1-2) with the nearest-point
// collision rule (Sec. III-D).
//
// One thread per point: a streaming, coalesced 16-byte float4 load, fp32
// range and boundary sign tests (no transcendental decides a bin), then a
// 32-bit atomicMin of the range's bit pattern into the frame's range image.
// Positive finite floats order like their bit patterns, so the minimum bit
// pattern is the nearest point; the empty pixel is 0xFFFFFFFF.
#include "lcc_internal.cuh"

namespace lcc {

constexpr int kBinThreads = 256;
constexpr int kBinPerThread = 4;

// Chunk cb of kBinThreads * kBinPerThread points (chunks are numbered over the batch's
// frames, blk_prefix[f] = first chunk of frame f); a CTA takes chunks blockIdx.x,
// blockIdx.x + gridDim.x, ... so that a capped grid covers them all.
__global__ void __launch_bounds__(kBinThreads) k_bin(Geometry g, Scratch s, Batch b, long long chunks) {
    __shared__ int s_frame;
    __shared__ unsigned s_cnt[kBinThreads / 32][3];
    for (long long cb = blockIdx.x; cb < chunks; cb += gridDim.x) {
        __syncthreads();   // s_frame of the previous chunk has been read by every thread
        if (threadIdx.x == 0) {
            int f = 0;
            while (f + 1 < b.nframes && b.blk_prefix[f + 1] <= cb) f++;
            s_frame = f;
        }
        __syncthreads();
        const int f = s_frame;
        const long long n = b.n[f];
        const long long base = (cb - b.blk_prefix[f]) * (kBinThreads * kBinPerThread);
        uint32_t *rimg = s.rimg + (size_t)b.slot[f] * g.H * g.W;
        const float4 *pts = b.pts[f];
        unsigned invalid = 0, fov = 0, binned = 0;
#pragma unroll
        for (int k = 0; k < kBinPerThread; k++) {
            const long long idx = base + (long long)k * kBinThreads + threadIdx.x;
            if (idx < n) {
                const float4 p = __ldcs(pts + idx);
                float r;
                int pix;
                const int res = bin_point(g, p.x, p.y, p.z, r, pix);
                if (res == 0) {
                    atomicMin(rimg + pix, __float_as_uint(r));
                    binned++;
                } else if (res == 1) {
                    invalid++;
                } else {
                    fov++;
                }
            }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
            invalid += __shfl_xor_sync(0xffffffffu, invalid, off);
            fov += __shfl_xor_sync(0xffffffffu, fov, off);
            binned += __shfl_xor_sync(0xffffffffu, binned, off);
        }
        // one set of counter updates per chunk: the frame's counters are shared by all its chunks
        if ((threadIdx.x & 31) == 0) {
            s_cnt[threadIdx.x >> 5][0] = invalid;
            s_cnt[threadIdx.x >> 5][1] = fov;
            s_cnt[threadIdx.x >> 5][2] = binned;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            unsigned long long v = 0;
#pragma unroll
            for (int w = 0; w < kBinThreads / 32; w++) v += s_cnt[w][threadIdx.x];
            DevStats *st = s.stats + b.slot[f];
            unsigned long long *dst = threadIdx.x == 0 ? &st->invalid : (threadIdx.x == 1 ? &st->fov : &st->binned);
            if (v) atomicAdd(dst, v);
            if (threadIdx.x == 0 && base == 0) atomicAdd(&st->points_in, (unsigned long long)n);
        }
    }
}

cudaError_t launch_bin(const Geometry &g, const Scratch &s, const Batch &b, long long total_blocks,
                       cudaStream_t st, long long max_blocks) {
    if (total_blocks <= 0) return cudaSuccess;
    const long long grid = max_blocks > 0 && total_blocks > max_blocks ? max_blocks : total_blocks;
    k_bin<<<(unsigned)grid, kBinThreads, 0, st>>>(g, s, b, total_blocks);
    return cudaGetLastError();
}

// Export of a range image: fp32 range (0 = empty), occupancy bitmap, and the
// pixel is reset to empty for the next frame.
__global__ void __launch_bounds__(256) k_range_export(Geometry g, uint32_t *rimg, float *range, uint32_t *valid) {
    const long long npx = (long long)g.H * g.W;
    const long long p = (long long)blockIdx.x * 256 + threadIdx.x;
    const uint32_t bits = p < npx ? rimg[p] : kEmptyBits;
    const bool v = bits_valid(bits);
    if (p < npx) {
        if (range) range[p] = v ? __uint_as_float(bits) : 0.0f;
        rimg[p] = kEmptyBits;
    }
    const uint32_t word = __ballot_sync(0xffffffffu, v);
    if (valid && (threadIdx.x & 31) == 0 && p < npx) valid[p >> 5] = word;
}

cudaError_t launch_range_image(const Geometry &g, const uint32_t *rimg, float *range, uint32_t *valid,
                               cudaStream_t st) {
    const long long npx = (long long)g.H * g.W;
    k_range_export<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(g, const_cast<uint32_t *>(rimg), range, valid);
    return cudaGetLastError();
}

}  // namespace lcc
