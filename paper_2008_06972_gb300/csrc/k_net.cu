// Learned tile proposal (not in the paper): a small convolutional net that
// predicts, for an 8x8 tile of the range image, whether the iterative plane
// fit of Sec. III-C will succeed and which plane it will find.  The encoder
// uses the prediction to seed its first fit round and to skip tiles that will
// not fit; the plain fit still decides every plane that codes points.
//
// Net: input 4x8x8 (r - r_anchor, p - p_anchor; empty pixels 0), conv3x3
// pad 1 4->32, ReLU, 32->64, ReLU, 64->64, ReLU, global average pool, linear
// 64->32, ReLU, linear 32->5 (logit, normal, offset relative to the anchor).
// BF16 operands with FP32 accumulation on the tensor cores; activations are
// rounded to BF16 after each ReLU, as are the pooled vector, the hidden head
// activation and the convolution gradients.
//
// Every convolution is an implicit GEMM: rows are pixels, columns output
// channels, and the reduction runs over the 9 taps x input channels, read
// straight from a zero-bordered 10x10 copy of the tile in shared memory (no
// im2col buffer).  The forward pass (inference and training) runs on tcgen05
// with TMEM accumulators, two tiles per 128-row MMA.  The backward pass runs
// on tcgen05 as well: the input-gradient convolution is the same GEMM with the
// taps mirrored and the channel roles swapped; the weight gradient is a GEMM
// whose reduction runs over the pixels of all tiles (one accumulator per CTA,
// summed across CTAs in a fixed order), the taps' shifts taken from where the
// staged operands start.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "lcc.h"
#include "lcc_ctx.cuh"

using namespace lcc;
using namespace lcc::api;

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kPX = 64;                       // pixels of an 8x8 tile
constexpr int C0 = 4, C1 = 32, C2 = 64, C3 = 64, HID = 32, NOUT = 5;
constexpr int K1 = 48;                        // conv1 on tcgen05 as one contraction: 9 taps x 4 channels, 3 k-steps

// offsets of the flat parameter vector: W1[32,4,3,3] b1 W2[64,32,3,3] b2 W3[64,64,3,3] b3 F1[32,64] c1 F2[5,32] c2
constexpr int OW1 = 0, OB1 = OW1 + C1 * C0 * 9, OW2 = OB1 + C1, OB2 = OW2 + C2 * C1 * 9, OW3 = OB2 + C2,
              OB3 = OW3 + C3 * C2 * 9, OF1 = OB3 + C3, OC1 = OF1 + HID * C3, OF2 = OC1 + HID, OC2 = OF2 + NOUT * HID,
              NPARAM = OC2 + NOUT;
static_assert(NPARAM == 58853, "parameter count");

// device copies of the weights in the layouts the kernels read
struct NetDev {
    const float *theta;                      // fp32 master parameters
    float *F1b, *F2b;                        // head weights rounded to bf16 values
    bf16 *T1, *T2, *T3;                      // tcgen05 B operands: [tap][ci/8][cout][8], core-matrix order
    bf16 *TB3, *TB2;                         // tcgen05 B operands of the input gradients: [tap][co/8][ci][8]
};

struct NetAct {                              // per-tile training activations
    bf16 *a1, *a2, *a3;                      // [T][64][C]
    float *g, *h, *o;                        // [T][64], [T][32], [T][5]
    float *da3c;                             // [T][64]  dL/d(pooled input) / 64
    float *hdy, *hdo, *hlt;                  // [T][32], [T][8], [T]: head gradient terms and loss per tile
    bf16 *dz1t, *dz2t, *dz3t;                // [T][C][64] pre-activation gradients, pixel-contiguous
};

__device__ __forceinline__ float bfround(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// ------------------------------------------------------------------ weights --

__global__ void k_net_prep(NetDev nd) {
    const float *th = nd.theta;
    const int total = HID * C3 + NOUT * HID;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int j = i;
        if (j < HID * C3) {
            nd.F1b[j] = bfround(th[OF1 + j]);
            continue;
        }
        j -= HID * C3;
        nd.F2b[j] = bfround(th[OF2 + j]);
    }
    // tcgen05 layouts: conv2/conv3 element (tap, c8, co, e) = W[co][ci = 8 c8 + e][tap]; conv1 is
    // one contraction over k = tap * 4 + ci (im2col, 36 of K1 = 48 used): element (c8, co, e) =
    // W1[co][ci][tap] for k = 8 c8 + e
    // the input gradients' B operands: element (tap, c8, ci, e) = W[co = 8 c8 + e][ci][8 - tap]
    const int m1 = (K1 / 8) * C1 * 8, m2 = 9 * (C1 / 8) * C2 * 8, m3 = 9 * (C2 / 8) * C3 * 8;
    const int m4 = 9 * (C3 / 8) * C2 * 8, m5 = 9 * (C2 / 8) * C1 * 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m1 + m2 + m3 + m4 + m5; i += gridDim.x * blockDim.x) {
        int j = i;
        if (j < m1) {
            const int e = j % 8, co = (j / 8) % C1, c8 = j / (8 * C1);
            const int k = 8 * c8 + e, tap = k / C0, ci = k % C0;
            nd.T1[j] = __float2bfloat16_rn(k < 9 * C0 ? th[OW1 + co * C0 * 9 + ci * 9 + tap] : 0.f);
            continue;
        }
        j -= m1;
        if (j < m2) {
            const int e = j % 8, co = (j / 8) % C2, c8 = (j / (8 * C2)) % (C1 / 8), tap = j / (8 * C2 * (C1 / 8));
            nd.T2[j] = __float2bfloat16_rn(th[OW2 + co * C1 * 9 + (8 * c8 + e) * 9 + tap]);
            continue;
        }
        j -= m2;
        if (j < m3) {
            const int e = j % 8, co = (j / 8) % C3, c8 = (j / (8 * C3)) % (C2 / 8), tap = j / (8 * C3 * (C2 / 8));
            nd.T3[j] = __float2bfloat16_rn(th[OW3 + co * C2 * 9 + (8 * c8 + e) * 9 + tap]);
            continue;
        }
        j -= m3;
        if (j < m4) {
            const int e = j % 8, ci = (j / 8) % C2, c8 = (j / (8 * C2)) % (C3 / 8), tap = j / (8 * C2 * (C3 / 8));
            nd.TB3[j] = __float2bfloat16_rn(th[OW3 + (8 * c8 + e) * C2 * 9 + ci * 9 + (8 - tap)]);
            continue;
        }
        j -= m4;
        const int e = j % 8, ci = (j / 8) % C1, c8 = (j / (8 * C1)) % (C2 / 8), tap = j / (8 * C1 * (C2 / 8));
        nd.TB2[j] = __float2bfloat16_rn(th[OW2 + (8 * c8 + e) * C1 * 9 + ci * 9 + (8 - tap)]);
    }
}

// ------------------------------------------------------------------ inputs --

// Net input of every 8x8 tile of the frames binned into slots 0.. (frame = blockIdx.y).  With
// kReset the range image is reset to empty afterwards (the standalone input call); without it the
// image stays for the encode that follows (the plan's seeded key frames, whose pack resets it).
// One warp per tile, two pixels per lane.
// The inputs of one tile (one warp, two pixels per lane); returns whether the tile has the 3
// valid pixels a fit needs (the same on every lane).
template <bool kReset>
__device__ __forceinline__ bool net_inputs_tile(const Geometry &g, uint32_t *rimg0, bf16 *x0, float4 *anchor0, int tile,
                                                int lane) {
    // frame blockIdx.y: its range image is slot blockIdx.y, its tiles follow the previous frames'
    uint32_t *rimg = rimg0 + (size_t)blockIdx.y * g.H * g.W;
    bf16 *x = x0 + (size_t)blockIdx.y * g.NT * kPX * C0;
    float4 *anchor = anchor0 + (size_t)blockIdx.y * g.NT;
    const int i0 = (tile / g.TC) * 8, j0 = (tile % g.TC) * 8;
    float r[2], p[2][3];
    bool v[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int q = lane + 32 * h, i = i0 + q / 8, j = j0 + q % 8;
        const bool in = i < g.H && j < g.W;
        const uint32_t bits = in ? rimg[(size_t)i * g.W + j] : kEmptyBits;
        v[h] = bits_valid(bits);
        r[h] = v[h] ? __uint_as_float(bits) : 0.f;
        p[h][0] = p[h][1] = p[h][2] = 0.f;
        if (v[h]) {
            float ux, uy, uz;
            beam(g, i, j, ux, uy, uz);
            p[h][0] = __fmul_rn(r[h], ux);
            p[h][1] = __fmul_rn(r[h], uy);
            p[h][2] = __fmul_rn(r[h], uz);
        }
        if (kReset && in) rimg[(size_t)i * g.W + j] = kEmptyBits;
    }
    const unsigned b0 = __ballot_sync(0xffffffffu, v[0]), b1 = __ballot_sync(0xffffffffu, v[1]);
    float ra = 0.f, pa0 = 0.f, pa1 = 0.f, pa2 = 0.f;
    if (b0 | b1) {
        const int first = b0 ? __ffs(b0) - 1 : 32 + __ffs(b1) - 1;
        const int src = first & 31, hh = first >> 5;
        ra = __shfl_sync(0xffffffffu, hh ? r[1] : r[0], src);
        pa0 = __shfl_sync(0xffffffffu, hh ? p[1][0] : p[0][0], src);
        pa1 = __shfl_sync(0xffffffffu, hh ? p[1][1] : p[0][1], src);
        pa2 = __shfl_sync(0xffffffffu, hh ? p[1][2] : p[0][2], src);
    }
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int q = lane + 32 * h;
        bf16 c[4];
        if (v[h]) {
            c[0] = __float2bfloat16_rn(__fsub_rn(r[h], ra));
            c[1] = __float2bfloat16_rn(__fsub_rn(p[h][0], pa0));
            c[2] = __float2bfloat16_rn(__fsub_rn(p[h][1], pa1));
            c[3] = __float2bfloat16_rn(__fsub_rn(p[h][2], pa2));
        } else {
            c[0] = c[1] = c[2] = c[3] = __float2bfloat16_rn(0.f);
        }
        *reinterpret_cast<uint2 *>(x + ((size_t)tile * kPX + q) * C0) = make_uint2(pack2(c[0], c[1]), pack2(c[2], c[3]));
    }
    if (lane == 0) anchor[tile] = make_float4(pa0, pa1, pa2, ra);
    // with need0: whether the tile can be fitted at all (3 valid pixels), the only tiles whose
    // proposals the seeded fit reads
    return __popc(b0) + __popc(b1) >= 3;
}

template <bool kReset>
__global__ void k_net_inputs(Geometry g, uint32_t *rimg0, bf16 *x0, float4 *anchor0, uint8_t *need0 = nullptr,
                             DevStats *stats0 = nullptr) {
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const bool live = tile < g.NT;
    const bool needed = live && net_inputs_tile<kReset>(g, rimg0, x0, anchor0, tile, lane);
    // with need0: whether the tile can be fitted at all, the only tiles whose proposals the
    // seeded fit reads; with stats0 the frame's count of them (frame blockIdx.y is slot blockIdx.y)
    if (need0 && live && lane == 0) need0[(size_t)blockIdx.y * g.NT + tile] = needed ? 1 : 0;
    if (need0 && stats0) {   // block-uniform condition: every thread reaches the barrier
        const int cnt = __syncthreads_count(needed && lane == 0);
        if (threadIdx.x == 0 && cnt) atomicAdd(&stats0[blockIdx.y].net_tiles, (unsigned long long)cnt);
    }
}

// The pairs of tiles (2p, 2p + 1) of which at least one is needed, appended to pairs; *npairs
// (zero before the launch) ends as their number.  A thread takes kPairsPer consecutive pairs;
// a block scan orders a block's pairs, and one atomic per block places the block's run (runs
// land in any order: a pair's outputs do not depend on where in the list it is).
// Training labels of one encoded frame, a thread per tile: (fit flag, unit normal, offset of the
// plane relative to the tile's anchor, d - n.a), zeros for tiles that did not fit.  The offset is
// formed in FP64 with separately rounded products and sums, n_x a_x + n_y a_y + n_z a_z added left
// to right, then rounded to fp32 once.
__global__ void k_net_labels(const TileRec *recs, const float4 *anchor, int NT, float *labels) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NT) return;
    const TileRec &r = recs[t];
    const bool fit = r.status == S_FIT;
    const float4 pl = r.plane, a = anchor[t];
    const double s = __dadd_rn(__dadd_rn(__dmul_rn((double)pl.x, (double)a.x), __dmul_rn((double)pl.y, (double)a.y)),
                               __dmul_rn((double)pl.z, (double)a.z));
    float *y = labels + (size_t)t * NOUT;
    y[0] = fit ? 1.0f : 0.0f;
    y[1] = fit ? pl.x : 0.0f;
    y[2] = fit ? pl.y : 0.0f;
    y[3] = fit ? pl.z : 0.0f;
    y[4] = fit ? (float)__dsub_rn((double)pl.w, s) : 0.0f;
}

constexpr int kPairsThreads = 256, kPairsPer = 8;
__global__ void __launch_bounds__(kPairsThreads) k_net_pairs(const uint8_t *need, long long T, uint32_t *pairs,
                                                             uint32_t *npairs) {
    __shared__ uint32_t s_warp[kPairsThreads / 32];
    __shared__ uint32_t s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long P = (T + 1) / 2;
    const long long p0 = ((long long)blockIdx.x * kPairsThreads + tid) * kPairsPer;
    uint32_t mask = 0;
#pragma unroll
    for (int k = 0; k < kPairsPer; k++) {
        const long long p = p0 + k;
        if (p < P && (need[2 * p] || (2 * p + 1 < T && need[2 * p + 1]))) mask |= 1u << k;
    }
    const uint32_t own = __popc(mask);
    uint32_t x = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < kPairsThreads / 32; w++) {
        before += w < warp ? s_warp[w] : 0u;
        total += s_warp[w];
    }
    if (tid == 0) s_base = total ? atomicAdd(npairs, total) : 0u;
    __syncthreads();
    uint32_t pos = s_base + before + x - own;
    for (uint32_t m = mask; m; m &= m - 1) pairs[pos++] = (uint32_t)(p0 + __ffs(m) - 1);
}

// ------------------------------------------------------------------ forward on tcgen05 --
//
// Two tiles per MMA: M = 128 GEMM rows ordered (tile row y, tile, pixel x),
// so that every 8-row core matrix of A is 8 consecutive pixels of one row of
// one tile.  Activations live in shared memory as [channel/8][y 0..9][tile][x
// 0..9][8 channels] with a zero border, i.e. K-major core matrices whose
// 8-row groups are 160 B apart; the 3x3 tap (ky, kx) is then the same
// descriptor started (ky*20 + kx)*16 bytes further, so the nine taps of a
// convolution are nine accumulating MMAs per 16 input channels, with no im2col.
// One thread issues tcgen05.mma into a 128-lane x 64-column fp32 TMEM
// accumulator; epilogue warps read their 32 lanes back (tcgen05.ld) for the
// bias/ReLU/BF16 epilogue into the next layer's copy.

constexpr int TPOS = 10 * 2 * 10;              // padded positions per 8-channel chunk
constexpr int TCHUNK = TPOS * 16;              // bytes per chunk (3200)
constexpr int TW1 = (K1 / 8) * C1 * 16, TW2 = 9 * (C1 / 8) * C2 * 16, TW3 = 9 * (C2 / 8) * C3 * 16;
// One activation buffer per pair slot, shared by the layer input (2 chunks: 4 channels and
// zeros), the first activations (4 chunks) and the second (8 chunks): each is dead once the
// convolution reading it has committed, which is before the next one is written.
constexpr int TACT = (C2 / 8) * TCHUNK;
constexpr int kTcSlots = 3;                     // pairs of tiles in flight per CTA
constexpr int TG = 2 * C3 * 4;
constexpr int TPAR = (C1 + C2 + C3 + HID * C3 + HID + NOUT * HID + NOUT + 3) / 4 * 16;   // biases, head (fp32)
constexpr size_t kTcSmem = (size_t)TW1 + TW2 + TW3 + kTcSlots * (size_t)(TACT + TG) + TPAR + 128;   // + barriers
constexpr uint32_t kTmemCols = 256;             // one 64-column accumulator per pair slot (3 x 64, rounded up)
constexpr long long kSpinLimit = 1ll << 22;
static_assert(kTcSmem <= 227 * 1024, "shared memory of the tcgen05 forward");
static_assert((1 + 4 * kTcSlots) * 8 + 8 <= 128, "the forward's barriers, TMEM address and failure flag fit");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle (start, leading = K-direction
// core-matrix stride, stride = M/N-direction 8-row group stride, version 1)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: fp32 accumulator, bf16 A and B, both K-major
__host__ __device__ constexpr uint32_t mma_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

// bounded wait on an mbarrier phase; false if the limit was reached
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit = kSpinLimit) {
    for (long long it = 0; it < limit; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// byte offset of (chunk, y, tile, x) in an activation copy
__device__ __forceinline__ int tpos(int c8, int y, int tile, int x) { return c8 * TCHUNK + ((y * 2 + tile) * 10 + x) * 16; }

// One convolution: nine taps x (CIN/16) k-steps of M=128, N=COUT MMAs (one thread).  The
// descriptors differ only in their start-address field, so each MMA's pair is the base pair
// plus compile-time offsets (all addresses stay below 256 KB: no carry out of the field).
template <int CIN, int COUT>
__device__ __forceinline__ void tc_conv(uint32_t tmem, uint32_t act, uint32_t wts) {
    constexpr uint32_t idesc = mma_idesc(128, COUT);
    constexpr int KCH = CIN < 16 ? 16 : CIN;   // conv1: 4 real channels padded to one k-step
    const uint64_t a0 = smem_desc(act, TCHUNK, 160);
    const uint64_t b0 = smem_desc(wts, COUT * 16, 128);
#pragma unroll
    for (int tap = 0; tap < 9; tap++) {
#pragma unroll
        for (int ks = 0; ks < KCH / 16; ks++) {
            const uint64_t a = a0 + (uint64_t)((((tap / 3) * 20 + tap % 3) * 16 + 2 * ks * TCHUNK) >> 4);
            const uint64_t b = b0 + (uint64_t)((tap * (KCH / 8) * COUT * 16 + 2 * ks * COUT * 16) >> 4);
            tc_mma(tmem, a, b, idesc, (tap | ks) ? 1u : 0u);
        }
    }
}

// Conv1 as one contraction over the im2col rows (k = tap * 4 + ci, written by the epilogue at
// each pixel's own position): three k-steps of M=128, N=32 MMAs.
__device__ __forceinline__ void tc_conv1(uint32_t tmem, uint32_t act, uint32_t wts) {
    constexpr uint32_t idesc = mma_idesc(128, C1);
    const uint64_t a0 = smem_desc(act, TCHUNK, 160) + (uint64_t)(((1 * 20 + 1) * 16) >> 4);
    const uint64_t b0 = smem_desc(wts, C1 * 16, 128);
#pragma unroll
    for (int ks = 0; ks < K1 / 16; ks++)
        tc_mma(tmem, a0 + (uint64_t)((2 * ks * TCHUNK) >> 4), b0 + (uint64_t)((2 * ks * C1 * 16) >> 4), idesc,
               ks ? 1u : 0u);
}

// bulk copy global -> shared (TMA engine), completion counted on an mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// Warp-specialised: kTcSlots pair slots, each with its own group of four epilogue warps (one
// per TMEM lane quadrant), its activation buffer and its 64 TMEM columns, and one MMA warp.
// A group runs its own pairs of tiles (the CTA's pairs s, s + 3, s + 6, ...) through input,
// three convolutions, pooling and head; an mbarrier the group arrives on hands a layer's input
// (and the emptied accumulator) to the MMA warp, and an mbarrier armed by tcgen05.commit hands
// the finished layer back.  The MMA warp serves whichever slot is ready, so one pair's
// epilogue, pooling and head overlap the other pairs' convolutions.
constexpr int kTcEpiWarps = 4 * kTcSlots;
constexpr int kTcThreads = (kTcEpiWarps + 1) * 32;    // the input-gradient kernel: + the MMA warp
constexpr int kFwdThreads = (kTcEpiWarps + 2) * 32;   // the forward: + the MMA warp and the head warp

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}
// non-blocking test of an mbarrier phase (the MMA warp polls several barriers in turn, so it must
// not be suspended on one that is not ready)
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    return done != 0;
}
// barrier of one slot's four epilogue warps (ids 1..kTcSlots; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int slot) {
    asm volatile("bar.sync %0, 128;\n" ::"r"(slot + 1) : "memory");
}

template <bool kTrain>
__global__ void __launch_bounds__(kFwdThreads, 1) k_net_fwd_tc(NetDev nd, const bf16 *x, long long T, float *out,
                                                              int *err, NetAct act, const uint32_t *pairs = nullptr,
                                                              const uint32_t *npairs = nullptr) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sW1 = sm, *sW2 = sW1 + TW1, *sW3 = sW2 + TW2;
    uint8_t *sAct = sW3 + TW3;                                         // [slot][TACT]
    float *sG = reinterpret_cast<float *>(sAct + kTcSlots * TACT);     // [slot][tile][64] pooled vectors
    float *sPar = sG + kTcSlots * 2 * C3;                              // b1 b2 b3 F1b c1 F2b c2
    float *sB1 = sPar, *sB2 = sB1 + C1, *sB3 = sB2 + C2, *sF1 = sB3 + C3, *sC1 = sF1 + HID * C3;
    float *sF2 = sC1 + HID, *sC2 = sF2 + NOUT * HID;
    // barriers: [0] weights, [1 + s] layer done (tcgen05.commit), [1 + kTcSlots + s] layer input ready,
    // [1 + 2 kTcSlots + s] pooled vectors ready (the slot's four warps), [1 + 3 kTcSlots + s] pooled
    // vectors read (the head warp)
    uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<uint8_t *>(sPar) + TPAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1 + 4 * kTcSlots);
    int *s_fail = reinterpret_cast<int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float *th = nd.theta;
    if (tid == 0) {
        for (int i = 0; i < 1 + kTcSlots; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar + i)) : "memory");
        for (int i = 1 + kTcSlots; i < 1 + 3 * kTcSlots; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(bar + i)) : "memory");
        for (int i = 1 + 3 * kTcSlots; i < 1 + 4 * kTcSlots; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar + i)) : "memory");
        *s_fail = 0;
    }
    {
        uint4 *z = reinterpret_cast<uint4 *>(sAct);
        for (int i = tid; i < kTcSlots * TACT / 16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
        for (int i = tid; i < C1; i += blockDim.x) sB1[i] = th[OB1 + i];
        for (int i = tid; i < C2; i += blockDim.x) sB2[i] = th[OB2 + i];
        for (int i = tid; i < C3; i += blockDim.x) sB3[i] = th[OB3 + i];
        for (int i = tid; i < HID * C3; i += blockDim.x) sF1[(i % C3) * HID + i / C3] = nd.F1b[i];   // [c][j]
        for (int i = tid; i < HID; i += blockDim.x) sC1[i] = th[OC1 + i];
        for (int i = tid; i < NOUT * HID; i += blockDim.x) sF2[i] = nd.F2b[i];
        for (int i = tid; i < NOUT; i += blockDim.x) sC2[i] = th[OC2 + i];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {   // weights by the TMA engine, counted on barrier 0
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                     "r"((uint32_t)(TW1 + TW2 + TW3))
                     : "memory");
        bulk_g2s(smem_u32(sW1), nd.T1, TW1, smem_u32(bar));
        bulk_g2s(smem_u32(sW2), nd.T2, TW2, smem_u32(bar));
        bulk_g2s(smem_u32(sW3), nd.T3, TW3, smem_u32(bar));
    }
    if (!mbar_wait(smem_u32(bar), 0)) {
        atomicExch(s_fail, 1);
        if (err) atomicExch(err, 1);
    }
    proxy_fence();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;
    const long long G = gridDim.x;
    // pair slots i = 0..NP-1: pair i itself, or with a pair list the pair pairs[i] (its count
    // written by the kernel before this one)
    const long long NP = pairs ? (long long)*npairs : (T + 1) / 2;
    if (warp == kTcEpiWarps) {
        // ---- MMA warp: one lane issues the convolutions of every slot, whichever is ready ----
        if (lane == 0) {
            const uint32_t aW1 = smem_u32(sW1), aW2 = smem_u32(sW2), aW3 = smem_u32(sW3);
            long long pa[kTcSlots];
            int layer[kTcSlots];
            uint32_t ph = 0u;   // bit s: parity of slot s's next input-ready wait
            int live = 0;
#pragma unroll
            for (int sl = 0; sl < kTcSlots; sl++) {
                pa[sl] = blockIdx.x + sl * G;
                layer[sl] = 0;
                live += pa[sl] < NP ? 1 : 0;
            }
            long long idle = 0;
            while (live > 0 && !*(volatile int *)s_fail) {
                bool progressed = false;
#pragma unroll
                for (int sl = 0; sl < kTcSlots; sl++) {
                    if (pa[sl] >= NP || !mbar_try(smem_u32(bar + 1 + kTcSlots + sl), (ph >> sl) & 1u)) continue;
                    ph ^= 1u << sl;
                    tc_after_sync();
                    const uint32_t base = smem_u32(sAct + sl * TACT);
                    const uint32_t d = tmem + (uint32_t)(sl * 64);
                    if (layer[sl] == 0) tc_conv1(d, base, aW1);
                    else if (layer[sl] == 1) tc_conv<C1, C2>(d, base, aW2);
                    else tc_conv<C2, C3>(d, base, aW3);
                    tc_commit(smem_u32(bar + 1 + sl));
                    if (++layer[sl] == 3) {
                        layer[sl] = 0;
                        pa[sl] += kTcSlots * G;
                        if (pa[sl] >= NP) live--;
                    }
                    progressed = true;
                }
                if (!progressed) __nanosleep(20);   // leave the issue slots to the epilogue warps meanwhile
                idle = progressed ? 0 : idle + 1;
                if (idle > kSpinLimit) {   // nothing became ready for too long: give up, report
                    atomicExch(s_fail, 1);
                    if (err) atomicExch(err, 1);
                }
            }
        }
        __syncwarp();
    } else if (warp == kTcEpiWarps + 1) {
        // ---- head warp: the pairs in the CTA's order (pair k in slot k mod kTcSlots); lane j holds
        //      hidden unit j's F1 row in registers ----
        float f1[C3];
#pragma unroll
        for (int c = 0; c < C3; c++) f1[c] = sF1[c * HID + lane];
        float f2[NOUT];
#pragma unroll
        for (int i = 0; i < NOUT; i++) f2[i] = sF2[i * HID + lane];
        const float c1 = sC1[lane];
        uint32_t ph = 0u;   // bit s: parity of slot s's next pooled-ready wait
        long long k = 0;
        for (long long i = blockIdx.x; i < NP; i += G, k++) {
            const int sl = (int)(k % kTcSlots);
            if (*(volatile int *)s_fail) break;
            if (!mbar_wait(smem_u32(bar + 1 + 2 * kTcSlots + sl), (ph >> sl) & 1u)) {
                atomicExch(s_fail, 1);
                if (err) atomicExch(err, 1);
                break;
            }
            ph ^= 1u << sl;
            const long long pa = pairs ? (long long)pairs[i] : i;
            const float *gsl = sG + sl * 2 * C3;
#pragma unroll 1
            for (int t2 = 0; t2 < 2; t2++) {
                const long long ht = pa * 2 + t2;
                if (ht >= T) continue;
                const float *g2 = gsl + t2 * C3;
                // four interleaved partial sums (a quarter of the dependent chain); g2 read as
                // broadcast 16-byte loads
                float y4[4] = {c1, 0.f, 0.f, 0.f};
#pragma unroll
                for (int c = 0; c < C3; c += 4) {
                    const float4 gv = *reinterpret_cast<const float4 *>(g2 + c);
                    y4[0] = fmaf(f1[c], gv.x, y4[0]);
                    y4[1] = fmaf(f1[c + 1], gv.y, y4[1]);
                    y4[2] = fmaf(f1[c + 2], gv.z, y4[2]);
                    y4[3] = fmaf(f1[c + 3], gv.w, y4[3]);
                }
                const float yv = (y4[0] + y4[1]) + (y4[2] + y4[3]);
                const float hj = bfround(fmaxf(yv, 0.f));
                float o[NOUT];
#pragma unroll
                for (int q = 0; q < NOUT; q++) {
                    float sacc = f2[q] * hj;
#pragma unroll
                    for (int off = 16; off; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
                    o[q] = sacc + sC2[q];
                }
                if (lane < NOUT) out[(size_t)ht * NOUT + lane] = o[lane];
                if (kTrain) {
                    act.h[(size_t)ht * HID + lane] = hj;
                    act.g[(size_t)ht * C3 + lane] = g2[lane];
                    act.g[(size_t)ht * C3 + lane + 32] = g2[lane + 32];
                    if (lane < NOUT) act.o[(size_t)ht * NOUT + lane] = o[lane];
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(bar + 1 + 3 * kTcSlots + sl));   // the slot's vectors are read
        }
        __syncwarp();
    } else {
        // ---- epilogue group of slot sl: row = 32 quad + lane -> (y, tile, x) ----
        const int sl = warp >> 2, quad = warp & 3;
        const int row = quad * 32 + lane, grp = row >> 3, px = row & 7, py = grp >> 1, tl = grp & 1;
        const int gt = tid - sl * 128;   // thread index within the group
        uint8_t *buf = sAct + sl * TACT;
        const uint32_t bar_done = smem_u32(bar + 1 + sl), bar_in = smem_u32(bar + 1 + kTcSlots + sl);
        const uint32_t bar_pooled = smem_u32(bar + 1 + 2 * kTcSlots + sl), bar_headdone = smem_u32(bar + 1 + 3 * kTcSlots + sl);
        uint32_t ph = 0u, hph = 0u;
        auto wait = [&](uint32_t mbar, uint32_t parity) {   // bounded; gives up at once after any expiry
            if (*(volatile int *)s_fail) return;
            if (!mbar_wait(mbar, parity)) {
                atomicExch(s_fail, 1);
                if (err) atomicExch(err, 1);
            }
        };
        auto handoff = [&]() {   // this warp's rows of the slot's next input are written
            proxy_fence();
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_in);
        };
        const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(sl * 64);
        float *gs = sG + sl * 2 * C3;
        // this thread's input pixel of pair pa (loaded one pair ahead, so that the global load's
        // latency overlaps the previous pair's layers)
        auto pair_of = [&](long long i) { return pairs ? (long long)pairs[i] : i; };
        auto load_in = [&](long long i) {   // this thread's input pixel of pair slot i
            uint2 v = make_uint2(0u, 0u);
            if (i < NP) {
                const long long tile = pair_of(i) * 2 + tl;
                if (tile < T) v = *reinterpret_cast<const uint2 *>(x + ((size_t)tile * kPX + py * 8 + px) * C0);
            }
            return v;
        };
        // the pair's input: the pixel's 4 channels into chunk 6 (zero border), then conv1's im2col
        // row (k = tap * 4 + ci, 36 values and 12 zeros) into chunks 0..5 at the pixel's position,
        // handed to the MMA warp; chunk 6 is free until the second layer's output is written
        auto put_input = [&](uint2 v) {
            *reinterpret_cast<uint4 *>(buf + tpos(6, py + 1, tl, px + 1)) = make_uint4(v.x, v.y, 0u, 0u);
            group_sync(sl);
#pragma unroll
            for (int c8 = 0; c8 < K1 / 8; c8++) {
                uint2 t0 = make_uint2(0u, 0u), t1 = make_uint2(0u, 0u);
                if (2 * c8 < 9) {
                    const int tap = 2 * c8;
                    t0 = *reinterpret_cast<const uint2 *>(buf + tpos(6, py + tap / 3, tl, px + tap % 3));
                }
                if (2 * c8 + 1 < 9) {
                    const int tap = 2 * c8 + 1;
                    t1 = *reinterpret_cast<const uint2 *>(buf + tpos(6, py + tap / 3, tl, px + tap % 3));
                }
                *reinterpret_cast<uint4 *>(buf + tpos(c8, py + 1, tl, px + 1)) = make_uint4(t0.x, t0.y, t1.x, t1.y);
            }
            handoff();
        };
        const long long i0 = blockIdx.x + sl * G;
        if (i0 < NP) put_input(load_in(i0));
        uint2 vin = load_in(i0 + kTcSlots * G);
        for (long long i = i0; i < NP; i += kTcSlots * G) {
            const long long tile = pair_of(i) * 2 + tl;
#pragma unroll 1
            for (int layer = 0; layer < 3; layer++) {
                wait(bar_done, ph);
                ph ^= 1u;
                tc_after_sync();
                const int cout = layer == 0 ? C1 : C2;
                const float *bias = layer == 0 ? sB1 : layer == 1 ? sB2 : sB3;
#pragma unroll 1
                for (int c0 = 0; c0 < cout; c0 += 8) {   // 8 columns per load: 14 warps need <= 128 registers
                    float v[8];
                    tc_ld8(trow + (uint32_t)c0, v);
                    // the 8 biases as two broadcast 16-byte loads (bias arrays are 16-byte aligned)
                    const float4 bl = *reinterpret_cast<const float4 *>(bias + c0),
                                 bh = *reinterpret_cast<const float4 *>(bias + c0 + 4);
                    const float bv[8] = {bl.x, bl.y, bl.z, bl.w, bh.x, bh.y, bh.z, bh.w};
                    tc_wait_ld();
#pragma unroll
                    for (int i = 0; i < 8; i++) v[i] = fmaxf(v[i] + bv[i], 0.f);
                    uint32_t w[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                        w[q] = *reinterpret_cast<const uint32_t *>(&b2);
                    }
                    if (kTrain && tile < T) {   // activations for the backward pass: [tile][pixel][channel]
                        bf16 *ao = layer == 0 ? act.a1 + ((size_t)tile * kPX + py * 8 + px) * C1
                                              : (layer == 1 ? act.a2 : act.a3) + ((size_t)tile * kPX + py * 8 + px) * C2;
                        *reinterpret_cast<uint4 *>(ao + c0) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                    // the next layer's input (or, after the last layer, the activations to pool) in
                    // place of this layer's input (already read by the MMAs)
                    *reinterpret_cast<uint4 *>(buf + tpos(c0 / 8, py + 1, tl, px + 1)) = make_uint4(w[0], w[1], w[2], w[3]);
                }
                if (layer < 2) handoff();   // the next layer's input is in place, the accumulator is read
                else tc_before_sync();
            }
            group_sync(sl);
            if (i != i0) {   // the head warp has read this slot's previous pooled vectors
                wait(bar_headdone, hph);
                hph ^= 1u;
            }
            {   // pooling: thread (tile t2, channel chunk c8, column x) sums its column's 8 pixels of
                // 8 channels (16-byte loads, 8 lanes on consecutive positions), then a reduce-scatter
                // over the 8 columns leaves lane x with channel 8 c8 + x
                const int t2 = gt >> 6, c8 = (gt >> 3) & 7, x = gt & 7;
                float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int y = 0; y < 8; y++) {
                    const uint4 q = *reinterpret_cast<const uint4 *>(buf + tpos(c8, y + 1, t2, x + 1));
                    const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        a[2 * k] += __uint_as_float(u[k] << 16);
                        a[2 * k + 1] += __uint_as_float(u[k] & 0xFFFF0000u);
                    }
                }
                const bool h4 = x & 4, h2 = x & 2, h1 = x & 1;
                float b4[4], b2[2];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const float send = h4 ? a[i] : a[i + 4];
                    b4[i] = (h4 ? a[i + 4] : a[i]) + __shfl_xor_sync(0xffffffffu, send, 4);
                }
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    const float send = h2 ? b4[i] : b4[i + 2];
                    b2[i] = (h2 ? b4[i + 2] : b4[i]) + __shfl_xor_sync(0xffffffffu, send, 2);
                }
                const float b1 = (h1 ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, h1 ? b2[0] : b2[1], 1);
                gs[t2 * C3 + 8 * c8 + x] = bfround(b1 * (1.0f / kPX));
            }
            group_sync(sl);   // pooled vectors complete; the activations are read, so the buffer is free
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_pooled);   // the head warp takes the pair's pooled vectors
            if (i + kTcSlots * G < NP) {   // the next pair's input goes to the MMA warp
                put_input(vin);
                vin = load_in(i + 2 * kTcSlots * G);
            }
        }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Failure detection without a fault: an mbarrier that nothing arrives on, waited on with the
// same bounded wait the tcgen05 kernels use; the expired wait sets the error word and the
// kernel returns normally.
__global__ void k_bounded_wait_selftest(long long limit, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar)) : "memory");
    __syncthreads();
    if (!mbar_wait(smem_u32(&bar), 0, limit) && threadIdx.x == 0) atomicExch(err, 1);
}

// ------------------------------------------------------------------ backward: loss and head --

constexpr float kBeta = 0.02f, kNormEps = 1e-12f;

// One warp per tile: the loss term, dL/d(output) (dout, scaled by 1/T), the hidden layer's
// gradient dy = F2b^T dout through its ReLU, and dL/d(pooled) / 64 per channel; the per-tile
// terms go to global memory and k_net_head_sums forms the head's weight gradients from them.
constexpr int kHeadWarps = 8;
constexpr int HDO = 8;   // dout row stride (5 used)

__global__ void __launch_bounds__(kHeadWarps * 32) k_net_head_bwd(NetDev nd, const float *labels, long long T,
                                                                   NetAct act) {
    const int lane = threadIdx.x & 31;
    const long long tile = (long long)blockIdx.x * kHeadWarps + (threadIdx.x >> 5);
    if (tile >= T) return;
    const float invT = 1.0f / (float)T;
    const float *o = act.o + (size_t)tile * NOUT;
    const float *y = labels + (size_t)tile * NOUT;
    const float lg = o[0], v0 = o[1], v1 = o[2], v2 = o[3], dd = o[4];
    const float fit = y[0], n0 = y[1], n1 = y[2], n2 = y[3], drel = y[4];
    const float s = sqrtf(v0 * v0 + v1 * v1 + v2 * v2 + kNormEps);
    const float vn = v0 * n0 + v1 * n1 + v2 * n2;
    const float cs = vn / s;
    const float xd = dd - drel, ax = fabsf(xd);
    const float sl1 = ax < kBeta ? 0.5f * xd * xd / kBeta : ax - 0.5f * kBeta;
    const float bce = fmaxf(lg, 0.f) - fit * lg + log1pf(expf(-fabsf(lg)));
    float dout[NOUT];
    dout[0] = (1.f / (1.f + expf(-lg)) - fit) * invT;
    const float sg = cs > 0.f ? 1.f : (cs < 0.f ? -1.f : 0.f);
    const float k3 = vn / (s * s * s);
    dout[1] = -fit * sg * (n0 / s - k3 * v0) * invT;
    dout[2] = -fit * sg * (n1 / s - k3 * v1) * invT;
    dout[3] = -fit * sg * (n2 / s - k3 * v2) * invT;
    dout[4] = fit * fminf(fmaxf(xd / kBeta, -1.f), 1.f) * invT;
    const float hj = act.h[(size_t)tile * HID + lane];
    float dh = 0.f;
#pragma unroll
    for (int i = 0; i < NOUT; i++) dh = fmaf(__ldg(nd.F2b + i * HID + lane), dout[i], dh);
    const float dy = hj > 0.f ? dh : 0.f;
    act.hdy[(size_t)tile * HID + lane] = dy;
    if (lane < NOUT) act.hdo[(size_t)tile * HDO + lane] = dout[lane];
    if (lane == 0) act.hlt[tile] = bce + fit * (1.f - fabsf(cs)) + fit * sl1;
    // dg[c] = sum_j F1b[j][c] dy_j: lane c and c + 32 gather the 32 hidden units
    float dg0 = 0.f, dg1 = 0.f;
#pragma unroll 8
    for (int j = 0; j < HID; j++) {
        const float dyj = __shfl_sync(0xffffffffu, dy, j);
        dg0 = fmaf(__ldg(nd.F1b + j * C3 + lane), dyj, dg0);
        dg1 = fmaf(__ldg(nd.F1b + j * C3 + lane + 32), dyj, dg1);
    }
    act.da3c[(size_t)tile * C3 + lane] = dg0 * (1.0f / kPX);
    act.da3c[(size_t)tile * C3 + lane + 32] = dg1 * (1.0f / kPX);
}

// The head's weight gradients and the loss as sums over tiles: dF1[j][c] = sum dy[j] g[c],
// dc1[j] = sum dy[j], dF2[i][j] = sum dout[i] h[j], dc2[i] = sum dout[i], loss = sum of the terms.
// Each block sums its chunks of kHeadChunk tiles (staged in shared memory) in tile order and
// stores its partial sums; k_net_head_reduce adds the blocks' partials in block order.
constexpr int kHeadChunk = 64, kHeadSumThreads = 256;
constexpr int HS_F1 = 0, HS_C1 = HS_F1 + HID * C3, HS_F2 = HS_C1 + HID, HS_C2 = HS_F2 + NOUT * HID,
              HS_LOSS = HS_C2 + NOUT, HS_N = HS_LOSS + 1;

__global__ void __launch_bounds__(kHeadSumThreads) k_net_head_sums(long long T, NetAct act, float *part) {
    __shared__ float sdy[kHeadChunk][HID], sg[kHeadChunk][C3], sh[kHeadChunk][HID], sdo[kHeadChunk][HDO],
        slt[kHeadChunk];
    const int tid = threadIdx.x, c = tid % C3, j0 = tid / C3;   // dF1 rows j0, j0 + 4, ..., column c
    float f1[HID / 4];
#pragma unroll
    for (int k = 0; k < HID / 4; k++) f1[k] = 0.f;
    float ex = 0.f;   // the one other sum of this thread (dc1, dF2, dc2 or the loss), if any
    for (long long t0 = (long long)blockIdx.x * kHeadChunk; t0 < T; t0 += (long long)gridDim.x * kHeadChunk) {
        const int nt = T - t0 < kHeadChunk ? (int)(T - t0) : kHeadChunk;
        __syncthreads();
        for (int i = tid; i < kHeadChunk * C3; i += kHeadSumThreads) {
            const int t = i / C3;
            sg[t][i % C3] = t < nt ? act.g[(size_t)(t0 + t) * C3 + i % C3] : 0.f;
        }
        for (int i = tid; i < kHeadChunk * HID; i += kHeadSumThreads) {
            const int t = i / HID;
            sdy[t][i % HID] = t < nt ? act.hdy[(size_t)(t0 + t) * HID + i % HID] : 0.f;
            sh[t][i % HID] = t < nt ? act.h[(size_t)(t0 + t) * HID + i % HID] : 0.f;
        }
        for (int i = tid; i < kHeadChunk * HDO; i += kHeadSumThreads) {
            const int t = i / HDO;
            sdo[t][i % HDO] = t < nt && i % HDO < NOUT ? act.hdo[(size_t)(t0 + t) * HDO + i % HDO] : 0.f;
        }
        if (tid < kHeadChunk) slt[tid] = tid < nt ? act.hlt[t0 + tid] : 0.f;
        __syncthreads();
        for (int t = 0; t < nt; t++) {
            const float gc = sg[t][c];
#pragma unroll
            for (int k = 0; k < HID / 4; k++) f1[k] = fmaf(sdy[t][j0 + 4 * k], gc, f1[k]);
        }
        if (tid < HID) {
            for (int t = 0; t < nt; t++) ex += sdy[t][tid];
        } else if (tid < HID + NOUT * HID) {
            const int i = (tid - HID) / HID, jj = (tid - HID) % HID;
            for (int t = 0; t < nt; t++) ex = fmaf(sdo[t][i], sh[t][jj], ex);
        } else if (tid < HID + NOUT * HID + NOUT) {
            for (int t = 0; t < nt; t++) ex += sdo[t][tid - HID - NOUT * HID];
        } else if (tid == HID + NOUT * HID + NOUT) {
            for (int t = 0; t < nt; t++) ex += slt[t];
        }
    }
    float *dst = part + (size_t)blockIdx.x * HS_N;
#pragma unroll
    for (int k = 0; k < HID / 4; k++) dst[HS_F1 + (j0 + 4 * k) * C3 + c] = f1[k];
    if (tid < HS_N - HS_C1) dst[HS_C1 + tid] = ex;   // dc1, dF2, dc2 and the loss follow dF1 in this order
}

__global__ void k_net_head_reduce(const float *part, int nparts, float invT, float *grad, float *loss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= HS_N) return;
    float s = 0.f;
    for (int b = 0; b < nparts; b++) s += part[(size_t)b * HS_N + k];
    if (k < HS_C1) grad[OF1 + k] += s;
    else if (k < HS_F2) grad[OC1 + (k - HS_C1)] += s;
    else if (k < HS_C2) grad[OF2 + (k - HS_F2)] += s;
    else if (k < HS_LOSS) grad[OC2 + (k - HS_C2)] += s;
    else *loss += s * invT;
}

// ------------------------------------------------------------------ backward: input gradients on tcgen05 --
//
// The input gradient of a 3x3 convolution is a 3x3 convolution of its output gradient with the
// taps mirrored and the channel roles swapped: da[p][ci] = sum over taps and co of
// dz[p + off(tap)][co] * W[co][ci][8 - tap].  So it runs on the forward's machinery: per pair of
// tiles the output gradient dz3 (the pooled gradient through the last ReLU) is written into the
// padded copy, conv3' (B: [tap][co/8][ci][8] = W3[co][ci][8 - tap]) accumulates da2 in TMEM,
// the epilogue applies conv2's ReLU mask into dz2 (the next input, and its pixel-contiguous global
// copy for the weight gradients), conv2' gives da1 and the epilogue dz1.  Bias gradients are the
// column sums of dz3, dz2 and dz1, reduced over each warp's rows by shuffles into shared sums.
constexpr int TWB3 = 9 * (C3 / 8) * C2 * 16, TWB2 = 9 * (C2 / 8) * C1 * 16;
constexpr int NDB = C3 + C2 + C1;   // bias-gradient sums per slot: db3, db2, db1
constexpr size_t kTcBwdSmem = (size_t)TWB3 + TWB2 + kTcSlots * (size_t)TACT + kTcSlots * NDB * 4 + 128;
static_assert(kTcBwdSmem <= 227 * 1024, "shared memory of the tcgen05 input-gradient kernel");

// Sum over the warp's 32 rows of 8 channel values (one per lane and channel): a reduce-scatter
// leaves the full sum of channel 4 [lane & 16] + 2 [lane & 8] + [lane & 4] on lanes whose two low
// bits are zero, which add it to sums[c0 + that channel].
__device__ __forceinline__ void colsum8(const float (&v)[8], float *sums, int c0, int lane) {
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
    float b4[4], b2[2];
#pragma unroll
    for (int i = 0; i < 4; i++)
        b4[i] = (h16 ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, h16 ? v[i] : v[i + 4], 16);
#pragma unroll
    for (int i = 0; i < 2; i++)
        b2[i] = (h8 ? b4[i + 2] : b4[i]) + __shfl_xor_sync(0xffffffffu, h8 ? b4[i] : b4[i + 2], 8);
    float b1 = (h4 ? b2[1] : b2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? b2[0] : b2[1], 4);
    b1 += __shfl_xor_sync(0xffffffffu, b1, 2);
    b1 += __shfl_xor_sync(0xffffffffu, b1, 1);
    if ((lane & 3) == 0) atomicAdd(sums + c0 + (h16 ? 4 : 0) + (h8 ? 2 : 0) + (h4 ? 1 : 0), b1);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_net_bwd_tc(NetDev nd, long long T, NetAct act, float *grad, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sWB3 = sm, *sWB2 = sWB3 + TWB3;
    uint8_t *sAct = sWB2 + TWB2;                                       // [slot][TACT]
    float *sDB = reinterpret_cast<float *>(sAct + kTcSlots * TACT);    // [slot][NDB]
    // barriers: [0] weights, [1 + s] layer done (tcgen05.commit), [1 + kTcSlots + s] layer input ready
    uint64_t *bar = reinterpret_cast<uint64_t *>(sDB + kTcSlots * NDB);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1 + 2 * kTcSlots);
    int *s_fail = reinterpret_cast<int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < 1 + kTcSlots; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar + i)) : "memory");
        for (int i = 1 + kTcSlots; i < 1 + 2 * kTcSlots; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;\n" ::"r"(smem_u32(bar + i)) : "memory");
        *s_fail = 0;
    }
    {
        uint4 *z = reinterpret_cast<uint4 *>(sAct);
        for (int i = tid; i < kTcSlots * TACT / 16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
        for (int i = tid; i < kTcSlots * NDB; i += blockDim.x) sDB[i] = 0.f;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {   // weights by the TMA engine, counted on barrier 0
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                     "r"((uint32_t)(TWB3 + TWB2))
                     : "memory");
        bulk_g2s(smem_u32(sWB3), nd.TB3, TWB3, smem_u32(bar));
        bulk_g2s(smem_u32(sWB2), nd.TB2, TWB2, smem_u32(bar));
    }
    if (!mbar_wait(smem_u32(bar), 0)) {
        atomicExch(s_fail, 1);
        if (err) atomicExch(err, 1);
    }
    proxy_fence();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;
    const long long G = gridDim.x, NP = (T + 1) / 2;
    if (warp == kTcEpiWarps) {
        // ---- MMA warp: conv3' then conv2' for every slot, whichever is ready ----
        if (lane == 0) {
            const uint32_t aWB3 = smem_u32(sWB3), aWB2 = smem_u32(sWB2);
            long long pa[kTcSlots];
            int layer[kTcSlots];
            uint32_t ph = 0u;
            int live = 0;
#pragma unroll
            for (int sl = 0; sl < kTcSlots; sl++) {
                pa[sl] = blockIdx.x + sl * G;
                layer[sl] = 0;
                live += pa[sl] < NP ? 1 : 0;
            }
            long long idle = 0;
            while (live > 0 && !*(volatile int *)s_fail) {
                bool progressed = false;
#pragma unroll
                for (int sl = 0; sl < kTcSlots; sl++) {
                    if (pa[sl] >= NP || !mbar_try(smem_u32(bar + 1 + kTcSlots + sl), (ph >> sl) & 1u)) continue;
                    ph ^= 1u << sl;
                    tc_after_sync();
                    const uint32_t base = smem_u32(sAct + sl * TACT);
                    const uint32_t d = tmem + (uint32_t)(sl * 64);
                    if (layer[sl] == 0) tc_conv<C3, C2>(d, base, aWB3);
                    else tc_conv<C2, C1>(d, base, aWB2);
                    tc_commit(smem_u32(bar + 1 + sl));
                    if (++layer[sl] == 2) {
                        layer[sl] = 0;
                        pa[sl] += kTcSlots * G;
                        if (pa[sl] >= NP) live--;
                    }
                    progressed = true;
                }
                if (!progressed) __nanosleep(20);
                idle = progressed ? 0 : idle + 1;
                if (idle > kSpinLimit) {
                    atomicExch(s_fail, 1);
                    if (err) atomicExch(err, 1);
                }
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue group of slot sl: row = 32 quad + lane -> (y, tile, x) ----
        const int sl = warp >> 2, quad = warp & 3;
        const int row = quad * 32 + lane, grp = row >> 3, px = row & 7, py = grp >> 1, tl = grp & 1;
        const int pix = py * 8 + px;
        uint8_t *buf = sAct + sl * TACT;
        float *db = sDB + sl * NDB;
        const uint32_t bar_done = smem_u32(bar + 1 + sl), bar_in = smem_u32(bar + 1 + kTcSlots + sl);
        uint32_t ph = 0u;
        auto wait = [&](uint32_t mbar, uint32_t parity) {
            if (*(volatile int *)s_fail) return;
            if (!mbar_wait(mbar, parity)) {
                atomicExch(s_fail, 1);
                if (err) atomicExch(err, 1);
            }
        };
        auto handoff = [&]() {
            proxy_fence();
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_in);
        };
        const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(sl * 64);
        // dz = bf16(da * [a > 0]) for 8 channels of this pixel: into the padded copy (when the next
        // convolution reads it), the pixel-contiguous global copy, and the bias sums
        auto emit = [&](const float (&da)[8], const bf16 *a, int C, int c0, bool in, bool pad, bf16 *dzt, float *sums) {
            uint4 av = make_uint4(0u, 0u, 0u, 0u);
            if (in) av = *reinterpret_cast<const uint4 *>(a + c0);
            const uint32_t aw[4] = {av.x, av.y, av.z, av.w};
            float d[8];
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float lo = __uint_as_float(aw[q] << 16), hi = __uint_as_float(aw[q] & 0xFFFF0000u);
                d[2 * q] = bfround(in && lo > 0.f ? da[2 * q] : 0.f);
                d[2 * q + 1] = bfround(in && hi > 0.f ? da[2 * q + 1] : 0.f);
                const __nv_bfloat162 b2 = __floats2bfloat162_rn(d[2 * q], d[2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t *>(&b2);
            }
            if (pad) *reinterpret_cast<uint4 *>(buf + tpos(c0 / 8, py + 1, tl, px + 1)) = make_uint4(w[0], w[1], w[2], w[3]);
            if (in)
#pragma unroll
                for (int i = 0; i < 8; i++) dzt[(size_t)(c0 + i) * kPX + pix] = __float2bfloat16_rn(d[i]);
            colsum8(d, sums, c0, lane);
            (void)C;
        };
        for (long long pa = blockIdx.x + sl * G; pa < NP; pa += kTcSlots * G) {
            const long long tile = pa * 2 + tl;
            const bool in = tile < T;
            const size_t tp = (size_t)(in ? tile : 0);
            {   // dz3: the pooled gradient of every pixel through the last ReLU
                const float *da3 = act.da3c + tp * C3;
                const bf16 *a3 = act.a3 + (tp * kPX + pix) * C3;
                bf16 *dzt = act.dz3t + tp * C3 * kPX;
#pragma unroll 1
                for (int c0 = 0; c0 < C3; c0 += 8) {
                    float da[8];
                    if (in) {
                        const float4 u = *reinterpret_cast<const float4 *>(da3 + c0), v = *reinterpret_cast<const float4 *>(da3 + c0 + 4);
                        da[0] = u.x; da[1] = u.y; da[2] = u.z; da[3] = u.w; da[4] = v.x; da[5] = v.y; da[6] = v.z; da[7] = v.w;
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; i++) da[i] = 0.f;
                    }
                    emit(da, a3, C3, c0, in, true, dzt, db);
                }
            }
            handoff();
#pragma unroll 1
            for (int layer = 0; layer < 2; layer++) {
                wait(bar_done, ph);
                ph ^= 1u;
                tc_after_sync();
                const int C = layer == 0 ? C2 : C1;
                const bf16 *a = (layer == 0 ? act.a2 : act.a1) + (tp * kPX + pix) * C;
                bf16 *dzt = (layer == 0 ? act.dz2t : act.dz1t) + tp * C * kPX;
                float *sums = db + (layer == 0 ? C3 : C3 + C2);
#pragma unroll 1
                for (int c0 = 0; c0 < C; c0 += 8) {
                    float v[8];
                    tc_ld8(trow + (uint32_t)c0, v);
                    tc_wait_ld();
                    emit(v, a, C, c0, in, layer == 0, dzt, sums);
                }
                if (layer == 0) handoff();   // dz2 is in place and the accumulator is read
                else tc_before_sync();
            }
        }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
    for (int c = tid; c < NDB; c += blockDim.x) {   // the slots' bias sums into the gradient
        float v = 0.f;
        for (int sl2 = 0; sl2 < kTcSlots; sl2++) v += sDB[sl2 * NDB + c];
        const int off = c < C3 ? OB3 + c : (c < C3 + C2 ? OB2 + (c - C3) : OB1 + (c - C3 - C2));
        if (v != 0.f) atomicAdd(grad + off, v);
    }
}

// ------------------------------------------------------------------ backward: weight gradients on tcgen05 --
//
// dW[co][ci][ky][kx] = sum over tiles and pixels p = (y, x) of dz[co][p] * a[ci][y + ky - 1][x + kx - 1]
// (zero outside the tile): a GEMM whose reduction runs over pixels.  Both operands are staged in
// shared memory K-major with the pixels as K; a "core" is one 8-pixel row of the tile (one core
// matrix wide in K):
//   P: rows (dx, ci), dx = -1, 0, +1: the input activations of channel ci shifted by dx along
//      each row (zero fill), cores 0..9 (8 and 9 stay zero);
//   Z: rows co, the pre-activation gradient, cores -1..9 (-1, 8 and 9 stay zero).
// Within a core the 8-row groups are kWgSbo = 144 bytes apart (128 + 16, so that the 16-byte
// stores of a quarter-warp fall in different banks) and the next core starts where the core's
// last group ends: an operand with more rows than a core holds continues into the next core, one
// tile row further down.  So the row shift dy comes from the core an operand starts at and the
// column shift dx from P's row blocks:
//   conv2, conv3 (A = P, B = Z, N = 3 CO): B starts one core early, its three row blocks are dz
//   one row above, level with and below A's rows (ky = 2, 1, 0); A starts at group 0 (and for
//   conv3's 192 rows at group 16 as well), so one or two M = 128 MMAs per k-step cover all dx;
//   conv1 (A = Z, B = P, M = 128, N = 32): A's row blocks are dz at ky = 2, 1, 0 (and an unused
//   fourth), B's rows are (dx, ci) with ci padded to 8.
// Rows and columns that hold no tap (the operand's spill into the next core, padding channels)
// are computed and ignored.  Every CTA accumulates its tiles in TMEM and stores the accumulator
// (lanes contiguous); k_net_wgrad_reduce adds the CTAs' copies in CTA order into the gradient.
constexpr int kWgSbo = 144;
constexpr int kWgTeams = 4, kWgTeamWarps = 2;                   // a team of warps fills one slot
constexpr int kWgProdWarps = kWgTeams * kWgTeamWarps;
constexpr int kWgThreads = (kWgProdWarps + 1) * 32;             // + the MMA warp

template <int CI, int CO>
struct Wg {
    static constexpr int CIP = CI < 8 ? 8 : CI;
    static constexpr int RP = 3 * CIP, GP = RP / 8, GZ = CO / 8;   // P rows; 8-row groups per core
    static constexpr int LBP = GP * kWgSbo, LBZ = GZ * kWgSbo;     // bytes per core
    static constexpr int PB = 10 * LBP, ZB = 11 * LBZ, SLOT = PB + ZB;
    static constexpr bool kAP = CI >= 16;                          // A = P; else A = Z
    static constexpr int N = kAP ? 3 * CO : 32;
    static constexpr int NM = kAP ? (RP + 127) / 128 : 1;          // MMAs per k-step
    static constexpr int DCOLS = NM * N, DSZ = 128 * DCOLS;        // accumulator columns, floats
    static constexpr uint32_t TCOLS = DCOLS <= 32 ? 32 : DCOLS <= 64 ? 64 : DCOLS <= 128 ? 128 : DCOLS <= 256 ? 256 : 512;
    static constexpr size_t SMEM = (size_t)kWgTeams * SLOT + (2 * kWgTeams + 1) * 8 + 16;
    static_assert(kAP ? (CI % 8 == 0 && CO % 8 == 0 && N <= 256) : (CI <= 8 && CO == 32), "operand shapes");
    static_assert(DCOLS <= 512 && SMEM <= 227 * 1024, "accumulator and staging fit");
};

__device__ __forceinline__ void st16(uint8_t *p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    *reinterpret_cast<uint4 *>(p) = make_uint4(a, b, c, d);
}

// The three shifted copies (dx = -1, 0, +1) of one row of 8 pixels (w: 4 words, 2 pixels each)
// at p, p + step and p + 2 step.
__device__ __forceinline__ void put_shifts(uint8_t *p, int step, const uint32_t (&w)[4]) {
    const uint32_t s1 = __byte_perm(w[0], w[1], 0x5432), s2 = __byte_perm(w[1], w[2], 0x5432),
                   s3 = __byte_perm(w[2], w[3], 0x5432);
    st16(p, w[0] << 16, s1, s2, s3);            // value at x is a[x - 1]
    st16(p + step, w[0], w[1], w[2], w[3]);
    st16(p + 2 * step, s1, s2, s3, w[3] >> 16); // value at x is a[x + 1]
}

template <int CI, int CO>
__global__ void __launch_bounds__(kWgThreads, 1) k_net_wgrad_tc(const bf16 *a, const bf16 *dzt, long long T, float *part,
                                                                 int *err) {
    using C = Wg<CI, CO>;
    extern __shared__ __align__(1024) uint8_t sm[];
    // barriers: [t] slot t filled (its team's warps), [kWgTeams + t] slot t read (tcgen05.commit),
    // [2 kWgTeams] all MMAs done
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kWgTeams * C::SLOT);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2 * kWgTeams + 1);
    int *s_fail = reinterpret_cast<int *>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < kWgTeams; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar + i)), "r"(kWgTeamWarps) : "memory");
        for (int i = kWgTeams; i < 2 * kWgTeams + 1; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar + i)) : "memory");
        *s_fail = 0;
    }
    {   // zero cores and padding rows stay as written here
        uint4 *z = reinterpret_cast<uint4 *>(sm);
        for (int i = tid; i < kWgTeams * C::SLOT / 16; i += blockDim.x) z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    proxy_fence();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tmem_slot;
    const long long G = gridDim.x;
    const long long ntl = (T - blockIdx.x + G - 1) / G;   // this CTA's tiles blockIdx.x + j G (>= 1: grid <= T)
    auto fail = [&]() {
        atomicExch(s_fail, 1);
        if (err) atomicExch(err, 1);
    };
    const uint32_t bar_done = smem_u32(bar + 2 * kWgTeams);
    if (warp == kWgProdWarps) {
        // ---- MMA warp: the tiles in order, slot j % kWgTeams ----
        if (lane == 0) {
            constexpr uint32_t idesc = mma_idesc(128, C::N);
            for (long long j = 0; j < ntl && !*(volatile int *)s_fail; j++) {
                const int s = (int)(j % kWgTeams);
                if (!mbar_wait(smem_u32(bar + s), (uint32_t)((j / kWgTeams) & 1))) {
                    fail();
                    break;
                }
                tc_after_sync();
                const uint32_t P = smem_u32(sm + s * C::SLOT), Z = P + C::PB;
#pragma unroll
                for (int ks = 0; ks < 4; ks++) {
                    const int kc = 2 * ks;   // first core of the k-step; Z's position kc is core kc - 1
#pragma unroll
                    for (int jm = 0; jm < C::NM; jm++) {
                        const uint64_t ad = C::kAP ? smem_desc(P + kc * C::LBP + jm * 16 * kWgSbo, C::LBP, kWgSbo)
                                                   : smem_desc(Z + kc * C::LBZ, C::LBZ, kWgSbo);
                        const uint64_t bd = C::kAP ? smem_desc(Z + kc * C::LBZ, C::LBZ, kWgSbo)
                                                   : smem_desc(P + kc * C::LBP, C::LBP, kWgSbo);
                        tc_mma(tmem + (uint32_t)(jm * C::N), ad, bd, idesc, (j | ks) ? 1u : 0u);
                    }
                }
                tc_commit(smem_u32(bar + kWgTeams + s));
            }
            tc_commit(bar_done);
        }
        __syncwarp();
    } else {
        // ---- team t = warp / kWgTeamWarps fills slot t with the tiles j = t, t + kWgTeams, ... ----
        const int team = warp / kWgTeamWarps, tt = tid % (kWgTeamWarps * 32), tw = warp % kWgTeamWarps;
        uint8_t *P = sm + team * C::SLOT, *Z = P + C::PB;
        for (long long j = team; j < ntl; j += kWgTeams) {
            if (*(volatile int *)s_fail) break;
            if (j >= kWgTeams && !mbar_wait(smem_u32(bar + kWgTeams + team), (uint32_t)((j / kWgTeams - 1) & 1))) {
                fail();
                break;
            }
            const long long tile = blockIdx.x + j * G;
            if constexpr (C::kAP) {
                constexpr int NC8 = CI / 8;
                for (int it = tt; it < 8 * NC8; it += kWgTeamWarps * 32) {
                    const int c8 = it % NC8, y = it / NC8;
                    const uint4 *src = reinterpret_cast<const uint4 *>(a + ((size_t)tile * kPX + y * 8) * CI) + c8;
                    uint32_t r[8][4];
#pragma unroll
                    for (int x = 0; x < 8; x++) {
                        const uint4 v = __ldg(src + x * NC8);
                        r[x][0] = v.x; r[x][1] = v.y; r[x][2] = v.z; r[x][3] = v.w;
                    }
                    uint8_t *row = P + y * C::LBP + c8 * kWgSbo;
#pragma unroll
                    for (int q = 0; q < 4; q++) {   // channels 2q and 2q + 1 of the group
                        uint32_t lo[4], hi[4];
#pragma unroll
                        for (int m = 0; m < 4; m++) {
                            lo[m] = __byte_perm(r[2 * m][q], r[2 * m + 1][q], 0x5410);
                            hi[m] = __byte_perm(r[2 * m][q], r[2 * m + 1][q], 0x7632);
                        }
                        put_shifts(row + (2 * q) * 16, NC8 * kWgSbo, lo);
                        put_shifts(row + (2 * q + 1) * 16, NC8 * kWgSbo, hi);
                    }
                }
            } else {
                if (tt < 8 * CI) {   // one channel of one row of 8 pixels per thread
                    const int ci = tt % CI, y = tt / CI;
                    const unsigned short *src =
                        reinterpret_cast<const unsigned short *>(a) + ((size_t)tile * kPX + y * 8) * CI + ci;
                    uint32_t w[4];
#pragma unroll
                    for (int m = 0; m < 4; m++)
                        w[m] = (uint32_t)__ldg(src + (2 * m) * CI) | ((uint32_t)__ldg(src + (2 * m + 1) * CI) << 16);
                    put_shifts(P + y * C::LBP + ci * 16, kWgSbo, w);
                }
            }
            {   // dz rows: a block of 8 channels x 4 rows per warp instruction (64 contiguous bytes per channel)
                constexpr int NBLK = (CO / 8) * 2;
                for (int b = tw; b < NBLK; b += kWgTeamWarps) {
                    const int chi = b % (CO / 8), y = (b / (CO / 8)) * 4 + (lane >> 3), co = chi * 8 + (lane & 7);
                    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(dzt + ((size_t)tile * CO + co) * kPX + y * 8));
                    *reinterpret_cast<uint4 *>(Z + (y + 1) * C::LBZ + chi * kWgSbo + (lane & 7) * 16) = v;
                }
            }
            proxy_fence();
            tc_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(bar + team));
        }
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4).. and every other 8-column chunk ----
        if (!*(volatile int *)s_fail && !mbar_wait(bar_done, 0)) fail();
        tc_after_sync();
        if (!*(volatile int *)s_fail) {
            const int quad = warp & 3, half = warp >> 2;
            float *dst = part + (size_t)blockIdx.x * C::DSZ + quad * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
            for (int c0 = half * 8; c0 < C::DCOLS; c0 += 16) {
                float v[8];
                tc_ld8(trow + (uint32_t)c0, v);
                tc_wait_ld();
#pragma unroll
                for (int i = 0; i < 8; i++) dst[(size_t)(c0 + i) * 128] = v[i];
            }
        }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(C::TCOLS) : "memory");
}

// The CTAs' accumulators summed in CTA order into the gradient: element (MMA jm, column n, row m)
// maps back to (co, ci, ky, kx) through the staging above; the elements that hold no tap are
// skipped, every tap is held by exactly one element.
template <int CI, int CO>
__global__ void k_net_wgrad_reduce(const float *part, int nparts, float *grad, int wofs) {
    using C = Wg<CI, CO>;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= C::DSZ) return;
    const int m = e % 128, col = e / 128, jm = col / C::N, n = col % C::N;
    int co, ci, ky, kx;
    if (C::kAP) {
        const int r = jm * 128 + m;   // P row (dx + 1) CI + ci of the k-step's first core
        if (r >= C::RP) return;
        kx = r / CI;
        ci = r % CI;
        ky = 2 - n / CO;
        co = n % CO;
    } else {
        if (m >= 3 * CO || n >= 24 || n % 8 >= CI) return;
        ky = 2 - m / CO;
        co = m % CO;
        kx = n / 8;
        ci = n % 8;
    }
    float s = 0.f;
    for (int c = 0; c < nparts; c++) s += part[(size_t)c * C::DSZ + e];
    grad[wofs + (co * CI + ci) * 9 + ky * 3 + kx] += s;
}

// ------------------------------------------------------------------ optimiser --

__global__ void k_net_adam(float *theta, const float *grad, float *m, float *v, int n, float lr, float bc1, float bc2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

}  // namespace

// ------------------------------------------------------------------ C ABI --

struct lcc_net {
    cudaStream_t stream = nullptr;
    int64_t max_tiles = 0;
    int sms = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
    int *err = nullptr;                      // set by a kernel whose bounded wait ran out
    float *wpart = nullptr;                  // per-CTA weight-gradient accumulators [sms][Wg::DSZ]
    NetDev nd{};
    NetAct act{};
    void *wbuf = nullptr, *abuf = nullptr;
};

namespace {

lcc_status net_prep(lcc_net *net) {
    k_net_prep<<<152, 256, 0, net->stream>>>(net->nd);
    return cudaGetLastError() == cudaSuccess ? LCC_OK : LCC_ERR_CUDA;
}

template <typename K>
lcc_status smem_attr(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess
               ? LCC_OK
               : LCC_ERR_CUDA;
}

template <int CI, int CO>
lcc_status wgrad_tc(lcc_net *net, const bf16 *a, const bf16 *dzt, int64_t ntiles, int grid, int wofs) {
    using C = Wg<CI, CO>;
    k_net_wgrad_tc<CI, CO><<<grid, kWgThreads, C::SMEM, net->stream>>>(a, dzt, ntiles, net->wpart, net->err);
    k_net_wgrad_reduce<CI, CO><<<(C::DSZ + 255) / 256, 256, 0, net->stream>>>(net->wpart, grid, net->grad, wofs);
    return cudaGetLastError() == cudaSuccess ? LCC_OK : LCC_ERR_CUDA;
}

// tcgen05 forward; with `train` it also keeps the activations the backward pass reads
// With a pair list (pair_list, its count at *npairs on the device) only the listed pairs of
// tiles are run; the grid is sized for all (ntiles + 1) / 2 pairs.
lcc_status forward_tc(lcc_net *net, const uint16_t *d_x, int64_t ntiles, float *d_out, bool train,
                      const uint32_t *pair_list = nullptr, const uint32_t *npairs = nullptr) {
    const int64_t pairs = (ntiles + 1) / 2;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(pairs, net->sms));
    const bf16 *x = reinterpret_cast<const bf16 *>(d_x);
    if (train)
        k_net_fwd_tc<true><<<grid, kFwdThreads, kTcSmem, net->stream>>>(net->nd, x, ntiles, d_out, net->err, net->act,
                                                                        pair_list, npairs);
    else
        k_net_fwd_tc<false><<<grid, kFwdThreads, kTcSmem, net->stream>>>(net->nd, x, ntiles, d_out, net->err, net->act,
                                                                         pair_list, npairs);
    return cudaGetLastError() == cudaSuccess ? LCC_OK : LCC_ERR_CUDA;
}

lcc_status backward(lcc_net *net, const uint16_t *d_x, const float *d_labels, int64_t ntiles) {
    cudaStream_t st = net->stream;
    LCC_CUDA(cudaMemsetAsync(net->grad, 0, sizeof(float) * NPARAM, st));
    LCC_CUDA(cudaMemsetAsync(net->loss, 0, sizeof(float), st));
    lcc_status s = forward_tc(net, d_x, ntiles, net->act.o, true);
    if (s != LCC_OK) return s;
    k_net_head_bwd<<<(unsigned)((ntiles + kHeadWarps - 1) / kHeadWarps), kHeadWarps * 32, 0, st>>>(net->nd, d_labels,
                                                                                                  ntiles, net->act);
    {   // the head's weight gradients and the loss, summed per block and then across blocks in order
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((ntiles + kHeadChunk - 1) / kHeadChunk, net->sms));
        k_net_head_sums<<<blocks, kHeadSumThreads, 0, st>>>(ntiles, net->act, net->wpart);
        k_net_head_reduce<<<(HS_N + 255) / 256, 256, 0, st>>>(net->wpart, blocks, 1.0f / (float)ntiles, net->grad,
                                                            net->loss);
    }
    {   // input gradients on tcgen05: one CTA per SM over pairs of tiles
        const int64_t pairs = (ntiles + 1) / 2;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(pairs, net->sms));
        k_net_bwd_tc<<<grid, kTcThreads, kTcBwdSmem, st>>>(net->nd, ntiles, net->act, net->grad, net->err);
    }
    {   // weight gradients on tcgen05, then the CTAs' accumulators summed (one buffer, reused in order)
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, net->sms));
        s = wgrad_tc<C2, C3>(net, net->act.a2, net->act.dz3t, ntiles, grid, OW3);
        if (s == LCC_OK) s = wgrad_tc<C1, C2>(net, net->act.a1, net->act.dz2t, ntiles, grid, OW2);
        if (s == LCC_OK) s = wgrad_tc<C0, C1>(net, reinterpret_cast<const bf16 *>(d_x), net->act.dz1t, ntiles, grid, OW1);
        if (s != LCC_OK) return s;
    }
    return cudaGetLastError() == cudaSuccess ? LCC_OK : LCC_ERR_CUDA;
}

}  // namespace

namespace lcc {
namespace api {

lcc_status net_inputs_slots(lcc_ctx *c, int nframes, uint16_t *d_x, float4 *d_anchor, uint8_t *d_need) {
    if (c->g.th != 8 || c->g.tw != 8 || nframes < 1 || nframes > c->slots) return LCC_ERR_UNSUPPORTED;
    const int wpb = 8;
    k_net_inputs<false><<<dim3((c->g.NT + wpb - 1) / wpb, nframes), wpb * 32, 0, c->stream>>>(
        c->g, c->s.rimg, reinterpret_cast<bf16 *>(d_x), d_anchor, d_need, c->s.stats);
    return cudaGetLastError() == cudaSuccess ? LCC_OK : LCC_ERR_CUDA;
}

lcc_status net_pairs(const uint8_t *d_need, int64_t ntiles, uint32_t *d_pairs, uint32_t *d_npairs, cudaStream_t st) {
    if (ntiles <= 0) return LCC_OK;
    LCC_CUDA(cudaMemsetAsync(d_npairs, 0, sizeof(uint32_t), st));
    const int64_t per_block = (int64_t)kPairsThreads * kPairsPer, pairs = (ntiles + 1) / 2;
    k_net_pairs<<<(unsigned)((pairs + per_block - 1) / per_block), kPairsThreads, 0, st>>>(d_need, ntiles, d_pairs,
                                                                                            d_npairs);
    return cudaGetLastError() == cudaSuccess ? LCC_OK : LCC_ERR_CUDA;
}

lcc_status net_forward_on(lcc_net *net, const uint16_t *d_x, int64_t ntiles, float *d_out, cudaStream_t st,
                          const uint32_t *d_pairs, const uint32_t *d_npairs) {
    if (ntiles <= 0) return LCC_OK;
    cudaStream_t own = net->stream;
    net->stream = st;
    const lcc_status s = forward_tc(net, d_x, ntiles, d_out, false, d_pairs, d_npairs);
    net->stream = own;
    return s;
}

lcc_status net_latched(lcc_net *net) {
    int e = 0;
    if (cudaMemcpy(&e, net->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LCC_ERR_CUDA;
    if (!e) return LCC_OK;
    cudaMemset(net->err, 0, sizeof(int));
    return LCC_ERR_TIMEOUT;
}

}  // namespace api
}  // namespace lcc

extern "C" {

lcc_status lcc_net_create(lcc_net **out, const float *h_params, int64_t max_tiles, void *cuda_stream) {
    if (!out || !h_params || max_tiles < 1 || max_tiles > ((int64_t)1 << 24)) return LCC_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return LCC_ERR_NO_DEVICE;
    if (!(prop.major == 10 && prop.minor == 3)) return LCC_ERR_NO_DEVICE;
    lcc_net *net = new (std::nothrow) lcc_net();
    if (!net) return LCC_ERR_CUDA;
    net->stream = (cudaStream_t)cuda_stream;
    net->max_tiles = max_tiles;
    net->sms = prop.multiProcessorCount;
    const size_t wb[] = {sizeof(float) * NPARAM * 4 + 256,   // theta, grad, m, v
                         (size_t)TW1 + TW2 + TW3 + TWB3 + TWB2,
                         sizeof(float) * (HID * C3 + NOUT * HID), 256};
    size_t wtotal = 0;
    for (size_t b : wb) wtotal += align256(b);
    const size_t T = (size_t)max_tiles;
    const size_t ab[] = {sizeof(bf16) * T * kPX * C1, sizeof(bf16) * T * kPX * C2, sizeof(bf16) * T * kPX * C3,
                         sizeof(float) * T * C3,      sizeof(float) * T * HID,      sizeof(float) * T * NOUT,
                         sizeof(float) * T * C3,      sizeof(bf16) * T * C1 * kPX,  sizeof(bf16) * T * C2 * kPX,
                         sizeof(bf16) * T * C3 * kPX, sizeof(float) * (size_t)net->sms * Wg<C2, C3>::DSZ,
                         sizeof(float) * T * HID,     sizeof(float) * T * HDO,      sizeof(float) * T};
    size_t atotal = 0;
    for (size_t b : ab) atotal += align256(b);
    if (cudaMalloc(&net->wbuf, wtotal) != cudaSuccess || cudaMalloc(&net->abuf, atotal) != cudaSuccess) {
        lcc_net_destroy(net);
        return LCC_ERR_CUDA;
    }
    char *w = (char *)net->wbuf;
    net->theta = (float *)w;
    net->grad = net->theta + NPARAM;
    net->m = net->grad + NPARAM;
    net->v = net->m + NPARAM;
    w += align256(wb[0]);
    net->nd.theta = net->theta;
    net->nd.T1 = (bf16 *)w;
    net->nd.T2 = net->nd.T1 + TW1 / 2;
    net->nd.T3 = net->nd.T2 + TW2 / 2;
    net->nd.TB3 = net->nd.T3 + TW3 / 2;
    net->nd.TB2 = net->nd.TB3 + TWB3 / 2;
    w += align256(wb[1]);
    net->nd.F1b = (float *)w;
    net->nd.F2b = net->nd.F1b + HID * C3;
    w += align256(wb[2]);
    net->loss = (float *)w;
    net->err = (int *)(w + 64);
    char *a = (char *)net->abuf;
    void **slots[] = {(void **)&net->act.a1, (void **)&net->act.a2, (void **)&net->act.a3, (void **)&net->act.g,
                      (void **)&net->act.h,  (void **)&net->act.o,  (void **)&net->act.da3c, (void **)&net->act.dz1t,
                      (void **)&net->act.dz2t, (void **)&net->act.dz3t, (void **)&net->wpart,
                      (void **)&net->act.hdy, (void **)&net->act.hdo, (void **)&net->act.hlt};
    for (int i = 0; i < 14; i++) {
        *slots[i] = a;
        a += align256(ab[i]);
    }
    if (smem_attr(k_net_bwd_tc, kTcBwdSmem) != LCC_OK ||
        smem_attr(k_net_fwd_tc<false>, kTcSmem) != LCC_OK ||
        smem_attr(k_net_fwd_tc<true>, kTcSmem) != LCC_OK ||
        smem_attr(k_net_wgrad_tc<C2, C3>, Wg<C2, C3>::SMEM) != LCC_OK ||
        smem_attr(k_net_wgrad_tc<C1, C2>, Wg<C1, C2>::SMEM) != LCC_OK ||
        smem_attr(k_net_wgrad_tc<C0, C1>, Wg<C0, C1>::SMEM) != LCC_OK ||
        cudaMemcpy(net->theta, h_params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(net->m, 0, sizeof(float) * 2 * NPARAM) != cudaSuccess ||
        cudaMemset(net->err, 0, sizeof(int)) != cudaSuccess || net_prep(net) != LCC_OK ||
        cudaDeviceSynchronize() != cudaSuccess) {
        lcc_net_destroy(net);
        return LCC_ERR_CUDA;
    }
    *out = net;
    return LCC_OK;
}

void lcc_net_destroy(lcc_net *net) {
    if (!net) return;
    cudaStreamSynchronize(net->stream);
    cudaFree(net->wbuf);
    cudaFree(net->abuf);
    delete net;
}

int64_t lcc_net_num_params(void) { return NPARAM; }

lcc_status lcc_net_get_params(lcc_net *net, float *h_params) {
    if (!net || !h_params) return LCC_ERR_INVALID_ARG;
    LCC_CUDA(cudaMemcpyAsync(h_params, net->theta, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, net->stream));
    LCC_CUDA(cudaStreamSynchronize(net->stream));
    return LCC_OK;
}

lcc_status lcc_net_set_params(lcc_net *net, const float *h_params) {
    if (!net || !h_params) return LCC_ERR_INVALID_ARG;
    LCC_CUDA(cudaMemcpyAsync(net->theta, h_params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, net->stream));
    LCC_CUDA(cudaMemsetAsync(net->m, 0, sizeof(float) * 2 * NPARAM, net->stream));
    lcc_status s = net_prep(net);
    if (s != LCC_OK) return s;
    LCC_CUDA(cudaStreamSynchronize(net->stream));
    return LCC_OK;
}

lcc_status lcc_net_tile_inputs_batch(lcc_ctx *c, int32_t nframes, const float *const *d_pts, const int64_t *n,
                                     uint16_t *d_x, float *d_anchor) {
    if (!c || !d_x || !d_anchor || !d_pts || !n) return LCC_ERR_INVALID_ARG;
    if (c->g.th != 8 || c->g.tw != 8) return LCC_ERR_UNSUPPORTED;
    if (nframes < 1 || nframes > c->slots || ((uintptr_t)d_x & 7u) || ((uintptr_t)d_anchor & 15u))
        return LCC_ERR_INVALID_ARG;
    for (int f = 0; f < nframes; f++)
        if (n[f] < 0 || (n[f] > 0 && (!d_pts[f] || ((uintptr_t)d_pts[f] & 15u)))) return LCC_ERR_INVALID_ARG;
    int slots[kMaxBatch];
    for (int f = 0; f < nframes; f++) slots[f] = f;
    lcc_status st = bin_frames(c, nframes, slots, d_pts, n);
    if (st != LCC_OK) return st;
    const int wpb = 8;
    k_net_inputs<true><<<dim3((c->g.NT + wpb - 1) / wpb, nframes), wpb * 32, 0, c->stream>>>(
        c->g, c->s.rimg, reinterpret_cast<bf16 *>(d_x), reinterpret_cast<float4 *>(d_anchor));
    return cudaGetLastError() == cudaSuccess ? LCC_OK : LCC_ERR_CUDA;
}

lcc_status lcc_net_tile_inputs(lcc_ctx *c, const float *d_pts, int64_t n, uint16_t *d_x, float *d_anchor) {
    return lcc_net_tile_inputs_batch(c, 1, &d_pts, &n, d_x, d_anchor);
}

lcc_status lcc_net_tile_labels(lcc_ctx *c, int32_t frame, const float *d_anchor, float *d_labels) {
    if (!c || !d_anchor || !d_labels || frame < 0 || frame >= c->last_nframes || ((uintptr_t)d_anchor & 15u))
        return LCC_ERR_INVALID_ARG;
    const int NT = c->g.NT;
    k_net_labels<<<(NT + 255) / 256, 256, 0, c->stream>>>(c->s.tiles + (size_t)frame * NT,
                                                          reinterpret_cast<const float4 *>(d_anchor), NT, d_labels);
    return cudaGetLastError() == cudaSuccess ? LCC_OK : LCC_ERR_CUDA;
}

lcc_status lcc_net_forward(lcc_net *net, const uint16_t *d_x, int64_t ntiles, float *d_out) {
    if (!net || !d_x || !d_out || ntiles < 0 || ((uintptr_t)d_x & 7u)) return LCC_ERR_INVALID_ARG;
    if (ntiles == 0) return LCC_OK;
    return forward_tc(net, d_x, ntiles, d_out, false);
}

lcc_status lcc_selftest_bounded_wait(int64_t limit, void *cuda_stream) {
    if (limit < 1 || limit > ((int64_t)1 << 30)) return LCC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int *d_err = nullptr;
    LCC_CUDA(cudaMalloc(&d_err, sizeof(int)));
    int e = 0;
    const bool ok = cudaMemsetAsync(d_err, 0, sizeof(int), st) == cudaSuccess &&
                    (k_bounded_wait_selftest<<<1, 32, 0, st>>>(limit, d_err), cudaGetLastError() == cudaSuccess) &&
                    cudaMemcpyAsync(&e, d_err, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
                    cudaStreamSynchronize(st) == cudaSuccess;
    cudaFree(d_err);
    if (!ok) return LCC_ERR_CUDA;
    return e ? LCC_ERR_TIMEOUT : LCC_OK;
}

lcc_status lcc_net_sync(lcc_net *net) {
    if (!net) return LCC_ERR_INVALID_ARG;
    LCC_CUDA(cudaStreamSynchronize(net->stream));
    int e = 0;
    LCC_CUDA(cudaMemcpy(&e, net->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        cudaMemset(net->err, 0, sizeof(int));
        return LCC_ERR_TIMEOUT;
    }
    return LCC_OK;
}

lcc_status lcc_net_gradient(lcc_net *net, const uint16_t *d_x, const float *d_labels, int64_t ntiles, float *d_grad,
                            float *d_loss) {
    if (!net || !d_x || !d_labels || ntiles < 1 || ntiles > net->max_tiles || ((uintptr_t)d_x & 7u))
        return LCC_ERR_INVALID_ARG;
    lcc_status s = backward(net, d_x, d_labels, ntiles);
    if (s != LCC_OK) return s;
    if (d_grad)
        LCC_CUDA(cudaMemcpyAsync(d_grad, net->grad, sizeof(float) * NPARAM, cudaMemcpyDeviceToDevice, net->stream));
    if (d_loss) LCC_CUDA(cudaMemcpyAsync(d_loss, net->loss, sizeof(float), cudaMemcpyDeviceToDevice, net->stream));
    return LCC_OK;
}

lcc_status lcc_net_train_step(lcc_net *net, const uint16_t *d_x, const float *d_labels, int64_t ntiles, float lr,
                              int32_t step, float *d_loss) {
    if (!net || step < 1 || !(lr > 0)) return LCC_ERR_INVALID_ARG;
    lcc_status s = lcc_net_gradient(net, d_x, d_labels, ntiles, nullptr, d_loss);
    if (s != LCC_OK) return s;
    const float bc1 = 1.f - powf(0.9f, (float)step), bc2 = 1.f - powf(0.999f, (float)step);
    k_net_adam<<<64, 256, 0, net->stream>>>(net->theta, net->grad, net->m, net->v, NPARAM, lr, bc1, bc2);
    if (cudaGetLastError() != cudaSuccess) return LCC_ERR_CUDA;
    return net_prep(net);
}

}  // extern "C"
