// Lossless entropy stage (Sec. III-A, its last paragraph): the planes and residual maps left by
// spatial and temporal coding pass through a lossless coder, Huffman coding being the one named.
//
// The stage is a lossless transform of a fixed-width frame stream into an entropy stream and
// back.  Sections, in stream order: the occupancy bitmap as 8-bit symbols (its bytes), the tile
// codes as 4-bit symbols, the run planes and temporal records copied, the fitted bits as 8-bit
// symbols, the residual and raw codes as symbols of their own width.  A symbol section of width
// <= 12 with at least one symbol gets its own canonical Huffman code when the coded form (4-bit
// length table, one offset word per 1024-symbol chunk, word-padded chunks of codes) is smaller
// than the copy.  Code lengths: Huffman's construction over the symbols that occur sorted by
// (count, symbol), the two lightest nodes joined at each step, a leaf before an internal node of
// equal weight; lengths above 15 halve every count (rounding up) and the construction runs
// again.  Canonical codes: consecutive in (length, symbol) order, the first code of each length
// from the DEFLATE rule.  A code's bits go most significant first to increasing bit positions
// (LSB-first words).
//
// Entropy stream: the fixed-width stream's 64-byte header; word 16 "LCE1"; word 17 the stream's
// bytes; words 18..45 one descriptor per section (mode | width << 8, count, alphabet, words);
// then the sections.
//
// Kernels.  Encode: k_ent_build (a CTA per frame and symbol section: histogram, sort, Huffman
// lengths, canonical codes, chunk sizes, the copy-or-code decision), k_ent_layout (a warp per
// frame: section offsets, capacity, header, length tables, chunk offsets), k_ent_write (a thread
// per 1024-symbol chunk writes its codes; the copied sections move a block of words per CTA).
// Decode: k_ent_dec_prep (a CTA per frame and section: validation, canonical decode tables),
// k_ent_dec (a thread per chunk decodes into the fixed-width section; copies as above).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "lcc_ctx.cuh"

namespace lcc {
namespace ent {

constexpr uint32_t kEntMagic = 0x3145434Cu;   // "LCE1"
constexpr int kChunk = 1024;
constexpr int kMaxLen = 15;
constexpr int kMaxWidth = 12;
constexpr int kMaxAlph = 1 << kMaxWidth;
constexpr int kSecs = 7;
constexpr int kEntHeaderWords = 16 + 2 + kSecs * 4;
constexpr int kBuildThreads = 1024;
constexpr int kWriteThreads = 128;
constexpr int kCopyWords = 1024;   // words a CTA copies per step of a copied section

struct Layout {            // a fixed-width stream's sections, from its header
    uint32_t width[kSecs];  // symbol width (0: a section that is always copied)
    uint32_t count[kSecs];  // symbols
    uint32_t words[kSecs];  // 32-bit words in the fixed-width stream
    uint32_t off[kSecs];    // word offset after the 64-byte header
    uint32_t total;         // bytes
};

struct Sec {               // one section of one frame in the entropy stream
    uint32_t mode;          // 0 copy, 1 Huffman
    uint32_t alph;
    uint32_t nch;
    uint32_t words;         // words in the entropy stream
    uint32_t ent_off;       // word offset in the entropy stream
    uint32_t per_len[kMaxLen + 1];
    uint32_t first[kMaxLen + 1];
    uint32_t index[kMaxLen + 2];
};

struct Frame {
    Sec sec[kSecs];
    Layout L;
    uint32_t ok;
};

struct Scratch {
    Frame *frame;          // [slots]
    uint8_t *len;          // [slots][7][kMaxAlph]
    uint16_t *rcode;       // [slots][7][kMaxAlph] codes with their bits reversed (LSB = first bit)
    uint16_t *sorted;      // [slots][7][kMaxAlph] symbols in (length, symbol) order (decoder)
    uint32_t *chunk;       // [slots][7][max_chunks] chunk words, then chunk offsets (in place)
    uint32_t max_chunks;
};

struct EntBatch {
    const uint8_t *in[kMaxBatch];
    uint8_t *out[kMaxBatch];
    unsigned long long in_size[kMaxBatch];   // bytes readable at in[f]
    unsigned long long out_cap[kMaxBatch];
    unsigned long long *out_bytes;            // device, one per frame
    uint32_t rows, cols;
};

__device__ __forceinline__ uint32_t words_of_bits(unsigned long long bits) { return (uint32_t)((bits + 31) / 32); }

// Section layout of the fixed-width stream whose header is h (16-byte aligned); false if the
// header is not one of this sensor's streams or its sizes disagree.
__device__ bool parse_fixed(const uint8_t *h, unsigned long long avail, uint32_t rows, uint32_t cols, Layout &L) {
    if (avail < (unsigned long long)kHeaderBytes) return false;
    const uint32_t *w = reinterpret_cast<const uint32_t *>(h);
    if (w[0] != kMagic || (w[1] & 0xFFFFu) != (uint32_t)kVersion) return false;
    const uint32_t flags = w[1] >> 24;
    if ((w[2] & 0xFFFFu) != rows || (w[2] >> 16) != cols) return false;
    const uint32_t w_res = (w[3] >> 16) & 0xFFu, w_raw = w[3] >> 24;
    const uint32_t n_tiles = w[6], n_runs = w[8], n_temp = w[9], n_cand = w[10], n_fit = w[11], n_raw = w[12];
    const unsigned long long npx = (unsigned long long)rows * cols;
    if (w_res > 32 || w_raw > 32 || n_tiles > npx || n_runs > n_tiles || n_temp > n_tiles || n_cand > npx ||
        n_fit > n_cand || n_raw > npx)
        return false;
    const uint32_t bw = words_of_bits(npx), fw = words_of_bits(n_cand);
    const uint32_t res_cnt = (flags & 2u) ? 0u : n_fit;
    const uint32_t width[kSecs] = {8, 4, 0, 0, 8, w_res, w_raw};
    const uint32_t count[kSecs] = {4 * bw, n_tiles, 0, 0, 4 * fw, res_cnt, n_raw};
    const uint32_t words[kSecs] = {bw,
                                   words_of_bits(4ull * n_tiles),
                                   ((flags & 16u) ? 3u : 4u) * n_runs,   // three-coefficient planes: 3 words
                                   2 * n_temp,
                                   fw,
                                   words_of_bits((unsigned long long)res_cnt * w_res),
                                   words_of_bits((unsigned long long)n_raw * w_raw)};
    unsigned long long o = 0;
    for (int s = 0; s < kSecs; s++) {
        L.width[s] = width[s];
        L.count[s] = count[s];
        L.words[s] = words[s];
        L.off[s] = (uint32_t)o;
        o += words[s];
    }
    const unsigned long long total = (unsigned long long)kHeaderBytes + 4 * o;
    if (total != w[14] || total > avail) return false;
    L.total = (uint32_t)total;
    return true;
}

__device__ __forceinline__ bool coded_width(uint32_t w) { return w >= 1 && w <= (uint32_t)kMaxWidth; }

// Symbol i of a section of width w (LSB-first in words; the symbol lies inside the section).
__device__ __forceinline__ uint32_t get_sym(const uint32_t *sec, uint32_t w, uint32_t i) {
    const unsigned long long p = (unsigned long long)i * w;
    const uint32_t wi = (uint32_t)(p >> 5), sh = (uint32_t)(p & 31);
    uint32_t v = sec[wi] >> sh;
    if (sh + w > 32) v |= sec[wi + 1] << (32 - sh);
    return v & ((1u << w) - 1u);
}

// m symbols of a section of width w from symbol `first` on, in order: first is a multiple of 32,
// so the run starts on a word (32 symbols of w bits fill w words); words are read one ahead of
// their use.
struct SymReader {
    const uint32_t *in;
    uint32_t words, ip, nxt, w, m;
    unsigned long long buf;
    int nb;
    __device__ SymReader(const uint32_t *sec, uint32_t w_, uint32_t first, uint32_t m_) {
        w = w_;
        m = m_;
        in = sec + (size_t)first * w / 32;
        words = (uint32_t)(((unsigned long long)m * w + 31) / 32);
        ip = 0;
        nxt = words ? in[0] : 0u;
        buf = 0;
        nb = 0;
    }
    __device__ __forceinline__ uint32_t next() {
        if (nb < (int)w) {
            buf |= (unsigned long long)nxt << nb;
            nb += 32;
            ip++;
            nxt = ip < words ? in[ip] : 0u;
        }
        const uint32_t v = (uint32_t)buf & ((1u << w) - 1u);
        buf >>= w;
        nb -= (int)w;
        return v;
    }
};

__device__ uint32_t block_sum(uint32_t v, uint32_t *red) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += red[k];
    __syncthreads();
    return t;
}

__device__ uint32_t block_max(uint32_t v, uint32_t *red) {
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t = max(t, red[k]);
    __syncthreads();
    return t;
}

// Exclusive prefix sum over the block (threads in order); *total receives the sum.
__device__ uint32_t block_excl(uint32_t v, uint32_t *red, uint32_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) red[wid] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
        if (k < wid) before += red[k];
        all += red[k];
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

// Ascending bitonic sort of keys[0, P), P a power of two up to 4 blockDim (the textbook
// network, every compare-exchange of it).  Each thread holds E = max(1, P / blockDim) consecutive
// keys in registers, so a warp holds 32 E consecutive keys: the steps whose partner distance j is
// below 32 E exchange in registers and by shuffles; only the longer ones go through shared memory
// with a barrier.  keys must be in shared memory and complete (barrier before the call); they are
// sorted in place and complete after it.
__device__ void bitonic_sort(unsigned long long *keys, uint32_t P) {
    const uint32_t T = blockDim.x, t = threadIdx.x;
    const uint32_t E = P > T ? P / T : 1u;      // 1, 2 or 4
    const uint32_t base = t * E, WR = 32u * E;   // first key of the thread, keys per warp
    unsigned long long r[4];
#pragma unroll
    for (int e = 0; e < 4; e++) r[e] = (uint32_t)e < E && base + e < P ? keys[base + e] : ~0ull;
    // one compare-exchange in registers: lo keeps the smaller key when up
    auto cx = [](unsigned long long &lo, unsigned long long &hi, bool up) {
        if ((lo > hi) == up) {
            const unsigned long long x = lo;
            lo = hi;
            hi = x;
        }
    };
    for (uint32_t k = 2; k <= P; k <<= 1) {
        uint32_t j = k >> 1;
        if (j >= WR) {
#pragma unroll
            for (int e = 0; e < 4; e++)
                if ((uint32_t)e < E && base + e < P) keys[base + e] = r[e];
            __syncthreads();
            for (; j >= WR; j >>= 1) {
                for (uint32_t i = t; i < P; i += T) {
                    const uint32_t l = i ^ j;
                    if (l > i) {
                        const unsigned long long a = keys[i], b = keys[l];
                        const bool up = (i & k) == 0;
                        if ((a > b) == up) {
                            keys[i] = b;
                            keys[l] = a;
                        }
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int e = 0; e < 4; e++) r[e] = (uint32_t)e < E && base + e < P ? keys[base + e] : ~0ull;
        }
        for (; j > 0; j >>= 1) {
            if (j >= E) {   // partner: the same slot of lane ^ (j / E)
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    if ((uint32_t)e >= E) break;
                    const uint32_t i = base + e;
                    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, r[e], j / E);
                    const bool up = (i & k) == 0, lower = (i & j) == 0;
                    r[e] = up == lower ? (r[e] < o ? r[e] : o) : (r[e] > o ? r[e] : o);
                }
            } else if (j == 2) {   // E == 4: slots (0, 2) and (1, 3)
                cx(r[0], r[2], (base & k) == 0);
                cx(r[1], r[3], ((base + 1) & k) == 0);
            } else {               // j == 1, E >= 2: slots (0, 1) and (2, 3)
                cx(r[0], r[1], (base & k) == 0);
                if (E == 4) cx(r[2], r[3], ((base + 2) & k) == 0);
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 4; e++)
        if ((uint32_t)e < E && base + e < P) keys[base + e] = r[e];
    __syncthreads();
}

// Canonical tables of a length table (any thread count): per length the number of codes, the
// first code and the index of its first symbol in (length, symbol) order.  Thread 0 only.
__device__ void canonical_tables(const uint32_t *per_len, uint32_t *first, uint32_t *index) {
    uint32_t code = 0;
    index[0] = index[1] = 0;
    first[0] = 0;
    for (int l = 1; l <= kMaxLen; l++) {
        code = l > 1 ? (code + per_len[l - 1]) << 1 : 0u;
        first[l] = code;
        index[l + 1] = index[l] + per_len[l];
    }
}

// Every used symbol's position in (length, symbol) order, handed to place(symbol, length,
// position).  A thread takes a run of consecutive symbols; for each length that has symbols, a
// block-wide exclusive scan of the threads' counts of that length gives each thread its first
// position (index[l] is the position of the first symbol of length l).  red: 32 words.  Called
// by every thread of the block; it starts with a barrier, so len and index may have been written
// by any thread just before the call.
template <class F>
__device__ void place_by_length(const uint8_t *len, uint32_t alph, const uint32_t *index, uint32_t *red,
                                F &&place) {
    __syncthreads();
    const uint32_t T = blockDim.x, t = threadIdx.x;
    const uint32_t per = (alph + T - 1) / T, s0 = min(alph, t * per), s1 = min(alph, s0 + per);
    for (uint32_t l = 1; l <= (uint32_t)kMaxLen; l++) {
        if (index[l + 1] == index[l]) continue;   // no symbol of this length (the same in every thread)
        uint32_t own = 0;
        for (uint32_t v = s0; v < s1; v++) own += len[v] == l ? 1u : 0u;
        uint32_t total;
        uint32_t pos = index[l] + block_excl(own, red, &total);
        for (uint32_t v = s0; v < s1; v++)
            if (len[v] == l) place(v, l, pos++);
    }
    __syncthreads();
}

// One warp copies the words holding symbols [b0, b0 + m) of a section of width w (b0 a multiple
// of 32, so its first symbol starts a word; m <= 1024) into buf, all of its loads in flight at
// once; the words are in buf for every lane after the call.
__device__ __forceinline__ void stage_symbols(const uint32_t *sec, uint32_t w, uint32_t b0, uint32_t m, uint32_t *buf) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nw = (uint32_t)(((unsigned long long)m * w + 31) / 32);
    const uint32_t *src = sec + (size_t)b0 / 32 * w;
    uint32_t v[kMaxWidth];
#pragma unroll
    for (int k = 0; k < kMaxWidth; k++) {
        const uint32_t i = lane + 32u * k;
        v[k] = i < nw ? src[i] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kMaxWidth; k++) {
        const uint32_t i = lane + 32u * k;
        if (i < nw) buf[i] = v[k];
    }
    __syncwarp();
}

struct BuildSmem {
    unsigned long long keys[kMaxAlph];
    uint32_t hist[kMaxAlph];        // counts; then the internal nodes' weights
    uint16_t leaf_parent[kMaxAlph];
    uint16_t node_parent[kMaxAlph];
    uint16_t node_depth[kMaxAlph];
    uint32_t lw[kMaxAlph];          // leaf weights in queue order
    uint32_t tw[kMaxAlph];          // a batch's items in pick order (their weights)
    uint32_t stage[kBuildThreads / 32][32 * kMaxWidth];   // per warp: the words of 1024 symbols
    uint8_t len[kMaxAlph];
    uint32_t red[32];
    uint32_t last_leaf;
    uint32_t per_len[kMaxLen + 1];
    uint32_t first[kMaxLen + 1];
    uint32_t index[kMaxLen + 2];
};

// Huffman's two-queue construction over the n >= 2 leaf weights S.lw (sorted by (count,
// symbol)): node k's weight goes to S.hist[k], every leaf's and node's parent to S.leaf_parent /
// S.node_parent.  Picks follow the two-queue rule (the lighter front; a leaf first on equal
// weights), and they are taken a batch at a time: with m the weight of the next node to be made
// (its two picks), every remaining node made so far (node weights never decrease, so they are
// all <= m) and every remaining leaf of weight <= m is picked before any node made from here on
// (a later node weighs >= m; a leaf wins ties and older nodes are ahead in their queue).  Those
// items, in pick order (a merge of the two sorted queue segments, ranks by binary search),
// pair up into the next nodes; an odd last item stays at its queue's front.  The smallest pair
// grows at least like a Fibonacci sequence from batch to batch, so the batches number
// O(log of the total count); after kMaxBatches one thread makes the remaining joins one by one.
// All threads of the block call this.
constexpr int kMaxBatches = 48;

__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t v) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t lower_bound_u32(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t v) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <class Smem>
__device__ void huffman_joins(Smem &S, uint32_t n) {
    const uint32_t tid = threadIdx.x;
    constexpr uint32_t kNone = 0xFFFFFFFFu;
    uint32_t li = 0, ni = 0, nk = 0;   // leaf front, node front, nodes made (the same in every thread)
    for (int batch = 0; batch < kMaxBatches && nk + 1 < n; batch++) {
        const uint32_t l0 = li < n ? S.lw[li] : kNone, l1 = li + 1 < n ? S.lw[li + 1] : kNone;
        const uint32_t n0 = ni < nk ? S.hist[ni] : kNone, n1 = ni + 1 < nk ? S.hist[ni + 1] : kNone;
        const uint32_t m = l0 <= n0 ? l0 + (l1 <= n0 ? l1 : n0) : n0 + (l0 <= n1 ? l0 : n1);
        const uint32_t a = upper_bound_u32(S.lw, li, n, m) - li, b = nk - ni;
        const uint32_t T = a + b, P = T >> 1;
        for (uint32_t e = tid; e < T; e += blockDim.x) {
            uint32_t w, r;
            if (e < a) {   // a leaf goes after the nodes strictly lighter than it
                w = S.lw[li + e];
                r = e + (lower_bound_u32(S.hist, ni, nk, w) - ni);
            } else {       // a node goes after the leaves no heavier than it
                w = S.hist[ni + e - a];
                r = (e - a) + (upper_bound_u32(S.lw, li, li + a, w) - li);
            }
            S.tw[r] = w;
            if (r < 2 * P) {
                if (e < a) S.leaf_parent[li + e] = (uint16_t)(nk + (r >> 1));
                else S.node_parent[ni + e - a] = (uint16_t)(nk + (r >> 1));
            } else {       // the odd last item
                S.last_leaf = e < a ? 1u : 0u;
            }
        }
        __syncthreads();
        const bool leaf_left = (T & 1) && S.last_leaf;   // read before the next batch can write it
        for (uint32_t q = tid; q < P; q += blockDim.x) S.hist[nk + q] = S.tw[2 * q] + S.tw[2 * q + 1];
        __syncthreads();
        li += (T & 1) && leaf_left ? a - 1 : a;
        ni += (T & 1) && !leaf_left ? b - 1 : b;
        nk += P;
    }
    if (tid == 0 && nk + 1 < n) {
        // the two-queue rule one join at a time; each queue's front weight is kept in a register
        // (kNone: empty) and the second one loaded a join ahead
        uint32_t wl = li < n ? S.lw[li] : kNone, wl2 = li + 1 < n ? S.lw[li + 1] : kNone;
        uint32_t wn = ni < nk ? S.hist[ni] : kNone, wn2 = ni + 1 < nk ? S.hist[ni + 1] : kNone;
        for (uint32_t k = nk; k + 1 < n; k++) {
            uint32_t wsum = 0;
#pragma unroll
            for (int pick = 0; pick < 2; pick++) {
                if (wl <= wn) {
                    wsum += wl;
                    S.leaf_parent[li++] = (uint16_t)k;
                    wl = wl2;
                    wl2 = li + 1 < n ? S.lw[li + 1] : kNone;
                } else {
                    wsum += wn;
                    S.node_parent[ni++] = (uint16_t)k;
                    wn = wn2;
                    wn2 = ni + 1 < k ? S.hist[ni + 1] : kNone;
                }
            }
            S.hist[k] = wsum;
            if (ni == k) wn = wsum;
            else if (ni + 1 == k) wn2 = wsum;
        }
    }
    __syncthreads();
}

// grid (5 symbol sections, nframes), kBuildThreads threads
__global__ void __launch_bounds__(kBuildThreads) k_ent_build(EntBatch b, Scratch sc, unsigned *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BuildSmem &S = *reinterpret_cast<BuildSmem *>(smem_raw);
    const int sid_of[5] = {0, 1, 4, 5, 6};
    const int s = sid_of[blockIdx.x], f = blockIdx.y;
    const int tid = threadIdx.x;
    Frame &F = sc.frame[f];
    Layout L;
    const bool valid = parse_fixed(b.in[f], b.in_size[f], b.rows, b.cols, L);
    if (!valid) {
        if (blockIdx.x == 0 && tid == 0) {
            F.ok = 0;
            atomicOr(err, E_CORRUPT);
        }
        return;
    }
    if (blockIdx.x == 0 && tid == 0) {
        F.L = L;
        for (int k = 2; k <= 3; k++) {   // the run planes and temporal records are copied
            F.sec[k].mode = 0;
            F.sec[k].alph = 0;
            F.sec[k].nch = 0;
            F.sec[k].words = L.words[k];
        }
    }
    Sec &out = F.sec[s];
    const uint32_t w = L.width[s], cnt = L.count[s];
    if (!coded_width(w) || cnt == 0) {
        if (tid == 0) {
            out.mode = 0;
            out.alph = 0;
            out.nch = 0;
            out.words = L.words[s];
        }
        return;
    }
    const uint32_t *sec = reinterpret_cast<const uint32_t *>(b.in[f] + kHeaderBytes) + L.off[s];
    // histogram, a warp per block of 1024 symbols staged in shared memory.  Widths up to 4: each
    // lane counts its 32 consecutive symbols in registers (16-bit fields; a lane sees at most
    // 32 symbols per block, so the fields cannot overflow below 2^21 blocks); widths 5..8: lanes
    // holding the same symbol add once (__match_any) into the warp's own copy of the histogram
    // (the sorting keys' space, not in use yet); wider: one shared atomic per symbol (large
    // alphabets rarely collide)
    constexpr uint32_t kPrivAlph = 256, kNone = 0xFFFFFFFFu;
    static_assert(sizeof(S.keys) >= 32 * kPrivAlph * sizeof(uint32_t), "per-warp histograms");
    const uint32_t lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const bool regc = w <= 4, priv = w > 4 && w <= 8;
    uint32_t *wh = reinterpret_cast<uint32_t *>(S.keys);
    uint32_t *wbuf = S.stage[warp];
    for (int i = tid; i < kMaxAlph; i += blockDim.x) {
        S.hist[i] = 0;
        S.len[i] = 0;
    }
    if (priv)
        for (int i = tid; i < 32 * (int)kPrivAlph; i += blockDim.x) wh[i] = 0;
    __syncthreads();
    uint32_t *hh = priv ? wh + warp * kPrivAlph : S.hist;
    uint32_t c2[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};   // symbol 2k in the low half of c2[k], 2k + 1 in the high
    const uint32_t nblk = (cnt + kChunk - 1) / kChunk;
    for (uint32_t blk = warp; blk < nblk; blk += nwarp) {
        const uint32_t b0 = blk * kChunk, m = min(cnt - b0, (uint32_t)kChunk);
        stage_symbols(sec, w, b0, m, wbuf);
        if (regc) {
            const uint32_t s0 = 32 * lane;
            SymReader rd(wbuf, w, s0, s0 < m ? min(m - s0, 32u) : 0u);
            for (uint32_t i = 0; i < rd.m; i++) {
                const uint32_t v = rd.next(), q = v >> 1, inc = 1u << ((v & 1u) << 4);
#pragma unroll
                for (int k = 0; k < 8; k++) c2[k] += q == (uint32_t)k ? inc : 0u;
            }
        } else {
            for (uint32_t k = 0; k < 32; k++) {
                const uint32_t i = 32 * k + lane;
                const uint32_t v = i < m ? get_sym(wbuf, w, i) : kNone;
                if (priv) {
                    const unsigned same = __match_any_sync(0xFFFFFFFFu, v);
                    if (v != kNone && lane == (uint32_t)__ffs(same) - 1) atomicAdd(&hh[v], (uint32_t)__popc(same));
                } else if (v != kNone) {
                    atomicAdd(&hh[v], 1u);
                }
            }
        }
        __syncwarp();   // the staged words are read before the next block overwrites them
    }
    if (regc) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            uint32_t lo = c2[k] & 0xFFFFu, hi = c2[k] >> 16;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                lo += __shfl_xor_sync(0xFFFFFFFFu, lo, o);
                hi += __shfl_xor_sync(0xFFFFFFFFu, hi, o);
            }
            if (lane == 0) {
                if (lo) atomicAdd(&S.hist[2 * k], lo);
                if (hi) atomicAdd(&S.hist[2 * k + 1], hi);
            }
        }
    }
    __syncthreads();
    if (priv) {
        for (uint32_t v = tid; v < kPrivAlph; v += blockDim.x) {
            uint32_t t = 0;
            for (int k = 0; k < 32; k++) t += wh[k * kPrivAlph + v];
            S.hist[v] = t;
        }
        __syncthreads();
    }
    uint32_t top = 0;
    for (uint32_t v = tid; v < (1u << w); v += blockDim.x)
        if (S.hist[v]) top = v + 1;
    const uint32_t alph = block_max(top, S.red);
    // used symbols as (count << 12 | symbol), in symbol order
    const uint32_t per = (alph + blockDim.x - 1) / blockDim.x;
    const uint32_t s0 = min(alph, tid * per), s1 = min(alph, s0 + per);
    uint32_t own = 0;
    for (uint32_t v = s0; v < s1; v++) own += S.hist[v] != 0;
    uint32_t n = 0;
    uint32_t pos = block_excl(own, S.red, &n);
    for (uint32_t v = s0; v < s1; v++)
        if (S.hist[v]) S.keys[pos++] = (unsigned long long)S.hist[v] << 12 | v;
    __syncthreads();
    if (n == 1) {
        if (tid == 0) S.len[S.keys[0] & 0xFFFu] = 1;
    } else {
        uint32_t P = 2;
        while (P < n) P <<= 1;
        for (;;) {
            for (uint32_t i = n + tid; i < P; i += blockDim.x) S.keys[i] = ~0ull;
            __syncthreads();
            bitonic_sort(S.keys, P);
            for (uint32_t i = tid; i < n; i += blockDim.x) S.lw[i] = (uint32_t)(S.keys[i] >> 12);
            __syncthreads();
            huffman_joins(S, n);
            // node depths by pointer jumping (children are made before parents, the root last):
            // node_parent becomes an ancestor pointer and node_depth the edges up to it
            for (uint32_t k = tid; k + 1 < n; k += blockDim.x) {
                const bool root = k + 2 == n;
                if (root) S.node_parent[k] = (uint16_t)k;
                S.node_depth[k] = root ? 0 : 1;
            }
            __syncthreads();
            // (2^12 >= the 4095 nodes a tree can have; the rounds stop once every pointer is the root)
            for (int r = 0; r < kMaxWidth; r++) {
                constexpr int kPer = kMaxAlph / kBuildThreads;   // nodes a thread holds (registers)
                uint16_t na[kPer], nd[kPer];
                int moved = 0;
#pragma unroll
                for (int q = 0; q < kPer; q++) {
                    const uint32_t k = tid + q * kBuildThreads;
                    if (k + 1 < n) {
                        const uint16_t a = S.node_parent[k];
                        na[q] = S.node_parent[a];
                        nd[q] = S.node_depth[k] + S.node_depth[a];
                        moved |= na[q] != a;
                    }
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < kPer; q++) {
                    const uint32_t k = tid + q * kBuildThreads;
                    if (k + 1 < n) {
                        S.node_parent[k] = na[q];
                        S.node_depth[k] = nd[q];
                    }
                }
                if (!__syncthreads_or(moved)) break;
            }
            uint32_t deep = 0;
            for (uint32_t i = tid; i < n; i += blockDim.x) deep = max(deep, (uint32_t)S.node_depth[S.leaf_parent[i]] + 1);
            if (block_max(deep, S.red) <= (uint32_t)kMaxLen) break;
            // too deep: halve every count (rounding up) and build again
            for (uint32_t i = tid; i < n; i += blockDim.x) {
                const unsigned long long c = S.keys[i] >> 12;
                S.keys[i] = ((c + 1) >> 1) << 12 | (S.keys[i] & 0xFFFu);
            }
            __syncthreads();
        }
        for (uint32_t i = tid; i < n; i += blockDim.x)
            S.len[S.keys[i] & 0xFFFu] = (uint8_t)(S.node_depth[S.leaf_parent[i]] + 1);
    }
    __syncthreads();
    // canonical codes: rank in (length, symbol) order.  Codes per length: a thread counts its (at
    // most 4) symbols in 4-bit fields of one register, the fields are widened to bytes (even and
    // odd lengths apart) and summed over the warp, and each warp adds its 15 counts once (a shared
    // atomic per symbol queued thousands of symbols on a dozen counters)
    if (tid <= kMaxLen) S.per_len[tid] = 0;
    __syncthreads();
    {
        static_assert(kMaxAlph / kBuildThreads <= 4 && 32 * 4 < 256, "per-length fields");
        unsigned long long c4 = 0ull;   // field l - 1: symbols of length l
        for (uint32_t v = tid; v < alph; v += blockDim.x) {
            const uint32_t l = S.len[v];
            if (l) c4 += 1ull << (4 * (l - 1));
        }
        unsigned long long ev = c4 & 0x0F0F0F0F0F0F0F0Full, od = (c4 >> 4) & 0x0F0F0F0F0F0F0F0Full;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            ev += __shfl_xor_sync(0xFFFFFFFFu, ev, o);
            od += __shfl_xor_sync(0xFFFFFFFFu, od, o);
        }
        if (lane == 0)
            for (int l = 1; l <= kMaxLen; l++) {
                const uint32_t q = (uint32_t)((((l - 1) & 1) ? od : ev) >> (8 * ((l - 1) >> 1))) & 0xFFu;
                if (q) atomicAdd(&S.per_len[l], q);
            }
    }
    __syncthreads();
    if (tid == 0) canonical_tables(S.per_len, S.first, S.index);
    __syncthreads();
    const size_t tab = ((size_t)f * kSecs + s) * kMaxAlph;
    place_by_length(S.len, alph, S.index, S.red, [&](uint32_t v, uint32_t l, uint32_t pos) {
        const uint32_t code = S.first[l] + (pos - S.index[l]);
        sc.rcode[tab + v] = (uint16_t)(__brev(code) >> (32 - l));
    });
    for (uint32_t v = tid; v < alph; v += blockDim.x) sc.len[tab + v] = S.len[v];
    // chunk sizes
    const uint32_t nch = (cnt + kChunk - 1) / kChunk;
    uint32_t *cw = sc.chunk + ((size_t)f * kSecs + s) * sc.max_chunks;
    uint32_t mine = 0;
    for (uint32_t c = warp; c < nch; c += nwarp) {   // a warp per chunk (staged), 32 symbols a lane
        const uint32_t c0 = c * kChunk, m = min(cnt - c0, (uint32_t)kChunk), s0 = 32 * lane;
        stage_symbols(sec, w, c0, m, wbuf);
        SymReader rd(wbuf, w, s0, s0 < m ? min(m - s0, 32u) : 0u);
        uint32_t bits = 0;
        for (uint32_t i = 0; i < rd.m; i++) bits += S.len[rd.next()];
        for (int o = 16; o; o >>= 1) bits += __shfl_xor_sync(0xFFFFFFFFu, bits, o);
        if (lane == 0) {
            cw[c] = (bits + 31) / 32;
            mine += (bits + 31) / 32;
        }
        __syncwarp();
    }
    const uint32_t payload = block_sum(mine, S.red);
    if (tid == 0) {
        const uint32_t coded = (alph + 7) / 8 + nch + payload;
        out.mode = coded < L.words[s] ? 1u : 0u;
        out.alph = out.mode ? alph : 0u;
        out.nch = out.mode ? nch : 0u;
        out.words = out.mode ? coded : L.words[s];
    }
}

// grid nframes, 32 * kSecs threads: every warp derives the section offsets; warp 0 writes the
// header and descriptors, warp s the length table and chunk offsets of section s
__global__ void __launch_bounds__(32 * kSecs) k_ent_layout(EntBatch b, Scratch sc, unsigned *err, int nframes) {
    const int f = blockIdx.x, lane = threadIdx.x & 31, s = threadIdx.x >> 5;
    if (f >= nframes) return;
    Frame &F = sc.frame[f];
    Layout L;
    if (!parse_fixed(b.in[f], b.in_size[f], b.rows, b.cols, L)) {
        if (threadIdx.x == 0) b.out_bytes[f] = 0;
        return;
    }
    uint32_t eo[kSecs];
    uint32_t off = kEntHeaderWords;
    for (int k = 0; k < kSecs; k++) {
        eo[k] = off;
        off += F.sec[k].words;
    }
    const unsigned long long total = 4ull * off;
    if (total > b.out_cap[f]) {
        if (threadIdx.x == 0) {
            F.ok = 0;
            b.out_bytes[f] = total;
            atomicOr(err, E_CAPACITY);
        }
        return;
    }
    uint32_t *o = reinterpret_cast<uint32_t *>(b.out[f]);
    if (s == 0) {
        const uint32_t *h = reinterpret_cast<const uint32_t *>(b.in[f]);
        if (lane < 16) o[lane] = h[lane];
        if (lane == 16) o[16] = kEntMagic;
        if (lane == 17) o[17] = (uint32_t)total;
        if (lane < kSecs) {
            F.sec[lane].ent_off = eo[lane];
            const Sec &D = F.sec[lane];
            o[18 + 4 * lane] = D.mode ? (1u | L.width[lane] << 8) : 0u;
            o[19 + 4 * lane] = D.mode ? L.count[lane] : L.words[lane];
            o[20 + 4 * lane] = D.alph;
            o[21 + 4 * lane] = D.words;
        }
        if (lane == 0) {
            F.ok = 1;
            b.out_bytes[f] = total;
        }
    }
    const Sec &S = F.sec[s];
    if (!S.mode) return;
    uint32_t *dst = o + eo[s];
    // 4-bit length table: eight byte lengths from two 32-bit loads per word (the table's base is
    // kMaxAlph-aligned); bytes past the alphabet are stale from earlier calls and masked out
    const uint32_t *len4 = reinterpret_cast<const uint32_t *>(sc.len + ((size_t)f * kSecs + s) * kMaxAlph);
    const uint32_t tw = (S.alph + 7) / 8;
#pragma unroll 4
    for (uint32_t j = lane; j < tw; j += 32) {
        const unsigned long long v8 = (unsigned long long)len4[2 * j] | ((unsigned long long)len4[2 * j + 1] << 32);
        uint32_t v = 0;
#pragma unroll
        for (uint32_t k = 0; k < 8; k++)
            if (8 * j + k < S.alph) v |= ((uint32_t)(v8 >> (8 * k)) & 15u) << (4 * k);
        dst[j] = v;
    }
    // chunk offsets: exclusive prefix of the chunk sizes, kept in place for the writer
    uint32_t *cw = sc.chunk + ((size_t)f * kSecs + s) * sc.max_chunks;
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < S.nch; c0 += 32) {
        const uint32_t c = c0 + lane;
        const uint32_t v = c < S.nch ? cw[c] : 0u;
        uint32_t x = v;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= d) x += y;
        }
        if (c < S.nch) {
            cw[c] = carry + x - v;
            dst[tw + c] = carry + x - v;
        }
        carry += __shfl_sync(0xFFFFFFFFu, x, 31);
    }
}

// grid (G, 7 sections, nframes), kWriteThreads threads: chunks and copied words with stride G
__global__ void __launch_bounds__(kWriteThreads) k_ent_write(EntBatch b, Scratch sc) {
    const int s = blockIdx.y, f = blockIdx.z;
    const Frame &F = sc.frame[f];
    if (!F.ok) return;
    const Sec &S = F.sec[s];
    const Layout &L = F.L;
    const uint32_t *sec = reinterpret_cast<const uint32_t *>(b.in[f] + kHeaderBytes) + L.off[s];
    uint32_t *dst = reinterpret_cast<uint32_t *>(b.out[f]) + S.ent_off;
    if (!S.mode) {
        for (uint32_t base = blockIdx.x * kCopyWords; base < L.words[s]; base += gridDim.x * kCopyWords) {
            const uint32_t e = min(L.words[s], base + kCopyWords);
            for (uint32_t i = base + threadIdx.x; i < e; i += blockDim.x) dst[i] = sec[i];
        }
        return;
    }
    constexpr int kWarps = kWriteThreads / 32;
    if (blockIdx.x * kWarps >= S.nch) return;
    // the section's codes in shared memory: reversed code | length << 16; a chunk buffer per warp
    __shared__ uint32_t s_code[kMaxAlph];
    __shared__ uint32_t s_buf[kWarps][kChunk * kMaxLen / 32];
    __shared__ uint32_t s_sym[kWarps][32 * kMaxWidth];   // the chunk's fixed-width words (staged once)
    const size_t tab = ((size_t)f * kSecs + s) * kMaxAlph;
    {   // four entries per thread and step: 8-byte code loads and 4-byte length loads (the tables'
        // bases are kMaxAlph-aligned; entries past the alphabet are loaded but never looked up)
        const uint2 *rc4 = reinterpret_cast<const uint2 *>(sc.rcode + tab);
        const uint32_t *ln4 = reinterpret_cast<const uint32_t *>(sc.len + tab);
        for (uint32_t v4 = threadIdx.x; v4 < (S.alph + 3) / 4; v4 += blockDim.x) {
            const uint2 rc = rc4[v4];
            const uint32_t ln = ln4[v4];
            s_code[4 * v4] = (rc.x & 0xFFFFu) | (ln & 0xFFu) << 16;
            s_code[4 * v4 + 1] = (rc.x >> 16) | ((ln >> 8) & 0xFFu) << 16;
            s_code[4 * v4 + 2] = (rc.y & 0xFFFFu) | ((ln >> 16) & 0xFFu) << 16;
            s_code[4 * v4 + 3] = (rc.y >> 16) | (ln >> 24) << 16;
        }
    }
    __syncthreads();
    const uint32_t *coff = sc.chunk + ((size_t)f * kSecs + s) * sc.max_chunks;
    const uint32_t w = L.width[s], cnt = L.count[s];
    uint32_t *pay = dst + (S.alph + 7) / 8 + S.nch;
    // a warp per chunk: each lane sizes its 32 symbols, an exclusive scan gives its first bit,
    // the lanes place their codes in the warp's buffer, the warp stores the chunk's words
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *buf = s_buf[warp];
    for (uint32_t c = blockIdx.x * kWarps + warp; c < S.nch; c += gridDim.x * kWarps) {
        const uint32_t c0 = c * kChunk, m = min(cnt - c0, (uint32_t)kChunk), s0 = 32 * lane;
        const uint32_t ml = s0 < m ? min(m - s0, 32u) : 0u;
        stage_symbols(sec, w, c0, m, s_sym[warp]);
        uint32_t bits = 0;
        {
            SymReader rd(s_sym[warp], w, s0, ml);
            for (uint32_t i = 0; i < ml; i++) bits += s_code[rd.next()] >> 16;
        }
        uint32_t x = bits;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= d) x += y;
        }
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, x, 31), nwords = (total + 31) / 32;
        for (uint32_t j = lane; j < nwords; j += 32) buf[j] = 0u;
        __syncwarp();
        {
            SymReader rd(s_sym[warp], w, s0, ml);
            uint32_t p = x - bits;
            for (uint32_t i = 0; i < ml; i++) {
                const uint32_t cl = s_code[rd.next()], code = cl & 0xFFFFu, len = cl >> 16;
                const uint32_t wi = p >> 5, sh = p & 31;
                atomicOr(&buf[wi], code << sh);
                if (sh + len > 32) atomicOr(&buf[wi + 1], code >> (32 - sh));
                p += len;
            }
        }
        __syncwarp();
        uint32_t *o = pay + coff[c];
        for (uint32_t j = lane; j < nwords; j += 32) o[j] = buf[j];
        __syncwarp();
    }
}

// ---- decoder ----

struct DecSmem {
    uint8_t len[kMaxAlph];
    uint32_t red[32];
    uint32_t last_leaf;
    uint32_t per_len[kMaxLen + 1];
    uint32_t first[kMaxLen + 1];
    uint32_t index[kMaxLen + 2];
    uint32_t bad;
};

// Descriptor words of section s and the section's word offset; false if they cannot be this
// frame's (layout L, stream of ent_words words).
__device__ bool read_desc(const uint32_t *e, uint32_t ent_words, const Layout &L, int s, uint32_t &mode,
                          uint32_t &alph, uint32_t &words, uint32_t &off) {
    uint32_t o = kEntHeaderWords;
    for (int k = 0; k < s; k++) o += e[21 + 4 * k];
    const uint32_t mw = e[18 + 4 * s], count = e[19 + 4 * s];
    alph = e[20 + 4 * s];
    words = e[21 + 4 * s];
    off = o;
    if ((unsigned long long)o + words > ent_words) return false;
    if (mw == 0) {
        mode = 0;
        return count == L.words[s] && words == L.words[s] && alph == 0;
    }
    mode = 1;
    if (mw != (1u | L.width[s] << 8) || !coded_width(L.width[s]) || count != L.count[s] || alph < 1 ||
        alph > (1u << L.width[s]))
        return false;
    const uint32_t nch = (count + kChunk - 1) / kChunk;
    return (unsigned long long)(alph + 7) / 8 + nch <= words;
}

// grid (7 sections, nframes), 256 threads
__global__ void __launch_bounds__(256) k_ent_dec_prep(EntBatch b, Scratch sc, unsigned *err) {
    __shared__ DecSmem S;
    const int s = blockIdx.x, f = blockIdx.y, tid = threadIdx.x;
    Frame &F = sc.frame[f];
    const uint32_t *e = reinterpret_cast<const uint32_t *>(b.in[f]);
    if (tid == 0) S.bad = 0;
    __syncthreads();
    // header checks (every block repeats them; all read the same words)
    Layout L;
    bool ok = b.in_size[f] >= 4ull * kEntHeaderWords && e[16] == kEntMagic && e[17] % 4 == 0 &&
              e[17] >= 4u * kEntHeaderWords && e[17] <= b.in_size[f];
    if (ok) {
        // the fixed-width header with a body of the size it states
        ok = parse_fixed(b.in[f], ~0ull, b.rows, b.cols, L) && L.total <= b.out_cap[f];
    }
    uint32_t mode = 0, alph = 0, words = 0, off = 0;
    if (ok) {
        const uint32_t ew = e[17] / 4;
        unsigned long long sum = kEntHeaderWords;
        for (int k = 0; k < kSecs; k++) sum += e[21 + 4 * k];
        ok = sum == ew && read_desc(e, ew, L, s, mode, alph, words, off);
    }
    if (!ok) {
        if (tid == 0) {
            atomicOr(&F.ok, 2u);   // bit 1: corrupt
            atomicOr(err, E_CORRUPT);
        }
        return;
    }
    Sec &D = F.sec[s];
    if (tid == 0) {
        D.mode = mode;
        D.alph = alph;
        D.words = words;
        D.ent_off = off;
        D.nch = mode ? (L.count[s] + kChunk - 1) / kChunk : 0u;
        if (s == 0) F.L = L;
    }
    if (s == 0 && tid < 16) reinterpret_cast<uint32_t *>(b.out[f])[tid] = e[tid];
    if (s == 0 && tid == 0) b.out_bytes[f] = L.total;
    if (!mode) return;
    // length table, Kraft sum, canonical tables, symbols in (length, symbol) order
    const uint32_t *sec = e + off;
    for (uint32_t v = tid; v < alph; v += blockDim.x) S.len[v] = (sec[v / 8] >> (4 * (v % 8))) & 15u;
    if (tid <= kMaxLen) S.per_len[tid] = 0;
    __syncthreads();
    uint32_t kraft = 0;
    for (uint32_t v = tid; v < alph; v += blockDim.x)
        if (S.len[v]) {
            atomicAdd(&S.per_len[S.len[v]], 1u);
            kraft += 1u << (kMaxLen - S.len[v]);
        }
    kraft = block_sum(kraft, S.red);
    if (kraft == 0 || kraft > (1u << kMaxLen)) {
        if (tid == 0) {
            atomicOr(&F.ok, 2u);
            atomicOr(err, E_CORRUPT);
        }
        return;
    }
    if (tid == 0) {
        canonical_tables(S.per_len, S.first, S.index);
        for (int l = 0; l <= kMaxLen; l++) {
            D.per_len[l] = S.per_len[l];
            D.first[l] = S.first[l];
        }
        for (int l = 0; l <= kMaxLen + 1; l++) D.index[l] = S.index[l];
    }
    uint16_t *sorted = sc.sorted + ((size_t)f * kSecs + s) * kMaxAlph;
    place_by_length(S.len, alph, S.index, S.red,
                    [&](uint32_t v, uint32_t, uint32_t pos) { sorted[pos] = (uint16_t)v; });
    // chunk offsets non-decreasing, inside the payload
    const uint32_t nch = (L.count[s] + kChunk - 1) / kChunk, tw = (alph + 7) / 8;
    const uint32_t pay = words - tw - nch;
    const uint32_t *co = sec + tw;
    uint32_t badc = 0;
    for (uint32_t c = tid; c < nch; c += blockDim.x) {
        const uint32_t hi = c + 1 < nch ? co[c + 1] : pay;
        if (co[c] > hi || hi > pay) badc = 1;
    }
    if (block_sum(badc, S.red) && tid == 0) {
        atomicOr(&F.ok, 2u);
        atomicOr(err, E_CORRUPT);
    }
}

constexpr int kPeek = 9;   // codes up to this length resolve in one table lookup

// grid (G, 7 sections, nframes), kWriteThreads threads
__global__ void __launch_bounds__(kWriteThreads) k_ent_dec(EntBatch b, Scratch sc, unsigned *err_word) {
    __shared__ uint16_t s_sym[kMaxAlph];          // symbols in (length, symbol) order
    __shared__ uint32_t s_peek[1 << kPeek];       // first kPeek bits -> symbol | length << 16 (0: longer)
    __shared__ uint32_t s_lim[kMaxLen + 1], s_first[kMaxLen + 1], s_index[kMaxLen + 2];
    const int s = blockIdx.y, f = blockIdx.z;
    const Frame &F = sc.frame[f];
    if (F.ok & 2u) return;
    const Sec &D = F.sec[s];
    const Layout &L = F.L;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(b.in[f]) + D.ent_off;
    uint32_t *dst = reinterpret_cast<uint32_t *>(b.out[f] + kHeaderBytes) + L.off[s];
    if (!D.mode) {
        for (uint32_t base = blockIdx.x * kCopyWords; base < L.words[s]; base += gridDim.x * kCopyWords) {
            const uint32_t e = min(L.words[s], base + kCopyWords);
            for (uint32_t i = base + threadIdx.x; i < e; i += blockDim.x) dst[i] = src[i];
        }
        return;
    }
    if (blockIdx.x * (kWriteThreads / 32) >= D.nch) return;
    // canonical decode tables: per length the left-justified limit (codes of length l are the
    // 15-bit windows in [limit(l - 1), limit(l))), and a direct table for the short codes
    if (threadIdx.x == 0) {
        for (int l = 1; l <= kMaxLen; l++) s_lim[l] = (D.first[l] + D.per_len[l]) << (kMaxLen - l);
    }
    if (threadIdx.x <= kMaxLen) s_first[threadIdx.x] = D.first[threadIdx.x];
    if (threadIdx.x <= kMaxLen + 1) s_index[threadIdx.x] = D.index[threadIdx.x];
    const uint32_t nused = D.index[kMaxLen + 1];
    const uint16_t *sorted = sc.sorted + ((size_t)f * kSecs + s) * kMaxAlph;
    for (uint32_t i = threadIdx.x; i < nused; i += blockDim.x) s_sym[i] = sorted[i];
    for (uint32_t i = threadIdx.x; i < (1u << kPeek); i += blockDim.x) s_peek[i] = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nused; i += blockDim.x) {
        int l = 1;
        while (l < kMaxLen && s_index[l + 1] <= i) l++;
        if (l > kPeek) continue;
        const uint32_t code = s_first[l] + (i - s_index[l]);
        const uint32_t lo = code << (kPeek - l), hi = (code + 1) << (kPeek - l);
        for (uint32_t x = lo; x < hi; x++) s_peek[x] = (uint32_t)s_sym[i] | (uint32_t)l << 16;
    }
    __syncthreads();
    const uint32_t w = L.width[s], cnt = L.count[s];
    const uint32_t tw = (D.alph + 7) / 8, nch = D.nch;
    const uint32_t *co = src + tw;
    const uint32_t *pay = co + nch;
    const uint32_t pay_words = D.words - tw - nch;
    constexpr int kWarps = kWriteThreads / 32;
    __shared__ uint32_t s_out[kWarps][kChunk * kMaxWidth / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *obuf = s_out[warp];
    // a warp per chunk.  Lane j decodes the codes that start in its 1/32 of the chunk's bits.
    // Its true first bit is where lane j - 1's codes end, found by rounds of speculative decode:
    // lane 0 starts exactly, each round every lane decodes from its current start and the next
    // lane takes its end; once no start changes every start is a code boundary (at most 32
    // rounds; Huffman codes resynchronise within a few codes, so usually two or three).
    for (uint32_t c = blockIdx.x * kWarps + warp; c < nch; c += gridDim.x * kWarps) {
        const uint32_t beg = co[c], end = c + 1 < nch ? co[c + 1] : pay_words;   // validated by the prep
        const uint32_t *cw = pay + beg;
        const uint32_t cwords = end - beg, nbits = 32 * cwords;
        const uint32_t m = min(cnt - c * kChunk, (uint32_t)kChunk);
        const uint32_t span = (nbits + 31) / 32;
        const uint32_t limit = lane == 31 ? nbits : min(nbits, (lane + 1) * span);   // codes starting below
        // one code at bit p of the chunk: symbol | length << 16, 0 if no code starts there
        auto code_at = [&](uint32_t p) -> uint32_t {
            const uint32_t wi = p >> 5, sh = p & 31;
            const unsigned long long lo = wi < cwords ? cw[wi] : 0u, hi = wi + 1 < cwords ? cw[wi + 1] : 0u;
            const uint32_t v = __brev((uint32_t)((lo | hi << 32) >> sh) & 0x7FFFu) >> (32 - kMaxLen);
            const uint32_t pk = s_peek[v >> (kMaxLen - kPeek)];
            if (pk) return pk;
            uint32_t l = kPeek + 1;
            while (l <= (uint32_t)kMaxLen && v >= s_lim[l]) l++;
            if (l > (uint32_t)kMaxLen) return 0u;
            return (uint32_t)s_sym[s_index[l] + (v >> (kMaxLen - l)) - s_first[l]] | l << 16;
        };
        uint32_t start = lane == 0 ? 0u : min(nbits, lane * span), n = 0;
        bool bad = false;
        for (int round = 0; round < 32; round++) {
            uint32_t p = start;
            n = 0;
            bad = false;
            while (p < limit) {
                const uint32_t sl = code_at(p);
                if (!sl || n == (uint32_t)kChunk) {
                    bad = true;
                    break;
                }
                p += sl >> 16;
                n++;
            }
            uint32_t next = __shfl_up_sync(0xFFFFFFFFu, p, 1);
            if (lane == 0) next = 0u;
            const bool moved = next != start;
            start = next;
            if (!__any_sync(0xFFFFFFFFu, moved)) break;
        }
        // symbols before each lane's first one; the chunk's word padding may decode into codes
        // past the m-th symbol, which are dropped
        uint32_t x = n;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
            if (lane >= d) x += y;
        }
        const uint32_t before = x - n, total = __shfl_sync(0xFFFFFFFFu, x, 31);
        const uint32_t mine = before >= m ? 0u : min(n, m - before);
        bool err = total < m || (bad && before + n < m);
        const uint32_t owords = (m * w + 31) / 32;
        for (uint32_t j = lane; j < owords; j += 32) obuf[j] = 0u;
        __syncwarp();
        uint32_t p = start;
        for (uint32_t i = 0; i < mine && !err; i++) {
            const uint32_t sl = code_at(p);
            if (!sl || p + (sl >> 16) > nbits) {   // no code, or one that runs past the chunk
                err = true;
                break;
            }
            p += sl >> 16;
            const uint32_t bit = (before + i) * w, wi = bit >> 5, sh = bit & 31, sym = sl & 0xFFFFu;
            atomicOr(&obuf[wi], sym << sh);
            if (sh + w > 32) atomicOr(&obuf[wi + 1], sym >> (32 - sh));
        }
        if (__any_sync(0xFFFFFFFFu, err)) {
            if (lane == 0) atomicOr(err_word, E_CORRUPT);
            __syncwarp();
            continue;
        }
        __syncwarp();
        uint32_t *o = dst + (size_t)c * kChunk * w / 32;   // 1024 symbols of w bits fill whole words
        for (uint32_t j = lane; j < owords; j += 32) o[j] = obuf[j];
        __syncwarp();
    }
}

}  // namespace ent
}  // namespace lcc

// ---- host side ----

namespace {

using namespace lcc;
using namespace lcc::api;

lcc_status ent_scratch(lcc_ctx *c, ent::Scratch &sc) {
    const uint64_t npx = (uint64_t)c->g.H * c->g.W;
    const uint32_t max_chunks = (uint32_t)((npx + 64 + ent::kChunk - 1) / ent::kChunk);
    const size_t slots = (size_t)c->slots;
    const size_t per = (size_t)ent::kSecs * ent::kMaxAlph;
    const size_t bytes = align256(slots * sizeof(ent::Frame)) + align256(slots * per) +
                         2 * align256(slots * per * 2) + align256(slots * ent::kSecs * max_chunks * 4);
    if (!c->d_ent) {
        if (cudaMalloc(&c->d_ent, bytes) != cudaSuccess) {
            c->d_ent = nullptr;
            return LCC_ERR_CUDA;
        }
    }
    unsigned char *p = static_cast<unsigned char *>(c->d_ent);
    sc.frame = reinterpret_cast<ent::Frame *>(p);
    p += align256(slots * sizeof(ent::Frame));
    sc.len = p;
    p += align256(slots * per);
    sc.rcode = reinterpret_cast<uint16_t *>(p);
    p += align256(slots * per * 2);
    sc.sorted = reinterpret_cast<uint16_t *>(p);
    p += align256(slots * per * 2);
    sc.chunk = reinterpret_cast<uint32_t *>(p);
    sc.max_chunks = max_chunks;
    return LCC_OK;
}

int grid_x(lcc_ctx *c, const ent::Scratch &sc) {
    const uint64_t words = c->max_bytes / 4;
    const uint64_t by_copy = (words + ent::kCopyWords - 1) / ent::kCopyWords;
    const uint64_t by_chunk = (sc.max_chunks + ent::kWriteThreads - 1) / ent::kWriteThreads;
    uint64_t g = by_copy > by_chunk ? by_copy : by_chunk;
    return (int)(g < 1 ? 1 : (g > 64 ? 64 : g));
}

lcc_status fill_batch(lcc_ctx *c, ent::EntBatch &b, int nframes, const uint8_t *const *d_in, const uint64_t *in_size,
                      uint8_t *const *d_out, const uint64_t *out_cap, uint64_t *d_out_bytes) {
    memset(&b, 0, sizeof(b));
    for (int f = 0; f < nframes; f++) {
        if (!d_in[f] || !d_out[f] || !aligned16(d_in[f]) || !aligned16(d_out[f])) return LCC_ERR_INVALID_ARG;
        b.in[f] = d_in[f];
        b.out[f] = d_out[f];
        b.in_size[f] = in_size[f];
        b.out_cap[f] = out_cap[f];
    }
    b.out_bytes = reinterpret_cast<unsigned long long *>(d_out_bytes);
    b.rows = (uint32_t)c->g.H;
    b.cols = (uint32_t)c->g.W;
    return LCC_OK;
}

}  // namespace

extern "C" {

lcc_status lcc_entropy_encode(lcc_ctx *c, int32_t nframes, const uint8_t *const *d_in, const uint64_t *in_size,
                              uint8_t *const *d_out, const uint64_t *out_cap, uint64_t *d_out_bytes) {
    if (!c || !d_in || !in_size || !d_out || !out_cap || !d_out_bytes || nframes < 1 || nframes > c->slots ||
        !aligned16(d_out_bytes))
        return LCC_ERR_INVALID_ARG;
    ent::EntBatch b;
    lcc_status st = fill_batch(c, b, nframes, d_in, in_size, d_out, out_cap, d_out_bytes);
    if (st != LCC_OK) return st;
    ent::Scratch sc;
    if ((st = ent_scratch(c, sc)) != LCC_OK) return st;
    const size_t smem = sizeof(ent::BuildSmem);
    LCC_CUDA(cudaFuncSetAttribute(ent::k_ent_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    LCC_LAUNCH(c, 10, (ent::k_ent_build<<<dim3(5, nframes), ent::kBuildThreads, smem, c->stream>>>(b, sc, c->s.err),
                       cudaGetLastError()));
    LCC_LAUNCH(c, 11, (ent::k_ent_layout<<<nframes, 32 * ent::kSecs, 0, c->stream>>>(b, sc, c->s.err, nframes), cudaGetLastError()));
    LCC_LAUNCH(c, 12, (ent::k_ent_write<<<dim3(grid_x(c, sc), ent::kSecs, nframes), ent::kWriteThreads, 0, c->stream>>>(
                           b, sc),
                       cudaGetLastError()));
    return LCC_OK;
}

lcc_status lcc_entropy_decode(lcc_ctx *c, int32_t nframes, const uint8_t *const *d_in, const uint64_t *in_bytes,
                              uint8_t *const *d_out, const uint64_t *out_cap, uint64_t *d_out_bytes) {
    if (!c || !d_in || !in_bytes || !d_out || !out_cap || !d_out_bytes || nframes < 1 || nframes > c->slots ||
        !aligned16(d_out_bytes))
        return LCC_ERR_INVALID_ARG;
    ent::EntBatch b;
    lcc_status st = fill_batch(c, b, nframes, d_in, in_bytes, d_out, out_cap, d_out_bytes);
    if (st != LCC_OK) return st;
    ent::Scratch sc;
    if ((st = ent_scratch(c, sc)) != LCC_OK) return st;
    // clear the frames' state words (bit 1 marks a corrupt frame)
    for (int f = 0; f < nframes; f++)
        LCC_CUDA(cudaMemsetAsync(&sc.frame[f].ok, 0, sizeof(uint32_t), c->stream));
    LCC_LAUNCH(c, 13, (ent::k_ent_dec_prep<<<dim3(ent::kSecs, nframes), 256, 0, c->stream>>>(b, sc, c->s.err),
                       cudaGetLastError()));
    LCC_LAUNCH(c, 13, (ent::k_ent_dec<<<dim3(grid_x(c, sc), ent::kSecs, nframes), ent::kWriteThreads, 0, c->stream>>>(
                           b, sc, c->s.err),
                       cudaGetLastError()));
    return LCC_OK;
}

}  // extern "C"
