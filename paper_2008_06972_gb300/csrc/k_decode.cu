// Decoder: validates a stream, resolves each tile's plane and stream
// offsets, then reconstructs every pixel by ray casting onto its plane
// (Sec. III-C): r = d / (n.u) + k q for plane-coded pixels, r = m q for raw
// ones, and the point is r * u.  A corrupt stream latches E_CORRUPT and leaves
// the outputs unspecified; no read leaves the stream's declared sections.
#include <algorithm>

#include "lcc_internal.cuh"

namespace lcc {

constexpr int kPrepThreads = 1024;
constexpr int kDecWarps = 8;

// Stream-level decode state written by the prep kernel.
struct DecState {
    uint32_t ok;
    uint32_t sec[8];
    float q;
    int32_t k_max, w_res, w_raw;
    int32_t no_delta;   // plane-coded points carry no residual code
    int32_t raw_exact;  // raw codes are the fp32 range bits
};

__device__ __forceinline__ uint32_t rd_u32(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

__device__ __forceinline__ uint32_t dwords(uint64_t bits) { return (uint32_t)((bits + 31) >> 5); }

// Set bits of the LSB-first bit string w in [pos, pos + len).
__device__ __forceinline__ uint32_t popc_range(const uint32_t *w, uint64_t pos, uint32_t len) {
    uint32_t n = 0;
    while (len) {
        const uint32_t sh = (uint32_t)(pos & 31), take = min(32u - sh, len);
        const uint32_t m = take == 32 ? 0xFFFFFFFFu : ((1u << take) - 1u);
        n += __popc((w[pos >> 5] >> sh) & m);
        pos += take;
        len -= take;
    }
    return n;
}

template <int N>
__device__ __forceinline__ void block_scan(uint32_t (&v)[N], uint32_t (&excl)[N], uint32_t (&tot)[N],
                                           uint32_t (*s_warp)[N]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc[N];
#pragma unroll
    for (int q = 0; q < N; q++) {
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
        for (int q = 0; q < N; q++) s_warp[warp][q] = inc[q];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < N; q++) {
            uint32_t x = s_warp[lane][q];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x += y;
            }
            s_warp[lane][q] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < N; q++) {
        excl[q] = (warp ? s_warp[warp - 1][q] : 0u) + inc[q] - v[q];
        tot[q] = s_warp[31][q];
    }
    __syncthreads();
}

// One CTA per stream (frame f = blockIdx.y of the batch).
__global__ void __launch_bounds__(kPrepThreads) k_decode_prep(Geometry g, DecBatch db, const float4 *kf, Poses ps,
                                                               float4 *kf_out, uint32_t *err, int expect_kind) {
    const int frame = blockIdx.y;
    const uint8_t *bits = db.bits[frame];
    const unsigned long long nbytes = db.nbytes[frame];
    DecTile *dt = db.dt[frame];
    DecState *state = reinterpret_cast<DecState *>(dt + g.NT);
    __shared__ uint32_t s_warp5[32][5];
    __shared__ uint32_t s_warp2[32][2];
    __shared__ uint32_t s_h[16];
    __shared__ uint32_t s_sec[8];
    __shared__ int s_bad;
    __shared__ uint32_t s_carry[7];
    __shared__ int s_last_start;
    const int tid = threadIdx.x;
    if (tid == 0) {
        int bad = nbytes < (unsigned long long)kHeaderBytes;
        if (!bad) {
            for (int q = 0; q < 16; q++) s_h[q] = rd_u32(bits + 4 * q);
            const uint32_t kind = (s_h[1] >> 16) & 0xff, flags = s_h[1] >> 24;
            bad |= s_h[0] != kMagic || (s_h[1] & 0xffff) != (uint32_t)kVersion || (flags & ~31u) ||
                   ((flags & 8u) && kind != 1);
            bad |= (int)(s_h[2] & 0xffff) != g.H || (int)(s_h[2] >> 16) != g.W;
            bad |= (int)(s_h[3] & 0xff) != g.th || (int)((s_h[3] >> 8) & 0xff) != g.tw;
            const uint32_t w_res = (s_h[3] >> 16) & 0xff, w_raw = s_h[3] >> 24;
            bad |= w_res == 0 || w_res > 16 || w_raw == 0 || ((flags & 4u) ? w_raw != 32 : w_raw > 24);
            bad |= s_h[6] != (uint32_t)g.NT || kind > 1 || (expect_kind >= 0 && kind != (uint32_t)expect_kind);
            bad |= !(__uint_as_float(s_h[5]) > 0.0f);
            if (kind == 1 && kf == nullptr) bad = 1;
            s_sec[0] = 0;
            s_sec[1] = s_sec[0] + dwords((uint64_t)g.H * g.W);
            s_sec[2] = s_sec[1] + dwords((uint64_t)g.NT * 4);
            s_sec[3] = s_sec[2] + ((flags & 16u) ? 3u : 4u) * s_h[8];   // three-coefficient planes: 3 words
            s_sec[4] = s_sec[3] + 2u * s_h[9];
            s_sec[5] = s_sec[4] + dwords(s_h[10]);
            s_sec[6] = s_sec[5] + ((flags & 2u) ? 0u : dwords((uint64_t)s_h[11] * w_res));   // no deltas: none
            s_sec[7] = s_sec[6] + dwords((uint64_t)s_h[12] * w_raw);
            const unsigned long long total = (unsigned long long)kHeaderBytes + 4ull * s_sec[7];
            bad |= total != s_h[14] || total > nbytes || s_h[8] > (uint32_t)g.NT || s_h[9] > (uint32_t)g.NT ||
                   s_h[10] > (uint32_t)(g.H * g.W) || s_h[11] > s_h[10] || s_h[12] > (uint32_t)(g.H * g.W);
        }
        s_bad = bad;
        s_last_start = -1;
        for (int q = 0; q < 7; q++) s_carry[q] = 0;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            state->ok = 0;
            atomicOr(err, E_CORRUPT);
        }
        return;
    }
    const uint32_t *w = reinterpret_cast<const uint32_t *>(bits + kHeaderBytes);
    const uint32_t *bm = w + s_sec[0], *tcw = w + s_sec[1], *runw = w + s_sec[2], *tmpw = w + s_sec[3],
                   *fitw = w + s_sec[4];
    const uint32_t n_runs = s_h[8], n_temp = s_h[9], n_cand = s_h[10];
    const uint32_t kind = (s_h[1] >> 16) & 0xff, hflags = s_h[1] >> 24;
    int bad = 0;
    for (int base = 0; base < g.NT; base += kPrepThreads) {
        const int t = base + tid;
        uint32_t mode = 0, nv = 0;
        int axis = -1;   // three-coefficient run start: its dominant axis (tile code 6 + axis)
        const int tr = t / g.TC, tc = t % g.TC;
        if (t < g.NT) {
            mode = (tcw[t >> 3] >> (4 * (t & 7))) & 15u;
            if (mode >= T_RUN_START3 && mode < T_RUN_START3 + 3u) {
                if (!(hflags & 16u)) bad = 1;
                axis = (int)(mode - T_RUN_START3);
                mode = T_RUN_START;
            } else if (mode == T_RUN_START && (hflags & 16u)) {
                bad = 1;
            }
            const int j0 = tc * g.tw, wdt = min(g.tw, g.W - j0);
            for (int rr = 0; rr < g.th; rr++) {
                const int i = tr * g.th + rr;
                if (i >= g.H) break;
                nv += popc_range(bm, (uint64_t)i * g.W + j0, (uint32_t)wdt);
            }
            if (mode > T_TEMPORAL_CONT) bad = 1;
            if (mode == T_EMPTY && nv) bad = 1;
            if (mode == T_RUN_CONT || mode == T_TEMPORAL_CONT) {   // continues the run to its left
                uint32_t pm = tc ? (tcw[(t - 1) >> 3] >> (4 * ((t - 1) & 7))) & 15u : 0u;
                if (pm >= T_RUN_START3 && pm < T_RUN_START3 + 3u) pm = T_RUN_START;
                const bool ok = mode == T_RUN_CONT ? (pm == T_RUN_START || pm == T_RUN_CONT)
                                                   : ((hflags & 8u) && (pm == T_TEMPORAL || pm == T_TEMPORAL_CONT));
                if (tc == 0 || !ok) bad = 1;
            }
        }
        const bool coded = mode >= T_RUN_START && mode <= T_TEMPORAL_CONT;
        uint32_t v5[5] = {coded ? nv : 0u, mode == T_RUN_START ? 1u : 0u, mode == T_TEMPORAL ? 1u : 0u,
                          mode == T_RAW ? nv : 0u, nv};
        uint32_t e5[5], t5[5];
        block_scan<5>(v5, e5, t5, s_warp5);
        const uint32_t off_cand = s_carry[0] + e5[0];
        const uint32_t run_idx = s_carry[1] + e5[1];
        const uint32_t tmp_idx = s_carry[2] + e5[2];
        // plane-coded pixels of the tile: popcount of its fitted bits
        uint32_t fitted = 0;
        if (coded && nv) {
            if (off_cand + nv > n_cand) {
                bad = 1;
            } else {
                fitted = popc_range(fitw, off_cand, nv);
            }
        }
        uint32_t v2[2] = {fitted, v5[3] + (coded ? nv - fitted : 0u)};
        uint32_t e2[2], t2[2];
        block_scan<2>(v2, e2, t2, s_warp2);
        float4 pl = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < g.NT) {
            if (mode == T_RUN_START) {
                if (run_idx >= n_runs) bad = 1;
                else if (hflags & 16u)
                    pl = plane_from3(make_float4(__uint_as_float(runw[3 * run_idx]), __uint_as_float(runw[3 * run_idx + 1]),
                                                 __uint_as_float(runw[3 * run_idx + 2]), (float)(axis < 0 ? 0 : axis)));
                else pl = make_float4(__uint_as_float(runw[4 * run_idx]), __uint_as_float(runw[4 * run_idx + 1]),
                                      __uint_as_float(runw[4 * run_idx + 2]), __uint_as_float(runw[4 * run_idx + 3]));
            } else if (mode == T_TEMPORAL) {
                if (kind != 1 || tmp_idx >= n_temp) {
                    bad = 1;
                } else {
                    const uint32_t kref = tmpw[2 * tmp_idx];
                    const float c = __uint_as_float(tmpw[2 * tmp_idx + 1]);
                    if (kref >= (uint32_t)g.NT) {
                        bad = 1;
                    } else {
                        const float4 kp = kf[kref];
                        if (kp.x == 0.f && kp.y == 0.f && kp.z == 0.f) bad = 1;
                        float o[3];
                        rotate_normal(ps.m[frame], kp.x, kp.y, kp.z, o);
                        pl = make_float4(o[0], o[1], o[2], c);
                    }
                }
            }
            DecTile d;
            d.plane = pl;
            d.off_cand = off_cand;
            d.off_fit = s_carry[5] + e2[0];
            d.off_raw = s_carry[6] + e2[1];
            d.mode = (uint8_t)mode;
            d.n_valid = (uint8_t)nv;
            d.pad0 = d.pad1 = 0;
            dt[t] = d;
        }
        __syncthreads();
        // run continuations (spatial or temporal) take the plane of the last run start at or before
        // them: a continuation follows its own kind of start with only continuations between
        {
            __shared__ int s_ms[32];
            int x = (t < g.NT && (mode == T_RUN_START || mode == T_TEMPORAL)) ? t : -1;
            const int lane = tid & 31, wp = tid >> 5;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, off);
                if (lane >= off) x = max(x, y);
            }
            if (lane == 31) s_ms[wp] = x;
            __syncthreads();
            if (wp == 0) {
                int y = s_ms[lane];
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int z = __shfl_up_sync(0xffffffffu, y, off);
                    if (lane >= off) y = max(y, z);
                }
                s_ms[lane] = y;
            }
            __syncthreads();
            const int start = max(max(x, wp ? s_ms[wp - 1] : -1), s_last_start);
            if (t < g.NT && (mode == T_RUN_CONT || mode == T_TEMPORAL_CONT)) {
                if (start < 0) bad = 1;
                else dt[t].plane = dt[start].plane;
            }
            if (kf_out && t < g.NT) kf_out[t] = (mode == T_RUN_START || mode == T_RUN_CONT) ? dt[t].plane
                                                                                              : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncthreads();
            if (tid == 0) s_last_start = max(s_last_start, s_ms[31]);
        }
        if (tid == 0) {
            for (int q = 0; q < 5; q++) s_carry[q] += t5[q];
            s_carry[5] += t2[0];
            s_carry[6] += t2[1];
        }
        __syncthreads();
    }
    bad = __syncthreads_or(bad);
    if (tid == 0) {
        bad |= s_carry[0] != n_cand || s_carry[1] != n_runs || s_carry[2] != n_temp || s_carry[4] != s_h[7] ||
               s_carry[5] != s_h[11] || s_carry[6] != s_h[12];
        DecState st;
        st.ok = bad ? 0u : 1u;
        for (int q = 0; q < 8; q++) st.sec[q] = s_sec[q];
        st.q = __uint_as_float(s_h[5]);
        st.k_max = (int32_t)s_h[13];
        st.w_res = (int32_t)((s_h[3] >> 16) & 0xff);
        st.w_raw = (int32_t)(s_h[3] >> 24);
        st.no_delta = (int32_t)((s_h[1] >> 25) & 1u);
        st.raw_exact = (int32_t)((s_h[1] >> 26) & 1u);
        *state = st;
        if (bad) atomicOr(err, E_CORRUPT);
    }
}

template <int TH_, int TW_>
__global__ void __launch_bounds__(kDecWarps * 32) k_decode_px(Geometry g, DecBatch db, uint32_t *err) {
    const int frame = blockIdx.y;
    const uint8_t *bits = db.bits[frame];
    const DecTile *dt = db.dt[frame];
    const DecState *state = reinterpret_cast<const DecState *>(dt + g.NT);
    float *range = db.range[frame];
    float4 *xyz = db.xyz[frame];
    constexpr int PX = TH_ * TW_;
    constexpr int LPT = PX < 32 ? PX : 32, PPL = PX / LPT, TPW = 32 / LPT;
    const unsigned FULL = 0xffffffffu;
    const DecState st = *state;
    if (!st.ok) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = lane / LPT, sl = lane % LPT;
    const int t = (blockIdx.x * kDecWarps + warp) * TPW + seg;
    const bool tile_ok = t < g.NT;
    const int tr = tile_ok ? t / g.TC : 0, tc = tile_ok ? t % g.TC : 0;
    const uint32_t segmask = (LPT == 32) ? FULL : (((1u << LPT) - 1u) << (seg * LPT));
    const uint32_t below = segmask & ((1u << lane) - 1u);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(bits + kHeaderBytes);
    DecTile d;
    if (tile_ok) d = dt[t];
    else { d.mode = T_EMPTY; d.off_cand = d.off_fit = d.off_raw = 0; d.plane = make_float4(0.f, 0.f, 0.f, 0.f); }
    const bool coded = d.mode >= T_RUN_START;
    bool v[PPL], fb[PPL];
    int vrank[PPL], ii[PPL], jj[PPL];
    int vacc = 0;
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        const int k = sl + LPT * m;
        ii[m] = tr * TH_ + k / TW_;
        jj[m] = tc * TW_ + k % TW_;
        const bool in = tile_ok && ii[m] < g.H && jj[m] < g.W;
        const uint64_t p = (uint64_t)ii[m] * g.W + jj[m];
        v[m] = in && ((w[st.sec[0] + (p >> 5)] >> (p & 31)) & 1u);
        const uint32_t vb = __ballot_sync(FULL, v[m]) & segmask;
        vrank[m] = vacc + __popc(vb & below);
        vacc += __popc(vb);
        fb[m] = false;
        if (v[m] && coded) {
            const uint32_t pos = d.off_cand + vrank[m];
            fb[m] = (w[st.sec[4] + (pos >> 5)] >> (pos & 31)) & 1u;
        }
    }
    int facc = 0;
    bool bad = false;
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        const uint32_t fmask = __ballot_sync(FULL, fb[m]) & segmask;
        const int frank = facc + __popc(fmask & below);
        facc += __popc(fmask);
        const bool in = tile_ok && ii[m] < g.H && jj[m] < g.W;
        if (!in) continue;
        const size_t p = (size_t)ii[m] * g.W + jj[m];
        float r = 0.f;
        float ux, uy, uz;
        beam(g, ii[m], jj[m], ux, uy, uz);
        if (v[m]) {
            if (fb[m]) {
                const int k = st.no_delta ? 0
                              : (int)get_bits(w + st.sec[5], (uint64_t)(d.off_fit + frank) * st.w_res, st.w_res) -
                                    st.k_max;
                const float dot = fmaf(d.plane.x, ux, fmaf(d.plane.y, uy, __fmul_rn(d.plane.z, uz)));
                if (!(dot > 1e-3f)) bad = true;
                r = fmaf((float)k, st.q, __fdiv_rn(d.plane.w, dot));
            } else {
                const int rrank = vrank[m] - frank;
                const uint32_t mm = get_bits(w + st.sec[6], (uint64_t)(d.off_raw + rrank) * st.w_raw, st.w_raw);
                r = st.raw_exact ? __uint_as_float(mm) : __fmul_rn((float)mm, st.q);
            }
        }
        if (range) range[p] = r;
        if (xyz) xyz[p] = v[m] ? make_float4(__fmul_rn(r, ux), __fmul_rn(r, uy), __fmul_rn(r, uz), 0.f)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (bad) atomicOr(err, E_CORRUPT);
}

cudaError_t launch_decode_prep(const Geometry &g, const DecBatch &db, int nframes, const float4 *kf,
                               const Poses &poses, float4 *kf_out, uint32_t *err, int expect_kind, cudaStream_t st) {
    if (nframes <= 0) return cudaSuccess;
    k_decode_prep<<<dim3(1, nframes), kPrepThreads, 0, st>>>(g, db, kf, poses, kf_out, err, expect_kind);
    return cudaGetLastError();
}

template <int TH_, int TW_>
static cudaError_t launch_px_t(const Geometry &g, const DecBatch &db, int nframes, uint32_t *err, cudaStream_t st) {
    constexpr int PX = TH_ * TW_;
    constexpr int TPW = 32 / (PX < 32 ? PX : 32);
    const int tpb = kDecWarps * TPW;
    k_decode_px<TH_, TW_><<<dim3((g.NT + tpb - 1) / tpb, nframes), kDecWarps * 32, 0, st>>>(g, db, err);
    return cudaGetLastError();
}

cudaError_t launch_decode_px(const Geometry &g, const DecBatch &db, int nframes, uint32_t *err, cudaStream_t st) {
    if (nframes <= 0) return cudaSuccess;
    if (g.th == 4 && g.tw == 4) return launch_px_t<4, 4>(g, db, nframes, err, st);
    if (g.th == 4 && g.tw == 8) return launch_px_t<4, 8>(g, db, nframes, err, st);
    if (g.th == 8 && g.tw == 8) return launch_px_t<8, 8>(g, db, nframes, err, st);
    if (g.th == 8 && g.tw == 16) return launch_px_t<8, 16>(g, db, nframes, err, st);
    return cudaErrorInvalidValue;
}

// Largest |a - b| over pixels occupied in either image; a pixel occupied in only one of them
// counts as +inf.  Non-negative floats order like their bit patterns, so an unsigned atomicMax
// on the bits is a float max.
__global__ void __launch_bounds__(256) k_maxdiff(const float *a, const float *b, long long n, uint32_t *out) {
    float m = 0.f;
    for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
        const float x = a[i], y = b[i];
        if (x > 0.f || y > 0.f) m = fmaxf(m, (x > 0.f && y > 0.f) ? fabsf(x - y) : __int_as_float(0x7f800000));
    }
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

cudaError_t launch_maxdiff(const float *a, const float *b, long long n, uint32_t *out, cudaStream_t st) {
    const long long blocks = std::min<long long>((n + 255) / 256, 152 * 8);
    if (blocks > 0) k_maxdiff<<<(unsigned)blocks, 256, 0, st>>>(a, b, n, out);
    return cudaGetLastError();
}

}  // namespace lcc
