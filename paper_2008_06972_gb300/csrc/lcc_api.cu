// C ABI of the lcc library: context and scratch management, argument
// checks, batched launches of the encode/decode kernels on the context
// stream, statistics and per-kernel timing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lcc.h"
#include "lcc_ctx.cuh"

using namespace lcc;

namespace lcc {
namespace api {

const char *kKernelNames[] = {"bin",        "fit",          "merge",      "rounds",    "pack",
                              "decode_prep", "decode_px",    "range_export", "lookbehind", "temporal",
                              "ent_build",  "ent_layout",   "ent_write",  "ent_decode", "net_inputs", "net_fwd"};

cudaEvent_t get_event(lcc_ctx *c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int prof_begin(lcc_ctx *c, int name, int count) {
    if (!c->prof) return -1;
    ProfRec r{name, get_event(c), get_event(c), count};
    cudaEventRecord(r.a, c->stream);
    c->pending.push_back(r);
    return (int)c->pending.size() - 1;
}

void prof_end(lcc_ctx *c, int idx) {
    if (idx < 0) return;
    cudaEventRecord(c->pending[idx].b, c->stream);
}

void prof_collect(lcc_ctx *c) {
    for (auto &r : c->pending) {
        float ms = 0.f;
        bool base = false;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            c->launches[r.name] += r.count;
            c->ms[r.name] += ms;
            if (!c->prof_base) {
                c->prof_base = r.a;
                base = true;
            }
            float t0 = 0.f, t1 = 0.f;
            if (c->timeline.size() < kMaxTimeline && cudaEventElapsedTime(&t0, c->prof_base, r.a) == cudaSuccess &&
                cudaEventElapsedTime(&t1, c->prof_base, r.b) == cudaSuccess)
                c->timeline.push_back(TimelineRec{r.name, t0, t1});
        }
        if (!base) c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->pending.clear();
}

void prof_reset(lcc_ctx *c) {
    for (int k = 0; k < kNumKernels; k++) {
        c->launches[k] = 0;
        c->ms[k] = 0.0;
    }
    if (c->prof_base) c->pool.push_back(c->prof_base);
    c->prof_base = nullptr;
    c->timeline.clear();
}

bool tile_supported(int th, int tw) {
    return (th == 4 && tw == 4) || (th == 4 && tw == 8) || (th == 8 && tw == 8) || (th == 8 && tw == 16);
}

// Sensor tables from the grid definition of Sec. III-B, fp64 libm rounded to fp32.
void make_tables(const lcc_sensor &s, std::vector<float> &t) {
    const int H = s.rows, W = s.cols;
    t.assign((size_t)4 * H + 2 + (size_t)4 * W, 0.f);
    float *ce = t.data(), *se = ce + H, *ct = se + H, *st = ct + W, *rbc = st + W, *rbs = rbc + H + 1,
          *cbc = rbs + H + 1, *cbs = cbc + W;
    const double deg = M_PI / 180.0;
    const double d_el = (s.elev_max_deg - s.elev_min_deg) / H;
    const double d_az = 2.0 * M_PI / W;
    for (int i = 0; i < H; i++) {
        const double e = (s.elev_max_deg - (i + 0.5) * d_el) * deg;
        ce[i] = (float)std::cos(e);
        se[i] = (float)std::sin(e);
    }
    for (int k = 0; k <= H; k++) row_boundary(s, k, rbc + k, rbs + k);
    for (int j = 0; j < W; j++) {
        const double a = -M_PI + (j + 0.5) * d_az;
        ct[j] = (float)std::cos(a);
        st[j] = (float)std::sin(a);
        col_boundary(s, j, cbc + j, cbs + j);
    }
}

int bits_for(int max_value) {
    int w = 1;
    while ((1 << w) < max_value + 1) w++;
    return w;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

void public_stats(const DevStats &d, lcc_stats *out) {
    out->points_in = (int64_t)d.points_in;
    out->points_invalid = (int64_t)d.invalid;
    out->points_fov = (int64_t)d.fov;
    out->points_binned = (int64_t)d.binned;
    out->pixels_valid = (int64_t)d.valid;
    out->tiles_empty = (int64_t)d.empty;
    out->tiles_raw = (int64_t)d.raw_tiles;
    out->tiles_run_start = (int64_t)d.run_start;
    out->tiles_run_cont = (int64_t)d.run_cont;
    out->tiles_temporal = (int64_t)d.temporal;
    for (int q = 0; q < 8; q++) out->fit_rounds[q] = (int64_t)d.rounds[q];
    out->tiles_borderline = (int64_t)d.borderline;
    out->cand = (int64_t)d.cand;
    out->fitted = (int64_t)d.fitted;
    out->raw = (int64_t)d.raw;
    out->bytes = d.bytes;
    out->tiles_temporal_cont = (int64_t)d.temporal_cont;
    out->tiles_net = (int64_t)d.net_tiles;
}

lcc_status latched(lcc_ctx *c) {
    uint32_t e = 0;
    if (cudaMemcpy(&e, c->s.err, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return LCC_ERR_CUDA;
    if (e) cudaMemset(c->s.err, 0, 4);
    if (e & E_CORRUPT) return LCC_ERR_CORRUPT;
    if (e & E_CAPACITY) return LCC_ERR_CAPACITY;
    if (e & E_TIMEOUT) return LCC_ERR_TIMEOUT;
    if (e) return LCC_ERR_CUDA;
    return LCC_OK;
}

void prepare_batch(Batch &b, Poses &p, int kind, int nframes, const int *slots, uint8_t *const *d_out,
                   const uint64_t *cap, const double *poses, const float4 *const *kf, float4 *const *kf_out,
                   unsigned long long *const *nbytes_out, const float *const *prop = nullptr,
                   float skip_logit = 0.f) {
    memset(&b, 0, sizeof(b));
    b.skip_logit = skip_logit;
    b.nframes = nframes;
    b.kind = kind;
    for (int f = 0; f < nframes; f++) {
        b.slot[f] = slots[f];
        b.out[f] = d_out[f];
        b.cap[f] = cap[f];
        b.kf[f] = kf ? kf[f] : nullptr;
        b.kf_out[f] = kf_out ? kf_out[f] : nullptr;
        b.nbytes_out[f] = nbytes_out ? nbytes_out[f] : nullptr;
        b.prop[f] = prop ? prop[f] : nullptr;
    }
    memset(&p, 0, sizeof(p));
    if (poses)
        for (int f = 0; f < nframes; f++) memcpy(p.m[f], poses + 16 * f, 16 * sizeof(double));
}

// Everything after the first fit pass: further rounds (unless already run) and the run
// pre-test, merge (which also lays out each frame's stream), pack.
lcc_status encode_tail(lcc_ctx *c, const Batch &b, bool rounds_done = false) {
    if (!rounds_done && c->g.schedule >= 1)
        LCC_LAUNCH_N(c, 3, queued_round_kernels(c->g, b), launch_queued_rounds(c->g, c->s, b, c->stream));
    if (c->g.merge && c->g.lookahead > 0) LCC_LAUNCH(c, 8, launch_lookbehind(c->g, c->s, b, c->stream));
    LCC_LAUNCH(c, 2, launch_merge(c->g, c->s, b, c->stream));
    LCC_LAUNCH(c, 4, launch_pack(c->g, c->s, b, c->stream));
    return LCC_OK;
}

lcc_status encode_batch(lcc_ctx *c, int kind, int nframes, const int *slots, uint8_t *const *d_out,
                        const uint64_t *cap, const double *poses, const float4 *const *kf, float4 *const *kf_out,
                        unsigned long long *const *nbytes_out, const float *const *prop, float skip_logit) {
    if (nframes <= 0) return LCC_OK;
    Batch b;
    Poses p;
    prepare_batch(b, p, kind, nframes, slots, d_out, cap, poses, kf, kf_out, nbytes_out, prop, skip_logit);
    if (kind == 1 && kf && c->g.schedule >= 4) {
        // P frames, spatial fits first: every tile's first round in the first pass (one thread per
        // tile, no temporal test), the queued tiles' remaining rounds and the run pre-test, then the
        // temporal test with a lane group per tile (a tile that passes becomes temporal exactly as
        // if its spatial fit had never run), merge and pack: the order of lcc_encode_sequence's P
        // frames, the same streams as the temporal-first order
        Batch bs = b;
        for (int f = 0; f < nframes; f++) bs.kf[f] = nullptr;
        LCC_LAUNCH(c, 1, launch_fit(c->g, c->s, bs, p, c->stream));
        LCC_LAUNCH_N(c, 3, queued_round_kernels(c->g, bs), launch_queued_rounds(c->g, c->s, bs, c->stream));
        const bool pretest = c->g.merge && c->g.lookahead > 0;
        if (pretest) LCC_LAUNCH(c, 8, launch_lookbehind(c->g, c->s, b, c->stream));
        LCC_LAUNCH(c, 9, launch_temporal(c->g, c->s, b, p, c->stream));
        // with temporal runs, the candidates that became temporal are tested again against their
        // relaxed planes
        if (pretest && c->g.truns) LCC_LAUNCH(c, 8, launch_lookbehind(c->g, c->s, b, c->stream, true));
        LCC_LAUNCH(c, 2, launch_merge(c->g, c->s, b, c->stream));
        LCC_LAUNCH(c, 4, launch_pack(c->g, c->s, b, c->stream));
        return LCC_OK;
    }
    LCC_LAUNCH(c, 1, launch_fit(c->g, c->s, b, p, c->stream));
    return encode_tail(c, b);
}

lcc_status bin_frames(lcc_ctx *c, int nframes, const int *slots, const float *const *d_pts, const int64_t *n,
                      long long max_blocks) {
    Batch b;
    memset(&b, 0, sizeof(b));
    b.nframes = nframes;
    long long blocks = 0;
    const long long per_block = 256 * 4;
    for (int f = 0; f < nframes; f++) {
        b.slot[f] = slots[f];
        b.pts[f] = reinterpret_cast<const float4 *>(d_pts[f]);
        b.n[f] = n[f];
        b.blk_prefix[f] = blocks;
        blocks += (n[f] + per_block - 1) / per_block;
    }
    bool contiguous = true;
    for (int f = 0; f < nframes; f++) contiguous = contiguous && slots[f] == slots[0] + f;
    if (contiguous) {
        LCC_CUDA(cudaMemsetAsync(c->s.stats + slots[0], 0, sizeof(DevStats) * nframes, c->stream));
    } else {
        for (int f = 0; f < nframes; f++)
            LCC_CUDA(cudaMemsetAsync(c->s.stats + slots[f], 0, sizeof(DevStats), c->stream));
    }
    b.blk_prefix[nframes] = blocks;
    LCC_LAUNCH(c, 0, launch_bin(c->g, c->s, b, blocks, c->stream, max_blocks));
    return LCC_OK;
}

lcc_status copy_bytes(lcc_ctx *c, int nframes, const int *slots, uint64_t *out_bytes) {
    if (!out_bytes) return LCC_OK;
    bool contiguous = true;
    for (int f = 0; f < nframes; f++) contiguous = contiguous && slots[f] == slots[0] + f;
    if (contiguous) {
        LCC_CUDA(cudaMemcpyAsync(out_bytes, c->s.bytes + slots[0], sizeof(uint64_t) * nframes, cudaMemcpyDefault,
                                 c->stream));
    } else {
        for (int f = 0; f < nframes; f++)
            LCC_CUDA(cudaMemcpyAsync(out_bytes + f, c->s.bytes + slots[f], sizeof(uint64_t), cudaMemcpyDefault,
                                     c->stream));
    }
    return LCC_OK;
}

lcc_status check_frames(lcc_ctx *c, int nframes, const float *const *d_pts, const int64_t *n,
                        uint8_t *const *d_out, const uint64_t *cap) {
    if (nframes < 1 || nframes > c->slots || !d_pts || !n || !d_out || !cap) return LCC_ERR_INVALID_ARG;
    for (int f = 0; f < nframes; f++) {
        if (n[f] < 0 || n[f] > (int64_t)1 << 31) return LCC_ERR_INVALID_ARG;
        if (n[f] > 0 && (!d_pts[f] || !aligned16(d_pts[f]))) return LCC_ERR_INVALID_ARG;
        if (!d_out[f] || !aligned16(d_out[f]) || cap[f] < (uint64_t)kHeaderBytes) return LCC_ERR_INVALID_ARG;
    }
    return LCC_OK;
}

}  // namespace api
}  // namespace lcc

using namespace lcc::api;

extern "C" {

const char *lcc_status_string(lcc_status s) {
    switch (s) {
    case LCC_OK: return "ok";
    case LCC_ERR_INVALID_ARG: return "invalid argument";
    case LCC_ERR_CAPACITY: return "output buffer too small";
    case LCC_ERR_CUDA: return "CUDA runtime error";
    case LCC_ERR_TIMEOUT: return "device wait timed out";
    case LCC_ERR_CORRUPT: return "corrupt stream";
    case LCC_ERR_UNSUPPORTED: return "unsupported";
    case LCC_ERR_NO_DEVICE: return "no sm_103 GPU";
    }
    return "unknown";
}

void lcc_default_params(lcc_params *p) {
    if (!p) return;
    p->tile_h = 4;
    p->tile_w = 4;
    p->fit_thr_m = 0.05f;
    p->quant_m = 0.02f;
    p->max_refits = 3;
    p->min_inlier_frac = 0.75f;
    p->merge_runs = 1;
    p->max_batch = 16;
    p->lookahead = 16;
    p->solver = 0;
    p->fit_schedule = 3;
    p->no_delta = 0;
    p->raw_exact = 0;
    p->temporal_candidates = 1;
    p->temporal_runs = 1;
    p->plane3 = 0;
}

lcc_status lcc_create(lcc_ctx **out, const lcc_sensor *sensor, const lcc_params *params, void *cuda_stream) {
    if (!out || !sensor || !params) return LCC_ERR_INVALID_ARG;
    *out = nullptr;
    const lcc_sensor &s = *sensor;
    const lcc_params &p = *params;
    if (s.rows < 1 || s.cols < 2 || s.rows > 65535 || s.cols > 65535 || !(s.elev_max_deg > s.elev_min_deg) ||
        (int64_t)s.rows * s.cols > (1 << 26) ||
        s.elev_max_deg > 90.0 || s.elev_min_deg < -90.0 || !(s.max_range_m > 0))
        return LCC_ERR_INVALID_ARG;
    if (!tile_supported(p.tile_h, p.tile_w)) return LCC_ERR_UNSUPPORTED;
    if (!(p.fit_thr_m >= 0) || !(p.quant_m > 0) || p.max_refits < 0 || p.max_refits > 6 ||
        !(p.min_inlier_frac >= 0) || p.max_batch < 1 || p.max_batch > kMaxBatch || p.lookahead < 0 ||
        p.lookahead > 32 || p.solver < 0 || p.solver > 1 || p.fit_schedule < 0 ||
        p.fit_schedule > 6 || p.no_delta < 0 || p.no_delta > 1 || p.raw_exact < 0 || p.raw_exact > 1 ||
        p.temporal_candidates < 0 || p.temporal_candidates > 4 || p.temporal_runs < 0 || p.temporal_runs > 1 ||
        p.plane3 < 0 || p.plane3 > 1)
        return LCC_ERR_INVALID_ARG;
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return LCC_ERR_NO_DEVICE;
    if (!(prop.major == 10 && prop.minor == 3)) return LCC_ERR_NO_DEVICE;

    lcc_ctx *c = new (std::nothrow) lcc_ctx();
    if (!c) return LCC_ERR_CUDA;
    c->sensor = s;
    c->prm = p;
    c->num_sms = prop.multiProcessorCount;
    c->stream = (cudaStream_t)cuda_stream;
    Geometry &g = c->g;
    g.H = s.rows;
    g.W = s.cols;
    g.th = p.tile_h;
    g.tw = p.tile_w;
    g.tpx = p.tile_h * p.tile_w;
    g.TR = (s.rows + p.tile_h - 1) / p.tile_h;
    g.TC = (s.cols + p.tile_w - 1) / p.tile_w;
    g.NT = g.TR * g.TC;
    g.thr = p.fit_thr_m;
    g.q = p.quant_m;
    g.rmax = (float)s.max_range_m;
    g.fmin = p.min_inlier_frac;
    g.R = p.max_refits;
    g.merge = p.merge_runs ? 1 : 0;
    g.lookahead = p.merge_runs ? p.lookahead : 0;
    g.solver = p.solver;
    g.schedule = p.fit_schedule;
    g.no_delta = p.no_delta;
    g.raw_exact = p.raw_exact;
    g.tcand = p.temporal_candidates;
    g.truns = p.temporal_runs && p.merge_runs ? 1 : 0;
    g.plane3 = p.plane3 ? 1 : 0;
    g.first_rounds = p.fit_schedule == 5 ? 0 : std::min(p.fit_schedule >= 3 ? 1 : p.fit_schedule, p.max_refits + 1);
    g.k_max = (int)floorf(p.fit_thr_m / p.quant_m + 0.5f) + 1;
    g.w_res = bits_for(2 * g.k_max);
    const int m_max = (int)floorf((float)s.max_range_m / p.quant_m + 0.5f) + 1;
    g.w_raw = p.raw_exact ? 32 : bits_for(m_max);   // lossless raw pixels: the range's fp32 bits
    g.elev_max_rad = (float)(s.elev_max_deg * (M_PI / 180.0));
    g.inv_d_el = (float)(s.rows / ((s.elev_max_deg - s.elev_min_deg) * (M_PI / 180.0)));
    g.inv_d_az = (float)(s.cols / (2.0 * M_PI));
    // the run walker keeps one tile row in shared memory
    if (g.w_res > 16 || (g.w_raw > 24 && !g.raw_exact) || merge_smem_bytes(g.TC) > 200 * 1024 || g.TC > 65535) {
        delete c;
        return LCC_ERR_UNSUPPORTED;
    }
    make_tables(s, c->h_tables);
    const int H = s.rows, W = s.cols;
    if (cudaMalloc(&c->d_tables, c->h_tables.size() * sizeof(float)) != cudaSuccess) {
        delete c;
        return LCC_ERR_CUDA;
    }
    cudaMemcpy(c->d_tables, c->h_tables.data(), c->h_tables.size() * sizeof(float), cudaMemcpyHostToDevice);
    const float *tb = (const float *)c->d_tables;
    g.ce = tb;
    g.se = g.ce + H;
    g.ct = g.se + H;
    g.st = g.ct + W;
    g.rbc = g.st + W;
    g.rbs = g.rbc + H + 1;
    g.cbc = g.rbs + H + 1;
    g.cbs = g.cbc + W;

    c->slots = p.max_batch;
    const size_t npx = (size_t)H * W, nt = (size_t)g.NT, sl = (size_t)c->slots;
    const size_t o_rimg = 0;
    const size_t o_tiles = o_rimg + align256(sl * npx * 4);
    const size_t o_codes = o_tiles + align256(sl * nt * sizeof(TileRec));
    const size_t o_offs = o_codes + align256(sl * nt * sizeof(TileCode));
    const size_t o_layout = o_offs + align256(sl * nt * sizeof(TileOff));
    const size_t o_stats = o_layout + align256(sl * sizeof(FrameLayout));
    const size_t o_bytes = o_stats + align256(sl * sizeof(DevStats));
    const size_t o_err = o_bytes + align256(sl * 8);
    const size_t o_dec = o_err + 256;
    const size_t o_lbcnt = o_dec + align256(sl * (nt + 4) * sizeof(DecTile));   // decoder state per slot
    const size_t o_rowtot = o_lbcnt + align256(sl * nt * 32);
    const size_t o_rowbase = o_rowtot + align256(sl * (size_t)g.TR * 32);
    const size_t o_queue = o_rowbase + align256(sl * (size_t)g.TR * 32);
    const size_t o_qcount = o_queue + align256(4 * sl * nt * 4);
    const size_t o_rowdone = o_qcount + 256;
    const size_t o_kplanes = o_rowdone + align256(sl * 4);
    const size_t o_coef = o_kplanes + align256(nt * sizeof(float4));
    const size_t total = o_coef + (p.plane3 ? align256(sl * nt * sizeof(float4)) : 0);
    if (cudaMalloc(&c->d_scratch, total) != cudaSuccess) {
        cudaFree(c->d_tables);
        delete c;
        return LCC_ERR_CUDA;
    }
    char *base = (char *)c->d_scratch;
    c->s.rimg = (uint32_t *)(base + o_rimg);
    c->s.tiles = (TileRec *)(base + o_tiles);
    c->s.codes = (TileCode *)(base + o_codes);
    c->s.offs = (TileOff *)(base + o_offs);
    c->s.layout = (FrameLayout *)(base + o_layout);
    c->s.stats = (DevStats *)(base + o_stats);
    c->s.bytes = (unsigned long long *)(base + o_bytes);
    c->s.err = (uint32_t *)(base + o_err);
    c->d_dec = (DecTile *)(base + o_dec);
    c->s.lbcnt = (uint8_t *)(base + o_lbcnt);
    c->s.rowtot = (uint32_t *)(base + o_rowtot);
    c->s.rowbase = (uint32_t *)(base + o_rowbase);
    c->s.queue = (uint32_t *)(base + o_queue);
    c->s.qcount = (uint32_t *)(base + o_qcount);
    c->s.rowdone = (uint32_t *)(base + o_rowdone);
    c->d_kplanes = (float4 *)(base + o_kplanes);
    c->s.coef = p.plane3 ? (float4 *)(base + o_coef) : nullptr;
    c->s.qcap = (uint32_t)(sl * nt);
    cudaMemset(c->d_scratch, 0, total);
    cudaMemset(c->s.rimg, 0xFF, sl * npx * 4);
    int prio_hi = 0;
    if (cudaHostAlloc(&c->h_pinned, sizeof(unsigned long long) * (kMaxBatch + 1), cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceGetStreamPriorityRange(nullptr, &prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->kstream, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_kplanes, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_kdone, cudaEventDisableTiming) != cudaSuccess) {
        lcc_destroy(c);
        return LCC_ERR_CUDA;
    }
    c->max_bytes = (uint64_t)kHeaderBytes +
                   4ull * ((npx + 31) / 32 + (nt * 4 + 31) / 32 + 4 * nt + 2 * nt + (npx + 31) / 32 +
                           (npx * g.w_res + 31) / 32 + (npx * g.w_raw + 31) / 32 + 4);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        lcc_destroy(c);
        return LCC_ERR_CUDA;
    }
    *out = c;
    return LCC_OK;
}

lcc_status lcc_destroy(lcc_ctx *c) {
    if (!c) return LCC_ERR_INVALID_ARG;
    cudaStreamSynchronize(c->stream);
    for (auto &r : c->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    if (c->prof_base) cudaEventDestroy(c->prof_base);
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->kstream) {
        cudaStreamSynchronize(c->kstream);
        cudaStreamDestroy(c->kstream);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_kplanes) cudaEventDestroy(c->ev_kplanes);
    if (c->ev_kdone) cudaEventDestroy(c->ev_kdone);
    cudaFree(c->d_tables);
    cudaFree(c->d_scratch);
    cudaFree(c->d_ent);
    cudaFree(c->d_stage_pts);
    cudaFree(c->d_stage_out);
    cudaFree(c->d_stage_bytes);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    delete c;
    return LCC_OK;
}

uint64_t lcc_max_encoded_bytes(const lcc_ctx *c) { return c ? c->max_bytes : 0; }

int64_t lcc_num_tiles(const lcc_ctx *c) { return c ? c->g.NT : 0; }

lcc_status lcc_tables(const lcc_ctx *c, float *ce, float *se, float *ct, float *st, float *rbc, float *rbs,
                      float *cbc, float *cbs) {
    if (!c) return LCC_ERR_INVALID_ARG;
    const int H = c->g.H, W = c->g.W;
    const float *t = c->h_tables.data();
    float *dst[8] = {ce, se, ct, st, rbc, rbs, cbc, cbs};
    const int len[8] = {H, H, W, W, H + 1, H + 1, W, W};
    for (int k = 0; k < 8; k++) {
        if (dst[k]) memcpy(dst[k], t, sizeof(float) * len[k]);
        t += len[k];
    }
    return LCC_OK;
}

lcc_status lcc_range_image(lcc_ctx *c, const float *d_pts, int64_t n, float *d_range, uint32_t *d_valid) {
    if (!c || n < 0 || (n > 0 && (!d_pts || !aligned16(d_pts)))) return LCC_ERR_INVALID_ARG;
    const int slot = 0;
    lcc_status st = bin_frames(c, 1, &slot, &d_pts, &n);
    if (st != LCC_OK) return st;
    LCC_LAUNCH(c, 7, launch_range_image(c->g, c->s.rimg, d_range, d_valid, c->stream));
    c->last_nframes = 1;
    return LCC_OK;
}

lcc_status lcc_keyframe_create(lcc_ctx *c, lcc_keyframe **out) {
    if (!c || !out) return LCC_ERR_INVALID_ARG;
    lcc_keyframe *k = new (std::nothrow) lcc_keyframe();
    if (!k) return LCC_ERR_CUDA;
    k->ctx = c;
    k->nt = c->g.NT;
    if (cudaMalloc(&k->planes, sizeof(float4) * k->nt) != cudaSuccess) {
        delete k;
        return LCC_ERR_CUDA;
    }
    cudaMemsetAsync(k->planes, 0, sizeof(float4) * k->nt, c->stream);
    *out = k;
    return LCC_OK;
}

void lcc_keyframe_free(lcc_keyframe *k) {
    if (!k) return;
    cudaStreamSynchronize(k->ctx->stream);
    cudaFree(k->planes);
    delete k;
}

lcc_status lcc_encode_keyframe(lcc_ctx *c, const float *d_pts, int64_t n, lcc_keyframe *kf, uint8_t *d_out,
                               uint64_t cap, uint64_t *out_bytes) {
    if (!c) return LCC_ERR_INVALID_ARG;
    if (kf && kf->ctx != c) return LCC_ERR_INVALID_ARG;
    lcc_status st = check_frames(c, 1, &d_pts, &n, &d_out, &cap);
    if (st != LCC_OK) return st;
    const int slot = 0;
    if ((st = bin_frames(c, 1, &slot, &d_pts, &n)) != LCC_OK) return st;
    float4 *kfo = kf ? kf->planes : nullptr;
    if ((st = encode_batch(c, 0, 1, &slot, &d_out, &cap, nullptr, nullptr, &kfo)) != LCC_OK) return st;
    c->last_nframes = 1;
    return copy_bytes(c, 1, &slot, out_bytes);
}

lcc_status lcc_encode_keyframe_seeded(lcc_ctx *c, const float *d_pts, int64_t n, const float *d_prop,
                                      float skip_logit, lcc_keyframe *kf, uint8_t *d_out, uint64_t cap,
                                      uint64_t *out_bytes) {
    if (!c || !d_prop || ((uintptr_t)d_prop & 3u) || !(skip_logit == skip_logit)) return LCC_ERR_INVALID_ARG;
    if (kf && kf->ctx != c) return LCC_ERR_INVALID_ARG;
    lcc_status st = check_frames(c, 1, &d_pts, &n, &d_out, &cap);
    if (st != LCC_OK) return st;
    const int slot = 0;
    if ((st = bin_frames(c, 1, &slot, &d_pts, &n)) != LCC_OK) return st;
    float4 *kfo = kf ? kf->planes : nullptr;
    if ((st = encode_batch(c, 0, 1, &slot, &d_out, &cap, nullptr, nullptr, &kfo, nullptr, &d_prop, skip_logit)) !=
        LCC_OK)
        return st;
    c->last_nframes = 1;
    return copy_bytes(c, 1, &slot, out_bytes);
}

lcc_status lcc_encode_keyframes(lcc_ctx *c, int32_t nframes, const float *const *d_pts, const int64_t *n,
                                const float *const *d_prop, float skip_logit, uint8_t *const *d_out,
                                const uint64_t *cap, uint64_t *out_bytes) {
    if (!c || !(skip_logit == skip_logit)) return LCC_ERR_INVALID_ARG;
    lcc_status st = check_frames(c, nframes, d_pts, n, d_out, cap);
    if (st != LCC_OK) return st;
    if (d_prop)
        for (int f = 0; f < nframes; f++)
            if (!d_prop[f] || ((uintptr_t)d_prop[f] & 3u)) return LCC_ERR_INVALID_ARG;
    int slots[kMaxBatch];
    for (int f = 0; f < nframes; f++) slots[f] = f;
    if ((st = bin_frames(c, nframes, slots, d_pts, n)) != LCC_OK) return st;
    if ((st = encode_batch(c, 0, nframes, slots, d_out, cap, nullptr, nullptr, nullptr, nullptr, d_prop,
                           skip_logit)) != LCC_OK)
        return st;
    c->last_nframes = nframes;
    return copy_bytes(c, nframes, slots, out_bytes);
}

lcc_status lcc_encode_pframes(lcc_ctx *c, const lcc_keyframe *kf, int32_t nframes, const double *poses,
                              const float *const *d_pts, const int64_t *n, uint8_t *const *d_out,
                              const uint64_t *cap, uint64_t *out_bytes) {
    if (!c || !kf || kf->ctx != c || !poses) return LCC_ERR_INVALID_ARG;
    lcc_status st = check_frames(c, nframes, d_pts, n, d_out, cap);
    if (st != LCC_OK) return st;
    int slots[kMaxBatch];
    const float4 *kfi[kMaxBatch];
    for (int f = 0; f < nframes; f++) {
        slots[f] = f;
        kfi[f] = kf->planes;
    }
    if ((st = bin_frames(c, nframes, slots, d_pts, n)) != LCC_OK) return st;
    if ((st = encode_batch(c, 1, nframes, slots, d_out, cap, poses, kfi, nullptr)) != LCC_OK) return st;
    c->last_nframes = nframes;
    return copy_bytes(c, nframes, slots, out_bytes);
}

lcc_status lcc_encode_pframe(lcc_ctx *c, const lcc_keyframe *kf, const double pose[16], const float *d_pts,
                             int64_t n, uint8_t *d_out, uint64_t cap, uint64_t *out_bytes) {
    return lcc_encode_pframes(c, kf, 1, pose, &d_pts, &n, &d_out, &cap, out_bytes);
}

}  // extern "C"

namespace {

// The sequence encode.  With h_pts, frame f's points are first copied from host memory into
// d_pts[f]: the key frame's copy on the context stream, the P frames' copies on the side stream
// where their binning and first fit pass follow, so the copies overlap the key frame's encode.
lcc_status encode_sequence(lcc_ctx *c, int32_t nframes, int32_t key_index, const double *poses,
                           const float *const *d_pts, const int64_t *n, uint8_t *const *d_out, const uint64_t *cap,
                           uint64_t *out_bytes, lcc_keyframe *kf, const float *const *h_pts,
                           bool via_link = false) {
    if (!c || !poses || key_index < 0 || key_index >= nframes) return LCC_ERR_INVALID_ARG;
    // points read in place over the host link: a binning grid of two CTAs per SM keeps enough
    // reads in flight for the link and leaves the rest of the SMs to the key frame's kernels
    const long long bin_cap = via_link ? 2LL * c->num_sms : 0LL;
    if (kf && kf->ctx != c) return LCC_ERR_INVALID_ARG;
    lcc_status st = check_frames(c, nframes, d_pts, n, d_out, cap);
    if (st != LCC_OK) return st;
    const bool overlap = nframes > 1;
    auto h2d = [&](int f, cudaStream_t sm) -> bool {
        return !h_pts || n[f] == 0 ||
               cudaMemcpyAsync(const_cast<float *>(d_pts[f]), h_pts[f], (size_t)n[f] * 16, cudaMemcpyHostToDevice,
                               sm) == cudaSuccess;
    };
    lcc_keyframe local;
    lcc_keyframe *k = kf;
    if (!k) {
        // the key frame's planes must outlive the P pass: use the decoder scratch
        static_assert(sizeof(DecTile) >= sizeof(float4), "scratch size");
        local.ctx = c;
        local.nt = c->g.NT;
        local.planes = reinterpret_cast<float4 *>(c->d_dec);
        k = &local;
    }
    int slots[kMaxBatch];
    for (int f = 0; f < nframes; f++) slots[f] = f;
    if (!overlap) {
        for (int f = 0; f < nframes; f++)
            if (!h2d(f, c->stream)) return LCC_ERR_CUDA;
        if ((st = bin_frames(c, nframes, slots, d_pts, n)) != LCC_OK) return st;
    }
    const int kslot = key_index;
    uint8_t *kout = d_out[key_index];
    const uint64_t kcap = cap[key_index];
    int pslots[kMaxBatch];
    uint8_t *pout[kMaxBatch];
    uint64_t pcap[kMaxBatch];
    const float4 *kfi[kMaxBatch];
    std::vector<double> pposes;
    int np = 0;
    for (int f = 0; f < nframes; f++) {
        if (f == key_index) continue;
        pslots[np] = f;
        pout[np] = d_out[f];
        pcap[np] = cap[f];
        kfi[np] = k->planes;
        pposes.insert(pposes.end(), poses + 16 * f, poses + 16 * f + 16);
        np++;
    }
    float4 *kfo = k->planes;
    if (!overlap) {
        if ((st = encode_batch(c, 0, 1, &kslot, &kout, &kcap, nullptr, nullptr, &kfo)) != LCC_OK) return st;
        if ((st = encode_batch(c, 1, np, pslots, pout, pcap, pposes.data(), kfi, nullptr)) != LCC_OK) return st;
    } else {
        // The key frame's chain (binning, fit, run pre-test, merge, pack) runs on a private
        // stream of the highest priority, issued first, so that its blocks are dispatched ahead of
        // the P frames' whenever both wait for room on the SMs.  The P frames' binning, spatial fits
        // and run pre-test do not need the key frame and run on the side stream beside it.  Their
        // temporal test needs the key frame's coding planes, which its merge writes: the P frames'
        // temporal test, merge and pack follow on the side stream while the key frame's pack
        // finishes.  The calling stream then waits for both.
        Batch bk, bp;
        Poses pk, pp;
        prepare_batch(bk, pk, 0, 1, &kslot, &kout, &kcap, nullptr, nullptr, &kfo, nullptr);
        prepare_batch(bp, pp, 1, np, pslots, pout, pcap, pposes.data(), nullptr, nullptr, nullptr);
        bp.qset = 1;   // the P frames' queued rounds run beside the key frame's: their own queues
        const float *pdp[kMaxBatch];
        int64_t pn[kMaxBatch];
        for (int q = 0; q < np; q++) {
            pdp[q] = d_pts[pslots[q]];
            pn[q] = n[pslots[q]];
        }
        struct StreamGuard {   // launches (and their profiling events) go to c->stream
            lcc_ctx *c;
            cudaStream_t saved;
            ~StreamGuard() { c->stream = saved; }
        } guard{c, c->stream};
        const cudaStream_t main = c->stream;
        LCC_CUDA(cudaEventRecord(c->ev_fork, main));
        LCC_CUDA(cudaStreamWaitEvent(c->kstream, c->ev_fork, 0));
        LCC_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        // key frame: binning and fit
        c->stream = c->kstream;
        if (!h2d(key_index, c->kstream)) return LCC_ERR_CUDA;
        if ((st = bin_frames(c, 1, &kslot, &d_pts[key_index], &n[key_index], bin_cap)) != LCC_OK) return st;
        LCC_LAUNCH(c, 1, launch_fit(c->g, c->s, bk, pk, c->stream));
        // P frames: binning, spatial fits (and the rest of their rounds), run pre-test
        c->stream = c->side;
        for (int q = 0; q < np; q++)
            if (!h2d(pslots[q], c->side)) return LCC_ERR_CUDA;
        if ((st = bin_frames(c, np, pslots, pdp, pn, bin_cap)) != LCC_OK) return st;
        LCC_LAUNCH(c, 1, launch_fit(c->g, c->s, bp, pp, c->stream));
        if (c->g.schedule >= 1)
            LCC_LAUNCH_N(c, 3, queued_round_kernels(c->g, bp), launch_queued_rounds(c->g, c->s, bp, c->stream));
        const bool ppretest = c->g.merge && c->g.lookahead > 0;
        if (ppretest) LCC_LAUNCH(c, 8, launch_lookbehind(c->g, c->s, bp, c->stream));
        // key frame: the rest of its rounds and its pre-test, merge (its coding planes), pack
        c->stream = c->kstream;
        if (c->g.schedule >= 1)
            LCC_LAUNCH_N(c, 3, queued_round_kernels(c->g, bk), launch_queued_rounds(c->g, c->s, bk, c->stream));
        if (c->g.merge && c->g.lookahead > 0) LCC_LAUNCH(c, 8, launch_lookbehind(c->g, c->s, bk, c->stream));
        LCC_LAUNCH(c, 2, launch_merge(c->g, c->s, bk, c->stream));   // with the frame's stream layout
        LCC_CUDA(cudaEventRecord(c->ev_kplanes, c->kstream));
        LCC_LAUNCH(c, 4, launch_pack(c->g, c->s, bk, c->stream));
        LCC_CUDA(cudaEventRecord(c->ev_kdone, c->kstream));
        // P frames: temporal test against the key planes, merge, pack
        c->stream = c->side;
        LCC_CUDA(cudaStreamWaitEvent(c->side, c->ev_kplanes, 0));
        for (int f = 0; f < np; f++) bp.kf[f] = k->planes;
        LCC_LAUNCH(c, 9, launch_temporal(c->g, c->s, bp, pp, c->stream));
        // with temporal runs, the P tiles' candidates that became temporal are tested again against
        // their relaxed planes (a pass that skips every tile without such a candidate)
        if (ppretest && c->g.truns) LCC_LAUNCH(c, 8, launch_lookbehind(c->g, c->s, bp, c->stream, true));
        LCC_LAUNCH(c, 2, launch_merge(c->g, c->s, bp, c->stream));
        LCC_LAUNCH(c, 4, launch_pack(c->g, c->s, bp, c->stream));
        LCC_CUDA(cudaEventRecord(c->ev_join, c->side));
        LCC_CUDA(cudaStreamWaitEvent(main, c->ev_kdone, 0));
        LCC_CUDA(cudaStreamWaitEvent(main, c->ev_join, 0));
    }
    c->last_nframes = nframes;
    return copy_bytes(c, nframes, slots, out_bytes);
}

}  // namespace

extern "C" {

lcc_status lcc_encode_sequence(lcc_ctx *c, int32_t nframes, int32_t key_index, const double *poses,
                               const float *const *d_pts, const int64_t *n, uint8_t *const *d_out,
                               const uint64_t *cap, uint64_t *out_bytes, lcc_keyframe *kf) {
    return encode_sequence(c, nframes, key_index, poses, d_pts, n, d_out, cap, out_bytes, kf, nullptr);
}

}  // extern "C"

namespace {

// Device address of page-locked host memory (mapped into the device's address space under
// unified addressing), or NULL for memory the device cannot address.
void *device_view(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    return a.devicePointer;
}

struct CopyOut {
    const uint8_t *src[kMaxBatch];
    uint8_t *dst[kMaxBatch];
    unsigned long long cap[kMaxBatch];
    const unsigned long long *nbytes;
};

// Every frame's stream from the device staging buffer straight into the caller's page-locked
// host buffer (16-byte stores over the host link), sized by the stream length on the device.
__global__ void __launch_bounds__(256) k_copy_out(CopyOut co) {
    const int f = blockIdx.y;
    const unsigned long long nb = co.nbytes[f] <= co.cap[f] ? co.nbytes[f] : 0ull;
    const uint4 *src = reinterpret_cast<const uint4 *>(co.src[f]);
    uint4 *dst = reinterpret_cast<uint4 *>(co.dst[f]);
    const unsigned long long n16 = nb / 16;
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n16; i += gridDim.x * 256ull) dst[i] = src[i];
    const unsigned long long tail = nb - n16 * 16;   // streams are whole 32-bit words
    if (blockIdx.x == 0 && threadIdx.x < tail / 4)
        reinterpret_cast<uint32_t *>(co.dst[f] + n16 * 16)[threadIdx.x] =
            reinterpret_cast<const uint32_t *>(co.src[f] + n16 * 16)[threadIdx.x];
}

}  // namespace

extern "C" {

lcc_status lcc_encode_sequence_host(lcc_ctx *c, int32_t nframes, int32_t key_index, const double *poses,
                                    const float *const *h_pts, const int64_t *n, uint8_t *const *h_out,
                                    const uint64_t *cap, uint64_t *out_bytes) {
    if (!c || !h_pts || !n || !h_out || !cap || !out_bytes || nframes < 1 || nframes > c->slots)
        return LCC_ERR_INVALID_ARG;
    size_t pts_total = 0, out_total = 0;
    for (int f = 0; f < nframes; f++) {
        if (n[f] < 0) return LCC_ERR_INVALID_ARG;
        pts_total += align256((size_t)n[f] * 16);
        out_total += align256((size_t)cap[f]);
    }
    if (pts_total > c->stage_pts_cap) {
        cudaFree(c->d_stage_pts);
        c->d_stage_pts = nullptr;
        LCC_CUDA(cudaMalloc(&c->d_stage_pts, pts_total));
        c->stage_pts_cap = pts_total;
    }
    if (out_total > c->stage_out_cap) {
        cudaFree(c->d_stage_out);
        c->d_stage_out = nullptr;
        LCC_CUDA(cudaMalloc(&c->d_stage_out, out_total));
        c->stage_out_cap = out_total;
    }
    if (!c->d_stage_bytes) LCC_CUDA(cudaMalloc(&c->d_stage_bytes, sizeof(unsigned long long) * kMaxBatch));
    // Page-locked inputs are read by the binning kernel in place, over the host link (no staging
    // copy); page-locked outputs are written by one copy-out kernel (no second host round trip).
    bool in_mapped = true, out_mapped = true;
    const float *hv[kMaxBatch];
    uint8_t *ov[kMaxBatch];
    for (int f = 0; f < nframes; f++) {
        hv[f] = n[f] ? (const float *)device_view(h_pts[f]) : nullptr;
        in_mapped = in_mapped && (!n[f] || (hv[f] && aligned16(hv[f])));
        ov[f] = (uint8_t *)device_view(h_out[f]);
        out_mapped = out_mapped && ov[f] && aligned16(ov[f]);
    }
    const float *dp[kMaxBatch];
    uint8_t *dout[kMaxBatch];
    char *pp = (char *)c->d_stage_pts;
    uint8_t *po = c->d_stage_out;
    for (int f = 0; f < nframes; f++) {
        dp[f] = in_mapped ? hv[f] : (const float *)pp;
        pp += align256((size_t)n[f] * 16);
        dout[f] = po;
        po += align256((size_t)cap[f]);
    }
    lcc_status st = encode_sequence(c, nframes, key_index, poses, dp, n, dout, cap, (uint64_t *)c->d_stage_bytes,
                                    nullptr, in_mapped ? nullptr : h_pts, in_mapped);
    if (st != LCC_OK) return st;
    if (out_mapped) {
        CopyOut co;
        for (int f = 0; f < nframes; f++) {
            co.src[f] = dout[f];
            co.dst[f] = ov[f];
            co.cap[f] = cap[f];
        }
        co.nbytes = c->d_stage_bytes;
        k_copy_out<<<dim3(16, nframes), 256, 0, c->stream>>>(co);
        LCC_CUDA(cudaGetLastError());
        // sizes and the error word into page-locked memory, then the one host round trip
        LCC_CUDA(cudaMemcpyAsync(c->h_pinned, c->d_stage_bytes, sizeof(uint64_t) * nframes, cudaMemcpyDeviceToHost,
                                 c->stream));
        LCC_CUDA(cudaMemcpyAsync(c->h_pinned + kMaxBatch, c->s.err, 4, cudaMemcpyDeviceToHost, c->stream));
        LCC_CUDA(cudaStreamSynchronize(c->stream));
        memcpy(out_bytes, c->h_pinned, sizeof(uint64_t) * nframes);
        const uint32_t e = (uint32_t)(c->h_pinned[kMaxBatch] & 0xFFFFFFFFull);
        if (!e) return LCC_OK;
        return latched(c);   // reads and clears the error word
    } else {
        LCC_CUDA(cudaMemcpyAsync(out_bytes, c->d_stage_bytes, sizeof(uint64_t) * nframes, cudaMemcpyDeviceToHost,
                                 c->stream));
        LCC_CUDA(cudaStreamSynchronize(c->stream));
        for (int f = 0; f < nframes; f++) {
            const uint64_t nb = out_bytes[f] <= cap[f] ? out_bytes[f] : 0;
            if (nb) LCC_CUDA(cudaMemcpyAsync(h_out[f], dout[f], nb, cudaMemcpyDeviceToHost, c->stream));
        }
        LCC_CUDA(cudaStreamSynchronize(c->stream));
    }
    return latched(c);
}

lcc_status lcc_keyframe_from_stream(lcc_ctx *c, const uint8_t *d_bits, uint64_t nbytes, lcc_keyframe *kf) {
    if (!c || !kf || kf->ctx != c || !d_bits || !aligned16(d_bits)) return LCC_ERR_INVALID_ARG;
    Poses p;
    memset(&p, 0, sizeof(p));
    DecBatch db;
    memset(&db, 0, sizeof(db));
    db.bits[0] = d_bits;
    db.nbytes[0] = nbytes;
    db.dt[0] = dec_slot(c, 0);
    LCC_LAUNCH(c, 5, launch_decode_prep(c->g, db, 1, nullptr, p, kf->planes, c->s.err, 0, c->stream));
    return LCC_OK;
}

namespace {

// The occupancy bitmap of a stream is its first section: copied as it is (a stream too short to
// hold it is latched as corrupt by the prep kernel).
lcc_status copy_valid(lcc_ctx *c, const uint8_t *d_bits, uint64_t nbytes, uint32_t *d_valid) {
    if (!d_valid) return LCC_OK;
    const size_t words = ((size_t)c->g.H * c->g.W + 31) / 32;
    if (nbytes >= (uint64_t)kHeaderBytes + 4 * words)
        LCC_CUDA(cudaMemcpyAsync(d_valid, d_bits + kHeaderBytes, 4 * words, cudaMemcpyDeviceToDevice, c->stream));
    return LCC_OK;
}

}  // namespace

lcc_status lcc_decode(lcc_ctx *c, const uint8_t *d_bits, uint64_t nbytes, const lcc_keyframe *kf,
                      const double pose[16], float *d_range, float *d_xyz4, uint32_t *d_valid) {
    if (!c || !d_bits || !aligned16(d_bits)) return LCC_ERR_INVALID_ARG;
    if (kf && (kf->ctx != c || !pose)) return LCC_ERR_INVALID_ARG;
    if (d_xyz4 && !aligned16(d_xyz4)) return LCC_ERR_INVALID_ARG;
    Poses p;
    memset(&p, 0, sizeof(p));
    if (pose) memcpy(p.m[0], pose, 16 * sizeof(double));
    DecBatch db;
    memset(&db, 0, sizeof(db));
    db.bits[0] = d_bits;
    db.nbytes[0] = nbytes;
    db.dt[0] = dec_slot(c, 0);
    db.range[0] = d_range;
    db.xyz[0] = reinterpret_cast<float4 *>(d_xyz4);
    LCC_LAUNCH(c, 5, launch_decode_prep(c->g, db, 1, kf ? kf->planes : nullptr, p, nullptr, c->s.err, kf ? 1 : 0,
                                        c->stream));
    LCC_LAUNCH(c, 6, launch_decode_px(c->g, db, 1, c->s.err, c->stream));
    return copy_valid(c, d_bits, nbytes, d_valid);
}

lcc_status lcc_decode_sequence(lcc_ctx *c, int32_t nframes, int32_t key_index, const double *poses,
                               const uint8_t *const *d_bits, const uint64_t *nbytes, float *const *d_range,
                               float *const *d_xyz4, uint32_t *const *d_valid) {
    if (!c || !poses || !d_bits || !nbytes || nframes < 1 || nframes > c->slots || key_index < 0 ||
        key_index >= nframes)
        return LCC_ERR_INVALID_ARG;
    for (int f = 0; f < nframes; f++) {
        if (!d_bits[f] || !aligned16(d_bits[f])) return LCC_ERR_INVALID_ARG;
        if (d_xyz4 && d_xyz4[f] && !aligned16(d_xyz4[f])) return LCC_ERR_INVALID_ARG;
    }
    DecBatch dk, dp;
    memset(&dk, 0, sizeof(dk));
    memset(&dp, 0, sizeof(dp));
    Poses pk, pp;
    memset(&pk, 0, sizeof(pk));
    memset(&pp, 0, sizeof(pp));
    dk.bits[0] = d_bits[key_index];
    dk.nbytes[0] = nbytes[key_index];
    dk.dt[0] = dec_slot(c, key_index);
    dk.range[0] = d_range ? d_range[key_index] : nullptr;
    dk.xyz[0] = d_xyz4 ? reinterpret_cast<float4 *>(d_xyz4[key_index]) : nullptr;
    int np = 0;
    for (int f = 0; f < nframes; f++) {
        if (f == key_index) continue;
        dp.bits[np] = d_bits[f];
        dp.nbytes[np] = nbytes[f];
        dp.dt[np] = dec_slot(c, f);
        dp.range[np] = d_range ? d_range[f] : nullptr;
        dp.xyz[np] = d_xyz4 ? reinterpret_cast<float4 *>(d_xyz4[f]) : nullptr;
        memcpy(pp.m[np], poses + 16 * (size_t)f, 16 * sizeof(double));
        np++;
    }
    // the key frame's stream gives its coding planes, then all P streams are resolved against them
    // in one launch (a CTA per stream) and reconstructed in one launch
    LCC_LAUNCH(c, 5, launch_decode_prep(c->g, dk, 1, nullptr, pk, c->d_kplanes, c->s.err, 0, c->stream));
    LCC_LAUNCH(c, 6, launch_decode_px(c->g, dk, 1, c->s.err, c->stream));
    LCC_LAUNCH(c, 5, launch_decode_prep(c->g, dp, np, c->d_kplanes, pp, nullptr, c->s.err, 1, c->stream));
    LCC_LAUNCH(c, 6, launch_decode_px(c->g, dp, np, c->s.err, c->stream));
    if (d_valid)
        for (int f = 0; f < nframes; f++)
            if (d_valid[f]) {
                const lcc_status st = copy_valid(c, d_bits[f], nbytes[f], d_valid[f]);
                if (st != LCC_OK) return st;
            }
    return LCC_OK;
}

lcc_status lcc_sync(lcc_ctx *c) {
    if (!c) return LCC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LCC_ERR_CUDA;
    return latched(c);
}

lcc_status lcc_last_stats(lcc_ctx *c, int32_t frame, lcc_stats *out) {
    if (!c || !out || frame < 0 || frame >= c->last_nframes) return LCC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LCC_ERR_CUDA;
    DevStats d;
    LCC_CUDA(cudaMemcpy(&d, c->s.stats + frame, sizeof(d), cudaMemcpyDeviceToHost));
    public_stats(d, out);
    return LCC_OK;
}

lcc_status lcc_tile_records(lcc_ctx *c, int32_t frame, lcc_tile_info *h_out, int64_t cap) {
    if (!c || !h_out || frame < 0 || frame >= c->last_nframes || cap < c->g.NT) return LCC_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LCC_ERR_CUDA;
    LCC_CUDA(cudaMemcpy(h_out, c->s.tiles + (size_t)frame * c->g.NT, sizeof(TileRec) * c->g.NT,
                        cudaMemcpyDeviceToHost));
    return LCC_OK;
}

lcc_status lcc_tile_coefficients(lcc_ctx *c, int32_t frame, float *h_out, int64_t cap) {
    if (!c || !h_out || frame < 0 || frame >= c->last_nframes || cap < c->g.NT) return LCC_ERR_INVALID_ARG;
    if (!c->s.coef) return LCC_ERR_UNSUPPORTED;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return LCC_ERR_CUDA;
    LCC_CUDA(cudaMemcpy(h_out, c->s.coef + (size_t)frame * c->g.NT, sizeof(float4) * c->g.NT, cudaMemcpyDeviceToHost));
    return LCC_OK;
}

lcc_status lcc_set_profiling(lcc_ctx *c, int32_t enable) {
    if (!c) return LCC_ERR_INVALID_ARG;
    c->prof = enable != 0;
    prof_collect(c);
    prof_reset(c);
    return LCC_OK;
}

int32_t lcc_kernel_timeline(lcc_ctx *c, char names[][16], float *t0_ms, float *t1_ms, int32_t cap) {
    if (!c || cap < 0) return 0;
    prof_collect(c);
    const int32_t w = (int32_t)std::min<size_t>((size_t)cap, c->timeline.size());
    for (int32_t k = 0; k < w; k++) {
        const TimelineRec &r = c->timeline[k];
        if (names) {
            strncpy(names[k], kKernelNames[r.name], 15);
            names[k][15] = 0;
        }
        if (t0_ms) t0_ms[k] = r.t0;
        if (t1_ms) t1_ms[k] = r.t1;
    }
    return w;
}

int32_t lcc_kernel_times(lcc_ctx *c, char names[][16], int64_t *launches, double *ms, int32_t cap) {
    if (!c) return 0;
    prof_collect(c);
    int w = 0;
    for (int k = 0; k < kNumKernels && w < cap; k++) {
        if (!c->launches[k]) continue;
        if (names) {
            strncpy(names[w], kKernelNames[k], 15);
            names[w][15] = 0;
        }
        if (launches) launches[w] = c->launches[k];
        if (ms) ms[w] = c->ms[k];
        w++;
    }
    return w;
}

}  // extern "C"
