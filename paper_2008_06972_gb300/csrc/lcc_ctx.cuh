// Host-side state of an lcc context shared by the translation units of the
// C ABI (single-sequence calls in lcc_api.cu, the batch planner in
// lcc_plan.cu).  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "lcc.h"
#include "lcc_internal.cuh"

namespace lcc {
namespace api {

struct ProfRec {
    int name;
    cudaEvent_t a, b;
    int count;   // kernels launched between the two events
};

struct TimelineRec {
    int name;
    float t0, t1;   // ms after the first launch timed since profiling was (re)enabled
};
constexpr size_t kMaxTimeline = 65536;

constexpr int kNumKernels = 16;
extern const char *kKernelNames[];

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace api
}  // namespace lcc

struct lcc_keyframe {
    lcc_ctx *ctx;
    float4 *planes;
    int64_t nt;
};

struct lcc_ctx {
    lcc_sensor sensor;
    lcc_params prm;
    cudaStream_t stream = nullptr;
    cudaStream_t side = nullptr;          // second stream for work that overlaps the key frame
    cudaStream_t kstream = nullptr;   // key-frame chain of a sequence call (highest priority)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_kplanes = nullptr, ev_kdone = nullptr;
    lcc::Geometry g{};
    lcc::Scratch s{};
    void *d_tables = nullptr;
    void *d_scratch = nullptr;
    lcc::DecTile *d_dec = nullptr;      // decoder state: per slot NT DecTiles, then a DecState
    float4 *d_kplanes = nullptr;        // key-frame coding planes of lcc_decode_sequence
    void *d_ent = nullptr;              // entropy-stage scratch (allocated on first use)
    std::vector<float> h_tables;  // ce, se, ct, st, rbc, rbs, cbc, cbs
    int slots = 0;
    int num_sms = 0;   // SMs of the context's device
    uint64_t max_bytes = 0;
    int last_nframes = 0;
    // profiling
    bool prof = false;
    std::vector<lcc::api::ProfRec> pending;
    std::vector<cudaEvent_t> pool;
    int64_t launches[lcc::api::kNumKernels] = {};
    double ms[lcc::api::kNumKernels] = {};
    cudaEvent_t prof_base = nullptr;   // start event of the first timed launch
    std::vector<lcc::api::TimelineRec> timeline;
    // host-buffer staging
    void *d_stage_pts = nullptr;
    size_t stage_pts_cap = 0;
    uint8_t *d_stage_out = nullptr;
    size_t stage_out_cap = 0;
    unsigned long long *d_stage_bytes = nullptr;
    unsigned long long *h_pinned = nullptr;   // page-locked: stream sizes (kMaxBatch) + error word
};

// Decoder state of batch slot f (NT DecTiles, then the slot's DecState).
inline lcc::DecTile *dec_slot(lcc_ctx *c, int f) { return c->d_dec + (size_t)f * ((size_t)c->g.NT + 4); }

namespace lcc {
namespace api {

int prof_begin(lcc_ctx *c, int name, int count = 1);
void prof_end(lcc_ctx *c, int idx);
bool aligned16(const void *p);
// The device counters of one frame as the public statistics record.
void public_stats(const DevStats &d, lcc_stats *out);
// Reads and clears the device error word (synchronous).
lcc_status latched(lcc_ctx *c);
// Bin frames d_pts[f] into slots[f] (their stats are reset first).
lcc_status bin_frames(lcc_ctx *c, int nframes, const int *slots, const float *const *d_pts, const int64_t *n,
                      long long max_blocks = 0);
// Fit, merge, scan and pack frames already binned into slots[f].  kf[f] (P frames) is the key-frame
// plane table frame f is coded against; kf_out[f] (key frames) receives frame f's coding planes;
// nbytes_out[f], when given, receives frame f's stream size in device memory; prop[f], when given,
// seeds frame f's tile fits (with skip_logit).
lcc_status encode_batch(lcc_ctx *c, int kind, int nframes, const int *slots, uint8_t *const *d_out,
                        const uint64_t *cap, const double *poses, const float4 *const *kf, float4 *const *kf_out,
                        unsigned long long *const *nbytes_out = nullptr, const float *const *prop = nullptr,
                        float skip_logit = 0.f);
lcc_status check_frames(lcc_ctx *c, int nframes, const float *const *d_pts, const int64_t *n,
                        uint8_t *const *d_out, const uint64_t *cap);
// Net inputs (8x8 tiles) of the frames binned into slots 0..nframes-1 of c, on c's stream; the
// range images are kept for the encode that follows.  Frame f's tiles are rows f*NT.. of d_x.
// d_need (may be NULL): per tile, 1 if it has the 3 valid pixels a fit needs.
lcc_status net_inputs_slots(lcc_ctx *c, int nframes, uint16_t *d_x, float4 *d_anchor, uint8_t *d_need = nullptr);
// The pairs of tiles with a needed tile (d_pairs, (ntiles + 1) / 2 entries; their count at
// *d_npairs), on stream st.
lcc_status net_pairs(const uint8_t *d_need, int64_t ntiles, uint32_t *d_pairs, uint32_t *d_npairs, cudaStream_t st);
// Proposal-net inference on stream st instead of the net's own stream; with a pair list only the
// listed pairs' outputs are written.
lcc_status net_forward_on(lcc_net *net, const uint16_t *d_x, int64_t ntiles, float *d_out, cudaStream_t st,
                          const uint32_t *d_pairs = nullptr, const uint32_t *d_npairs = nullptr);
// Reads and clears the net's bounded-wait error flag (synchronous): LCC_ERR_TIMEOUT if it was set.
lcc_status net_latched(lcc_net *net);

}  // namespace api
}  // namespace lcc

#define LCC_LAUNCH(ctx, id, call)                                  \
    do {                                                           \
        const int _pi = lcc::api::prof_begin(ctx, id);             \
        const cudaError_t _e = (call);                             \
        lcc::api::prof_end(ctx, _pi);                              \
        if (_e != cudaSuccess) return LCC_ERR_CUDA;                \
    } while (0)

// The same for a call that launches n kernels (n = 0: timed, not counted).
#define LCC_LAUNCH_N(ctx, id, n, call)                             \
    do {                                                           \
        const int _pi = lcc::api::prof_begin(ctx, id, n);          \
        const cudaError_t _e = (call);                             \
        lcc::api::prof_end(ctx, _pi);                              \
        if (_e != cudaSuccess) return LCC_ERR_CUDA;                \
    } while (0)

#define LCC_CUDA(call)                                   \
    do {                                                 \
        if ((call) != cudaSuccess) return LCC_ERR_CUDA;  \
    } while (0)
