// Batched encode of a table of sequences (lcc_plan_*): key-frame grouping,
// chunking of frames into the contexts' slots, fork/join of resolution
// classes onto side streams, and capture of the whole enqueue as one CUDA
// graph that is replayed.  With a proposal net attached, every chunk of key
// frames of an 8x8-tile class runs the net's input and tcgen05 inference
// kernels between its binning and its (seeded) fit, inside the same graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "lcc.h"
#include "lcc_ctx.cuh"

using namespace lcc;
using namespace lcc::api;

namespace {

constexpr int kMaxPlanContexts = 8;

// One frame of the table, in the order the planner enqueues it.
struct PlanFrame {
    int seq, frame;       // position in the caller's table
    int table;            // key-frame plane table (index into the context's tables)
    const float *pts;     // where the device reads the points (device memory, or host memory's device view)
    const float *src;     // the caller's pointer
    bool host;            // the points are page-locked host memory
    int64_t n;
    uint8_t *out;
    uint64_t cap;
    unsigned long long *nbytes;
    double pose[16];
};

struct PlanClass {
    lcc_ctx *ctx = nullptr;
    cudaStream_t side = nullptr;     // side stream when the plan has several classes
    cudaEvent_t done = nullptr;
    cudaEvent_t first_bin = nullptr; // the class's first chunk is binned (the next class starts after it)
    float4 *tables = nullptr;        // ngroups x NT key-frame planes
    int ngroups = 0;
    std::vector<PlanFrame> keys, pframes;
    // learned proposals of the key frames (8x8-tile classes with a net attached)
    bool seeded = false;
    uint16_t *x = nullptr;           // net inputs of one chunk: slots x NT x 64 pixels x 4 bf16
    float4 *anchor = nullptr;        // slots x NT tile anchors
    float *prop = nullptr;           // slots x NT x 5 proposals (written for the listed pairs only)
    uint8_t *need = nullptr;         // slots x NT: the tile has the 3 valid pixels a fit needs
    uint32_t *pairs = nullptr;       // pairs of tiles with a needed tile, and their count
    uint32_t *npairs = nullptr;
    DevStats *stats = nullptr;       // per frame of the last encode, in enqueue order (keys, then P frames)
    // staging of host points by the copy engines (lcc_plan_set_staging): two device buffers of a
    // chunk each (slots x stage_n points), filled on the class's copy stream
    bool staged = false;
    cudaStream_t cstream = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
    float4 *stage = nullptr;
    int64_t stage_n = 0;
};

}  // namespace

struct lcc_plan {
    cudaStream_t stream = nullptr;   // the stream every context was created on (replays run here)
    cudaStream_t cap = nullptr;      // private stream the graph is recorded on (the legacy default
                                     // stream cannot be captured)
    cudaEvent_t fork = nullptr;
    std::vector<PlanClass> cls;
    std::vector<lcc_seq_desc> shape;  // nframes / key_interval / ctx per sequence (structure check)
    int64_t frames = 0, key_frames = 0, points = 0;
    int64_t launches = 0;            // kernel launches of one encode
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    lcc_net *net = nullptr;          // proposal net of the seeded key frames (not owned)
    bool staging = false;            // host points copied by the copy engines ahead of each chunk
    float skip_logit = 0.f;
    // host-output path (lcc_plan_encode_host): one copy item per frame, in table order
    struct CopyItem *d_items = nullptr;
    unsigned long long *d_sizes = nullptr, *h_sizes = nullptr;   // h_sizes page-locked
    int64_t items = 0;
};

// One frame of the host-output copy: its device stream and size, and the host buffer.
struct CopyItem {
    const uint8_t *src;
    uint8_t *dst;
    unsigned long long cap;
    const unsigned long long *nbytes;
};

namespace {

// Every frame's stream (its size read on the device) from its device buffer into the caller's
// page-locked host buffer, 16-byte stores over the host link; frame f = blockIdx.y + 65535 *
// blockIdx.z.  The sizes are gathered into `sizes` (table order) for one copy back.
__global__ void __launch_bounds__(256) k_plan_copy_out(const CopyItem *items, long long nitems,
                                                     unsigned long long *sizes) {
    const long long f = blockIdx.y + 65535ll * blockIdx.z;
    if (f >= nitems) return;
    const CopyItem it = items[f];
    const unsigned long long raw = *it.nbytes;
    const unsigned long long nb = raw <= it.cap ? raw : 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) sizes[f] = raw;
    const uint4 *src = reinterpret_cast<const uint4 *>(it.src);
    uint4 *dst = reinterpret_cast<uint4 *>(it.dst);
    const unsigned long long n16 = nb / 16;
    for (unsigned long long i = blockIdx.x * 256ull + threadIdx.x; i < n16; i += gridDim.x * 256ull) dst[i] = src[i];
    const unsigned long long tail = nb - n16 * 16;   // streams are whole 32-bit words
    if (blockIdx.x == 0 && threadIdx.x < tail / 4)
        reinterpret_cast<uint32_t *>(it.dst + n16 * 16)[threadIdx.x] =
            reinterpret_cast<const uint32_t *>(it.src + n16 * 16)[threadIdx.x];
}

// Group g of a sequence covers frames [g*I, min((g+1)*I, nframes)); its key frame is the
// group's middle frame start + floor(len/2) (Sec. III-C: K is the middle frame of the group).
int key_of(int frame, int nframes, int interval, int *group) {
    const int g = frame / interval, start = g * interval;
    const int len = std::min(interval, nframes - start);
    *group = g;
    return start + len / 2;
}

// Address the device reads a frame's points at: device (or managed) memory as given, page-locked
// host memory through its device view (read in place over the host link); NULL for host memory
// the device cannot address.
const float *points_view(const float *p, bool *host) {
    *host = false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    *host = a.type == cudaMemoryTypeHost;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<const float *>(a.devicePointer);
    return nullptr;
}

// Output buffers are written with device atomics: device memory only.
bool device_memory(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice;
}

// Builds the frame lists of every class from the sequence table; the plan is left untouched
// unless the whole table is valid (and, for check_only, has the plan's group structure).
lcc_status fill(lcc_plan *p, int32_t nseq, const lcc_seq_desc *seqs, bool check_only) {
    const size_t ncls = p->cls.size();
    std::vector<std::vector<PlanFrame>> keys_of(ncls), pfr_of(ncls);
    std::vector<int> group_base(ncls, 0);
    int64_t frames = 0, keys = 0, points = 0;
    for (int s = 0; s < nseq; s++) {
        const lcc_seq_desc &d = seqs[s];
        if (d.ctx < 0 || d.ctx >= (int)p->cls.size() || d.nframes < 1 || d.key_interval < 1 || !d.poses ||
            !d.d_pts || !d.n || !d.d_out || !d.cap || !d.d_nbytes)
            return LCC_ERR_INVALID_ARG;
        for (int f = 0; f < d.nframes; f++) {
            if (d.n[f] < 0 || d.n[f] > (int64_t)1 << 31) return LCC_ERR_INVALID_ARG;
            bool host = false;
            const float *pts = d.n[f] > 0 && d.d_pts[f] ? points_view(d.d_pts[f], &host) : nullptr;
            if (d.n[f] > 0 && (!pts || !aligned16(pts))) return LCC_ERR_INVALID_ARG;
            if (!d.d_out[f] || !aligned16(d.d_out[f]) || d.cap[f] < (uint64_t)kHeaderBytes ||
                !device_memory(d.d_out[f]))
                return LCC_ERR_INVALID_ARG;
            int grp = 0;
            const int k = key_of(f, d.nframes, d.key_interval, &grp);
            PlanFrame pf;
            pf.seq = s;
            pf.frame = f;
            pf.table = group_base[d.ctx] + grp;
            pf.pts = pts;
            pf.src = d.d_pts[f];
            pf.host = host;
            pf.n = d.n[f];
            pf.out = d.d_out[f];
            pf.cap = d.cap[f];
            pf.nbytes = reinterpret_cast<unsigned long long *>(d.d_nbytes + f);
            memcpy(pf.pose, d.poses + 16 * (size_t)f, sizeof(pf.pose));
            (k == f ? keys_of[d.ctx] : pfr_of[d.ctx]).push_back(pf);
            keys += k == f;
            points += d.n[f];
            frames++;
        }
        group_base[d.ctx] += (d.nframes + d.key_interval - 1) / d.key_interval;
    }
    if (check_only)
        for (size_t k = 0; k < ncls; k++)
            if (group_base[k] != p->cls[k].ngroups) return LCC_ERR_INVALID_ARG;
    for (size_t k = 0; k < ncls; k++) {
        p->cls[k].ngroups = group_base[k];
        p->cls[k].keys.swap(keys_of[k]);
        p->cls[k].pframes.swap(pfr_of[k]);
    }
    p->frames = frames;
    p->key_frames = keys;
    p->points = points;
    return LCC_OK;
}

// Enqueue one class: its key frames chunk by chunk, then its P frames, each chunk binned into
// slots 0..m-1 of the class context and encoded as one batch.  Seeded key-frame chunks run the
// net's input kernel on the binned slots and its inference between the binning and the fit.
lcc_status enqueue_class(PlanClass &pc, lcc_net *net, float skip_logit, int64_t *launches) {
    lcc_ctx *c = pc.ctx;
    const int NT = c->g.NT;
    int chunk = 0;                      // chunks of the class so far: staging buffer chunk % 2
    bool used[2] = {false, false};      // staging buffer b was filled for an earlier chunk of this encode
    for (int kind = 0; kind < 2; kind++) {
        const std::vector<PlanFrame> &list = kind == 0 ? pc.keys : pc.pframes;
        const bool seeded = kind == 0 && pc.seeded && net;
        for (size_t base = 0; base < list.size(); base += (size_t)c->slots) {
            const int m = (int)std::min<size_t>((size_t)c->slots, list.size() - base);
            int slots[kMaxBatch];
            const float *pts[kMaxBatch];
            int64_t n[kMaxBatch];
            uint8_t *out[kMaxBatch];
            uint64_t cap[kMaxBatch];
            const float4 *kf[kMaxBatch];
            float4 *kfo[kMaxBatch];
            unsigned long long *nb[kMaxBatch];
            const float *props[kMaxBatch];
            std::vector<double> poses((size_t)m * 16);
            for (int f = 0; f < m; f++) {
                const PlanFrame &pf = list[base + f];
                slots[f] = f;
                pts[f] = pf.pts;
                n[f] = pf.n;
                out[f] = pf.out;
                cap[f] = pf.cap;
                float4 *tab = pc.tables + (size_t)pf.table * NT;
                kf[f] = tab;
                kfo[f] = tab;
                nb[f] = pf.nbytes;
                props[f] = seeded ? pc.prop + (size_t)f * NT * 5 : nullptr;
                memcpy(poses.data() + 16 * (size_t)f, pf.pose, sizeof(pf.pose));
            }
            // staged class: the chunk's host points are copied (one copy per frame, copy stream) into
            // buffer b once the chunk two before it, which used b, is binned; the binning waits for them
            const int b = chunk++ & 1;
            bool staged = false;
            for (int f = 0; f < m; f++) staged = staged || (pc.staged && list[base + f].host && n[f] > 0);
            if (staged) {
                if (used[b]) LCC_CUDA(cudaStreamWaitEvent(pc.cstream, pc.consumed[b], 0));
                for (int f = 0; f < m; f++) {
                    const PlanFrame &pf = list[base + f];
                    if (!pf.host || pf.n <= 0) continue;
                    float4 *dst = pc.stage + ((size_t)b * c->slots + f) * (size_t)pc.stage_n;
                    LCC_CUDA(cudaMemcpyAsync(dst, pf.src, sizeof(float4) * (size_t)pf.n, cudaMemcpyHostToDevice,
                                             pc.cstream));
                    pts[f] = reinterpret_cast<const float *>(dst);
                }
                LCC_CUDA(cudaEventRecord(pc.copied[b], pc.cstream));
                LCC_CUDA(cudaStreamWaitEvent(c->stream, pc.copied[b], 0));
            }
            lcc_status st = bin_frames(c, m, slots, pts, n);
            if (st != LCC_OK) return st;
            if (staged) LCC_CUDA(cudaEventRecord(pc.consumed[b], c->stream));
            used[b] = staged;
            if (kind == 0 && base == 0 && pc.first_bin) LCC_CUDA(cudaEventRecord(pc.first_bin, c->stream));
            if (seeded) {
                // the net runs only on pairs of tiles with a tile that can be fitted: the seeded fit
                // reads no other tile's proposal (empty sky and sparse tiles are often half a frame)
                int pi = prof_begin(c, 14);
                st = net_inputs_slots(c, m, pc.x, pc.anchor, pc.need);
                if (st == LCC_OK) st = net_pairs(pc.need, (int64_t)m * NT, pc.pairs, pc.npairs, c->stream);
                prof_end(c, pi);
                if (st != LCC_OK) return st;
                pi = prof_begin(c, 15);
                st = net_forward_on(net, pc.x, (int64_t)m * NT, pc.prop, c->stream, pc.pairs, pc.npairs);
                prof_end(c, pi);
                if (st != LCC_OK) return st;
                *launches += 3;
            }
            st = encode_batch(c, kind, m, slots, out, cap, kind ? poses.data() : nullptr, kind ? kf : nullptr,
                              kind ? nullptr : kfo, nb, seeded ? props : nullptr, skip_logit);
            if (st != LCC_OK) return st;
            // the chunk's counters (reset by the next chunk's binning) into the plan's per-frame record
            LCC_CUDA(cudaMemcpyAsync(pc.stats + (kind ? pc.keys.size() : 0) + base, c->s.stats, sizeof(DevStats) * m,
                                     cudaMemcpyDeviceToDevice, c->stream));
            c->last_nframes = m;
            *launches += 1 + 3 + (c->g.lookahead > 0 ? 1 : 0) + (kind == 1 && c->g.schedule >= 4 ? 1 : 0) +
                         (kind == 1 && c->g.schedule >= 4 && c->g.truns && c->g.lookahead > 0 ? 1 : 0) +
                         (c->g.schedule >= 3 ? 1
                          : c->g.schedule >= 1 ? c->g.R + 1 - (kind == 1 ? 0 : c->g.first_rounds) : 0);
        }
    }
    return LCC_OK;
}

// Every launch of the plan, ordered after earlier work on `main`.  With several classes each
// class runs on its own side stream between a fork and a join event, so classes overlap on the
// GPU.  When a class's points are in host memory, the next class starts once it has binned its
// first chunk, so that the classes' binning (over the host link, or their staged copies) falls
// beside the other classes' fits and packs rather than beside their binning.  The contexts'
// launches go to the chosen stream for the duration of the call.
lcc_status enqueue(lcc_plan *p, cudaStream_t main) {
    int64_t launches = 0;
    const bool forked = p->cls.size() > 1;
    bool any_staged = false;
    for (const auto &pc : p->cls) any_staged = any_staged || pc.staged;
    if (forked || any_staged) LCC_CUDA(cudaEventRecord(p->fork, main));
    lcc_status st = LCC_OK;
    const PlanClass *prev = nullptr;
    for (auto &pc : p->cls) {
        if (forked && cudaStreamWaitEvent(pc.side, p->fork, 0) != cudaSuccess) return LCC_ERR_CUDA;
        if (pc.staged && cudaStreamWaitEvent(pc.cstream, p->fork, 0) != cudaSuccess) return LCC_ERR_CUDA;
        if (forked && prev && !prev->keys.empty() && prev->keys.front().host &&
            cudaStreamWaitEvent(pc.side, prev->first_bin, 0) != cudaSuccess)
            return LCC_ERR_CUDA;
        prev = &pc;
        pc.ctx->stream = forked ? pc.side : main;
        st = enqueue_class(pc, p->net, p->skip_logit, &launches);
        pc.ctx->stream = p->stream;
        if (forked && (cudaEventRecord(pc.done, pc.side) != cudaSuccess ||
                       cudaStreamWaitEvent(main, pc.done, 0) != cudaSuccess))
            return LCC_ERR_CUDA;
        if (st != LCC_OK) return st;
    }
    p->launches = launches;
    return LCC_OK;
}

void release(lcc_plan *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto &pc : p->cls) {
        if (pc.side) cudaStreamDestroy(pc.side);
        if (pc.done) cudaEventDestroy(pc.done);
        if (pc.first_bin) cudaEventDestroy(pc.first_bin);
        if (pc.cstream) cudaStreamDestroy(pc.cstream);
        for (int b = 0; b < 2; b++) {
            if (pc.copied[b]) cudaEventDestroy(pc.copied[b]);
            if (pc.consumed[b]) cudaEventDestroy(pc.consumed[b]);
        }
        cudaFree(pc.stage);
        cudaFree(pc.tables);
        cudaFree(pc.x);
        cudaFree(pc.anchor);
        cudaFree(pc.prop);
        cudaFree(pc.need);
        cudaFree(pc.pairs);
        cudaFree(pc.npairs);
        cudaFree(pc.stats);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->cap) cudaStreamDestroy(p->cap);
    cudaFree(p->d_items);
    cudaFree(p->d_sizes);
    if (p->h_sizes) cudaFreeHost(p->h_sizes);
    delete p;
}

// Staging buffers and copy streams of the classes with host points (when staging is on): two
// chunks of the context's slots at the class's largest host frame; grown when an update needs it.
lcc_status ensure_staging(lcc_plan *p) {
    for (auto &pc : p->cls) {
        int64_t need = 0;
        for (const auto *list : {&pc.keys, &pc.pframes})
            for (const auto &pf : *list)
                if (pf.host) need = std::max(need, pf.n);
        // the class reads its host points in place unless everything below is in place
        pc.staged = false;
        if (!p->staging || need == 0) continue;
        if (!pc.cstream) {
            if (cudaStreamCreateWithFlags(&pc.cstream, cudaStreamNonBlocking) != cudaSuccess) return LCC_ERR_CUDA;
            for (int b = 0; b < 2; b++)
                if (cudaEventCreateWithFlags(&pc.copied[b], cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&pc.consumed[b], cudaEventDisableTiming) != cudaSuccess)
                    return LCC_ERR_CUDA;
        }
        if (need > pc.stage_n) {
            LCC_CUDA(cudaStreamSynchronize(p->stream));   // a replay may still read the old buffers
            cudaFree(pc.stage);
            pc.stage = nullptr;
            pc.stage_n = 0;
            LCC_CUDA(cudaMalloc(&pc.stage, sizeof(float4) * 2 * (size_t)pc.ctx->slots * (size_t)need));
            pc.stage_n = need;
        }
        pc.staged = true;
    }
    return LCC_OK;
}

}  // namespace

extern "C" {

lcc_status lcc_plan_create(lcc_plan **out, int32_t nctx, lcc_ctx *const *ctxs, int32_t nseq,
                           const lcc_seq_desc *seqs) {
    if (!out || !ctxs || !seqs || nctx < 1 || nctx > kMaxPlanContexts || nseq < 1) return LCC_ERR_INVALID_ARG;
    *out = nullptr;
    for (int k = 0; k < nctx; k++) {
        if (!ctxs[k] || ctxs[k]->stream != ctxs[0]->stream) return LCC_ERR_INVALID_ARG;
        for (int j = 0; j < k; j++)
            if (ctxs[j] == ctxs[k]) return LCC_ERR_INVALID_ARG;
    }
    lcc_plan *p = new (std::nothrow) lcc_plan();
    if (!p) return LCC_ERR_CUDA;
    p->stream = ctxs[0]->stream;
    p->cls.resize(nctx);
    for (int k = 0; k < nctx; k++) p->cls[k].ctx = ctxs[k];
    lcc_status st = fill(p, nseq, seqs, false);
    if (st != LCC_OK) {
        release(p);
        return st;
    }
    p->shape.assign(seqs, seqs + nseq);
    bool ok = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &pc : p->cls) {
        ok = ok && cudaMalloc(&pc.tables, sizeof(float4) * (size_t)std::max(pc.ngroups, 1) * pc.ctx->g.NT) ==
                       cudaSuccess;
        ok = ok && cudaMemset(pc.tables, 0, sizeof(float4) * (size_t)std::max(pc.ngroups, 1) * pc.ctx->g.NT) ==
                       cudaSuccess;
        const size_t nfr = std::max<size_t>(pc.keys.size() + pc.pframes.size(), 1);
        ok = ok && cudaMalloc(&pc.stats, sizeof(DevStats) * nfr) == cudaSuccess &&
             cudaMemset(pc.stats, 0, sizeof(DevStats) * nfr) == cudaSuccess;
        if (nctx > 1) {
            ok = ok && cudaStreamCreateWithFlags(&pc.side, cudaStreamNonBlocking) == cudaSuccess;
            ok = ok && cudaEventCreateWithFlags(&pc.done, cudaEventDisableTiming) == cudaSuccess;
            ok = ok && cudaEventCreateWithFlags(&pc.first_bin, cudaEventDisableTiming) == cudaSuccess;
        }
    }
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
        release(p);
        return LCC_ERR_CUDA;
    }
    *out = p;
    return LCC_OK;
}

lcc_status lcc_plan_update(lcc_plan *p, int32_t nseq, const lcc_seq_desc *seqs) {
    if (!p || !seqs || nseq != (int32_t)p->shape.size()) return LCC_ERR_INVALID_ARG;
    for (int s = 0; s < nseq; s++)
        if (seqs[s].ctx != p->shape[s].ctx || seqs[s].nframes != p->shape[s].nframes ||
            seqs[s].key_interval != p->shape[s].key_interval)
            return LCC_ERR_INVALID_ARG;
    lcc_status st = fill(p, nseq, seqs, true);
    if (st != LCC_OK) return st;
    if ((st = ensure_staging(p)) != LCC_OK) return st;
    if (!p->exec) return LCC_OK;
    // re-record with the new pointers, counts and poses and update the executable graph in place
    return lcc_plan_capture(p);
}

lcc_status lcc_plan_set_proposals(lcc_plan *p, lcc_net *net, float skip_logit) {
    if (!p || (net && !(skip_logit == skip_logit))) return LCC_ERR_INVALID_ARG;
    if (net) {
        bool any = false;
        for (const auto &pc : p->cls) any = any || (pc.ctx->g.th == 8 && pc.ctx->g.tw == 8);
        if (!any) return LCC_ERR_UNSUPPORTED;
        for (auto &pc : p->cls) {
            if (pc.ctx->g.th != 8 || pc.ctx->g.tw != 8) continue;
            if (!pc.x) {
                const size_t tiles = (size_t)pc.ctx->slots * pc.ctx->g.NT;
                if (cudaMalloc(&pc.x, tiles * 64 * 4 * sizeof(uint16_t)) != cudaSuccess ||
                    cudaMalloc(&pc.anchor, tiles * sizeof(float4)) != cudaSuccess ||
                    cudaMalloc(&pc.prop, tiles * 5 * sizeof(float)) != cudaSuccess ||
                    cudaMalloc(&pc.need, tiles) != cudaSuccess ||
                    cudaMalloc(&pc.pairs, (tiles + 1) / 2 * sizeof(uint32_t)) != cudaSuccess ||
                    cudaMalloc(&pc.npairs, sizeof(uint32_t)) != cudaSuccess) {
                    cudaFree(pc.x);
                    cudaFree(pc.anchor);
                    cudaFree(pc.prop);
                    cudaFree(pc.need);
                    cudaFree(pc.pairs);
                    cudaFree(pc.npairs);
                    pc.x = nullptr;
                    pc.anchor = nullptr;
                    pc.prop = nullptr;
                    pc.need = nullptr;
                    pc.pairs = nullptr;
                    pc.npairs = nullptr;
                    return LCC_ERR_CUDA;
                }
            }
        }
    }
    for (auto &pc : p->cls) pc.seeded = net && pc.ctx->g.th == 8 && pc.ctx->g.tw == 8;
    p->net = net;
    p->skip_logit = skip_logit;
    if (!p->exec) return LCC_OK;
    // the captured graph no longer matches: re-record it and update the executable in place
    return lcc_plan_capture(p);
}

lcc_status lcc_plan_set_staging(lcc_plan *p, int32_t enable) {
    if (!p || enable < 0 || enable > 1) return LCC_ERR_INVALID_ARG;
    p->staging = enable != 0;
    const lcc_status st = ensure_staging(p);
    if (st != LCC_OK) return st;
    if (!p->exec) return LCC_OK;
    return lcc_plan_capture(p);
}

lcc_status lcc_plan_encode(lcc_plan *p) {
    if (!p) return LCC_ERR_INVALID_ARG;
    return enqueue(p, p->stream);
}

lcc_status lcc_plan_capture(lcc_plan *p) {
    if (!p) return LCC_ERR_INVALID_ARG;
    for (auto &pc : p->cls)
        if (pc.ctx->prof) return LCC_ERR_INVALID_ARG;  // profiling events cannot be collected from a graph
    LCC_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    const lcc_status st = enqueue(p, p->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->cap, &g);
    if (st != LCC_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != LCC_OK ? st : LCC_ERR_CUDA;
    }
    if (p->exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(p->exec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(p->exec);
            p->exec = nullptr;
        }
    }
    if (!p->exec && cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return LCC_ERR_CUDA;
    }
    if (p->graph) cudaGraphDestroy(p->graph);
    p->graph = g;
    return LCC_OK;
}

lcc_status lcc_plan_replay(lcc_plan *p) {
    if (!p || !p->exec) return LCC_ERR_INVALID_ARG;
    LCC_CUDA(cudaGraphLaunch(p->exec, p->stream));
    return LCC_OK;
}

lcc_status lcc_plan_sync(lcc_plan *p) {
    if (!p) return LCC_ERR_INVALID_ARG;
    LCC_CUDA(cudaStreamSynchronize(p->stream));
    lcc_status first = LCC_OK;
    for (auto &pc : p->cls) {
        const lcc_status st = latched(pc.ctx);
        if (first == LCC_OK) first = st;
    }
    if (p->net) {
        const lcc_status st = net_latched(p->net);
        if (first == LCC_OK) first = st;
    }
    return first;
}

lcc_status lcc_plan_encode_host(lcc_plan *p, uint8_t *const *h_out, uint64_t *h_nbytes) {
    if (!p || !h_out || !h_nbytes) return LCC_ERR_INVALID_ARG;
    // copy items in table order (sequence by sequence, frame by frame)
    std::vector<CopyItem> items;
    items.reserve((size_t)p->frames);
    std::vector<const PlanFrame *> order((size_t)p->frames, nullptr);
    {
        std::vector<int64_t> base(p->shape.size() + 1, 0);
        for (size_t s = 0; s < p->shape.size(); s++) base[s + 1] = base[s] + p->shape[s].nframes;
        for (const auto &pc : p->cls)
            for (const auto *list : {&pc.keys, &pc.pframes})
                for (const auto &pf : *list) order[(size_t)(base[pf.seq] + pf.frame)] = &pf;
    }
    for (int64_t f = 0; f < p->frames; f++) {
        const PlanFrame *pf = order[(size_t)f];
        if (!pf || !h_out[f]) return LCC_ERR_INVALID_ARG;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, h_out[f]) != cudaSuccess) {
            cudaGetLastError();
            return LCC_ERR_INVALID_ARG;
        }
        if (a.type != cudaMemoryTypeHost || !a.devicePointer || !aligned16(a.devicePointer))
            return LCC_ERR_INVALID_ARG;   // page-locked, device-mapped, 16-byte aligned host memory only
        items.push_back(CopyItem{pf->out, (uint8_t *)a.devicePointer, pf->cap, pf->nbytes});
    }
    if (p->items != p->frames) {
        cudaFree(p->d_items);
        cudaFree(p->d_sizes);
        if (p->h_sizes) cudaFreeHost(p->h_sizes);
        p->d_items = nullptr;
        p->d_sizes = p->h_sizes = nullptr;
        p->items = 0;
        LCC_CUDA(cudaMalloc(&p->d_items, sizeof(CopyItem) * (size_t)p->frames));
        LCC_CUDA(cudaMalloc(&p->d_sizes, sizeof(unsigned long long) * (size_t)p->frames));
        LCC_CUDA(cudaMallocHost(&p->h_sizes, sizeof(unsigned long long) * (size_t)p->frames));
        p->items = p->frames;
    }
    // the table is small (32 B per frame); it rides on the stream ahead of the encode
    LCC_CUDA(cudaMemcpyAsync(p->d_items, items.data(), sizeof(CopyItem) * items.size(), cudaMemcpyHostToDevice,
                             p->stream));
    lcc_status st = p->exec ? lcc_plan_replay(p) : lcc_plan_encode(p);
    if (st != LCC_OK) return st;
    const long long nf = (long long)p->frames;
    k_plan_copy_out<<<dim3(8, (unsigned)std::min<long long>(nf, 65535), (unsigned)((nf + 65534) / 65535)), 256, 0,
                      p->stream>>>(p->d_items, nf, p->d_sizes);
    LCC_CUDA(cudaGetLastError());
    LCC_CUDA(cudaMemcpyAsync(p->h_sizes, p->d_sizes, sizeof(unsigned long long) * (size_t)nf,
                             cudaMemcpyDeviceToHost, p->stream));
    st = lcc_plan_sync(p);
    memcpy(h_nbytes, p->h_sizes, sizeof(uint64_t) * (size_t)nf);
    return st;
}

lcc_status lcc_plan_stats(lcc_plan *p, int32_t seq, int32_t frame, lcc_stats *out) {
    if (!p || !out || seq >= (int32_t)p->shape.size() || (seq >= 0 && (frame < 0 || frame >= p->shape[seq].nframes)))
        return LCC_ERR_INVALID_ARG;
    LCC_CUDA(cudaStreamSynchronize(p->stream));
    DevStats sum;
    memset(&sum, 0, sizeof(sum));
    bool found = false;
    for (const auto &pc : p->cls) {
        const size_t nk = pc.keys.size(), n = nk + pc.pframes.size();
        if (!n) continue;
        std::vector<DevStats> h(n);
        LCC_CUDA(cudaMemcpy(h.data(), pc.stats, sizeof(DevStats) * n, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; i++) {
            const PlanFrame &pf = i < nk ? pc.keys[i] : pc.pframes[i - nk];
            if (seq >= 0 && (pf.seq != seq || pf.frame != frame)) continue;
            const unsigned long long *a = reinterpret_cast<const unsigned long long *>(&h[i]);
            unsigned long long *b = reinterpret_cast<unsigned long long *>(&sum);
            for (size_t w = 0; w < sizeof(DevStats) / sizeof(unsigned long long); w++) b[w] += a[w];
            found = true;
        }
    }
    if (!found && seq >= 0) return LCC_ERR_INVALID_ARG;
    public_stats(sum, out);
    return LCC_OK;
}

lcc_status lcc_plan_get_info(const lcc_plan *p, lcc_plan_info *out) {
    if (!p || !out) return LCC_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->frames = p->frames;
    out->key_frames = p->key_frames;
    out->points = p->points;
    out->launches = p->launches;
    out->classes = (int32_t)p->cls.size();
    out->captured = p->exec ? 1 : 0;
    for (const auto &pc : p->cls)
        if (pc.seeded && p->net) out->seeded_key_frames += (int64_t)pc.keys.size();
    size_t nodes = 0;
    if (p->graph && cudaGraphGetNodes(p->graph, nullptr, &nodes) != cudaSuccess) nodes = 0;
    out->graph_nodes = (int64_t)nodes;
    return LCC_OK;
}

void lcc_plan_destroy(lcc_plan *p) {
    if (!p) return;
    cudaStreamSynchronize(p->stream);
    release(p);
}

}  // extern "C"
