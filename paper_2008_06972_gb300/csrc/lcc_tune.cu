// Autotuner (lcc_autotune): encodes a sample key-frame group with every
// candidate schedule (tile shape x run-test horizon x fit schedule) the way a
// plan encodes its chunks (the key frame, then the P frames in one batched
// call against its planes), times it with CUDA events, decodes it to check the
// error bound, and picks the fastest candidate whose stream is within a slack
// of the smallest one.
#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "lcc.h"
#include "lcc_ctx.cuh"

using namespace lcc;

namespace {

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { cudaFree(p); }
    bool alloc(size_t n) { return cudaMalloc(&p, n) == cudaSuccess; }
};

// One candidate, measured on its own context; r is filled on success.
lcc_status measure(const lcc_sensor *sensor, const lcc_params &prm, int nframes, int key_index, const double *poses,
                   const float *const *d_pts, const int64_t *n, int reps, cudaStream_t stream,
                   lcc_tune_result *r) {
    lcc_ctx *c = nullptr;
    lcc_status st = lcc_create(&c, sensor, &prm, stream);
    if (st != LCC_OK) return st;
    struct Guard {
        lcc_ctx *c;
        lcc_keyframe *k = nullptr, *kd = nullptr;
        ~Guard() {
            lcc_keyframe_free(k);
            lcc_keyframe_free(kd);
            lcc_destroy(c);
        }
    } guard{c};
    const uint64_t cap = lcc_max_encoded_bytes(c);
    const size_t npx = (size_t)sensor->rows * sensor->cols;
    DevBuf out, nbytes, rref, rdec, err;
    if (!out.alloc(cap * nframes) || !nbytes.alloc(8 * (size_t)nframes) || !rref.alloc(4 * npx) ||
        !rdec.alloc(4 * npx) || !err.alloc(4))
        return LCC_ERR_CUDA;
    if ((st = lcc_keyframe_create(c, &guard.k)) != LCC_OK || (st = lcc_keyframe_create(c, &guard.kd)) != LCC_OK)
        return st;
    std::vector<uint8_t *> outs(nframes);
    std::vector<uint64_t> caps(nframes, cap);
    for (int f = 0; f < nframes; f++) outs[f] = (uint8_t *)out.p + cap * f;
    // the P frames in one batch, in frame order
    std::vector<const float *> pp;
    std::vector<int64_t> pn;
    std::vector<uint8_t *> po;
    std::vector<uint64_t> pc;
    std::vector<double> pposes;
    for (int f = 0; f < nframes; f++) {
        if (f == key_index) continue;
        pp.push_back(d_pts[f]);
        pn.push_back(n[f]);
        po.push_back(outs[f]);
        pc.push_back(cap);
        pposes.insert(pposes.end(), poses + 16 * (size_t)f, poses + 16 * (size_t)f + 16);
    }
    uint64_t *nb_dev = (uint64_t *)nbytes.p;   // key frame's size first, then the P frames'
    auto encode = [&]() {
        lcc_status e = lcc_encode_keyframe(c, d_pts[key_index], n[key_index], guard.k, outs[key_index], cap, nb_dev);
        if (e != LCC_OK || pp.empty()) return e;
        return lcc_encode_pframes(c, guard.k, (int32_t)pp.size(), pposes.data(), pp.data(), pn.data(), po.data(),
                                  pc.data(), nb_dev + 1);
    };
    if ((st = encode()) != LCC_OK || (st = lcc_sync(c)) != LCC_OK) return st;
    cudaEvent_t a, b;
    LCC_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return LCC_ERR_CUDA;
    }
    cudaEventRecord(a, stream);
    for (int k = 0; k < reps && st == LCC_OK; k++) st = encode();
    cudaEventRecord(b, stream);
    float ms = 0.f;
    const bool timed = cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != LCC_OK) return st;
    if (!timed) return LCC_ERR_CUDA;
    if ((st = lcc_sync(c)) != LCC_OK) return st;
    std::vector<uint64_t> nbk(nframes), nb(nframes);
    LCC_CUDA(cudaMemcpy(nbk.data(), nbytes.p, 8 * (size_t)nframes, cudaMemcpyDeviceToHost));
    for (int f = 0, q = 1; f < nframes; f++) nb[f] = f == key_index ? nbk[0] : nbk[q++];
    uint64_t total = 0;
    int64_t pts = 0;
    for (int f = 0; f < nframes; f++) {
        total += nb[f];
        pts += n[f];
    }
    // decode every frame and compare with the binned input
    LCC_CUDA(cudaMemsetAsync(err.p, 0, 4, stream));
    if ((st = lcc_keyframe_from_stream(c, outs[key_index], nb[key_index], guard.kd)) != LCC_OK) return st;
    for (int f = 0; f < nframes; f++) {
        if ((st = lcc_range_image(c, d_pts[f], n[f], (float *)rref.p, nullptr)) != LCC_OK) return st;
        const bool key = f == key_index;
        if ((st = lcc_decode(c, outs[f], nb[f], key ? nullptr : guard.kd, key ? nullptr : poses + 16 * (size_t)f,
                             (float *)rdec.p, nullptr, nullptr)) != LCC_OK)
            return st;
        LCC_CUDA(launch_maxdiff((const float *)rref.p, (const float *)rdec.p, (long long)npx, (uint32_t *)err.p,
                                stream));
    }
    if ((st = lcc_sync(c)) != LCC_OK) return st;
    float max_err = 0.f;
    LCC_CUDA(cudaMemcpy(&max_err, err.p, 4, cudaMemcpyDeviceToHost));
    r->ms = (double)ms / reps;
    r->mpts_per_s = (double)pts / (r->ms * 1e-3) / 1e6;
    r->bytes = total;
    r->max_err_m = max_err;
    return LCC_OK;
}

}  // namespace

extern "C" {

lcc_status lcc_autotune(const lcc_sensor *sensor, const lcc_params *base, int32_t nframes, int32_t key_index,
                        const double *poses, const float *const *d_pts, const int64_t *n, int32_t reps,
                        float max_err_m, float bytes_slack, uint32_t shapes, void *cuda_stream,
                        lcc_tune_result *results, int32_t cap, int32_t *nresults, lcc_params *best) {
    if (!sensor || !base || !poses || !d_pts || !n || !best || nframes < 1 || nframes > kMaxBatch ||
        key_index < 0 || key_index >= nframes || reps < 1 || !(max_err_m > 0) || !(bytes_slack >= 0) ||
        (cap > 0 && !results) || shapes > 15u)
        return LCC_ERR_INVALID_ARG;
    static const int kTiles[4][2] = {{4, 4}, {4, 8}, {8, 8}, {8, 16}};
    static const int kHorizon[3] = {8, 16, 32};
    if (!shapes) shapes = 15u;
    std::vector<lcc_tune_result> all;
    for (int ti = 0; ti < 4; ti++)
        for (int sched : {0, 3, 4, 5, 6})
            for (int h = 0; h < (base->merge_runs ? 3 : 1); h++) {
                if (!((shapes >> ti) & 1u)) continue;
                const int *t = kTiles[ti];
                lcc_params prm = *base;
                prm.tile_h = t[0];
                prm.tile_w = t[1];
                prm.fit_schedule = sched;
                prm.lookahead = base->merge_runs ? kHorizon[h] : 0;
                prm.max_batch = nframes;
                lcc_tune_result r;
                memset(&r, 0, sizeof(r));
                r.tile_h = prm.tile_h;
                r.tile_w = prm.tile_w;
                r.lookahead = prm.lookahead;
                r.fit_schedule = sched;
                r.status = measure(sensor, prm, nframes, key_index, poses, d_pts, n, reps,
                                   (cudaStream_t)cuda_stream, &r);
                if (r.status == LCC_ERR_CUDA || r.status == LCC_ERR_NO_DEVICE) return (lcc_status)r.status;
                all.push_back(r);
            }
    uint64_t min_bytes = UINT64_MAX;
    for (auto &r : all)
        if (r.status == LCC_OK && r.max_err_m <= max_err_m && r.bytes < min_bytes) min_bytes = r.bytes;
    int pick = -1;
    for (int i = 0; i < (int)all.size(); i++) {
        const auto &r = all[i];
        if (r.status != LCC_OK || r.max_err_m > max_err_m) continue;
        if ((double)r.bytes > (1.0 + bytes_slack) * (double)min_bytes) continue;
        if (pick < 0 || r.mpts_per_s > all[pick].mpts_per_s) pick = i;
    }
    if (nresults) *nresults = (int32_t)all.size();
    for (int i = 0; i < (int)all.size() && i < cap; i++) {
        results[i] = all[i];
        results[i].chosen = i == pick;
    }
    if (pick < 0) return LCC_ERR_UNSUPPORTED;
    *best = *base;
    best->tile_h = all[pick].tile_h;
    best->tile_w = all[pick].tile_w;
    best->lookahead = all[pick].lookahead;
    best->fit_schedule = all[pick].fit_schedule;
    return LCC_OK;
}

}  // extern "C"
