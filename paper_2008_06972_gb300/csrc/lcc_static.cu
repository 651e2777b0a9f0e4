// lcc_range_image_static: the range-image conversion of Sec. III-B (Eq. 1-2,
// nearest point per pixel) for callers that may not allocate: no context, no
// cudaMalloc/cudaFree, no allocating library call.  Its scratch (the range
// image being built, the boundary tables, the binning counters) is one
// fixed device array of this file.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

#include "lcc.h"
#include "lcc_internal.cuh"

using namespace lcc;

namespace {

constexpr int kStaticMaxRows = 512;
constexpr int kStaticMaxCols = 8192;
constexpr int64_t kStaticMaxPixels = 1 << 18;  // e.g. 128 x 2048
constexpr size_t kRimgBytes = (size_t)kStaticMaxPixels * 4;
constexpr size_t kTableFloats = 2 * (size_t)(kStaticMaxRows + 1) + 2 * (size_t)kStaticMaxCols;
constexpr size_t kTableOff = kRimgBytes;
constexpr size_t kStatsOff = kTableOff + ((kTableFloats * 4 + 255) & ~size_t(255));
constexpr size_t kStaticBytes = kStatsOff + 256;
static_assert(sizeof(DevStats) <= 256, "binning counters fit their slot");

// 1.2 MB: range image (1 MiB), row/column boundary tables, binning counters.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::atomic<unsigned char *> g_base[kMaxDevices];

// Address of the scratch array on the current device: resolved once per device by
// cudaGetSymbolAddress (with the device current), after checking that it is an sm_103 part.
lcc_status scratch_base(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LCC_ERR_NO_DEVICE;
    if (dev < 0 || dev >= kMaxDevices) return LCC_ERR_UNSUPPORTED;
    unsigned char *p = g_base[dev].load(std::memory_order_acquire);
    if (!p) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
            return LCC_ERR_NO_DEVICE;
        if (!(major == 10 && minor == 3)) return LCC_ERR_NO_DEVICE;
        void *sym = nullptr;
        if (cudaGetSymbolAddress(&sym, g_static_scratch) != cudaSuccess || !sym) return LCC_ERR_CUDA;
        p = static_cast<unsigned char *>(sym);
        g_base[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return LCC_OK;
}

// Boundary tables rbc, rbs (rows + 1 each), cbc, cbs (cols each), packed in that order, uploaded
// in chunks from a small stack buffer (pageable copies return once the chunk is staged).
lcc_status upload_tables(const lcc_sensor &s, float *dst, cudaStream_t st) {
    constexpr int kChunk = 2048;
    float buf[kChunk];
    const int H = s.rows, W = s.cols;
    const int64_t total = 2 * (int64_t)(H + 1) + 2 * (int64_t)W;
    for (int64_t base = 0; base < total; base += kChunk) {
        const int m = (int)std::min<int64_t>(kChunk, total - base);
        for (int q = 0; q < m; q++) {
            const int64_t e = base + q;
            float c, sn;
            if (e < 2 * (int64_t)(H + 1)) {
                row_boundary(s, (int)(e % (H + 1)), &c, &sn);
                buf[q] = e < H + 1 ? c : sn;
            } else {
                const int64_t e2 = e - 2 * (int64_t)(H + 1);
                col_boundary(s, (int)(e2 % W), &c, &sn);
                buf[q] = e2 < W ? c : sn;
            }
        }
        if (cudaMemcpyAsync(dst + base, buf, sizeof(float) * m, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return LCC_ERR_CUDA;
    }
    return LCC_OK;
}

}  // namespace

extern "C" lcc_status lcc_range_image_static(const lcc_sensor *sensor, const float *d_pts, int64_t n,
                                             float *d_range, uint32_t *d_valid, void *cuda_stream) {
    if (!sensor || n < 0 || n > ((int64_t)1 << 31) || (n > 0 && (!d_pts || ((uintptr_t)d_pts & 15u))))
        return LCC_ERR_INVALID_ARG;
    const lcc_sensor &s = *sensor;
    if (s.rows < 1 || s.cols < 2 || !(s.elev_max_deg > s.elev_min_deg) || s.elev_max_deg > 90.0 ||
        s.elev_min_deg < -90.0 || !(s.max_range_m > 0))
        return LCC_ERR_INVALID_ARG;
    if (s.rows > kStaticMaxRows || s.cols > kStaticMaxCols || (int64_t)s.rows * s.cols > kStaticMaxPixels)
        return LCC_ERR_UNSUPPORTED;
    unsigned char *base = nullptr;
    lcc_status st = scratch_base(&base);
    if (st != LCC_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int H = s.rows, W = s.cols;
    float *tab = reinterpret_cast<float *>(base + kTableOff);
    if ((st = upload_tables(s, tab, stream)) != LCC_OK) return st;

    Geometry g{};
    g.H = H;
    g.W = W;
    g.rmax = (float)s.max_range_m;
    g.elev_max_rad = (float)(s.elev_max_deg * (M_PI / 180.0));
    g.inv_d_el = (float)(s.rows / ((s.elev_max_deg - s.elev_min_deg) * (M_PI / 180.0)));
    g.inv_d_az = (float)(s.cols / (2.0 * M_PI));
    g.rbc = tab;
    g.rbs = tab + (H + 1);
    g.cbc = tab + 2 * (H + 1);
    g.cbs = g.cbc + W;
    Scratch sc{};
    sc.rimg = reinterpret_cast<uint32_t *>(base);
    sc.stats = reinterpret_cast<DevStats *>(base + kStatsOff);
    // the range image must start empty (all-ones bits) and the counters at zero
    if (cudaMemsetAsync(sc.rimg, 0xFF, (size_t)H * W * 4, stream) != cudaSuccess ||
        cudaMemsetAsync(sc.stats, 0, sizeof(DevStats), stream) != cudaSuccess)
        return LCC_ERR_CUDA;
    Batch b;
    memset(&b, 0, sizeof(b));
    b.nframes = 1;
    b.slot[0] = 0;
    b.pts[0] = reinterpret_cast<const float4 *>(d_pts);
    b.n[0] = n;
    const long long per_block = 256 * 4;
    const long long blocks = (n + per_block - 1) / per_block;
    b.blk_prefix[0] = 0;
    b.blk_prefix[1] = blocks;
    if (launch_bin(g, sc, b, blocks, stream) != cudaSuccess) return LCC_ERR_CUDA;
    if (launch_range_image(g, sc.rimg, d_range, d_valid, stream) != cudaSuccess) return LCC_ERR_CUDA;
    return LCC_OK;
}
