// lcc_range_image_static: the same range image as lcc_range_image, for callers
// that may not allocate: no context, no cudaMalloc/cudaFree, no allocating
// library call.  Its scratch (the range image being built, the boundary
// tables, the binning counters) is one fixed device array of this file.  The
// paper has no counterpart: this is an implementation entry point.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
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

// Per device: the context the scratch address was looked up in (its unique id, 0 = none), the
// address, and the sensor whose boundary tables the array holds (valid while `have_tables`).
struct DevState {
    unsigned long long ctx_id = 0;
    unsigned char *base = nullptr;
    bool have_tables = false;
    lcc_sensor tables_of{};
};
DevState g_dev[kMaxDevices];

using PfnCtxGetCurrent = CUresult (*)(CUcontext *);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 if there is none yet or the driver
// cannot tell): a cudaDeviceReset ends a device's context, and the next one gets a new id.
unsigned long long current_ctx_id() {
    static PfnCtxGetCurrent get_current = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PfnCtxGetCurrent>(fn);
    }();
    static PfnCtxGetId get_id = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PfnCtxGetId>(fn);
    }();
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Address of the scratch array on the current device.  Set-up (with the device current): check
// that it is an sm_103 part and look the address up with cudaGetSymbolAddress; done on the first
// call on a device and again whenever the device's context is not the one of the last set-up.
lcc_status scratch_base(DevState **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LCC_ERR_NO_DEVICE;
    if (dev < 0 || dev >= kMaxDevices) return LCC_ERR_UNSUPPORTED;
    DevState &d = g_dev[dev];
    const unsigned long long id = current_ctx_id();
    if (!d.base || id == 0 || id != d.ctx_id) {
        int major = 0, minor = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
            return LCC_ERR_NO_DEVICE;
        if (!(major == 10 && minor == 3)) return LCC_ERR_NO_DEVICE;
        void *sym = nullptr;
        if (cudaGetSymbolAddress(&sym, g_static_scratch) != cudaSuccess || !sym) return LCC_ERR_CUDA;
        d.base = static_cast<unsigned char *>(sym);
        d.ctx_id = current_ctx_id();   // the lookup above made the device's context current
        d.have_tables = false;         // a new context's array holds no tables yet
    }
    *out = &d;
    return LCC_OK;
}

bool same_sensor(const lcc_sensor &a, const lcc_sensor &b) {
    return a.rows == b.rows && a.cols == b.cols && a.elev_min_deg == b.elev_min_deg &&
           a.elev_max_deg == b.elev_max_deg && a.max_range_m == b.max_range_m;
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
    DevState *dev = nullptr;
    lcc_status st = scratch_base(&dev);
    if (st != LCC_OK) return st;
    unsigned char *base = dev->base;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    const int H = s.rows, W = s.cols;
    float *tab = reinterpret_cast<float *>(base + kTableOff);
    // the tables stay in the array between calls: upload them only for a sensor other than the
    // previous call's on this device (calls are serialised by the caller)
    if (!dev->have_tables || !same_sensor(dev->tables_of, s)) {
        dev->have_tables = false;
        if ((st = upload_tables(s, tab, stream)) != LCC_OK) return st;
        dev->tables_of = s;
        dev->have_tables = true;
    }

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
