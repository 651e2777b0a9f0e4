/*
 * lcc — GB300-native spatio-temporal LiDAR point-cloud compression.
 *
 * C ABI of the encoder/decoder described in "Real-Time Spatio-Temporal LiDAR
 * Point Cloud Compression" (Feng, Liu, Zhu): a key frame (K) is spatially
 * encoded by iterative plane fitting over range-image tiles (Sec. III-B,
 * III-C); predicted frames (P) are encoded against the key frame's planes
 * moved by the inter-frame pose, with the leftover tiles spatially encoded
 * (Sec. III-D).  All compute runs as CUDA kernels for sm_103a.
 *
 * Conventions
 *  - Pointers named d_* are device pointers; the caller owns them.  Host
 *    arrays are named h_* or are plain C arrays (poses, pointer tables).
 *  - Every call is asynchronous on the context's CUDA stream unless stated.
 *    Argument errors are returned at once.  Errors found on the device
 *    (output capacity, corrupt stream) are latched in the context and
 *    returned by lcc_sync().
 *  - One context per stream; a context is not thread-safe.
 *  - Points are float4 (x, y, z, unused), metres, sensor coordinates.
 *  - Poses are row-major 4x4 doubles M with p_K = R p + T (Eq. 6), mapping a
 *    P frame's coordinates into the key frame's.
 */
#ifndef LCC_H
#define LCC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LCC_OK = 0,
    LCC_ERR_INVALID_ARG = 1,  /* bad pointer, size or parameter */
    LCC_ERR_CAPACITY = 2,     /* an output buffer is too small; the needed size is reported */
    LCC_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    LCC_ERR_TIMEOUT = 4,      /* a bounded device wait gave up */
    LCC_ERR_CORRUPT = 5,      /* a stream failed validation while decoding */
    LCC_ERR_UNSUPPORTED = 6,  /* valid request this build does not handle */
    LCC_ERR_NO_DEVICE = 7     /* no usable sm_103 GPU */
} lcc_status;

/* Range-image geometry (Sec. III-B): rows = beams (row 0 = top), cols =
 * azimuth steps over 360 degrees starting at -180.  Row i spans elevations
 * (b_{i+1}, b_i], b_k = elev_max - k (elev_max - elev_min) / rows; column j
 * spans azimuths [-pi + j 2pi/cols, -pi + (j+1) 2pi/cols). */
typedef struct {
    int32_t rows, cols;
    double elev_min_deg, elev_max_deg;
    double max_range_m;
} lcc_sensor;

/* Encoder parameters. */
typedef struct {
    int32_t tile_h, tile_w;   /* unit tile (Sec. III-C); supported: 4x4, 4x8, 8x8, 8x16 */
    float fit_thr_m;          /* threshold on the along-ray residual |r - d/(n.u)| */
    float quant_m;            /* quantisation step q of residual and raw codes (decode error <= q/2) */
    int32_t max_refits;       /* refit rounds after the first plane fit (0..7) */
    float min_inlier_frac;    /* share of a tile's points a plane must keep (1.0 = all, the paper's rule) */
    int32_t merge_runs;       /* 1: grow runs of tiles horizontally with the run's plane (Sec. III-C) */
    int32_t max_batch;        /* frames per batched launch the context reserves scratch for (1..64) */
    int32_t lookahead;        /* run pre-test span: tiles to the left each tile is tested against (0..32) */
    int32_t solver;           /* 3x3 plane solve: 0 float-float on the FP32 pipes (default), 1 FP64 */
    int32_t fit_schedule;     /* 0: a thread runs all refit rounds of its tile; 1 or 2: a thread runs that
                                 many rounds, tiles needing another round are queued and re-run in
                                 dense warps, one kernel per round; 3: one round per thread, then the
                                 queued tiles' remaining rounds in one dense kernel; 4: as 3, and P
                                 frames encoded in batches (lcc_encode_pframes, plans) run their spatial
                                 fits first and the temporal test after them (one lane group per tile),
                                 the order lcc_encode_sequence always uses, which pays when few P tiles
                                 pass the temporal test; 5: as 4 with every round of every tile run by
                                 a group of lanes (a warp quarter for 8x8 tiles) splitting its pixels,
                                 the first pass only queueing the tiles; 6: as 4 with the queued tiles'
                                 remaining rounds run by one thread per tile (same results for every
                                 value) */
    int32_t no_delta;         /* 1: plane-coded points carry no residual code, the paper's default
                                 (Sec. III-C drops the deltas): they decode onto their plane, decode
                                 error <= fit_thr_m; 0 (default here): residual codes, error <= q/2 */
    int32_t raw_exact;        /* 1: raw (unfit) pixels carry their fp32 range bits instead of a
                                 q-quantised code, so they decode exactly (header flags bit 2, 32-bit
                                 raw codes); 0 (default): raw codes m = round(r / q) */
    int32_t temporal_candidates; /* K tiles a P tile's relaxed-plane test (Sec. III-D) may try, 1..4:
                                 the distinct K tiles its valid pixels fall in after Eq. 6, in raster
                                 order from the anchor's, the first that passes kept; 1 (default):
                                 the anchor's K tile only */
    int32_t temporal_runs;    /* 1 (default): P tiles that passed the relaxed-plane test grow runs to the
                                 right like spatial runs (Sec. III-D applies the same horizontal growing
                                 strategy): a following tile that passes the acceptance rule against
                                 the run start's relaxed plane (n', c') joins the run (tile code
                                 TEMPORAL_CONT = 5, no record of its own; header flags bit 3); spatial
                                 runs stop at temporal tiles.  Needs merge_runs.  0: each temporal
                                 tile carries its own record */
    int32_t plane3;           /* 1: planes in Eq. 3's three-coefficient form (Sec. III-C prints x + a y + b z
                                 = c, which misses planes with n_x = 0; here divided by the dominant
                                 component): every fitted plane becomes the unit-normal plane of its
                                 coefficients a = n_i/n_k, b = n_j/n_k, c = d/n_k (k the axis of the
                                 largest |n_k|, i, j the next axes), run records carry the 3
                                 coefficients (header flags bit 4) and a run start's tile code is
                                 6 + k.  0 (default): unit normal and offset, 4 words a run */
} lcc_params;

/* Per-frame statistics of the last encode (Fig. 11's categories and more). */
typedef struct {
    int64_t points_in;        /* points passed in */
    int64_t points_invalid;   /* non-finite, r <= 0 or r > max range */
    int64_t points_fov;       /* outside the vertical field of view */
    int64_t points_binned;    /* binned (before collisions) */
    int64_t pixels_valid;     /* occupied pixels; binned - valid = points lost to collisions */
    int64_t tiles_empty, tiles_raw, tiles_run_start, tiles_run_cont, tiles_temporal;
    int64_t fit_rounds[8];    /* tiles by number of plane fits (index = fits, 0..7) */
    int64_t tiles_borderline; /* tiles with a residual within 1e-6 m of the threshold in some round */
    int64_t cand, fitted, raw;/* candidate, plane-coded and raw-coded pixels */
    uint64_t bytes;           /* stream size */
    int64_t tiles_temporal_cont; /* tiles inside a temporal run (after its first tile) */
    int64_t tiles_net;        /* plans with a proposal net: key-frame tiles with the 3 valid pixels a
                                 fit needs, the tiles whose proposals the net computes */
} lcc_stats;

/* Per-tile record (debug and parity checks): the tile's own fit results. */
typedef struct {
    float plane[4];           /* own spatial plane n.p = d, or (n', c') for a temporal tile */
    float tplane[4];          /* temporal test plane (n', c') if a K tile was found */
    uint32_t kref;            /* K tile the anchor maps to, 0xFFFFFFFF if none */
    uint32_t ahead_mask;      /* run pre-test bits: bit j = this tile passes the plane of tile t-1-j
                                 (bit j and ahead_cnt[j] are meaningful where tile t-1-j has status 2;
                                 otherwise they are 0, or in lcc_encode_sequence's P frames may hold
                                 the test against that tile's spatial plane before it became temporal) */
    uint8_t status;           /* 0 empty, 1 fit failed, 2 fit ok, 3 temporal */
    uint8_t rounds;           /* spatial plane fits performed */
    uint8_t flags;            /* bit0 borderline, bit1 degenerate scatter, bit2 temporal tested,
                                 bit3 not fitted: its proposal logit was below the skip logit */
    uint8_t n_valid;          /* valid pixels */
    uint8_t n_inlier;         /* inliers of the final spatial (or temporal) plane */
    uint8_t t_rounds;         /* temporal offset fits */
    uint8_t t_inlier;         /* inliers of the temporal plane */
    uint8_t t_status;         /* 0 no K plane, 1 failed, 2 passed */
    uint8_t ahead_cnt[16];    /* inlier counts of the first 16 of those pre-tests */
} lcc_tile_info;

typedef struct lcc_ctx lcc_ctx;
typedef struct lcc_keyframe lcc_keyframe;

/* Human-readable name of a status. */
const char *lcc_status_string(lcc_status s);

/* Default parameters: 4x4 tiles, thr 0.05 m, q 0.02 m, 3 refits, f_min 0.75,
 * runs on (spatial and temporal), max_batch 16, lookahead 16, float-float
 * solver, fit schedule 3 (one round per thread, the few tiles needing more
 * finish in one dense launch). */
void lcc_default_params(lcc_params *p);

/* Create a context on the current device bound to cuda_stream (a
 * cudaStream_t, NULL = default stream).  Allocates device scratch for
 * max_batch frames.  Fails with LCC_ERR_NO_DEVICE without an sm_103 GPU. */
lcc_status lcc_create(lcc_ctx **out, const lcc_sensor *sensor, const lcc_params *params, void *cuda_stream);
lcc_status lcc_destroy(lcc_ctx *ctx);

/* Upper bound of one frame's stream size in bytes (for output buffers). */
uint64_t lcc_max_encoded_bytes(const lcc_ctx *ctx);

/* Number of tiles of one frame. */
int64_t lcc_num_tiles(const lcc_ctx *ctx);

/* Beam and boundary tables of the sensor (host copies, fp32): ce/se [rows]
 * (cos/sin of row-centre elevation), ct/st [cols] (column-centre azimuth),
 * rbc/rbs [rows+1] (row boundaries), cbc/cbs [cols] (column boundaries).
 * Beam of pixel (i,j) = (ce_i ct_j, ce_i st_j, se_i) in fp32.  Synchronous. */
lcc_status lcc_tables(const lcc_ctx *ctx, float *ce, float *se, float *ct, float *st,
                      float *rbc, float *rbs, float *cbc, float *cbs);

/* Eq. 1-2: range image of one frame.  d_range [rows*cols] fp32 (0 = empty,
 * nearest point wins on collision, Sec. III-D); d_valid [ceil(rows*cols/32)]
 * occupancy bitmap, raster order, LSB first.  Either output may be NULL. */
lcc_status lcc_range_image(lcc_ctx *ctx, const float *d_pts, int64_t n, float *d_range, uint32_t *d_valid);

/* Key-frame handles hold a frame's per-tile coding planes on the device. */
lcc_status lcc_keyframe_create(lcc_ctx *ctx, lcc_keyframe **out);
void lcc_keyframe_free(lcc_keyframe *kf);

/* Spatial encode of a key frame (Sec. III-B, III-C).  d_out receives up to
 * cap bytes; *out_bytes (host or device uint64, caller-owned) receives the
 * stream size once the stream syncs (the needed size if cap was too small;
 * lcc_sync then returns LCC_ERR_CAPACITY).  kf (nullable) receives the coding
 * planes for later P frames. */
lcc_status lcc_encode_keyframe(lcc_ctx *ctx, const float *d_pts, int64_t n, lcc_keyframe *kf,
                               uint8_t *d_out, uint64_t cap, uint64_t *out_bytes);

/* Temporal + spatial encode of one P frame against kf (Sec. III-D). */
lcc_status lcc_encode_pframe(lcc_ctx *ctx, const lcc_keyframe *kf, const double pose[16],
                             const float *d_pts, int64_t n, uint8_t *d_out, uint64_t cap,
                             uint64_t *out_bytes);

/* A key frame whose tile fits are seeded by proposals (the learned proposal of
 * the net below; not in the paper).  d_prop: device float [num_tiles][5] per
 * tile: planarity logit, unnormalised normal (3), plane offset relative to the
 * tile's anchor (its first valid pixel's point r*u).  A tile whose logit is
 * below skip_logit is not fitted (raw-coded); otherwise its first round fits
 * the pixels within fit_thr_m of the proposed plane (all valid pixels if fewer
 * than 3), and the rounds and the FIT rule are the plain ones, so every plane
 * that codes points passes the same threshold test.  Streams are in the same
 * format and decode with lcc_decode. */
lcc_status lcc_encode_keyframe_seeded(lcc_ctx *ctx, const float *d_pts, int64_t n, const float *d_prop,
                                      float skip_logit, lcc_keyframe *kf, uint8_t *d_out, uint64_t cap,
                                      uint64_t *out_bytes);

/* Batched key frames: nframes independent frames, each spatially coded (its own
 * key frame), in one launch per kernel.  d_prop: NULL for the plain fit, or a
 * host array of nframes device proposal tables as in lcc_encode_keyframe_seeded.
 * nframes <= max_batch; out_bytes: nframes uint64 (host or device). */
lcc_status lcc_encode_keyframes(lcc_ctx *ctx, int32_t nframes, const float *const *d_pts, const int64_t *n,
                                const float *const *d_prop, float skip_logit, uint8_t *const *d_out,
                                const uint64_t *cap, uint64_t *out_bytes);

/* Batched: nframes P frames against one key frame in one launch per kernel.
 * poses: nframes x 16 doubles; d_pts, n, d_out, cap: per-frame host arrays;
 * out_bytes: nframes uint64 (host or device).  nframes <= max_batch. */
lcc_status lcc_encode_pframes(lcc_ctx *ctx, const lcc_keyframe *kf, int32_t nframes, const double *poses,
                              const float *const *d_pts, const int64_t *n, uint8_t *const *d_out,
                              const uint64_t *cap, uint64_t *out_bytes);

/* A whole sequence (Fig. 1): frame key_index is the K frame, all others are P
 * frames; poses[f] maps frame f to the key frame (poses[key_index] unused).
 * The key frame's chain runs on a private high-priority stream; the P frames'
 * binning, spatial fits and run pre-test run on a second stream of the context
 * beside it (they do not need K), and their temporal test, merge and pack
 * follow once the key frame's merge has written its planes.  The streams are
 * byte-identical to encoding K and then the P frames in sequence.
 * nframes <= max_batch.  kf (nullable) receives the key frame's planes. */
lcc_status lcc_encode_sequence(lcc_ctx *ctx, int32_t nframes, int32_t key_index, const double *poses,
                               const float *const *d_pts, const int64_t *n, uint8_t *const *d_out,
                               const uint64_t *cap, uint64_t *out_bytes, lcc_keyframe *kf);

/* End-to-end variant with HOST buffers: copies the points host->device,
 * encodes the sequence and copies each stream device->host.  h_out[f] must
 * hold cap[f] bytes; out_bytes is a host array.  Synchronous. */
lcc_status lcc_encode_sequence_host(lcc_ctx *ctx, int32_t nframes, int32_t key_index, const double *poses,
                                    const float *const *h_pts, const int64_t *n, uint8_t *const *h_out,
                                    const uint64_t *cap, uint64_t *out_bytes);

/* Rebuild a key frame's planes from its stream (for decoding P frames). */
lcc_status lcc_keyframe_from_stream(lcc_ctx *ctx, const uint8_t *d_bits, uint64_t nbytes, lcc_keyframe *kf);

/* Decode one stream (ray casting, Sec. III-C).  kf and pose are required for
 * P-frame streams (NULL for K).  Outputs (any may be NULL): d_range
 * [rows*cols] fp32 (0 = empty), d_xyz4 [rows*cols] float4 (x, y, z, 0),
 * d_valid occupancy bitmap.  A corrupt stream latches LCC_ERR_CORRUPT. */
lcc_status lcc_decode(lcc_ctx *ctx, const uint8_t *d_bits, uint64_t nbytes, const lcc_keyframe *kf,
                      const double pose[16], float *d_range, float *d_xyz4, uint32_t *d_valid);

/* Decode a whole sequence encoded by lcc_encode_sequence (frame key_index is
 * its key frame, poses[16 f] the pose of frame f, as given to the encoder):
 * the key frame's stream is resolved first (its coding planes), then every P
 * stream against them, all P streams in one launch (one CTA each), and every
 * frame is reconstructed.  The same outputs as lcc_keyframe_from_stream plus
 * lcc_decode per frame.  d_range, d_xyz4 and d_valid are arrays of nframes
 * device pointers (each array, and each entry, may be NULL); nframes <=
 * max_batch.  The decoder's per-frame state lives in the context, so a
 * context decodes one sequence at a time.  Not in the paper as a call: its
 * decoder is per frame. */
lcc_status lcc_decode_sequence(lcc_ctx *ctx, int32_t nframes, int32_t key_index, const double *poses,
                               const uint8_t *const *d_bits, const uint64_t *nbytes, float *const *d_range,
                               float *const *d_xyz4, uint32_t *const *d_valid);

/* Lossless entropy stage (Sec. III-A, its last paragraph: planes and residual
 * maps pass through a lossless coder, Huffman coding being the one named).
 * lcc_entropy_encode turns each fixed-width frame stream d_in[f] (in_size[f]
 * readable bytes, at least the stream's own size) into an entropy stream at
 * d_out[f] (out_cap[f] bytes); lcc_entropy_decode gives the fixed-width stream
 * back, byte for byte.  Entropy stream: the fixed-width stream's 64-byte
 * header, word 16 "LCE1", word 17 its size in bytes, words 18..45 one
 * descriptor of 4 words per section (mode | width << 8, count, alphabet,
 * words), then the sections in stream order.  The bitmap and the fitted bits
 * are coded as bytes, the tile codes as 4-bit symbols, the residual and raw
 * codes at their width (at most 12 bits); the run planes and temporal records
 * are copied.  A symbol section gets its own canonical Huffman code (lengths
 * <= 15 from Huffman's construction over (count, symbol)-sorted leaves, a leaf
 * first on equal weights, counts halved until the depth fits; codes in
 * (length, symbol) order by the DEFLATE rule) when the coded form - a 4-bit
 * length per symbol of the alphabet, one word offset per 1024-symbol chunk,
 * then the word-padded chunks, each code's bits most significant first at
 * increasing LSB-first bit positions - is smaller than the copy.
 * Device buffers 16-byte aligned; out_bytes is a DEVICE array of nframes sizes
 * (the needed size on a capacity error).  Asynchronous on the context stream;
 * up to max_batch frames per call.  Errors latch (lcc_sync): LCC_ERR_CAPACITY,
 * LCC_ERR_CORRUPT (a stream that is not this sensor's, or a corrupt entropy
 * stream). */
lcc_status lcc_entropy_encode(lcc_ctx *ctx, int32_t nframes, const uint8_t *const *d_in, const uint64_t *in_size,
                              uint8_t *const *d_out, const uint64_t *out_cap, uint64_t *out_bytes);
lcc_status lcc_entropy_decode(lcc_ctx *ctx, int32_t nframes, const uint8_t *const *d_in, const uint64_t *in_bytes,
                              uint8_t *const *d_out, const uint64_t *out_cap, uint64_t *out_bytes);

/* Pose of a P frame from IMU samples (Sec. III-D, the equations of T and R before
 * Eq. 6): the 4x4 row-major M with p_K = R p_P + T for the frame taken at t_p,
 * the key frame taken at t_key.  Samples k = 0..n-1 at strictly increasing times
 * t[k] give the acceleration acc[3k..3k+2] (m/s^2, gravity removed) and rotation
 * rate gyro[3k..3k+2] (rad/s, about x, y, z), in the key frame's sensor axes;
 * each holds until the next sample.  v_key is the velocity at t_key.
 * Integration is first-order (explicit Euler) from t_key to t_p, forward or
 * backward, one step per (partial) sample interval, position before velocity;
 * T = the position reached, R = Rz(alpha) Ry(beta) Rx(gamma) in the paper's
 * printed form with (alpha, beta, gamma) = -(angle about z, y, x).  Host code,
 * synchronous; LCC_ERR_INVALID_ARG on NULL pointers, n < 1, non-increasing
 * times or non-finite t_key / t_p. */
lcc_status lcc_imu_pose(const double *t, const double *acc, const double *gyro, int32_t n, const double v_key[3],
                        double t_key, double t_p, double pose[16]);

/* Wait for the context's stream and return (then clear) any latched device error. */
lcc_status lcc_sync(lcc_ctx *ctx);

/* Statistics of frame `frame` (batch position) of the last encode call.  Synchronous. */
lcc_status lcc_last_stats(lcc_ctx *ctx, int32_t frame, lcc_stats *out);

/* Per-tile records of frame `frame` of the last encode call (host array of
 * at least lcc_num_tiles entries).  Synchronous. */
lcc_status lcc_tile_records(lcc_ctx *ctx, int32_t frame, lcc_tile_info *h_out, int64_t cap);

/* With plane3: the three-coefficient form (a, b, c, axis as a float) of each tile's last spatial
 * fit in frame `frame` of the last encode call (h_out: at least lcc_num_tiles x 4 floats; the
 * plane in the tile record is the unit-normal plane of these coefficients).  Synchronous;
 * LCC_ERR_UNSUPPORTED for a context without plane3. */
lcc_status lcc_tile_coefficients(lcc_ctx *ctx, int32_t frame, float *h_out, int64_t cap);

/* Kernel timing: when enabled, every kernel launch is bracketed by CUDA events
 * on the stream it runs on.  lcc_kernel_times returns, per kernel name, the
 * number of launches and summed milliseconds since the last reset
 * (synchronous; launches that overlap are each timed in full).  Names: "bin",
 * "fit" (first fit pass), "rounds" (queued fit rounds), "lookbehind" (run
 * pre-test), "temporal", "merge" (with the frame's stream layout), "pack",
 * "decode_prep", "decode_px", "range_export".  Returns the number of entries
 * written. */
lcc_status lcc_set_profiling(lcc_ctx *ctx, int32_t enable);
int32_t lcc_kernel_times(lcc_ctx *ctx, char names[][16], int64_t *launches, double *ms, int32_t cap);

/* Launch timeline: for each timed launch since profiling was last enabled
 * (in the order the launches were issued, up to 65536), its name and its
 * start and end in milliseconds after the start of the first timed launch,
 * across all the streams the context uses, so overlapping launches show as
 * overlapping intervals.  Synchronous; writes at most cap entries (names,
 * t0_ms and t1_ms may each be NULL) and returns the number written. */
int32_t lcc_kernel_timeline(lcc_ctx *ctx, char names[][16], float *t0_ms, float *t1_ms, int32_t cap);

/* ---- Learned tile proposal (net over 8x8 tiles) ----
 *
 * Not in the paper: a small convolutional net that predicts, for an 8x8 tile,
 * whether the iterative fit will succeed (logit) and the plane it will find
 * (unnormalised normal, offset relative to the tile's anchor = its first valid
 * pixel's point), used by lcc_encode_keyframe_seeded.  Input per tile: 64
 * pixels x 4 bf16 channels (r - r_anchor, p - p_anchor in metres, empty
 * pixels 0), pixel-major.  Layers: conv3x3 pad 1 4->32, 32->64, 64->64 (ReLU),
 * global average pool, linear 64->32 (ReLU), linear 32->5.  BF16 operands,
 * FP32 accumulation on the tensor cores.  Parameters: one fp32 vector of
 * lcc_net_num_params() = 58853 values, in the order W1[32,4,3,3], b1,
 * W2[64,32,3,3], b2, W3[64,64,3,3], b3, F1[32,64], c1, F2[5,32], c2.
 * Loss (mean over tiles): BCE-with-logits(logit, fit) + fit*(1 - |n_hat.n|) +
 * fit*SmoothL1_0.02m(offset - d_rel); labels per tile (fit, n[3], d_rel).
 * Optimiser: Adam (0.9, 0.999, 1e-8) on fp32 master weights. */
typedef struct lcc_net lcc_net;

int64_t lcc_net_num_params(void);
/* max_tiles bounds the tiles of one lcc_net_gradient / lcc_net_train_step call
 * (activations are kept per tile, about 41 KB each).  Synchronous. */
lcc_status lcc_net_create(lcc_net **out, const float *h_params, int64_t max_tiles, void *cuda_stream);
void lcc_net_destroy(lcc_net *net);
lcc_status lcc_net_get_params(lcc_net *net, float *h_params);   /* synchronous */
lcc_status lcc_net_set_params(lcc_net *net, const float *h_params);   /* also resets Adam moments */
/* Bins a frame (slot 0 of a context with 8x8 tiles) and writes the net input of
 * every tile: d_x [num_tiles][64][4] bf16 (as uint16), d_anchor [num_tiles]
 * float4 (anchor x, y, z, r).  LCC_ERR_UNSUPPORTED for other tile shapes. */
lcc_status lcc_net_tile_inputs(lcc_ctx *ctx, const float *d_pts, int64_t n, uint16_t *d_x, float *d_anchor);
/* The same for nframes frames (<= max_batch) in one binning launch and one input launch: frame f's
 * tiles are rows [f*num_tiles, (f+1)*num_tiles) of d_x and d_anchor. */
lcc_status lcc_net_tile_inputs_batch(lcc_ctx *ctx, int32_t nframes, const float *const *d_pts, const int64_t *n,
                                     uint16_t *d_x, float *d_anchor);
/* Training labels of frame `frame` of the context's last encode: d_labels [num_tiles][5] fp32
 * (fit flag 1 or 0, the plane's unit normal n[3], its offset relative to the tile's anchor
 * d - n.anchor formed in FP64 and rounded once; zeros for a tile whose status is not FIT), from
 * the tile records and d_anchor [num_tiles] float4 as lcc_net_tile_inputs writes it (16-byte
 * aligned).  Asynchronous on the context's stream.  LCC_ERR_INVALID_ARG for a frame outside the
 * last encode. */
lcc_status lcc_net_tile_labels(lcc_ctx *ctx, int32_t frame, const float *d_anchor, float *d_labels);
/* Outputs d_out [ntiles][5] fp32 (logit, v[3], d_rel), on the net's stream.
 * Inference runs on tcgen05 (TMEM accumulators, two tiles per MMA); its
 * waits are bounded, and one that ran out is reported by lcc_net_sync. */
lcc_status lcc_net_forward(lcc_net *net, const uint16_t *d_x, int64_t ntiles, float *d_out);
/* Waits for the net's stream; LCC_ERR_TIMEOUT if a kernel's bounded wait ran out (then cleared). */
lcc_status lcc_net_sync(lcc_net *net);
/* Gradient of the mean loss w.r.t. the parameters (d_grad: 58853 fp32, may be
 * NULL) and the loss (d_loss: 1 fp32, may be NULL); d_labels [ntiles][5]. */
lcc_status lcc_net_gradient(lcc_net *net, const uint16_t *d_x, const float *d_labels, int64_t ntiles, float *d_grad,
                            float *d_loss);
/* One training step: gradient, then an Adam update with learning rate lr at
 * step number `step` (from 1, for the bias correction). */
lcc_status lcc_net_train_step(lcc_net *net, const uint16_t *d_x, const float *d_labels, int64_t ntiles, float lr,
                              int32_t step, float *d_loss);

/* Self-test of the bounded device waits (failure detection without a fault):
 * one kernel waits, at most `limit` polls, on an mbarrier that nothing
 * arrives on, the same bounded wait the tcgen05 kernels use.  Returns
 * LCC_ERR_TIMEOUT when the wait expired as it must, the context stays usable.
 * Synchronous.  Not in the paper. */
lcc_status lcc_selftest_bounded_wait(int64_t limit, void *cuda_stream);

/* ---- Range image without a context or any allocation ----
 *
 * The paper has no counterpart: this is an implementation entry point.  It
 * writes the same outputs as lcc_range_image, bit for bit, for callers that
 * must not allocate device memory: a process whose device memory is fully
 * reserved up front by its own pool, or a latency-critical thread that cannot
 * take the implicit device-wide synchronisation of cudaFree or the cost of a
 * first allocation.  It makes no cudaMalloc, cudaFree or other allocating
 * call; its scratch is one fixed device array of about 1.2 MB (range image,
 * boundary tables, counters) in the library, which every GPU that loads the
 * library keeps until the process exits.
 *
 * Limits: rows <= 512, cols <= 8192, rows * cols <= 262144 (e.g. 128 x 2048);
 * larger sensors return LCC_ERR_UNSUPPORTED.  Invalid sensor or pointers
 * return LCC_ERR_INVALID_ARG.
 *
 * d_pts: n device float4 (x, y, z, unused), 16-byte aligned (may be NULL when
 * n = 0).  Outputs (either may be NULL): d_range [rows*cols] fp32 (0 =
 * empty), d_valid occupancy bitmap of ceil(rows*cols/32) words, bit p of word
 * p/32 set when pixel p holds a point.  The clearing and binning work runs
 * asynchronously on cuda_stream.  The sensor's boundary tables stay in the
 * array between calls: a call whose sensor differs from the previous call's on
 * the device (and the first call) copies them from host memory with pageable
 * cudaMemcpyAsync, and such a copy first waits for the work already queued on
 * cuda_stream, so that call returns only after that work has finished.
 *
 * Set-up: the first call on each device, with that device current, resolves
 * the array's address with cudaGetSymbolAddress (checked) and keeps it; make
 * that first call before any stream capture begins.  A cudaDeviceReset ends
 * the context the address belongs to, and the next call in the new context
 * repeats the set-up (and the table copy).
 * The array is shared by every call on a device: calls that overlap in time
 * (other streams, other threads) race on it and must be serialised by the
 * caller.  Each call clears what must start cleared (range image to empty,
 * counters to zero) on its stream before binning. */
lcc_status lcc_range_image_static(const lcc_sensor *sensor, const float *d_pts, int64_t n, float *d_range,
                                  uint32_t *d_valid, void *cuda_stream);

/* ---- Batched encode of many sequences, replayed as a CUDA graph ----
 *
 * The paper encodes one sequence at a time (Sec. III-C: frames are grouped,
 * the middle frame of each group is the key frame K, the others are P frames
 * coded against K's planes).  A plan applies that grouping to a whole table
 * of sequences of possibly different sensors: every sequence is bound to one
 * of up to 8 contexts (one per resolution / tile-shape class).  Per class,
 * all key frames are encoded first, then all P frames, in chunks of the
 * context's max_batch frames, each chunk one batched launch set.  With more
 * than one class, each class runs on its own stream between a fork and a
 * join, so the classes overlap on the GPU; when a class's points are in host
 * memory the next class starts once it has binned its first chunk, so that
 * one class's binning (over the host link) meets the others' fits and packs.
 * Sequences of one sensor may be spread over several contexts of the same
 * parameters to have their chunks overlap in this way.
 *
 * Key-frame groups: group g of a sequence covers frames [g*I, min((g+1)*I, n))
 * with I = key_interval; its key frame is the group's frame start + floor(len/2).
 * poses[f] (4x4 row-major doubles) maps frame f into the coordinates of its
 * group's key frame (p_K = R p + T, Eq. 6); the key frames' own entries are
 * ignored.  Stream f of a sequence is bit-identical to what
 * lcc_encode_sequence makes for that group (same params).
 *
 * Every context must have been created on the same stream.  The plan copies
 * the descriptors (pointer arrays, counts, poses) at create/update time; the
 * device buffers they point to must stay allocated while the plan is used.
 * The plan owns, per class, one key-frame plane table per group.  While a
 * plan call runs, its contexts must not be used by other calls. */
typedef struct lcc_seq_desc {
    int32_t ctx;              /* index into the plan's context array */
    int32_t nframes;          /* >= 1 */
    int32_t key_interval;     /* frames per key-frame group, >= 1 */
    int32_t reserved;
    const double *poses;      /* host, nframes x 16 */
    const float *const *d_pts;/* host array of nframes pointers to float4 (x, y, z, unused), 16-B aligned: device
                                 memory, or page-locked host memory (read in place over the host link) */
    const int64_t *n;         /* host array: points per frame */
    uint8_t *const *d_out;    /* host array of nframes device output buffers (device memory), 16-B aligned */
    const uint64_t *cap;      /* host array: capacity of each output buffer (bytes) */
    uint64_t *d_nbytes;       /* DEVICE array of nframes: stream size of each frame, written by the encode */
} lcc_seq_desc;

typedef struct lcc_plan lcc_plan;

typedef struct lcc_plan_info {
    int64_t frames, key_frames, points;
    int64_t launches;         /* kernel launches of one encode (after the first encode or capture) */
    int64_t graph_nodes;      /* nodes of the captured graph (0 before capture) */
    int32_t classes, captured;
    int64_t seeded_key_frames;/* key frames whose fits the attached proposal net seeds */
} lcc_plan_info;

/* Validates the table and allocates the key-frame plane tables (synchronous).
 * LCC_ERR_INVALID_ARG: bad descriptor, contexts on different streams, a context listed twice. */
lcc_status lcc_plan_create(lcc_plan **out, int32_t nctx, lcc_ctx *const *ctxs, int32_t nseq,
                           const lcc_seq_desc *seqs);
/* Replaces pointers, counts and poses; the structure (per sequence: ctx, nframes,
 * key_interval) must be unchanged.  A captured plan is re-recorded and its
 * executable graph updated in place. */
lcc_status lcc_plan_update(lcc_plan *plan, int32_t nseq, const lcc_seq_desc *seqs);
/* Learned proposals for the plan's key frames (not in the paper; the net is the one of
 * lcc_net_* below).  With net != NULL, every chunk of key frames of a class whose context has
 * 8x8 tiles is, after its binning, turned into net inputs (lcc_net_tile_inputs_batch's kernel,
 * the range images kept) and run through the tcgen05 inference, and its tile fits are seeded by
 * the proposals as in lcc_encode_keyframes (skip_logit as there), all on the class's stream and
 * inside the captured graph.  P frames keep the plain fit for the tiles their temporal test
 * leaves.  Streams are those lcc_encode_keyframes(..., proposals, skip_logit, ...) writes for
 * the same key frames, followed by the plain P-frame path.  Classes with other tile shapes stay
 * plain; LCC_ERR_UNSUPPORTED if no class has 8x8 tiles.  net == NULL detaches the net.  The plan
 * allocates the inputs and proposals of one chunk per class (about 550 B per tile of max_batch
 * frames) and does not own the net, which must outlive the plan's use.  A captured plan is
 * re-recorded and its executable graph updated in place.  A bounded wait of the inference that
 * ran out is reported by lcc_plan_sync (LCC_ERR_TIMEOUT). */
lcc_status lcc_plan_set_proposals(lcc_plan *plan, lcc_net *net, float skip_logit);
/* Staging of host points (not in the paper; an I/O choice).  enable = 1: the points of frames
 * that are page-locked host memory are copied by the copy engines, one cudaMemcpyAsync per
 * frame on a copy stream of the class, into one of two device buffers of a chunk (the class
 * context's max_batch frames, each the size of the class's largest such frame) ahead of that
 * chunk's binning, so that the copies of one chunk run while the previous chunk is encoded
 * and the binning reads device memory; a buffer is refilled only after the chunk that used it
 * is binned.  enable = 0 (the default): the binning kernels read such points in place over the
 * host link.  The streams are the same either way.  Allocates 2 x max_batch x (largest host
 * frame) x 16 bytes per class (grown by lcc_plan_update if a frame grows); device points are not
 * copied.  A captured plan is re-recorded.  LCC_ERR_INVALID_ARG for enable outside 0..1. */
lcc_status lcc_plan_set_staging(lcc_plan *plan, int32_t enable);
/* Enqueues one encode of the whole table (asynchronous, no graph). */
lcc_status lcc_plan_encode(lcc_plan *plan);
/* Records one encode of the table as a CUDA graph (nothing runs).  Not allowed while
 * profiling is enabled on one of the contexts (LCC_ERR_INVALID_ARG). */
lcc_status lcc_plan_capture(lcc_plan *plan);
/* Launches the captured graph on the contexts' stream (asynchronous). */
lcc_status lcc_plan_replay(lcc_plan *plan);
/* Waits for the stream, then returns (and clears) the first error latched by any context. */
lcc_status lcc_plan_sync(lcc_plan *plan);
/* End-to-end encode with HOST outputs: one encode of the table (the captured graph if there is
 * one, else eager launches), then every frame's stream is copied by one kernel into h_out[f] (a
 * host array of `frames` pointers in table order: sequence by sequence, frame by frame; each a
 * page-locked, device-mapped, 16-byte aligned host buffer of at least that frame's cap bytes),
 * and every stream size into h_nbytes (host array of `frames` entries, table order; the needed
 * size where a capacity error latched).  Synchronous: returns lcc_plan_sync's status.  The plan's
 * input points may be page-locked host memory mapped into the device (read in place by the
 * binning kernel over the host link).  LCC_ERR_INVALID_ARG for an output that is not
 * page-locked host memory. */
lcc_status lcc_plan_encode_host(lcc_plan *plan, uint8_t *const *h_out, uint64_t *h_nbytes);
lcc_status lcc_plan_get_info(const lcc_plan *plan, lcc_plan_info *out);
/* Statistics of frame `frame` of sequence `seq` of the last encode or replay, or (seq = -1) their
 * sum over every frame of the table (counts add up; bytes is the total stream size).  Waits for
 * the stream.  Synchronous. */
lcc_status lcc_plan_stats(lcc_plan *plan, int32_t seq, int32_t frame, lcc_stats *out);
void lcc_plan_destroy(lcc_plan *plan);

/* ---- Autotuner ----
 *
 * Not in the paper (its tile size is a fixed parameter).  Encodes a sample
 * key-frame group (nframes <= 64 device frames, key frame key_index, poses as
 * in lcc_encode_sequence) the way a plan encodes its chunks (the key frame by
 * lcc_encode_keyframe, then the P frames in one lcc_encode_pframes call
 * against its planes) with every candidate of tile shape {4x4, 4x8, 8x8,
 * 8x16} (those whose bit is set in `shapes`: bit 0 4x4, bit 1 4x8, bit 2 8x8,
 * bit 3 8x16; 0 = all four) x run-test horizon {8, 16, 32} (only 0 when
 * base->merge_runs is 0) x fit schedule {0, 3, 4, 5, 6}, each on a context of its own,
 * `reps` timed encodes per candidate (CUDA events on cuda_stream).  Every
 * frame is then decoded and compared with its binned input: candidates whose
 * max range error exceeds max_err_m are rejected.  Of the rest, those whose
 * total stream size is at most (1 + bytes_slack) x the smallest are eligible,
 * and the fastest of them is written to *best (base with tile_h, tile_w,
 * lookahead and fit_schedule replaced).  results (cap entries, may be NULL
 * when cap is 0) receives every candidate, *nresults their number.
 * Synchronous; allocates and frees its own buffers.  LCC_ERR_UNSUPPORTED when
 * no candidate is eligible. */
typedef struct lcc_tune_result {
    int32_t tile_h, tile_w, lookahead, fit_schedule;
    int32_t status;           /* LCC_OK, or why the candidate could not be measured */
    int32_t chosen;           /* 1 for the candidate written to *best */
    double ms;                /* mean device time of one encode of the sample */
    double mpts_per_s;
    uint64_t bytes;           /* total stream bytes of the sample */
    float max_err_m;          /* max |decoded range - binned input range| over occupied pixels */
    float reserved;
} lcc_tune_result;

lcc_status lcc_autotune(const lcc_sensor *sensor, const lcc_params *base, int32_t nframes, int32_t key_index,
                        const double *poses, const float *const *d_pts, const int64_t *n, int32_t reps,
                        float max_err_m, float bytes_slack, uint32_t shapes, void *cuda_stream,
                        lcc_tune_result *results, int32_t cap, int32_t *nresults, lcc_params *best);

#ifdef __cplusplus
}
#endif
#endif
