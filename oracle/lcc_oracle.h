/*
 * CPU ORACLE — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, single-threaded C restatement of the spatio-temporal LiDAR encoder
 * of "Real-Time Spatio-Temporal LiDAR Point Cloud Compression" (Feng, Liu,
 * Zhu).  Only the test-suite, the smoke check and the bench's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant with the GPU
 * library: both follow the same written definitions independently.
 *
 * Parity status of each entry point (how it is pinned by the CPU tests):
 *   orc_tables / orc_range_image  pinned: pixel-centre points, Eq. 2 in fp64
 *                                 away from boundaries, collision rule.
 *   orc_tls_fit                   pinned: numpy eigh, brute-force sphere search,
 *                                 exact recovery of noise-free planes.
 *   orc_fit_tiles                 pinned: noise-free planar tiles (1 round, exact
 *                                 plane), planted outliers (rounds, inlier set).
 *   orc_temporal_tiles            pinned: pure translation (c' = d - n.T), P == K.
 *   orc_pack / orc_decode         pinned: decode error <= q/2, raw round trip,
 *                                 greedy-run invariants (spatial and temporal runs),
 *                                 re-encode identity.
 */
#ifndef LCC_ORACLE_H
#define LCC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t rows, cols;          /* range image height (beams) and width (azimuth steps) */
    double elev_min_deg;         /* elevation of the bottom edge of the last row */
    double elev_max_deg;         /* elevation of the top edge of row 0 */
    double max_range_m;          /* points farther than this are dropped */
} orc_sensor;

typedef struct {
    int32_t tile_h, tile_w;      /* unit tile (Sec. III-C, e.g. 4x4) */
    float fit_thr_m;             /* plane-fit threshold on the along-ray residual */
    float quant_m;               /* quantisation step q of residual and raw codes */
    int32_t max_refits;          /* R: refit rounds after the first fit */
    float min_inlier_frac;       /* f_min: inlier share a plane needs (1.0 = all points) */
    int32_t merge_runs;          /* 1: grow runs of tiles horizontally (Sec. III-C) */
    int32_t no_delta;            /* 1: plane-coded points carry no residual code (Sec. III-C:
                                    the deltas are dropped, decode error <= threshold) */
    int32_t raw_exact;           /* 1: raw pixels carry their fp32 range bits, so unfit points
                                    are kept losslessly (header flags bit 2, 32-bit raw codes) */
    int32_t temporal_candidates; /* K tiles a P tile's relaxed-plane test may try (1..4): the
                                    distinct K tiles its valid pixels fall in, raster order from
                                    the anchor's; 1 (or 0) = the anchor's K tile only */
    int32_t temporal_runs;       /* 1: temporally coded tiles grow runs like spatial ones
                                    (Sec. III-D: the same horizontal growing strategy): a tile
                                    that passes the acceptance rule against the relaxed plane of
                                    the temporal tile to its left joins that tile's run (tile code
                                    TEMPORAL_CONT, no record of its own; header flags bit 3) */
    int32_t plane3;              /* 1: planes in Eq. 3's three-coefficient form (dominant axis):
                                    every fitted plane is replaced by the unit-normal plane of its
                                    coefficients a = n_i/n_k, b = n_j/n_k, c = d/n_k (k the axis of
                                    the largest |n_k|), and run records carry the coefficients (3
                                    words; header flags bit 4) with the axis in the run start's tile
                                    code (6 + k) */
} orc_params;

/* tile codes of the bitstream */
enum { ORC_T_EMPTY = 0, ORC_T_RAW = 1, ORC_T_RUN_START = 2, ORC_T_RUN_CONT = 3, ORC_T_TEMPORAL = 4,
       ORC_T_TEMPORAL_CONT = 5, ORC_T_RUN_START3 = 6 /* .. 8: plane3 run start, dominant axis x, y, z */ };
/* own-fit status */
enum { ORC_FIT_EMPTY = 0, ORC_FIT_FAIL = 1, ORC_FIT_OK = 2 };
/* errors */
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_CORRUPT = -2, ORC_ERR_CAPACITY = -3, ORC_ERR_INCONSISTENT = -4 };

typedef struct {
    int32_t status;              /* ORC_FIT_* */
    int32_t n_valid;             /* valid pixels in the tile */
    int32_t n_inlier;            /* inliers of the final plane */
    int32_t rounds;              /* TLS fits performed (1 .. R+1), 0 if none */
    int32_t borderline;          /* some |e| within 1e-6 m of thr, or the lambda cut within 0.1 % */
    int32_t degenerate;          /* the last fit had lambda_mid <= 1e-12 lambda_max */
    float plane[4];              /* stored fp32 plane n.x, n.y, n.z, d (n.p = d) */
    double plane64[4];           /* the fp64 plane before rounding */
    double lam[3];               /* eigenvalues of the last fit, ascending */
    float coef[3];               /* plane3: the plane's coefficients a, b, c */
    int32_t axis;                /* plane3: its dominant axis k (0 x, 1 y, 2 z) */
} orc_tile_fit;

typedef struct {
    int32_t status;              /* 0 no plane-coded K tile found, 1 tested and failed, 2 pass */
    int32_t kref;                /* K tile index the anchor maps to, -1 if none */
    int32_t n_valid, n_inlier, rounds, borderline;
    float plane[4];              /* n' (fp32, K normal rotated into P coordinates) and c' */
} orc_tile_temporal;

/* Beam and boundary tables (Sec. III-B).  Sizes: ce,se: rows; ct,st: cols;
 * rbc,rbs: rows+1 (row boundaries, top to bottom); cbc,cbs: cols. */
int orc_tables(const orc_sensor *s, float *ce, float *se, float *ct, float *st,
               float *rbc, float *rbs, float *cbc, float *cbs);

/* Eq. 1-2: bin points (float4 x,y,z,w) into the range image (fp32 r, 0 = empty).
 * point_pixel (nullable) gets the pixel index of each point or -1 if dropped.
 * stats[0..3] = binned points, dropped invalid, dropped out of FOV, valid pixels. */
int64_t orc_range_image(const orc_sensor *s, const float *pts, int64_t n, float *range,
                        int32_t *point_pixel, int64_t stats[4]);

/* Total-least-squares plane of n points (fp64, n x 3): the normal is the
 * eigenvector of the smallest eigenvalue of the centred scatter matrix. */
int orc_tls_fit(const double *p, int n, double normal[3], double *d, double lam[3]);

/* Per-tile iterative plane fit of the whole image (tiles row-major). */
int orc_fit_tiles(const orc_sensor *s, const orc_params *prm, const float *range, orc_tile_fit *out);

/* Per-tile fit seeded by a proposal per tile, prop[t] = (logit, v0, v1, v2,
 * d_rel) (the learned proposal; not in the paper): see fit_one_seeded. */
int orc_fit_tiles_seeded(const orc_sensor *s, const orc_params *prm, const float *range, const float *prop,
                         float skip_logit, orc_tile_fit *out);

/* Temporal test of every P tile against the warped K planes (Sec. III-D). */
int orc_temporal_tiles(const orc_sensor *s, const orc_params *prm, const float *range,
                       const float *kf_table, const double pose[16], orc_tile_temporal *out);

/* Greedy run merge, point coding and stream packing given per-tile results.
 * fit_plane/fit_ok: own spatial fit per tile; temporal_plane/temporal_kref
 * (both NULL for a key frame; kref -1 = not temporal).  Returns the stream size
 * in bytes; writes only if it fits in cap.  kf_table_out (nullable, ntiles x 4)
 * receives the coding plane of every plane-coded tile (zeros elsewhere);
 * modes_out (nullable) the tile codes. */
int64_t orc_pack(const orc_sensor *s, const orc_params *prm, int kind, const float *range,
                 const float *fit_plane, const uint8_t *fit_ok,
                 const float *temporal_plane, const int32_t *temporal_kref,
                 uint8_t *out, uint64_t cap, float *kf_table_out, uint8_t *modes_out);

/* orc_pack for plane3 streams: fit_coef (ntiles x 4: a, b, c, axis as a float) gives each
 * fitted tile's coefficients, whose unit-normal plane must equal fit_plane bit for bit. */
int64_t orc_pack3(const orc_sensor *s, const orc_params *prm, int kind, const float *range,
                  const float *fit_plane, const float *fit_coef, const uint8_t *fit_ok,
                  const float *temporal_plane, const int32_t *temporal_kref,
                  uint8_t *out, uint64_t cap, float *kf_table_out, uint8_t *modes_out);

/* Eq. 3 generalised to any dominant axis: the coefficients (a, b, c) and axis k of a unit-normal
 * plane, and the unit-normal plane of coefficients (both fp32, fixed operation order). */
void orc_plane_to3(const float pl[4], int *axis, float abc[3]);
void orc_plane_from3(int axis, const float abc[3], float pl[4]);

/* Full key-frame encode: bin, fit, merge, code, pack. */
int64_t orc_encode_keyframe(const orc_sensor *s, const orc_params *prm, const float *pts, int64_t n,
                            uint8_t *out, uint64_t cap, float *kf_table_out,
                            orc_tile_fit *fits_out, uint8_t *modes_out);

/* Full P-frame encode against a key-frame tile table; pose maps P to K
 * coordinates (row-major 4x4, p_K = R p + T). */
int64_t orc_encode_pframe(const orc_sensor *s, const orc_params *prm, const float *kf_table,
                          const double pose[16], const float *pts, int64_t n,
                          uint8_t *out, uint64_t cap, orc_tile_fit *fits_out,
                          orc_tile_temporal *temporal_out, uint8_t *modes_out);

/* Decode a stream: range (fp32, 0 = empty), xyz4 (x, y, z, 0), valid bitmap
 * (rows*cols bits).  kf_table/pose are needed for P-frame streams only. */
int orc_decode(const orc_sensor *s, const uint8_t *bits, uint64_t nbytes, const float *kf_table,
               const double pose[16], float *range, float *xyz4, uint32_t *valid);

/* Coding plane per tile (ntiles x 4) recovered from a key-frame stream. */
int orc_kf_table_from_stream(const orc_sensor *s, const uint8_t *bits, uint64_t nbytes, float *kf_table);

#ifdef __cplusplus
}
#endif
#endif
