/*
 * CPU ORACLE — TEST INFRASTRUCTURE ONLY (see lcc_oracle.h).
 *
 * Plain single-threaded C.  Every step follows the paper's description in the
 * paper's order; where the paper is silent the reading used is stated at the
 * step.  Compile with -ffp-contract=off: the fp32 expressions below are the
 * arithmetic contract (explicit fmaf, IEEE division and square root), and the
 * compiler must not fuse any other multiply and add.
 */
#include "lcc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define STREAM_MAGIC 0x3143434Cu /* "LCC1" */
#define STREAM_VERSION 1
#define HEADER_BYTES 64
#define MAX_TILE_PX 1024

/* ------------------------------------------------------------------------ */
/* Sensor tables (Sec. III-B, Eq. 2)                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    int rows, cols;
    float *ce, *se;   /* cos/sin of row-centre elevation */
    float *ct, *st;   /* cos/sin of column-centre azimuth */
    float *rbc, *rbs; /* cos/sin of row boundary elevations, rows+1 */
    float *cbc, *cbs; /* cos/sin of column boundary azimuths, cols */
} tables_t;

static int sensor_ok(const orc_sensor *s) {
    return s && s->rows >= 1 && s->cols >= 2 && s->rows <= 65535 && s->cols <= 65535 &&
           s->elev_max_deg > s->elev_min_deg && s->elev_max_deg <= 90.0 && s->elev_min_deg >= -90.0 &&
           s->max_range_m > 0;
}

/*
 * Eq. 2 maps azimuth and elevation to pixel coordinates with the sensor's
 * angular resolutions.  Reading (the printed equation has no offsets and an
 * ambiguous arctan): row 0 is the top beam; row i spans elevations
 * (b_{i+1}, b_i] with b_k = elev_max - k*(elev_max-elev_min)/rows; column j
 * spans azimuths [a_j, a_{j+1}) with a_j = -pi + j*2pi/cols.  Beam direction of
 * pixel (i,j) is the pixel centre.  Tables are fp64 libm values rounded to fp32.
 */
int orc_tables(const orc_sensor *s, float *ce, float *se, float *ct, float *st,
               float *rbc, float *rbs, float *cbc, float *cbs) {
    if (!sensor_ok(s)) return ORC_ERR_ARG;
    const double deg = M_PI / 180.0;
    const double d_el = (s->elev_max_deg - s->elev_min_deg) / s->rows;
    const double d_az = 2.0 * M_PI / s->cols;
    for (int i = 0; i < s->rows; i++) {
        double e = (s->elev_max_deg - (i + 0.5) * d_el) * deg;
        ce[i] = (float)cos(e);
        se[i] = (float)sin(e);
    }
    for (int k = 0; k <= s->rows; k++) {
        double e = (s->elev_max_deg - k * d_el) * deg;
        rbc[k] = (float)cos(e);
        rbs[k] = (float)sin(e);
    }
    for (int j = 0; j < s->cols; j++) {
        double a = -M_PI + (j + 0.5) * d_az;
        ct[j] = (float)cos(a);
        st[j] = (float)sin(a);
        double b = -M_PI + j * d_az;
        cbc[j] = (float)cos(b);
        cbs[j] = (float)sin(b);
    }
    return ORC_OK;
}

static int tables_make(const orc_sensor *s, tables_t *t) {
    memset(t, 0, sizeof(*t));
    if (!sensor_ok(s)) return ORC_ERR_ARG;
    t->rows = s->rows;
    t->cols = s->cols;
    t->ce = malloc(sizeof(float) * s->rows);
    t->se = malloc(sizeof(float) * s->rows);
    t->ct = malloc(sizeof(float) * s->cols);
    t->st = malloc(sizeof(float) * s->cols);
    t->rbc = malloc(sizeof(float) * (s->rows + 1));
    t->rbs = malloc(sizeof(float) * (s->rows + 1));
    t->cbc = malloc(sizeof(float) * s->cols);
    t->cbs = malloc(sizeof(float) * s->cols);
    return orc_tables(s, t->ce, t->se, t->ct, t->st, t->rbc, t->rbs, t->cbc, t->cbs);
}

static void tables_free(tables_t *t) {
    free(t->ce); free(t->se); free(t->ct); free(t->st);
    free(t->rbc); free(t->rbs); free(t->cbc); free(t->cbs);
}

/* Beam direction of pixel (i,j): fp32 products of the row and column tables. */
static void beam(const tables_t *T, int i, int j, float u[3]) {
    u[0] = T->ce[i] * T->ct[j];
    u[1] = T->ce[i] * T->st[j];
    u[2] = T->se[i];
}

/* Sign test against row boundary k: > 0 iff the point lies above b_k. */
static float row_side(const tables_t *T, int k, float z, float rho) {
    return fmaf(z, T->rbc[k], -(rho * T->rbs[k]));
}

/* Sign test against column boundary j: >= 0 iff the azimuth is at or past a_j
 * (within half a turn). */
static float col_side(const tables_t *T, int j, float x, float y) {
    return fmaf(y, T->cbc[j], -(x * T->cbs[j]));
}

/*
 * Eq. 1-2 for one point.  r = sqrt(x^2+y^2+z^2) in fp32.  The pixel is decided
 * by exact-sign tests against the boundary tables, never by a transcendental,
 * so any implementation with the same fp32 expressions bins identically.
 * Returns 0 (binned), 1 (invalid: non-finite, r <= 0 or r > max range) or
 * 2 (outside the field of view).
 */
static int bin_point(const orc_sensor *s, const tables_t *T, float x, float y, float z,
                     float *r_out, int *pix_out) {
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) return 1;
    float r = sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
    if (!(r > 0.0f) || !(r <= (float)s->max_range_m)) return 1;
    float rho = sqrtf(fmaf(x, x, y * y));
    const int H = s->rows, W = s->cols;
    if (row_side(T, 0, z, rho) > 0.0f) return 2;
    if (!(row_side(T, H, z, rho) > 0.0f)) return 2;
    int row = -1;
    for (int i = 0; i < H; i++) {
        if (!(row_side(T, i, z, rho) > 0.0f) && row_side(T, i + 1, z, rho) > 0.0f) {
            row = i;
            break;
        }
    }
    if (row < 0) return 2;
    /* Column: the unique j with side_j >= 0 and side_{j+1} < 0 (cyclic).  A
     * first guess from atan2 only shortens the search; a full scan decides if
     * the guess and its neighbours fail. */
    int col = -1;
    double a = atan2((double)y, (double)x);
    int j0 = (int)floor((a + M_PI) / (2.0 * M_PI / W));
    for (int dj = -1; dj <= 1 && col < 0; dj++) {
        int j = ((j0 + dj) % W + W) % W;
        if (col_side(T, j, x, y) >= 0.0f && col_side(T, (j + 1) % W, x, y) < 0.0f) col = j;
    }
    for (int j = 0; j < W && col < 0; j++)
        if (col_side(T, j, x, y) >= 0.0f && col_side(T, (j + 1) % W, x, y) < 0.0f) col = j;
    if (col < 0) return 2;
    *r_out = r;
    *pix_out = row * W + col;
    return 0;
}

/* Range image conversion with the collision rule of Sec. III-D: when several
 * points fall in one pixel the nearest is kept. */
int64_t orc_range_image(const orc_sensor *s, const float *pts, int64_t n, float *range,
                        int32_t *point_pixel, int64_t stats[4]) {
    tables_t T;
    if (tables_make(s, &T) != ORC_OK || n < 0) { tables_free(&T); return ORC_ERR_ARG; }
    const int64_t npx = (int64_t)s->rows * s->cols;
    for (int64_t p = 0; p < npx; p++) range[p] = 0.0f;
    int64_t st[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < n; i++) {
        float r;
        int pix;
        int res = bin_point(s, &T, pts[4 * i], pts[4 * i + 1], pts[4 * i + 2], &r, &pix);
        if (point_pixel) point_pixel[i] = (res == 0) ? pix : -1;
        if (res == 1) { st[1]++; continue; }
        if (res == 2) { st[2]++; continue; }
        st[0]++;
        if (range[pix] == 0.0f || r < range[pix]) range[pix] = r;
    }
    for (int64_t p = 0; p < npx; p++) st[3] += (range[p] > 0.0f);
    if (stats) memcpy(stats, st, sizeof(st));
    tables_free(&T);
    return st[3];
}

/* ------------------------------------------------------------------------ */
/* Plane fit (Sec. III-C)                                                    */
/* ------------------------------------------------------------------------ */

/* Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (fp64).
 * Eigenvectors are the columns of V. */
static void jacobi3(double A[3][3], double w[3], double V[3][3]) {
    static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) V[a][b] = (a == b) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; sweep++) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off == 0.0 || off <= 1e-40 * dia) break;
        for (int r = 0; r < 3; r++) {
            int p = P[r][0], q = P[r][1];
            if (A[p][q] == 0.0) continue;
            double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
            double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
            for (int k = 0; k < 3; k++) {
                double akp = A[k][p], akq = A[k][q];
                A[k][p] = c * akp - sn * akq;
                A[k][q] = sn * akp + c * akq;
            }
            for (int k = 0; k < 3; k++) {
                double apk = A[p][k], aqk = A[q][k];
                A[p][k] = c * apk - sn * aqk;
                A[q][k] = sn * apk + c * aqk;
            }
            for (int k = 0; k < 3; k++) {
                double vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - sn * vkq;
                V[k][q] = sn * vkp + c * vkq;
            }
        }
    }
    for (int a = 0; a < 3; a++) w[a] = A[a][a];
}

/*
 * Closed-form least-squares plane (Sec. III-C cites total least squares): the
 * plane through the centroid c whose normal is the eigenvector of the smallest
 * eigenvalue of the centred scatter matrix.  Stored as unit normal n and offset
 * d with n.p = d (reading: Eq. 3's x + a y + b z = c cannot hold planes with
 * n_x = 0).  Canonical sign: d >= 0; if |d| < 1e-9 the largest-magnitude
 * component of n is made positive.
 */
int orc_tls_fit(const double *p, int n, double normal[3], double *d, double lam[3]) {
    if (n < 3) return ORC_ERR_ARG;
    double c[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) c[a] += p[3 * i + a];
    for (int a = 0; a < 3; a++) c[a] /= n;
    double A[3][3] = {{0}};
    for (int i = 0; i < n; i++) {
        double q[3] = {p[3 * i] - c[0], p[3 * i + 1] - c[1], p[3 * i + 2] - c[2]};
        for (int a = 0; a < 3; a++)
            for (int b = a; b < 3; b++) A[a][b] += q[a] * q[b];
    }
    for (int a = 0; a < 3; a++)
        for (int b = a; b < 3; b++) {
            A[a][b] /= n;
            A[b][a] = A[a][b];
        }
    double w[3], V[3][3];
    jacobi3(A, w, V);
    int idx[3] = {0, 1, 2};
    for (int a = 0; a < 3; a++)
        for (int b = a + 1; b < 3; b++)
            if (w[idx[b]] < w[idx[a]]) { int t = idx[a]; idx[a] = idx[b]; idx[b] = t; }
    for (int a = 0; a < 3; a++) lam[a] = w[idx[a]];
    double nv[3] = {V[0][idx[0]], V[1][idx[0]], V[2][idx[0]]};
    double nn = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    for (int a = 0; a < 3; a++) nv[a] /= nn;
    double dd = nv[0] * c[0] + nv[1] * c[1] + nv[2] * c[2];
    int flip;
    if (fabs(dd) < 1e-9) {
        int m = 0;
        for (int a = 1; a < 3; a++)
            if (fabs(nv[a]) > fabs(nv[m])) m = a;
        flip = nv[m] < 0;
    } else {
        flip = dd < 0;
    }
    if (flip) {
        for (int a = 0; a < 3; a++) nv[a] = -nv[a];
        dd = -dd;
    }
    for (int a = 0; a < 3; a++) normal[a] = nv[a];
    *d = dd;
    return ORC_OK;
}

/* Along-ray residual test of one pixel against an fp32 plane: the decoder
 * ray-casts the pixel's beam onto the plane (Sec. III-C), r_hat = d / (n.u).
 * Returns 1 if inlier (|r - r_hat| <= thr); e_out gets the residual; grazing or
 * back-facing beams (n.u <= 1e-3) are outliers. */
static int residual(const float pl[4], const float u[3], float r, float thr, float *e_out) {
    float dot = fmaf(pl[0], u[0], fmaf(pl[1], u[1], pl[2] * u[2]));
    if (!(dot > 1e-3f)) {
        *e_out = INFINITY;
        return 0;
    }
    float rhat = pl[3] / dot;
    float e = r - rhat;
    *e_out = e;
    return fabsf(e) <= thr;
}

/*
 * Eq. 3 writes a plane as x + a y + b z = c, which cannot hold planes with n_x = 0.  Its
 * three-coefficient form is kept by dividing by the dominant component instead: with k the axis of
 * the largest |n_k| (the lowest index on ties) and i, j the next two axes in cyclic order,
 * a = n_i / n_k, b = n_j / n_k, c = d / n_k (IEEE fp32 divisions).  The plane a decoder gets back
 * is the unit-normal one: n_k = 1 / sqrt(a^2 + b^2 + 1), n_i = a n_k, n_j = b n_k, d = c n_k,
 * negated when d < 0 (a plane through the origin, |d| < 1e-9, keeps n_k > 0).
 */
void orc_plane_to3(const float pl[4], int *axis, float abc[3]) {
    int k = 0;
    float m = fabsf(pl[0]);
    if (fabsf(pl[1]) > m) { k = 1; m = fabsf(pl[1]); }
    if (fabsf(pl[2]) > m) k = 2;
    abc[0] = pl[(k + 1) % 3] / pl[k];
    abc[1] = pl[(k + 2) % 3] / pl[k];
    abc[2] = pl[3] / pl[k];
    *axis = k;
}

void orc_plane_from3(int axis, const float abc[3], float pl[4]) {
    const float inv = 1.0f / sqrtf(fmaf(abc[0], abc[0], fmaf(abc[1], abc[1], 1.0f)));
    pl[axis] = inv;
    pl[(axis + 1) % 3] = abc[0] * inv;
    pl[(axis + 2) % 3] = abc[1] * inv;
    pl[3] = abc[2] * inv;
    if (!(fabsf(pl[3]) < 1e-9f) && pl[3] < 0.0f)
        for (int a = 0; a < 4; a++) pl[a] = -pl[a];
}

typedef struct {
    int n;               /* pixels of the tile inside the image */
    int pix[MAX_TILE_PX];/* image pixel index, raster order within the tile */
    int valid[MAX_TILE_PX];
    float r[MAX_TILE_PX];
    float u[MAX_TILE_PX][3];
    float p[MAX_TILE_PX][3]; /* r * u in fp32 */
    int n_valid;
} tile_px_t;

static void tile_gather(const orc_sensor *s, const orc_params *prm, const tables_t *T,
                        const float *range, int t, tile_px_t *tp) {
    const int TW = (s->cols + prm->tile_w - 1) / prm->tile_w;
    const int tr = t / TW, tc = t % TW;
    const int i0 = tr * prm->tile_h, j0 = tc * prm->tile_w;
    tp->n = 0;
    tp->n_valid = 0;
    for (int i = i0; i < i0 + prm->tile_h && i < s->rows; i++)
        for (int j = j0; j < j0 + prm->tile_w && j < s->cols; j++) {
            int k = tp->n++;
            tp->pix[k] = i * s->cols + j;
            tp->r[k] = range[tp->pix[k]];
            tp->valid[k] = tp->r[k] > 0.0f;
            beam(T, i, j, tp->u[k]);
            for (int a = 0; a < 3; a++) tp->p[k][a] = tp->r[k] * tp->u[k][a];
            tp->n_valid += tp->valid[k];
        }
}

static int need_inliers(const orc_params *prm, int n_valid) {
    int need = (int)ceilf(prm->min_inlier_frac * (float)n_valid);
    return need < 3 ? 3 : need;
}

/* Inlier set of a tile against a plane; returns its size and flags pixels whose
 * |e| is within 1e-6 m of the threshold. */
static int inliers(const tile_px_t *tp, const float pl[4], float thr, int *in, int *border) {
    int cnt = 0;
    for (int k = 0; k < tp->n; k++) {
        in[k] = 0;
        if (!tp->valid[k]) continue;
        float e;
        in[k] = residual(pl, tp->u[k], tp->r[k], thr, &e);
        cnt += in[k];
        if (border && isfinite(e) && fabsf(fabsf(e) - thr) <= 1e-6f) *border = 1;
    }
    return cnt;
}

/*
 * Iterative plane fit of one tile (abstract: "iterative plane fitting";
 * outliers are dropped and the plane refit).  Reading of the rounds:
 * S = valid pixels; fit; then up to R times: I = inliers of the last plane
 * (any valid pixel may re-enter); stop if I == S or |I| < 3; else S = I, refit.
 * The tile is FIT iff it has >= 3 valid pixels, the last scatter matrix is not
 * degenerate (lambda_mid > 1e-12 lambda_max) and the last plane keeps at least
 * max(3, ceil(f_min * n_valid)) inliers.
 */
static void fit_one(const orc_params *prm, const tile_px_t *tp, orc_tile_fit *f) {
    memset(f, 0, sizeof(*f));
    f->n_valid = tp->n_valid;
    if (tp->n_valid == 0) { f->status = ORC_FIT_EMPTY; return; }
    f->status = ORC_FIT_FAIL;
    if (tp->n_valid < 3) return;
    int S[MAX_TILE_PX], I[MAX_TILE_PX];
    double buf[3 * MAX_TILE_PX];
    for (int k = 0; k < tp->n; k++) S[k] = tp->valid[k];
    int nS = tp->n_valid, nI = 0;
    for (;;) {
        int m = 0;
        for (int k = 0; k < tp->n; k++)
            if (S[k]) {
                for (int a = 0; a < 3; a++) buf[3 * m + a] = (double)tp->p[k][a];
                m++;
            }
        double nrm[3], d, lam[3];
        orc_tls_fit(buf, m, nrm, &d, lam);
        f->rounds++;
        for (int a = 0; a < 3; a++) f->lam[a] = lam[a];
        f->plane64[0] = nrm[0]; f->plane64[1] = nrm[1]; f->plane64[2] = nrm[2]; f->plane64[3] = d;
        for (int a = 0; a < 3; a++) f->plane[a] = (float)nrm[a];
        f->plane[3] = (float)d;
        if (prm->plane3) {   /* the fitted plane as Eq. 3's coefficients store it */
            orc_plane_to3(f->plane, &f->axis, f->coef);
            orc_plane_from3(f->axis, f->coef, f->plane);
        }
        if (lam[1] >= 0.999e-12 * lam[2] && lam[1] <= 1.001e-12 * lam[2]) f->borderline = 1;
        if (!(lam[1] > 1e-12 * lam[2])) { f->degenerate = 1; nI = 0; break; }
        nI = inliers(tp, f->plane, prm->fit_thr_m, I, &f->borderline);
        int same = (nI == nS);
        for (int k = 0; k < tp->n && same; k++) same = (I[k] == S[k]);
        if (same || f->rounds == prm->max_refits + 1 || nI < 3) break;
        memcpy(S, I, sizeof(int) * tp->n);
        nS = nI;
    }
    f->n_inlier = nI;
    if (!f->degenerate && nI >= need_inliers(prm, tp->n_valid)) f->status = ORC_FIT_OK;
}

/*
 * Seeded fit (a learned proposal per tile; not in the paper).  prop = (logit,
 * v0, v1, v2, d_rel): a planarity logit, an unnormalised normal and the plane
 * offset relative to the tile's anchor (its first valid pixel's point).
 *   - logit < skip_logit: the tile is not fitted (status FAIL, no round).
 *   - Otherwise the proposed plane, in fp32: n = v / |v| (sqrtf of an fma sum,
 *     IEEE divisions), d = d_rel + n.anchor (fma chain), both negated if d < 0.
 *     The first set S is the valid pixels within the threshold of that plane;
 *     with fewer than 3 of them (or |v| = 0) S is all valid pixels, as in the
 *     plain fit.  From S on, the rounds and the FIT rule are those of fit_one.
 */
static void fit_one_seeded(const orc_params *prm, const tile_px_t *tp, const float prop[5], float skip_logit,
                           orc_tile_fit *f) {
    memset(f, 0, sizeof(*f));
    f->n_valid = tp->n_valid;
    if (tp->n_valid == 0) { f->status = ORC_FIT_EMPTY; return; }
    f->status = ORC_FIT_FAIL;
    if (tp->n_valid < 3) return;
    if (prop[0] < skip_logit) return;
    int S[MAX_TILE_PX], I[MAX_TILE_PX];
    double buf[3 * MAX_TILE_PX];
    int nS = 0, nI = 0;
    const float nn = sqrtf(fmaf(prop[1], prop[1], fmaf(prop[2], prop[2], prop[3] * prop[3])));
    if (nn > 0.0f && isfinite(nn)) {
        int a0 = 0;
        while (!tp->valid[a0]) a0++;
        float pl[4] = {prop[1] / nn, prop[2] / nn, prop[3] / nn, 0.0f};
        pl[3] = prop[4] + fmaf(pl[0], tp->p[a0][0], fmaf(pl[1], tp->p[a0][1], pl[2] * tp->p[a0][2]));
        if (pl[3] < 0.0f)
            for (int a = 0; a < 4; a++) pl[a] = -pl[a];
        nS = inliers(tp, pl, prm->fit_thr_m, S, &f->borderline);
    }
    if (nS < 3) {
        for (int k = 0; k < tp->n; k++) S[k] = tp->valid[k];
        nS = tp->n_valid;
    }
    for (;;) {
        int m = 0;
        for (int k = 0; k < tp->n; k++)
            if (S[k]) {
                for (int a = 0; a < 3; a++) buf[3 * m + a] = (double)tp->p[k][a];
                m++;
            }
        double nrm[3], d, lam[3];
        orc_tls_fit(buf, m, nrm, &d, lam);
        f->rounds++;
        for (int a = 0; a < 3; a++) f->lam[a] = lam[a];
        f->plane64[0] = nrm[0]; f->plane64[1] = nrm[1]; f->plane64[2] = nrm[2]; f->plane64[3] = d;
        for (int a = 0; a < 3; a++) f->plane[a] = (float)nrm[a];
        f->plane[3] = (float)d;
        if (prm->plane3) {   /* the fitted plane as Eq. 3's coefficients store it */
            orc_plane_to3(f->plane, &f->axis, f->coef);
            orc_plane_from3(f->axis, f->coef, f->plane);
        }
        if (lam[1] >= 0.999e-12 * lam[2] && lam[1] <= 1.001e-12 * lam[2]) f->borderline = 1;
        if (!(lam[1] > 1e-12 * lam[2])) { f->degenerate = 1; nI = 0; break; }
        nI = inliers(tp, f->plane, prm->fit_thr_m, I, &f->borderline);
        int same = (nI == nS);
        for (int k = 0; k < tp->n && same; k++) same = (I[k] == S[k]);
        if (same || f->rounds == prm->max_refits + 1 || nI < 3) break;
        memcpy(S, I, sizeof(int) * tp->n);
        nS = nI;
    }
    f->n_inlier = nI;
    if (!f->degenerate && nI >= need_inliers(prm, tp->n_valid)) f->status = ORC_FIT_OK;
}

static int params_ok(const orc_sensor *s, const orc_params *p) {
    return sensor_ok(s) && p && p->tile_h >= 1 && p->tile_w >= 1 &&
           p->tile_h * p->tile_w <= MAX_TILE_PX && p->tile_h <= 255 && p->tile_w <= 255 &&
           p->fit_thr_m >= 0 && p->quant_m > 0 && p->max_refits >= 0 && p->min_inlier_frac >= 0 &&
           p->temporal_candidates >= 0 && p->temporal_candidates <= 4 && p->temporal_runs >= 0 &&
           p->temporal_runs <= 1 && p->plane3 >= 0 && p->plane3 <= 1;
}

int orc_fit_tiles(const orc_sensor *s, const orc_params *prm, const float *range, orc_tile_fit *out) {
    if (!params_ok(s, prm)) return ORC_ERR_ARG;
    tables_t T;
    tables_make(s, &T);
    const int TW = (s->cols + prm->tile_w - 1) / prm->tile_w;
    const int TH = (s->rows + prm->tile_h - 1) / prm->tile_h;
    tile_px_t *tp = malloc(sizeof(tile_px_t));
    for (int t = 0; t < TW * TH; t++) {
        tile_gather(s, prm, &T, range, t, tp);
        fit_one(prm, tp, &out[t]);
    }
    free(tp);
    tables_free(&T);
    return ORC_OK;
}

int orc_fit_tiles_seeded(const orc_sensor *s, const orc_params *prm, const float *range, const float *prop,
                         float skip_logit, orc_tile_fit *out) {
    if (!params_ok(s, prm) || !prop) return ORC_ERR_ARG;
    tables_t T;
    tables_make(s, &T);
    const int TW = (s->cols + prm->tile_w - 1) / prm->tile_w;
    const int TH = (s->rows + prm->tile_h - 1) / prm->tile_h;
    tile_px_t *tp = malloc(sizeof(tile_px_t));
    for (int t = 0; t < TW * TH; t++) {
        tile_gather(s, prm, &T, range, t, tp);
        fit_one_seeded(prm, tp, prop + 5 * (size_t)t, skip_logit, &out[t]);
    }
    free(tp);
    tables_free(&T);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Temporal test (Sec. III-D, Eq. 6)                                         */
/* ------------------------------------------------------------------------ */

/* n' = R^T n: a K-frame plane seen in P-frame coordinates (the P frame maps to
 * K by p_K = R p + T, Eq. 6), fp64 with a fixed operation order, rounded. */
static void rotate_normal(const double M[16], const float n[3], float out[3]) {
    for (int j = 0; j < 3; j++) {
        double t = M[0 * 4 + j] * (double)n[0];
        t = fma(M[1 * 4 + j], (double)n[1], t);
        t = fma(M[2 * 4 + j], (double)n[2], t);
        out[j] = (float)t;
    }
}

/* Eq. 6: p' = R p + T in fp64, rounded to fp32. */
static void transform_point(const double M[16], const float p[3], float out[3]) {
    for (int i = 0; i < 3; i++) {
        double t = M[i * 4 + 0] * (double)p[0];
        t = fma(M[i * 4 + 1], (double)p[1], t);
        t = fma(M[i * 4 + 2], (double)p[2], t);
        out[i] = (float)(t + M[i * 4 + 3]);
    }
}

/*
 * Relaxed-plane test of Sec. III-D.  Reading: the P frame stays in its own
 * coordinates and the K plane is moved instead (same test, no resampling).
 * The K tile is the one the tile's anchor (first valid pixel in raster order)
 * falls in after Eq. 6 and Eq. 1-2.  The normal n' is held fixed and only the
 * offset c' is refit as the mean of n'.p over the current set, with the same
 * drop-and-refit rounds and acceptance rule as the spatial fit.  With several
 * candidates the test runs against the distinct K tiles the tile's valid
 * pixels fall in, in raster order from the anchor's (K tiles without a plane
 * are skipped), until one passes; the record holds the passing test, or the
 * last one run, with the borderline flag of all of them.
 */
int orc_temporal_tiles(const orc_sensor *s, const orc_params *prm, const float *range,
                       const float *kf_table, const double pose[16], orc_tile_temporal *out) {
    if (!params_ok(s, prm) || !kf_table || !pose) return ORC_ERR_ARG;
    tables_t T;
    tables_make(s, &T);
    const int TW = (s->cols + prm->tile_w - 1) / prm->tile_w;
    const int TH = (s->rows + prm->tile_h - 1) / prm->tile_h;
    tile_px_t *tp = malloc(sizeof(tile_px_t));
    int S[MAX_TILE_PX], I[MAX_TILE_PX];
    for (int t = 0; t < TW * TH; t++) {
        orc_tile_temporal *o = &out[t];
        memset(o, 0, sizeof(*o));
        o->kref = -1;
        tile_gather(s, prm, &T, range, t, tp);
        o->n_valid = tp->n_valid;
        if (tp->n_valid == 0) continue;
        int a = 0;
        while (!tp->valid[a]) a++;
        /* candidate K tiles: those of the valid pixels (Eq. 6, then Eq. 1-2), distinct, in raster
         * order from the anchor's; none if the anchor falls outside the key frame's image */
        const int ncand_max = prm->temporal_candidates > 1 ? prm->temporal_candidates : 1;
        int cand[4], ncand = 0, tested = 0, border = 0;
        for (int k = a; k < tp->n && ncand < ncand_max; k++) {
            if (!tp->valid[k]) continue;
            float aK[3];
            transform_point(pose, tp->p[k], aK);
            float rK;
            int pixK;
            if (bin_point(s, &T, aK[0], aK[1], aK[2], &rK, &pixK) != 0) {
                if (k == a) break;
                continue;
            }
            const int kt = (pixK / s->cols / prm->tile_h) * TW + (pixK % s->cols) / prm->tile_w;
            int seen = 0;
            for (int q = 0; q < ncand; q++) seen |= cand[q] == kt;
            if (seen) continue;
            cand[ncand++] = kt;
            const float *kp = &kf_table[4 * kt];
            if (kp[0] == 0.0f && kp[1] == 0.0f && kp[2] == 0.0f) continue;
            /* the relaxed-plane test against this K tile; the record keeps the last one tested,
             * or the first that passes */
            tested = 1;
            o->kref = kt;
            o->status = 1;
            o->rounds = 0;
            o->borderline = 0;
            rotate_normal(pose, kp, o->plane);
            for (int q = 0; q < tp->n; q++) S[q] = tp->valid[q];
            int nS = tp->n_valid, nI = 0;
            for (;;) {
                double sum = 0.0;
                for (int q = 0; q < tp->n; q++) {
                    if (!S[q]) continue;
                    double dp = (double)o->plane[0] * (double)tp->p[q][0];
                    dp = fma((double)o->plane[1], (double)tp->p[q][1], dp);
                    dp = fma((double)o->plane[2], (double)tp->p[q][2], dp);
                    sum += dp;
                }
                o->plane[3] = (float)(sum / nS);
                o->rounds++;
                nI = inliers(tp, o->plane, prm->fit_thr_m, I, &o->borderline);
                int same = (nI == nS);
                for (int q = 0; q < tp->n && same; q++) same = (I[q] == S[q]);
                if (same || o->rounds == prm->max_refits + 1 || nI < 3) break;
                memcpy(S, I, sizeof(int) * tp->n);
                nS = nI;
            }
            border |= o->borderline;
            o->n_inlier = nI;
            if (tp->n_valid >= 3 && nI >= need_inliers(prm, tp->n_valid)) {
                o->status = 2;
                break;
            }
        }
        (void)tested;
        o->borderline = border;
    }
    free(tp);
    tables_free(&T);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Stream layout                                                             */
/* ------------------------------------------------------------------------ */

/* Residual codes: k = round-half-away(e / q), |k| <= k_max, stored as k + k_max.
 * Raw codes: m = round-half-away(r / q) <= m_max.  Widths in bits. */
static void code_widths(const orc_sensor *s, const orc_params *prm, int *k_max, int *w_res, int *w_raw) {
    *k_max = (int)floorf(prm->fit_thr_m / prm->quant_m + 0.5f) + 1;
    int w = 1;
    while ((1 << w) < 2 * *k_max + 1) w++;
    *w_res = w;
    int m_max = (int)floorf((float)s->max_range_m / prm->quant_m + 0.5f) + 1;
    w = 1;
    while ((1 << w) < m_max + 1) w++;
    *w_raw = prm->raw_exact ? 32 : w;   /* lossless raw pixels: the range's fp32 bits */
}

static int quant_res(float e, float q) {
    float k = floorf(fabsf(e) / q + 0.5f);
    return (e < 0.0f) ? -(int)k : (int)k;
}

static int quant_raw(float r, float q) { return (int)floorf(r / q + 0.5f); }

static void put_bits(uint32_t *words, uint64_t bitpos, uint32_t value, int width) {
    for (int k = 0; k < width; k++)
        if ((value >> k) & 1u) words[(bitpos + k) >> 5] |= 1u << ((bitpos + k) & 31);
}

static uint32_t get_bits(const uint32_t *words, uint64_t bitpos, int width) {
    uint32_t v = 0;
    for (int k = 0; k < width; k++)
        v |= ((words[(bitpos + k) >> 5] >> ((bitpos + k) & 31)) & 1u) << k;
    return v;
}

static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint64_t words_for(uint64_t bits) { return (bits + 31) / 32; }

typedef struct {
    uint32_t kind, flags, rows, cols, tile_h, tile_w, w_res, w_raw;
    float thr, q;
    uint32_t n_tiles, n_valid, n_runs, n_temporal, n_cand, n_fitted, n_raw;
    int32_t k_max;
    uint32_t total_bytes;
} header_t;

/* Section word offsets after the header: bitmap, tile codes (4 bits/tile),
 * run planes (4 words each), temporal records (2 words each), fitted bits,
 * residual codes, raw codes. */
static void section_offsets(const header_t *h, uint64_t off[8]) {
    off[0] = 0;
    off[1] = off[0] + words_for((uint64_t)h->rows * h->cols);
    off[2] = off[1] + words_for((uint64_t)h->n_tiles * 4);
    off[3] = off[2] + ((h->flags & 16u) ? 3ull : 4ull) * h->n_runs;
    off[4] = off[3] + 2ull * h->n_temporal;
    off[5] = off[4] + words_for(h->n_cand);
    off[6] = off[5] + ((h->flags & 2u) ? 0 : words_for((uint64_t)h->n_fitted * h->w_res));   /* no deltas */
    off[7] = off[6] + words_for((uint64_t)h->n_raw * h->w_raw);
}

static void wr32(uint8_t *b, uint32_t v) { b[0] = v; b[1] = v >> 8; b[2] = v >> 16; b[3] = v >> 24; }
static void wr16(uint8_t *b, uint32_t v) { b[0] = v; b[1] = v >> 8; }
static uint32_t rd32(const uint8_t *b) { return b[0] | (b[1] << 8) | (b[2] << 16) | ((uint32_t)b[3] << 24); }
static uint32_t rd16(const uint8_t *b) { return b[0] | (b[1] << 8); }

static void header_write(uint8_t *b, const header_t *h) {
    memset(b, 0, HEADER_BYTES);
    wr32(b + 0, STREAM_MAGIC);
    wr16(b + 4, STREAM_VERSION);
    b[6] = (uint8_t)h->kind;
    b[7] = (uint8_t)h->flags;
    wr16(b + 8, h->rows);
    wr16(b + 10, h->cols);
    b[12] = (uint8_t)h->tile_h;
    b[13] = (uint8_t)h->tile_w;
    b[14] = (uint8_t)h->w_res;
    b[15] = (uint8_t)h->w_raw;
    wr32(b + 16, f2u(h->thr));
    wr32(b + 20, f2u(h->q));
    wr32(b + 24, h->n_tiles);
    wr32(b + 28, h->n_valid);
    wr32(b + 32, h->n_runs);
    wr32(b + 36, h->n_temporal);
    wr32(b + 40, h->n_cand);
    wr32(b + 44, h->n_fitted);
    wr32(b + 48, h->n_raw);
    wr32(b + 52, (uint32_t)h->k_max);
    wr32(b + 56, h->total_bytes);
}

static int header_read(const uint8_t *b, uint64_t nbytes, header_t *h) {
    if (nbytes < HEADER_BYTES) return ORC_ERR_CORRUPT;
    if (rd32(b) != STREAM_MAGIC || rd16(b + 4) != STREAM_VERSION) return ORC_ERR_CORRUPT;
    h->kind = b[6];
    h->flags = b[7];
    h->rows = rd16(b + 8);
    h->cols = rd16(b + 10);
    h->tile_h = b[12];
    h->tile_w = b[13];
    h->w_res = b[14];
    h->w_raw = b[15];
    h->thr = u2f(rd32(b + 16));
    h->q = u2f(rd32(b + 20));
    h->n_tiles = rd32(b + 24);
    h->n_valid = rd32(b + 28);
    h->n_runs = rd32(b + 32);
    h->n_temporal = rd32(b + 36);
    h->n_cand = rd32(b + 40);
    h->n_fitted = rd32(b + 44);
    h->n_raw = rd32(b + 48);
    h->k_max = (int32_t)rd32(b + 52);
    h->total_bytes = rd32(b + 56);
    if (h->kind > 1 || (h->flags & ~31u) || ((h->flags & 8u) && h->kind != 1) || h->tile_h == 0 || h->tile_w == 0 || h->w_res == 0 || h->w_res > 16 ||
        h->w_raw == 0 || ((h->flags & 4u) ? h->w_raw != 32 : h->w_raw > 24) || !(h->q > 0))
        return ORC_ERR_CORRUPT;
    uint64_t off[8];
    section_offsets(h, off);
    if (h->total_bytes != HEADER_BYTES + 4 * off[7] || h->total_bytes > nbytes) return ORC_ERR_CORRUPT;
    return ORC_OK;
}

/* Does a tile pass the acceptance rule against a plane (run growth, Sec. III-C)? */
static int tile_passes(const orc_params *prm, const tile_px_t *tp, const float pl[4]) {
    int I[MAX_TILE_PX];
    if (tp->n_valid < 3) return 0;
    return inliers(tp, pl, prm->fit_thr_m, I, NULL) >= need_inliers(prm, tp->n_valid);
}

/*
 * Greedy horizontal run growth (Sec. III-C): a run starts at a tile whose own
 * fit succeeded and takes that plane; the next tile to the right joins while it
 * passes the acceptance rule against the run's plane (the plane "fit so far" is
 * not refit); on failure the process restarts at the failing tile.  In a P
 * frame the tiles that passed the relaxed-plane test are coded first
 * (Sec. III-D): each ends any spatial run before it, and with temporal_runs it
 * starts a temporal run that grows to the right by the same rule against its
 * relaxed plane (n', c'), over any tile that passes it; the tiles left over are
 * then coded spatially.  One left-to-right walk gives both: temporal runs take
 * every tile they reach, and spatial runs never cross a temporal tile.  Then
 * each valid pixel, in canonical order (tiles row-major, raster inside a tile),
 * is coded against its tile's plane: fitted bit + residual code if it passes
 * the threshold, raw range code otherwise; pixels of raw tiles get raw codes.
 */
int64_t orc_pack(const orc_sensor *s, const orc_params *prm, int kind, const float *range,
                 const float *fit_plane, const uint8_t *fit_ok,
                 const float *temporal_plane, const int32_t *temporal_kref,
                 uint8_t *out, uint64_t cap, float *kf_table_out, uint8_t *modes_out) {
    return orc_pack3(s, prm, kind, range, fit_plane, NULL, fit_ok, temporal_plane, temporal_kref, out, cap,
                     kf_table_out, modes_out);
}

int64_t orc_pack3(const orc_sensor *s, const orc_params *prm, int kind, const float *range,
                  const float *fit_plane, const float *fit_coef, const uint8_t *fit_ok,
                  const float *temporal_plane, const int32_t *temporal_kref,
                  uint8_t *out, uint64_t cap, float *kf_table_out, uint8_t *modes_out) {
    if (!params_ok(s, prm) || (kind != 0 && kind != 1) || (prm->plane3 && !fit_coef)) return ORC_ERR_ARG;
    tables_t T;
    tables_make(s, &T);
    const int TW = (s->cols + prm->tile_w - 1) / prm->tile_w;
    const int TH = (s->rows + prm->tile_h - 1) / prm->tile_h;
    const int NT = TW * TH;
    uint8_t *mode = calloc(NT, 1);
    float *cp = calloc((size_t)NT * 4, sizeof(float));
    tile_px_t *tp = malloc(sizeof(tile_px_t));
    int64_t ret = 0;
    header_t h;
    memset(&h, 0, sizeof(h));
    int k_max, w_res, w_raw;
    code_widths(s, prm, &k_max, &w_res, &w_raw);

    /* 1. tile modes and coding planes */
    for (int tr = 0; tr < TH && ret == 0; tr++) {
        int j = 0;
        while (j < TW) {
            int t = tr * TW + j;
            tile_gather(s, prm, &T, range, t, tp);
            if (temporal_kref && temporal_kref[t] >= 0) {
                mode[t] = ORC_T_TEMPORAL;
                memcpy(&cp[4 * t], &temporal_plane[4 * t], 16);
                if (!tile_passes(prm, tp, &cp[4 * t])) ret = ORC_ERR_INCONSISTENT;
                int k = j + 1;
                while (prm->merge_runs && prm->temporal_runs && k < TW) {
                    int t2 = tr * TW + k;
                    tile_gather(s, prm, &T, range, t2, tp);
                    if (!tile_passes(prm, tp, &cp[4 * t])) break;
                    mode[t2] = ORC_T_TEMPORAL_CONT;
                    memcpy(&cp[4 * t2], &cp[4 * t], 16);
                    k++;
                }
                j = k;
                continue;
            }
            if (!fit_ok[t]) {
                mode[t] = tp->n_valid ? ORC_T_RAW : ORC_T_EMPTY;
                j++;
                continue;
            }
            mode[t] = ORC_T_RUN_START;
            memcpy(&cp[4 * t], &fit_plane[4 * t], 16);
            if (!tile_passes(prm, tp, &cp[4 * t])) ret = ORC_ERR_INCONSISTENT;
            if (prm->plane3) {   /* the run record holds the coefficients: they must give this plane */
                float back[4];
                orc_plane_from3((int)fit_coef[4 * t + 3], &fit_coef[4 * t], back);
                if (memcmp(back, &cp[4 * t], 16) != 0 || fit_coef[4 * t + 3] < 0.0f || fit_coef[4 * t + 3] > 2.0f)
                    ret = ORC_ERR_INCONSISTENT;
            }
            int k = j + 1;
            while (prm->merge_runs && k < TW) {
                int t2 = tr * TW + k;
                if (temporal_kref && temporal_kref[t2] >= 0) break;
                tile_gather(s, prm, &T, range, t2, tp);
                if (!tile_passes(prm, tp, &cp[4 * t])) break;
                mode[t2] = ORC_T_RUN_CONT;
                memcpy(&cp[4 * t2], &cp[4 * t], 16);
                k++;
            }
            j = k;
        }
    }
    if (ret != 0) goto done;

    /* 2. counts */
    h.kind = kind;
    h.flags = (prm->merge_runs ? 1u : 0u) | (prm->no_delta ? 2u : 0u) | (prm->raw_exact ? 4u : 0u) |
              (kind == 1 && prm->merge_runs && prm->temporal_runs ? 8u : 0u) | (prm->plane3 ? 16u : 0u);
    h.rows = s->rows;
    h.cols = s->cols;
    h.tile_h = prm->tile_h;
    h.tile_w = prm->tile_w;
    h.w_res = w_res;
    h.w_raw = w_raw;
    h.thr = prm->fit_thr_m;
    h.q = prm->quant_m;
    h.n_tiles = NT;
    h.k_max = k_max;
    for (int t = 0; t < NT; t++) {
        tile_gather(s, prm, &T, range, t, tp);
        h.n_valid += tp->n_valid;
        h.n_runs += (mode[t] == ORC_T_RUN_START);
        h.n_temporal += (mode[t] == ORC_T_TEMPORAL);
        int coded = mode[t] >= ORC_T_RUN_START;
        for (int k = 0; k < tp->n; k++) {
            if (!tp->valid[k]) continue;
            if (coded) {
                float e;
                h.n_cand++;
                if (residual(&cp[4 * t], tp->u[k], tp->r[k], prm->fit_thr_m, &e)) h.n_fitted++;
                else h.n_raw++;
            } else {
                h.n_raw++;
            }
        }
    }
    uint64_t off[8];
    section_offsets(&h, off);
    h.total_bytes = (uint32_t)(HEADER_BYTES + 4 * off[7]);
    ret = h.total_bytes;
    if (kf_table_out)
        for (int t = 0; t < NT; t++) {
            int plane = mode[t] == ORC_T_RUN_START || mode[t] == ORC_T_RUN_CONT;
            for (int a = 0; a < 4; a++) kf_table_out[4 * t + a] = plane ? cp[4 * t + a] : 0.0f;
        }
    if (modes_out) memcpy(modes_out, mode, NT);
    if (!out || h.total_bytes > cap) goto done;

    /* 3. streams */
    {
        uint32_t *w = calloc(off[7] + 1, sizeof(uint32_t));
        for (int64_t p = 0; p < (int64_t)s->rows * s->cols; p++)
            if (range[p] > 0.0f) put_bits(w + off[0], (uint64_t)p, 1, 1);
        for (int t = 0; t < NT; t++) {   /* plane3: a run start's code names its dominant axis */
            const uint32_t code = (prm->plane3 && mode[t] == ORC_T_RUN_START)
                                      ? ORC_T_RUN_START3 + (uint32_t)fit_coef[4 * t + 3] : mode[t];
            put_bits(w + off[1], (uint64_t)t * 4, code, 4);
        }
        uint64_t ir = 0, itp = 0, ic = 0, ifit = 0, iraw = 0;
        for (int t = 0; t < NT; t++) {
            if (mode[t] == ORC_T_RUN_START) {
                if (prm->plane3) {   /* Eq. 3's coefficients; the axis is in the tile code */
                    for (int a = 0; a < 3; a++) w[off[2] + 3 * ir + a] = f2u(fit_coef[4 * t + a]);
                } else {
                    for (int a = 0; a < 4; a++) w[off[2] + 4 * ir + a] = f2u(cp[4 * t + a]);
                }
                ir++;
            }
            if (mode[t] == ORC_T_TEMPORAL) {
                w[off[3] + 2 * itp] = (uint32_t)temporal_kref[t];
                w[off[3] + 2 * itp + 1] = f2u(cp[4 * t + 3]);
                itp++;
            }
            tile_gather(s, prm, &T, range, t, tp);
            int coded = mode[t] >= ORC_T_RUN_START;
            for (int k = 0; k < tp->n; k++) {
                if (!tp->valid[k]) continue;
                float e;
                int in = coded && residual(&cp[4 * t], tp->u[k], tp->r[k], prm->fit_thr_m, &e);
                if (coded) put_bits(w + off[4], ic++, (uint32_t)in, 1);
                if (in) {
                    /* with deltas the residual code follows; without, the point is the plane's */
                    if (!prm->no_delta)
                        put_bits(w + off[5], ifit * w_res, (uint32_t)(quant_res(e, prm->quant_m) + k_max), w_res);
                    ifit++;
                } else {
                    put_bits(w + off[6], iraw * w_raw,
                             prm->raw_exact ? f2u(tp->r[k]) : (uint32_t)quant_raw(tp->r[k], prm->quant_m), w_raw);
                    iraw++;
                }
            }
        }
        header_write(out, &h);
        for (uint64_t i = 0; i < off[7]; i++) wr32(out + HEADER_BYTES + 4 * i, w[i]);
        free(w);
    }
done:
    free(tp);
    free(mode);
    free(cp);
    tables_free(&T);
    return ret;
}

/* ------------------------------------------------------------------------ */
/* Whole-frame encoders                                                      */
/* ------------------------------------------------------------------------ */

int64_t orc_encode_keyframe(const orc_sensor *s, const orc_params *prm, const float *pts, int64_t n,
                            uint8_t *out, uint64_t cap, float *kf_table_out,
                            orc_tile_fit *fits_out, uint8_t *modes_out) {
    if (!params_ok(s, prm)) return ORC_ERR_ARG;
    const int TW = (s->cols + prm->tile_w - 1) / prm->tile_w;
    const int TH = (s->rows + prm->tile_h - 1) / prm->tile_h;
    const int NT = TW * TH;
    float *range = malloc(sizeof(float) * (size_t)s->rows * s->cols);
    orc_tile_fit *fits = malloc(sizeof(orc_tile_fit) * NT);
    float *planes = malloc(sizeof(float) * 4 * NT);
    uint8_t *ok = malloc(NT);
    float *coef = malloc(sizeof(float) * 4 * NT);
    orc_range_image(s, pts, n, range, NULL, NULL);
    orc_fit_tiles(s, prm, range, fits);
    for (int t = 0; t < NT; t++) {
        memcpy(&planes[4 * t], fits[t].plane, 16);
        memcpy(&coef[4 * t], fits[t].coef, 12);
        coef[4 * t + 3] = (float)fits[t].axis;
        ok[t] = fits[t].status == ORC_FIT_OK;
    }
    int64_t r = orc_pack3(s, prm, 0, range, planes, coef, ok, NULL, NULL, out, cap, kf_table_out, modes_out);
    free(coef);
    if (fits_out) memcpy(fits_out, fits, sizeof(orc_tile_fit) * NT);
    free(range); free(fits); free(planes); free(ok);
    return r;
}

/* Sec. III-D: temporal test first; the tiles left over (the image I') are
 * spatially encoded exactly as a key frame. */
int64_t orc_encode_pframe(const orc_sensor *s, const orc_params *prm, const float *kf_table,
                          const double pose[16], const float *pts, int64_t n,
                          uint8_t *out, uint64_t cap, orc_tile_fit *fits_out,
                          orc_tile_temporal *temporal_out, uint8_t *modes_out) {
    if (!params_ok(s, prm) || !kf_table || !pose) return ORC_ERR_ARG;
    const int TW = (s->cols + prm->tile_w - 1) / prm->tile_w;
    const int TH = (s->rows + prm->tile_h - 1) / prm->tile_h;
    const int NT = TW * TH;
    float *range = malloc(sizeof(float) * (size_t)s->rows * s->cols);
    orc_tile_fit *fits = malloc(sizeof(orc_tile_fit) * NT);
    orc_tile_temporal *tmp = malloc(sizeof(orc_tile_temporal) * NT);
    float *planes = malloc(sizeof(float) * 4 * NT);
    float *tplanes = malloc(sizeof(float) * 4 * NT);
    int32_t *kref = malloc(sizeof(int32_t) * NT);
    uint8_t *ok = malloc(NT);
    float *coef = malloc(sizeof(float) * 4 * NT);
    orc_range_image(s, pts, n, range, NULL, NULL);
    orc_temporal_tiles(s, prm, range, kf_table, pose, tmp);
    orc_fit_tiles(s, prm, range, fits);
    for (int t = 0; t < NT; t++) {
        memcpy(&planes[4 * t], fits[t].plane, 16);
        memcpy(&coef[4 * t], fits[t].coef, 12);
        coef[4 * t + 3] = (float)fits[t].axis;
        memcpy(&tplanes[4 * t], tmp[t].plane, 16);
        kref[t] = (tmp[t].status == 2) ? tmp[t].kref : -1;
        ok[t] = fits[t].status == ORC_FIT_OK;
    }
    int64_t r = orc_pack3(s, prm, 1, range, planes, coef, ok, tplanes, kref, out, cap, NULL, modes_out);
    free(coef);
    if (fits_out) memcpy(fits_out, fits, sizeof(orc_tile_fit) * NT);
    if (temporal_out) memcpy(temporal_out, tmp, sizeof(orc_tile_temporal) * NT);
    free(range); free(fits); free(tmp); free(planes); free(tplanes); free(kref); free(ok);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Decoder (ray casting, Sec. III-C)                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    header_t h;
    const uint32_t *w; /* section words (host copy) */
    uint64_t off[8];
    uint32_t *copy;
} stream_t;

static int stream_open(const orc_sensor *s, const uint8_t *bits, uint64_t nbytes, stream_t *st) {
    memset(st, 0, sizeof(*st));
    int r = header_read(bits, nbytes, &st->h);
    if (r != ORC_OK) return r;
    const int TW = (s->cols + st->h.tile_w - 1) / st->h.tile_w;
    const int TH = (s->rows + st->h.tile_h - 1) / st->h.tile_h;
    if ((int)st->h.rows != s->rows || (int)st->h.cols != s->cols || (int)st->h.n_tiles != TW * TH)
        return ORC_ERR_CORRUPT;
    section_offsets(&st->h, st->off);
    st->copy = malloc(sizeof(uint32_t) * (st->off[7] + 1));
    for (uint64_t i = 0; i < st->off[7]; i++) st->copy[i] = rd32(bits + HEADER_BYTES + 4 * i);
    st->w = st->copy;
    return ORC_OK;
}

/* Walk the tile codes and assign each plane-coded tile its coding plane. */
static int stream_planes(const orc_sensor *s, const stream_t *st, const float *kf_table,
                         const double pose[16], float *cp, uint8_t *mode) {
    const int TW = (s->cols + st->h.tile_w - 1) / st->h.tile_w;
    const int NT = st->h.n_tiles;
    uint64_t ir = 0, itp = 0;
    for (int t = 0; t < NT; t++) {
        mode[t] = (uint8_t)get_bits(st->w + st->off[1], (uint64_t)t * 4, 4);
        int axis = -1;
        if (mode[t] >= ORC_T_RUN_START3 && mode[t] < ORC_T_RUN_START3 + 3) {
            if (!(st->h.flags & 16u)) return ORC_ERR_CORRUPT;
            axis = mode[t] - ORC_T_RUN_START3;
            mode[t] = ORC_T_RUN_START;
        } else if (mode[t] == ORC_T_RUN_START && (st->h.flags & 16u)) {
            return ORC_ERR_CORRUPT;   /* a 3-coefficient stream names every run start's axis */
        }
        switch (mode[t]) {
        case ORC_T_EMPTY:
        case ORC_T_RAW:
            break;
        case ORC_T_RUN_START:
            if (ir >= st->h.n_runs) return ORC_ERR_CORRUPT;
            if (st->h.flags & 16u) {   /* Eq. 3's coefficients along the tile code's axis */
                float abc[3];
                for (int a = 0; a < 3; a++) abc[a] = u2f(st->w[st->off[2] + 3 * ir + a]);
                orc_plane_from3(axis, abc, &cp[4 * t]);
            } else {
                for (int a = 0; a < 4; a++) cp[4 * t + a] = u2f(st->w[st->off[2] + 4 * ir + a]);
            }
            ir++;
            break;
        case ORC_T_RUN_CONT:
            if (t % TW == 0 || (mode[t - 1] != ORC_T_RUN_START && mode[t - 1] != ORC_T_RUN_CONT))
                return ORC_ERR_CORRUPT;
            memcpy(&cp[4 * t], &cp[4 * (t - 1)], 16);
            break;
        case ORC_T_TEMPORAL_CONT:
            /* continues the temporal run to its left (flags bit 3): the run start's plane */
            if (!(st->h.flags & 8u) || t % TW == 0 ||
                (mode[t - 1] != ORC_T_TEMPORAL && mode[t - 1] != ORC_T_TEMPORAL_CONT))
                return ORC_ERR_CORRUPT;
            memcpy(&cp[4 * t], &cp[4 * (t - 1)], 16);
            break;
        case ORC_T_TEMPORAL: {
            if (st->h.kind != 1 || !kf_table || !pose || itp >= st->h.n_temporal) return ORC_ERR_CORRUPT;
            uint32_t kref = st->w[st->off[3] + 2 * itp];
            float c = u2f(st->w[st->off[3] + 2 * itp + 1]);
            itp++;
            if (kref >= (uint32_t)NT) return ORC_ERR_CORRUPT;
            const float *kp = &kf_table[4 * kref];
            if (kp[0] == 0.0f && kp[1] == 0.0f && kp[2] == 0.0f) return ORC_ERR_CORRUPT;
            rotate_normal(pose, kp, &cp[4 * t]);
            cp[4 * t + 3] = c;
            break;
        }
        default:
            return ORC_ERR_CORRUPT;
        }
    }
    if (ir != st->h.n_runs || itp != st->h.n_temporal) return ORC_ERR_CORRUPT;
    return ORC_OK;
}

int orc_kf_table_from_stream(const orc_sensor *s, const uint8_t *bits, uint64_t nbytes, float *kf_table) {
    stream_t st;
    int r = stream_open(s, bits, nbytes, &st);
    if (r != ORC_OK) { free(st.copy); return r; }
    if (st.h.kind != 0) { free(st.copy); return ORC_ERR_CORRUPT; }
    const int NT = st.h.n_tiles;
    float *cp = calloc((size_t)NT * 4, sizeof(float));
    uint8_t *mode = calloc(NT, 1);
    r = stream_planes(s, &st, NULL, NULL, cp, mode);
    if (r == ORC_OK)
        for (int t = 0; t < NT; t++) {
            int plane = mode[t] == ORC_T_RUN_START || mode[t] == ORC_T_RUN_CONT;
            for (int a = 0; a < 4; a++) kf_table[4 * t + a] = plane ? cp[4 * t + a] : 0.0f;
        }
    free(cp); free(mode); free(st.copy);
    return r;
}

int orc_decode(const orc_sensor *s, const uint8_t *bits, uint64_t nbytes, const float *kf_table,
               const double pose[16], float *range, float *xyz4, uint32_t *valid) {
    stream_t st;
    int r = stream_open(s, bits, nbytes, &st);
    if (r != ORC_OK) { free(st.copy); return r; }
    tables_t T;
    tables_make(s, &T);
    const int NT = st.h.n_tiles;
    const int TW = (s->cols + st.h.tile_w - 1) / st.h.tile_w;
    const int64_t npx = (int64_t)s->rows * s->cols;
    float *cp = calloc((size_t)NT * 4, sizeof(float));
    uint8_t *mode = calloc(NT, 1);
    r = stream_planes(s, &st, kf_table, pose, cp, mode);
    if (r != ORC_OK) goto out;
    for (int64_t p = 0; p < npx; p++) {
        range[p] = 0.0f;
        if (xyz4) xyz4[4 * p] = xyz4[4 * p + 1] = xyz4[4 * p + 2] = xyz4[4 * p + 3] = 0.0f;
    }
    if (valid) memcpy(valid, st.w + st.off[0], sizeof(uint32_t) * words_for(npx));
    uint64_t ic = 0, ifit = 0, iraw = 0, nvalid = 0;
    for (int t = 0; t < NT && r == ORC_OK; t++) {
        const int tr = t / TW, tc = t % TW;
        const int coded = mode[t] >= ORC_T_RUN_START;
        for (int i = tr * st.h.tile_h; i < (tr + 1) * (int)st.h.tile_h && i < s->rows; i++)
            for (int j = tc * st.h.tile_w; j < (tc + 1) * (int)st.h.tile_w && j < s->cols; j++) {
                const int64_t p = (int64_t)i * s->cols + j;
                if (!get_bits(st.w + st.off[0], (uint64_t)p, 1)) continue;
                nvalid++;
                if (mode[t] == ORC_T_EMPTY) { r = ORC_ERR_CORRUPT; break; }
                float u[3];
                beam(&T, i, j, u);
                float rr;
                int fitted = 0;
                if (coded) {
                    if (ic >= st.h.n_cand) { r = ORC_ERR_CORRUPT; break; }
                    fitted = (int)get_bits(st.w + st.off[4], ic++, 1);
                }
                if (fitted) {
                    if (ifit >= st.h.n_fitted) { r = ORC_ERR_CORRUPT; break; }
                    int k = (st.h.flags & 2u) ? 0
                            : (int)get_bits(st.w + st.off[5], ifit * st.h.w_res, st.h.w_res) - st.h.k_max;
                    ifit++;
                    const float *pl = &cp[4 * t];
                    float dot = fmaf(pl[0], u[0], fmaf(pl[1], u[1], pl[2] * u[2]));
                    if (!(dot > 1e-3f)) { r = ORC_ERR_CORRUPT; break; }
                    rr = fmaf((float)k, st.h.q, pl[3] / dot);
                } else {
                    if (iraw >= st.h.n_raw) { r = ORC_ERR_CORRUPT; break; }
                    uint32_t m = get_bits(st.w + st.off[6], iraw * st.h.w_raw, st.h.w_raw);
                    iraw++;
                    rr = (st.h.flags & 4u) ? u2f(m) : (float)m * st.h.q;
                }
                range[p] = rr;
                if (xyz4) {
                    xyz4[4 * p] = rr * u[0];
                    xyz4[4 * p + 1] = rr * u[1];
                    xyz4[4 * p + 2] = rr * u[2];
                }
            }
    }
    if (r == ORC_OK && (ic != st.h.n_cand || ifit != st.h.n_fitted || iraw != st.h.n_raw ||
                        nvalid != st.h.n_valid))
        r = ORC_ERR_CORRUPT;
out:
    free(cp); free(mode); free(st.copy);
    tables_free(&T);
    return r;
}
