/*
 * Seeded synthetic LiDAR scenes and sequences (input generation only).
 *
 * This file simulates a spinning multi-beam LiDAR (HDL-64E-like geometry) by
 * ray casting against a procedural urban scene: a ground plane, axis-aligned
 * wall rectangles, car-sized boxes and thin vertical poles.  It holds none of
 * the compression method's arithmetic; both the CPU oracle and the GPU library
 * consume its output.  Every random draw comes from a counter-based hash of
 * (seed, stream, index), so output does not depend on thread count or order.
 *
 * Beam directions are placed at pixel centres of the sensor grid:
 *   elevation of row i  = elev_max - (i + 0.5) * (elev_max - elev_min) / rows
 *   azimuth of column j = -pi + (j + 0.5) * 2 pi / cols
 * (row 0 is the top beam), matching the range-image grid of Sec. III-B.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum { SYN_GROUND = 0, SYN_WALL_X = 1, SYN_WALL_Y = 2, SYN_BOX = 3, SYN_POLE = 4 };

/* One scene object.  Meaning of p[] by kind:
 *  GROUND : p0 = z of the plane
 *  WALL_X : plane x = p0, y in [p1,p2], z in [p3,p4]
 *  WALL_Y : plane y = p0, x in [p1,p2], z in [p3,p4]
 *  BOX    : x in [p0,p1], y in [p2,p3], z in [p4,p5]
 *  POLE   : centre (p0,p1), radius p2, z in [p3,p4]
 */
typedef struct {
    int32_t kind;
    int32_t pad;
    double p[6];
} syn_obj;

static uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Uniform double in [0,1) from (seed, stream, index). */
static double urand(uint64_t seed, uint64_t stream, uint64_t idx) {
    uint64_t h = mix64(seed ^ mix64(stream * 0x632BE59BD9B4E019ull + mix64(idx)));
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

/* Standard normal via Box-Muller on two counter-based uniforms. */
static double nrand(uint64_t seed, uint64_t stream, uint64_t idx) {
    double u1 = urand(seed, stream, 2 * idx);
    double u2 = urand(seed, stream, 2 * idx + 1);
    if (u1 < 1e-300) u1 = 1e-300;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/*
 * Build a scene.  Objects are scattered over a rectangle around a path that
 * runs along +x from x=0 to x=path_len (the ego trajectory of a sequence),
 * keeping a clear lane around y=0 for boxes and poles.  Walls are placed
 * 10-40 m from the path; with enclose != 0 the first four walls close a
 * courtyard around it.  Returns the object count.
 */
int syn_make_scene(uint64_t seed, int n_walls, int n_boxes, int n_poles,
                   double ground_z, double path_len, int enclose, syn_obj *out, int cap) {
    int n = 0;
    if (cap < 1) return -1;
    memset(out, 0, sizeof(syn_obj) * (size_t)cap);
    out[n].kind = SYN_GROUND;
    out[n].p[0] = ground_z;
    n++;
    int w0 = 0;
    if (enclose && n_walls >= 4) {
        /* four walls forming a closed courtyard around the path, 10-40 m away */
        for (int w = 0; w < 4 && n < cap; w++) {
            double dist = 10.0 + 30.0 * urand(seed, 10, (uint64_t)w);
            syn_obj *o = &out[n++];
            o->kind = (w < 2) ? SYN_WALL_X : SYN_WALL_Y;
            if (w == 0) o->p[0] = path_len + dist;
            if (w == 1) o->p[0] = -dist;
            if (w == 2) o->p[0] = dist;
            if (w == 3) o->p[0] = -dist;
            o->p[1] = -1e3;
            o->p[2] = 1e3;
            o->p[3] = ground_z;
            o->p[4] = ground_z + 30.0;
        }
        w0 = 4;
    }
    for (int w = w0; w < n_walls && n < cap; w++) {
        double u0 = urand(seed, 11, (uint64_t)w * 8 + 0);
        double u1 = urand(seed, 11, (uint64_t)w * 8 + 1);
        double u2 = urand(seed, 11, (uint64_t)w * 8 + 2);
        double u3 = urand(seed, 11, (uint64_t)w * 8 + 3);
        double u4 = urand(seed, 11, (uint64_t)w * 8 + 4);
        double dist = 10.0 + 30.0 * u1;
        double len = 8.0 + 30.0 * u2;
        double top = ground_z + 3.0 + 9.0 * u3;
        double side = (u4 < 0.5) ? -1.0 : 1.0;
        syn_obj *o = &out[n++];
        if (u0 < 0.6) {
            /* wall parallel to the path, at lateral distance dist */
            double xc = -40.0 + (path_len + 80.0) * urand(seed, 11, (uint64_t)w * 8 + 5);
            o->kind = SYN_WALL_Y;
            o->p[0] = side * dist;
            o->p[1] = xc - 0.5 * len;
            o->p[2] = xc + 0.5 * len;
        } else {
            /* wall across the path, ahead of or behind the trajectory */
            double yc = -30.0 + 60.0 * urand(seed, 11, (uint64_t)w * 8 + 5);
            o->kind = SYN_WALL_X;
            o->p[0] = (side > 0) ? (path_len + dist) : -dist;
            o->p[1] = yc - 0.5 * len;
            o->p[2] = yc + 0.5 * len;
        }
        o->p[3] = ground_z;
        o->p[4] = top;
    }
    for (int b = 0; b < n_boxes && n < cap; b++) {
        double u0 = urand(seed, 12, (uint64_t)b * 4 + 0);
        double u1 = urand(seed, 12, (uint64_t)b * 4 + 1);
        double u2 = urand(seed, 12, (uint64_t)b * 4 + 2);
        double xc = -35.0 + (path_len + 70.0) * u0;
        double yabs = 3.0 + 27.0 * u1;
        double yc = (u2 < 0.5) ? -yabs : yabs;
        int along = urand(seed, 12, (uint64_t)b * 4 + 3) < 0.7;
        double hx = along ? 2.25 : 0.9, hy = along ? 0.9 : 2.25;
        syn_obj *o = &out[n++];
        o->kind = SYN_BOX;
        o->p[0] = xc - hx; o->p[1] = xc + hx;
        o->p[2] = yc - hy; o->p[3] = yc + hy;
        o->p[4] = ground_z; o->p[5] = ground_z + 1.5;
    }
    for (int q = 0; q < n_poles && n < cap; q++) {
        double u0 = urand(seed, 13, (uint64_t)q * 4 + 0);
        double u1 = urand(seed, 13, (uint64_t)q * 4 + 1);
        double u2 = urand(seed, 13, (uint64_t)q * 4 + 2);
        double u3 = urand(seed, 13, (uint64_t)q * 4 + 3);
        double xc = -35.0 + (path_len + 70.0) * u0;
        double yabs = 2.5 + 27.5 * u1;
        syn_obj *o = &out[n++];
        o->kind = SYN_POLE;
        o->p[0] = xc;
        o->p[1] = (u2 < 0.5) ? -yabs : yabs;
        o->p[2] = 0.15;
        o->p[3] = ground_z;
        o->p[4] = ground_z + 3.0 + 3.0 * u3;
    }
    return n;
}

/* Ray (origin o, unit direction d) against one object: distance or +inf. */
static double hit_obj(const syn_obj *ob, const double o[3], const double d[3]) {
    const double INF = INFINITY;
    switch (ob->kind) {
    case SYN_GROUND: {
        if (d[2] >= -1e-12) return INF;
        double t = (ob->p[0] - o[2]) / d[2];
        return t > 0 ? t : INF;
    }
    case SYN_WALL_X:
    case SYN_WALL_Y: {
        int ax = (ob->kind == SYN_WALL_X) ? 0 : 1;
        int bx = 1 - ax;
        if (fabs(d[ax]) < 1e-12) return INF;
        double t = (ob->p[0] - o[ax]) / d[ax];
        if (t <= 0) return INF;
        double b = o[bx] + t * d[bx];
        double z = o[2] + t * d[2];
        if (b < ob->p[1] || b > ob->p[2] || z < ob->p[3] || z > ob->p[4]) return INF;
        return t;
    }
    case SYN_BOX: {
        double t0 = -INF, t1 = INF;
        for (int a = 0; a < 3; a++) {
            double lo = ob->p[2 * a], hi = ob->p[2 * a + 1];
            if (fabs(d[a]) < 1e-15) {
                if (o[a] < lo || o[a] > hi) return INF;
                continue;
            }
            double ta = (lo - o[a]) / d[a], tb = (hi - o[a]) / d[a];
            if (ta > tb) { double s = ta; ta = tb; tb = s; }
            if (ta > t0) t0 = ta;
            if (tb < t1) t1 = tb;
        }
        if (t1 < t0 || t1 <= 0) return INF;
        return t0 > 0 ? t0 : INF;
    }
    case SYN_POLE: {
        double ox = o[0] - ob->p[0], oy = o[1] - ob->p[1];
        double a = d[0] * d[0] + d[1] * d[1];
        if (a < 1e-18) return INF;
        double b = ox * d[0] + oy * d[1];
        double c = ox * ox + oy * oy - ob->p[2] * ob->p[2];
        double disc = b * b - a * c;
        if (disc < 0) return INF;
        double t = (-b - sqrt(disc)) / a;
        if (t <= 0) return INF;
        double z = o[2] + t * d[2];
        if (z < ob->p[3] || z > ob->p[4]) return INF;
        return t;
    }
    }
    return INF;
}

/*
 * Render one frame.  pose = sensor-to-world rotation R (row-major 3x3) and
 * translation t.  For every beam (row-major, ring by ring, the order of KITTI
 * scans) the nearest hit within [min_range, max_range] becomes one point
 * r * d_sensor with r = hit + N(0, sigma).  A beam is dropped with probability
 * dropout; with probability clutter its range is replaced by U(1, hit).
 * Writes float4 (x, y, z, 0) in sensor coordinates.  Returns the point count
 * (<= rows*cols) or -1 if cap is too small.
 */
int64_t syn_render(const syn_obj *objs, int n_obj, int rows, int cols,
                   double elev_min_deg, double elev_max_deg, double max_range,
                   const double R[9], const double t[3], double sigma,
                   double dropout, double clutter, uint64_t seed,
                   float *out_xyzw, int64_t cap) {
    const double deg = M_PI / 180.0;
    const double de = (elev_max_deg - elev_min_deg) / rows;
    const double da = 2.0 * M_PI / cols;
    const int64_t nbeam = (int64_t)rows * cols;
    if (cap < nbeam) return -1;
    int64_t n = 0;
    for (int i = 0; i < rows; i++) {
        double el = (elev_max_deg - (i + 0.5) * de) * deg;
        double ce = cos(el), se = sin(el);
        for (int j = 0; j < cols; j++) {
            uint64_t idx = (uint64_t)i * (uint64_t)cols + (uint64_t)j;
            if (dropout > 0 && urand(seed, 21, idx) < dropout) continue;
            double az = -M_PI + (j + 0.5) * da;
            double ds[3] = {ce * cos(az), ce * sin(az), se};
            double dw[3];
            for (int a = 0; a < 3; a++)
                dw[a] = R[3 * a + 0] * ds[0] + R[3 * a + 1] * ds[1] + R[3 * a + 2] * ds[2];
            double best = INFINITY;
            for (int k = 0; k < n_obj; k++) {
                double h = hit_obj(&objs[k], t, dw);
                if (h < best) best = h;
            }
            if (!(best <= max_range) || best < 0.5) continue;
            double r = best;
            if (clutter > 0 && urand(seed, 22, idx) < clutter)
                r = 1.0 + (best - 1.0) * urand(seed, 23, idx);
            if (sigma > 0) r += sigma * nrand(seed, 24, idx);
            if (!(r > 0.05) || r > max_range) continue;
            float *p = out_xyzw + 4 * n;
            p[0] = (float)(r * ds[0]);
            p[1] = (float)(r * ds[1]);
            p[2] = (float)(r * ds[2]);
            p[3] = 0.0f;
            n++;
        }
    }
    return n;
}
