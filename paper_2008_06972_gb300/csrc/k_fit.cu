// Per-tile plane fitting (Sec. III-C) and the relaxed-plane temporal test
// (Sec. III-D).
//
// First pass (k_fit_first): one thread owns one tile: it reads the tile's
// pixels from the range image (L2/L1), forms the points p = r * u_ij in fp32,
// and runs the fit itself, so every instruction of the plane solve carries up
// to 32 tiles.  Under the default schedule the pass runs one round; the few
// tiles that need more (5% on an HDL-64E frame) are queued and finish in one
// launch of k_fit_round with a group of lanes per tile, which splits each
// round's pixel work.  Both sum a tile's moments in the same order (pixel
// chunks summed left to right, FitLanes), so every schedule gives the same
// records.
//
// Spatial fit, per round: anchor-shifted moments q = p - a (a = the tile's
// first valid point) are accumulated in float-float (TwoSum / exact products),
// then the covariance is formed and the smallest eigenvector found (largest
// eigenpair by Newton + cross products, then an exact 2x2 Jacobi rotation in
// its orthogonal complement).  The solve runs in float-float on the FP32 pipes
// (ffmath.cuh, ~48-bit); params.solver = 1 selects the same method in FP64
// (solve_plane below), which GB300's FP64 latency makes ~10x slower per tile.
// The fp32 plane is tested on every valid pixel with the along-ray residual to
// give the next inlier set.
//
// Temporal test (P frames): the anchor is moved to key-frame coordinates
// (Eq. 6), binned (Eq. 1-2) into the key frame's grid, and the K tile's coding
// plane normal is rotated into P coordinates; the offset c' = mean(n'.p) is
// refit over the current set with the same rounds.  It runs before the
// spatial fit in the first pass (per thread), or after the spatial fits in
// k_temporal (a lane group per tile) when lcc_encode_sequence has fitted the P
// frames beside the key frame.
//
// Run pre-test (k_lookbehind): each tile tests itself against the planes of
// the fitted tiles to its left, so the run-growth walker rarely has to touch
// pixels.
#include <algorithm>

#include "ffmath.cuh"
#include "lcc_internal.cuh"

namespace lcc {

constexpr int kFitThreads = 128;

// FP64 reciprocal and reciprocal square root for the solver.  GB300 runs a
// dependent FP64 FMA in ~64 cycles but a correctly rounded FP64 division or
// square root in ~430-680 cycles, so these take the fp32 hardware estimate
// and refine it with Newton steps in FP64: relative error ~1e-15 (rcp64, two
// steps) and ~1.5e-14 (rsqrt64, one step), far below the fp32 rounding of
// the plane.  Arguments must be positive normal fp32 numbers after the cast.
__device__ __forceinline__ double rcp64(double x) {
    double y = (double)__frcp_rn((float)x);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

__device__ __forceinline__ double rsqrt64(double x) {
    const double y = (double)__frsqrt_rn((float)x);
    const double h = x * y;
    const double r = fma(-h, y, 1.0);   // 1 - x y^2
    return fma(0.5 * y, r, y);
}

// Scale a vector by roughly 1/max|v_i| so that its squared norm is fp32-safe.
__device__ __forceinline__ bool prescale(double &x, double &y, double &z) {
    const double m = fmax(fabs(x), fmax(fabs(y), fabs(z)));
    if (!(m > 1e-300)) return false;
    const double s = (double)__frcp_rn((float)fmin(fmax(m, 1e-30), 1e30));
    x *= s;
    y *= s;
    z *= s;
    return true;
}

// FP64 plane of the moments: returns true if the scatter matrix is degenerate.
//
// The smallest eigenvector of C is found without ever resolving the smallest
// eigenvalue from the characteristic polynomial (whose root is only accurate
// to eps*lambda_max^2/lambda_mid): the largest eigenpair is well conditioned,
// so lambda_max comes from Newton steps on det(C - l I) started above it from
// an fp32 trigonometric seed, and its eigenvector from the largest cross
// product of two rows of C - lambda_max I.  C is then projected onto the plane
// orthogonal to that vector and the 2x2 problem is solved by one exact Jacobi
// rotation, which gives lambda_min, lambda_mid and the normal with absolute
// accuracy ~eps*lambda_max, like a full Jacobi sweep.  The dependency chain is
// kept short (fixed Newton counts, no FP64 division or square root).
__device__ __noinline__ bool solve_plane(const double m1[3], const double m2[6], int n, float ax, float ay,
                                         float az, float4 &pl, float &ratio) {
    const double inv = rcp64((double)n);
    const double mx = m1[0] * inv, my = m1[1] * inv, mz = m1[2] * inv;
    const double cxx = fma(m2[0], inv, -mx * mx), cxy = fma(m2[1], inv, -mx * my), cxz = fma(m2[2], inv, -mx * mz);
    const double cyy = fma(m2[3], inv, -my * my), cyz = fma(m2[4], inv, -my * mz), czz = fma(m2[5], inv, -mz * mz);
    const double tr = cxx + cyy + czz;
    pl = make_float4(0.f, 0.f, 0.f, 0.f);
    ratio = 0.f;
    if (!(tr > 1e-30)) return true;
    // fp32 seed of the largest eigenvalue (trigonometric closed form)
    const float fxx = (float)cxx, fyy = (float)cyy, fzz = (float)czz;
    const float fxy = (float)cxy, fxz = (float)cxz, fyz = (float)cyz;
    const float q = (fxx + fyy + fzz) * (1.0f / 3.0f);
    const float p1 = fxy * fxy + fxz * fxz + fyz * fyz;
    const float dx = fxx - q, dy = fyy - q, dz = fzz - q;
    const float p2 = dx * dx + dy * dy + dz * dz + 2.0f * p1;
    float seed = q, spread = q;
    if (p2 > 0.0f) {
        const float pp = sqrtf(p2 * (1.0f / 6.0f));
        const float ip = 1.0f / pp;
        const float bxx = dx * ip, byy = dy * ip, bzz = dz * ip, bxy = fxy * ip, bxz = fxz * ip, byz = fyz * ip;
        const float detb = bxx * (byy * bzz - byz * byz) - bxy * (bxy * bzz - byz * bxz) + bxz * (bxy * byz - byy * bxz);
        const float rr = fminf(fmaxf(0.5f * detb, -1.0f), 1.0f);
        seed = q + 2.0f * pp * cosf(acosf(rr) * (1.0f / 3.0f));
        spread = pp;
    }
    // Newton on f(l) = det(C - l I) from above lambda_max: f is concave and
    // decreasing there, so the iterates fall onto the root; three steps take
    // the 3e-5 start offset to full precision (quadratic convergence).
    const double scale = (double)spread + 1e-30 * tr;
    double lam = (double)seed + 3e-5 * scale;
#pragma unroll
    for (int it = 0; it < 3; it++) {
        const double a = cxx - lam, b = cyy - lam, c = czz - lam;
        const double myz = fma(b, c, -cyz * cyz), mxz = fma(a, c, -cxz * cxz), mxy = fma(a, b, -cxy * cxy);
        const double det = fma(a, myz, fma(-cxy, fma(cxy, c, -cyz * cxz), cxz * fma(cxy, cyz, -b * cxz)));
        const double dsum = myz + mxz + mxy;  // -f'(l) > 0 above the largest root
        if (dsum > 0.0) lam = fma(det, (double)__frcp_rn((float)dsum), lam);
    }
    // eigenvector of lambda_max: largest cross product of two rows of C - lam I
    double v2x, v2y, v2z;
    {
        const double a = cxx - lam, b = cyy - lam, c = czz - lam;
        const double x0 = fma(cxy, cyz, -b * cxz), y0 = fma(cxz, cxy, -cyz * a), z0 = fma(b, a, -cxy * cxy);   // r0 x r1
        const double x1 = fma(cxy, c, -cxz * cyz), y1 = fma(cxz, cxz, -a * c), z1 = fma(a, cyz, -cxy * cxz);   // r0 x r2
        const double x2 = fma(b, c, -cyz * cyz), y2 = fma(cyz, cxz, -cxy * c), z2 = fma(cxy, cyz, -b * cxz);   // r1 x r2
        const double n0 = x0 * x0 + y0 * y0 + z0 * z0, n1 = x1 * x1 + y1 * y1 + z1 * z1,
                     n2 = x2 * x2 + y2 * y2 + z2 * z2;
        v2x = x2; v2y = y2; v2z = z2;
        double nn = n2;
        if (n1 > nn) { v2x = x1; v2y = y1; v2z = z1; nn = n1; }
        if (n0 > nn) { v2x = x0; v2y = y0; v2z = z0; nn = n0; }
        if (!(nn > 1e-24 * tr * tr * tr * tr)) {
            // C - lam I has rank <= 1 (lambda_mid ~ lambda_max): its largest row
            // is the normal direction; take any unit vector orthogonal to it.
            const double r0 = a * a + cxy * cxy + cxz * cxz, r1 = cxy * cxy + b * b + cyz * cyz,
                         r2 = cxz * cxz + cyz * cyz + c * c;
            double wx = a, wy = cxy, wz = cxz;
            if (r1 > r0 && r1 >= r2) { wx = cxy; wy = b; wz = cyz; }
            else if (r2 > r0 && r2 > r1) { wx = cxz; wy = cyz; wz = c; }
            const double aw = fabs(wx), bw = fabs(wy), cw = fabs(wz);
            if (aw <= bw && aw <= cw) { v2x = 0.0; v2y = wz; v2z = -wy; }
            else if (bw <= cw) { v2x = -wz; v2y = 0.0; v2z = wx; }
            else { v2x = wy; v2y = -wx; v2z = 0.0; }
        }
        if (!prescale(v2x, v2y, v2z)) return true;
        const double in = rsqrt64(v2x * v2x + v2y * v2y + v2z * v2z);
        v2x *= in; v2y *= in; v2z *= in;
    }
    // orthonormal basis (u, w) of the plane orthogonal to v2
    double ux, uy, uz;
    {
        const double ax2 = fabs(v2x), ay2 = fabs(v2y), az2 = fabs(v2z);
        if (ax2 <= ay2 && ax2 <= az2) { ux = 0.0; uy = v2z; uz = -v2y; }
        else if (ay2 <= az2) { ux = -v2z; uy = 0.0; uz = v2x; }
        else { ux = v2y; uy = -v2x; uz = 0.0; }
        const double in = rsqrt64(ux * ux + uy * uy + uz * uz);   // in [1/2, 1]: fp32-safe
        ux *= in; uy *= in; uz *= in;
    }
    const double wx = fma(v2y, uz, -v2z * uy), wy = fma(v2z, ux, -v2x * uz), wz = fma(v2x, uy, -v2y * ux);
    // B = [u w]^T C [u w]
    const double cux = cxx * ux + cxy * uy + cxz * uz, cuy = cxy * ux + cyy * uy + cyz * uz,
                 cuz = cxz * ux + cyz * uy + czz * uz;
    const double cwx = cxx * wx + cxy * wy + cxz * wz, cwy = cxy * wx + cyy * wy + cyz * wz,
                 cwz = cxz * wx + cyz * wy + czz * wz;
    const double b00 = ux * cux + uy * cuy + uz * cuz;
    const double b01 = ux * cwx + uy * cwy + uz * cwz;
    const double b11 = wx * cwx + wy * cwy + wz * cwz;
    // one Jacobi rotation diagonalises the 2x2 block
    double e0 = b00, e1 = b11, c0 = 1.0, s0 = 0.0;
    if (fabs(b01) > 1e-30 * tr) {
        const double tau = (b11 - b00) * (0.5 * rcp64(b01));
        const double at = fabs(tau);
        double t;
        if (at > 1e4) {
            // t = 1 / (|tau| + sqrt(tau^2 + 1)) = (1 - 1/(4 tau^2) + O(tau^-4)) / (2 |tau|)
            const double r = rcp64(at);
            t = 0.5 * r * fma(-0.25 * r, r, 1.0);
        } else {
            const double x = fma(at, at, 1.0);
            t = rcp64(at + x * rsqrt64(x));
        }
        if (tau < 0.0) t = -t;
        c0 = rsqrt64(fma(t, t, 1.0));
        s0 = t * c0;
        e0 = fma(-t, b01, b00);
        e1 = fma(t, b01, b11);
    }
    // eigenvectors in the (u, w) basis: (c, -s) for e0 and (s, c) for e1
    double nx, ny, nz, lmid;
    if (e0 <= e1) {
        nx = c0 * ux - s0 * wx; ny = c0 * uy - s0 * wy; nz = c0 * uz - s0 * wz;
        lmid = e1;
    } else {
        nx = s0 * ux + c0 * wx; ny = s0 * uy + c0 * wy; nz = s0 * uz + c0 * wz;
        lmid = e0;
    }
    const double lmax = lam;
    const bool degenerate = !(lmid > 1e-12 * lmax);   // lambda_mid <= 1e-12 lambda_max
    ratio = lmax > 0.0 ? (float)lmid / (float)lmax : 0.0f;
    {
        const double in = rsqrt64(nx * nx + ny * ny + nz * nz);   // ~1 already
        nx *= in; ny *= in; nz *= in;
    }
    double d = nx * ((double)ax + mx) + ny * ((double)ay + my) + nz * ((double)az + mz);
    bool flip;
    if (fabs(d) < 1e-9) {
        const double ux3 = fabs(nx), uy3 = fabs(ny), uz3 = fabs(nz);
        const double big = (ux3 >= uy3 && ux3 >= uz3) ? nx : ((uy3 >= uz3) ? ny : nz);
        flip = big < 0.0;
    } else {
        flip = d < 0.0;
    }
    if (flip) { nx = -nx; ny = -ny; nz = -nz; d = -d; }
    pl = make_float4((float)nx, (float)ny, (float)nz, (float)d);
    return degenerate;
}

// Moments of a point set (float-float), anchor and count: the solver input.
struct Moments {
    ff s1x, s1y, s1z, sxx, sxy, sxz, syy, syz, szz;
};

__device__ __forceinline__ Moments moments_zero() {
    Moments m;
    m.s1x = m.s1y = m.s1z = m.sxx = m.sxy = m.sxz = m.syy = m.syz = m.szz = {0.f, 0.f};
    return m;
}

// Running moment sums of one pixel chunk: per moment a sum hi of the terms' leading parts,
// whose rounding errors are caught exactly (TwoSum), and a plain sum lo of those errors and of
// the terms' own low parts (exact product errors, cross terms).  Cheaper than float-float
// addition per term; finished into normalised float-float by moments_finish.
struct MomentAcc {
    float h[9], l[9];
};

__device__ __forceinline__ MomentAcc macc_zero() {
    MomentAcc a;
#pragma unroll
    for (int i = 0; i < 9; i++) a.h[i] = a.l[i] = 0.f;
    return a;
}

// h + l += p + e, the rounding error of h + p kept exactly (Knuth's TwoSum)
__device__ __forceinline__ void macc_add(float &h, float &l, float p, float e) {
    const float s = __fadd_rn(h, p);
    const float bb = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    h = s;
    l = __fadd_rn(l, __fadd_rn(err, e));
}

// Adds the point p = r u, shifted by the anchor a (q = p - a exactly, as hi + lo), to m when it
// is in the set: q, and q_i q_j as p = fl(hi_i hi_j) plus its exact error and the cross terms by
// fma.  A pixel outside the set adds exact zeros, which leave every running sum and error term as
// it was, so the pixel loops need no branch.
__device__ __forceinline__ void moments_point(MomentAcc &m, bool in, float rr, float ux, float uy, float uz,
                                                 float ax, float ay, float az) {
    ff qx = two_sum(__fmul_rn(rr, ux), -ax), qy = two_sum(__fmul_rn(rr, uy), -ay),
       qz = two_sum(__fmul_rn(rr, uz), -az);
    if (!in) qx = qy = qz = {0.f, 0.f};
    macc_add(m.h[0], m.l[0], qx.hi, qx.lo);
    macc_add(m.h[1], m.l[1], qy.hi, qy.lo);
    macc_add(m.h[2], m.l[2], qz.hi, qz.lo);
    const ff *q[3] = {&qx, &qy, &qz};
    int k = 3;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = i; j < 3; j++, k++) {
            const float a = q[i]->hi, al = q[i]->lo, b = q[j]->hi, bl = q[j]->lo;
            const float p = __fmul_rn(a, b);
            const float e = fmaf(a, bl, fmaf(al, b, fmaf(a, b, -p)));
            macc_add(m.h[k], m.l[k], p, e);
        }
}

// The chunk's sums as normalised float-float moments.
__device__ __forceinline__ Moments moments_finish(const MomentAcc &a) {
    ff v[9];
#pragma unroll
    for (int i = 0; i < 9; i++) v[i] = two_sum(a.h[i], a.l[i]);   // exact whatever the magnitudes
    Moments m;
    m.s1x = v[0]; m.s1y = v[1]; m.s1z = v[2];
    m.sxx = v[3]; m.sxy = v[4]; m.sxz = v[5];
    m.syy = v[6]; m.syz = v[7]; m.szz = v[8];
    return m;
}

__device__ __forceinline__ Moments moments_add(const Moments &a, const Moments &b) {
    Moments m;
    m.s1x = ff_add(a.s1x, b.s1x);
    m.s1y = ff_add(a.s1y, b.s1y);
    m.s1z = ff_add(a.s1z, b.s1z);
    m.sxx = ff_add(a.sxx, b.sxx);
    m.sxy = ff_add(a.sxy, b.sxy);
    m.sxz = ff_add(a.sxz, b.sxz);
    m.syy = ff_add(a.syy, b.syy);
    m.syz = ff_add(a.syz, b.syz);
    m.szz = ff_add(a.szz, b.szz);
    return m;
}

__device__ __forceinline__ Moments moments_shfl(unsigned mask, const Moments &m, int src) {
    Moments o;
    o.s1x = {__shfl_sync(mask, m.s1x.hi, src), __shfl_sync(mask, m.s1x.lo, src)};
    o.s1y = {__shfl_sync(mask, m.s1y.hi, src), __shfl_sync(mask, m.s1y.lo, src)};
    o.s1z = {__shfl_sync(mask, m.s1z.hi, src), __shfl_sync(mask, m.s1z.lo, src)};
    o.sxx = {__shfl_sync(mask, m.sxx.hi, src), __shfl_sync(mask, m.sxx.lo, src)};
    o.sxy = {__shfl_sync(mask, m.sxy.hi, src), __shfl_sync(mask, m.sxy.lo, src)};
    o.sxz = {__shfl_sync(mask, m.sxz.hi, src), __shfl_sync(mask, m.sxz.lo, src)};
    o.syy = {__shfl_sync(mask, m.syy.hi, src), __shfl_sync(mask, m.syy.lo, src)};
    o.syz = {__shfl_sync(mask, m.syz.hi, src), __shfl_sync(mask, m.syz.lo, src)};
    o.szz = {__shfl_sync(mask, m.szz.hi, src), __shfl_sync(mask, m.szz.lo, src)};
    return o;
}

// Order of a tile's moment sums, shared by the per-thread fit (TileView) and the
// lane-group fit of the queued rounds (TileLanes), so both give the same bits:
// the pixels are split into L chunks of CH consecutive pixels (raster order),
// each chunk is summed in pixel order, and the chunk sums are added left to right.
template <int TH_, int TW_>
struct FitLanes {
    static constexpr int PX = TH_ * TW_;
    static constexpr int L = PX / 4 < 8 ? PX / 4 : 8;
    static constexpr int CH = PX / L;
};

// The plane solve of the moments (FP64 or float-float).
__device__ __forceinline__ bool solve_moments_raw(const Moments m, int n, float ax, float ay, float az, int solver,
                                                  float4 *pl, float *ratio) {
    if (solver == 1) {
        const double m1[3] = {ff_to_d(m.s1x), ff_to_d(m.s1y), ff_to_d(m.s1z)};
        const double m2[6] = {ff_to_d(m.sxx), ff_to_d(m.sxy), ff_to_d(m.sxz),
                              ff_to_d(m.syy), ff_to_d(m.syz), ff_to_d(m.szz)};
        return solve_plane(m1, m2, n, ax, ay, az, *pl, *ratio);
    }
    const ffm::f2 f1[3] = {{m.s1x.hi, m.s1x.lo}, {m.s1y.hi, m.s1y.lo}, {m.s1z.hi, m.s1z.lo}};
    const ffm::f2 f2m[6] = {{m.sxx.hi, m.sxx.lo}, {m.sxy.hi, m.sxy.lo}, {m.sxz.hi, m.sxz.lo},
                            {m.syy.hi, m.syy.lo}, {m.syz.hi, m.syz.lo}, {m.szz.hi, m.szz.lo}};
    float o4[4];
    const bool dg = ffm::solve_plane_ff(f1, f2m, n, ax, ay, az, o4, ratio);
    *pl = make_float4(o4[0], o4[1], o4[2], o4[3]);
    return dg;
}

// One plane solve; a single out-of-line copy keeps the instruction footprint
// of the kernels small (the kernels run few warps per SM, so cold instruction
// fetches, not arithmetic, bound them when code is duplicated).
__device__ __noinline__ bool solve_moments(const Moments m, int n, float ax, float ay, float az, int solver,
                                           int plane3, float4 *pl, float4 *coef, float *ratio) {
    const bool dg = solve_moments_raw(m, n, ax, ay, az, solver, pl, ratio);
    // three-coefficient planes: the fitted plane is the one its stored coefficients give back
    if (plane3 && (pl->x != 0.0f || pl->y != 0.0f || pl->z != 0.0f)) {
        *coef = plane_to3(*pl);
        *pl = plane_from3(*coef);
    }
    return dg;
}

// Pixel masks of a tile (up to 128 pixels).
struct Mask {
    unsigned long long w0, w1;
    __device__ __forceinline__ bool get(int k) const { return ((k < 64 ? w0 : w1) >> (k & 63)) & 1ull; }
    __device__ __forceinline__ void set(int k) {
        if (k < 64) w0 |= 1ull << k;
        else w1 |= 1ull << (k & 63);
    }
    __device__ __forceinline__ bool operator==(const Mask &o) const { return w0 == o.w0 && w1 == o.w1; }
};

// One tile seen by one thread: geometry, valid mask and anchor.  Pixel
// ranges are re-read from the range image (L1 hits) on each pass.
template <int TH_, int TW_>
struct TileView {
    static constexpr int PX = TH_ * TW_;
    const Geometry &g;
    const uint32_t *rimg;
    int t, tc, i0, j0;
    Mask V;
    int nv, first;
    float ax, ay, az;

    __device__ __forceinline__ TileView(const Geometry &g_, const uint32_t *rimg_, int t_)
        : g(g_), rimg(rimg_), t(t_) {
        const int tr = t / g.TC;
        tc = t % g.TC;
        i0 = tr * TH_;
        j0 = tc * TW_;
        nv = 0;
        first = -1;
        V.w0 = V.w1 = 0ull;
#pragma unroll 4
        for (int k = 0; k < PX; k++) {
            if (r(k) > 0.0f) {
                V.set(k);
                nv++;
                if (first < 0) first = k;
            }
        }
        ax = ay = az = 0.f;
        if (first >= 0) {
            float ux, uy, uz;
            u(first, ux, uy, uz);
            const float r0 = r(first);
            ax = __fmul_rn(r0, ux);
            ay = __fmul_rn(r0, uy);
            az = __fmul_rn(r0, uz);
        }
    }
    // range of pixel k (0 if empty or outside the image)
    __device__ __forceinline__ float r(int k) const {
        const int i = i0 + k / TW_, j = j0 + k % TW_;
        if (i >= g.H || j >= g.W) return 0.0f;
        const uint32_t bits = __ldg(rimg + (size_t)i * g.W + j);
        return bits_valid(bits) ? __uint_as_float(bits) : 0.0f;
    }
    __device__ __forceinline__ void u(int k, float &ux, float &uy, float &uz) const {
        beam(g, i0 + k / TW_, j0 + k % TW_, ux, uy, uz);
    }
    // inlier set of a plane over the valid pixels; returns its size
    __device__ __forceinline__ int inliers(const float4 &pl, Mask &I, bool &border) const {
        int cnt = 0;
        I.w0 = I.w1 = 0ull;
#pragma unroll 2
        for (int k = 0; k < PX; k++) {
            if (!V.get(k)) continue;
            float ux, uy, uz;
            u(k, ux, uy, uz);
            if (inlier_screened(pl, ux, uy, uz, r(k), g.thr, border)) {
                I.set(k);
                cnt++;
            }
        }
        return cnt;
    }
    // one total-least-squares fit over the set S (float-float moments, in the chunk order
    // of FitLanes)
    __device__ __forceinline__ bool fit(const Mask &S, int nS, float4 &pl, float4 &coef, float &ratio) const {
        constexpr int L = FitLanes<TH_, TW_>::L, CH = FitLanes<TH_, TW_>::CH;
        Moments m = moments_zero();
#pragma unroll 1
        for (int c = 0; c < L; c++) {
            MomentAcc acc = macc_zero();
#pragma unroll 2
            for (int k = c * CH; k < (c + 1) * CH; k++) {
                float ux, uy, uz;
                u(k, ux, uy, uz);
                moments_point(acc, S.get(k), r(k), ux, uy, uz, ax, ay, az);
            }
            const Moments part = moments_finish(acc);
            m = c == 0 ? part : moments_add(m, part);
        }
        return solve_moments(m, nS, ax, ay, az, g.solver, g.plane3, &pl, &coef, &ratio);
    }
};

// One tile seen by a group of L lanes (FitLanes; an aligned group of a warp):
// lane l owns the pixel chunk [l CH, (l + 1) CH).  Every member function is
// collective over the group and returns the same value on every lane.
template <int TH_, int TW_>
struct TileLanes {
    static constexpr int PX = TH_ * TW_;
    static constexpr int L = FitLanes<TH_, TW_>::L, CH = FitLanes<TH_, TW_>::CH;
    const Geometry &g;
    const uint32_t *rimg;
    int t, i0, j0, l, g0;
    unsigned gmask;
    Mask V;
    int nv, first;
    float ax, ay, az;

    __device__ __forceinline__ TileLanes(const Geometry &g_, const uint32_t *rimg_, int t_, int lane)
        : g(g_), rimg(rimg_), t(t_) {
        l = lane % L;
        g0 = lane - l;
        gmask = ((1u << L) - 1u) << g0;
        i0 = (t / g.TC) * TH_;
        j0 = (t % g.TC) * TW_;
        V.w0 = V.w1 = 0ull;
#pragma unroll 4
        for (int k = l * CH; k < (l + 1) * CH; k++)
            if (r(k) > 0.0f) V.set(k);
#pragma unroll
        for (int off = 1; off < L; off <<= 1) {
            V.w0 |= __shfl_xor_sync(gmask, V.w0, off);
            V.w1 |= __shfl_xor_sync(gmask, V.w1, off);
        }
        nv = __popcll(V.w0) + __popcll(V.w1);
        first = V.w0 ? __ffsll((long long)V.w0) - 1 : (V.w1 ? 64 + __ffsll((long long)V.w1) - 1 : -1);
        ax = ay = az = 0.f;
        if (first >= 0) {
            float ux, uy, uz;
            u(first, ux, uy, uz);
            const float r0 = r(first);
            ax = __fmul_rn(r0, ux);
            ay = __fmul_rn(r0, uy);
            az = __fmul_rn(r0, uz);
        }
    }
    __device__ __forceinline__ float r(int k) const {
        const int i = i0 + k / TW_, j = j0 + k % TW_;
        if (i >= g.H || j >= g.W) return 0.0f;
        const uint32_t bits = __ldg(rimg + (size_t)i * g.W + j);
        return bits_valid(bits) ? __uint_as_float(bits) : 0.0f;
    }
    __device__ __forceinline__ void u(int k, float &ux, float &uy, float &uz) const {
        beam(g, i0 + k / TW_, j0 + k % TW_, ux, uy, uz);
    }
    __device__ __forceinline__ int inliers(const float4 &pl, Mask &I, bool &border) const {
        I.w0 = I.w1 = 0ull;
        bool bd = false;
#pragma unroll 2
        for (int k = l * CH; k < (l + 1) * CH; k++) {
            if (!V.get(k)) continue;
            float ux, uy, uz;
            u(k, ux, uy, uz);
            if (inlier_screened(pl, ux, uy, uz, r(k), g.thr, bd)) I.set(k);
        }
#pragma unroll
        for (int off = 1; off < L; off <<= 1) {
            I.w0 |= __shfl_xor_sync(gmask, I.w0, off);
            I.w1 |= __shfl_xor_sync(gmask, I.w1, off);
        }
        if (__any_sync(gmask, bd)) border = true;
        return __popcll(I.w0) + __popcll(I.w1);
    }
    __device__ __forceinline__ bool fit(const Mask &S, int nS, float4 &pl, float4 &coef, float &ratio) const {
        MomentAcc acc = macc_zero();
#pragma unroll 2
        for (int k = l * CH; k < (l + 1) * CH; k++) {
            float ux, uy, uz;
            u(k, ux, uy, uz);
            moments_point(acc, S.get(k), r(k), ux, uy, uz, ax, ay, az);
        }
        const Moments part = moments_finish(acc);
        Moments m = moments_shfl(gmask, part, g0);
#pragma unroll
        for (int c = 1; c < L; c++) m = moments_add(m, moments_shfl(gmask, part, g0 + c));
        return solve_moments(m, nS, ax, ay, az, g.solver, g.plane3, &pl, &coef, &ratio);
    }
};

struct RecOut {
    float4 plane, tplane;
    float4 coef;          // plane3: the coefficients of the last spatial fit (kept in Scratch::coef)
    uint32_t kref, amask;
    uint8_t status, rounds, flags, nv, n_inl, t_rounds, t_inl, t_status;
    uint32_t acnt[4];
};

__device__ __forceinline__ void write_rec(TileRec *dst_rec, const RecOut &o) {
    uint4 *dst = reinterpret_cast<uint4 *>(dst_rec);
    dst[0] = make_uint4(__float_as_uint(o.plane.x), __float_as_uint(o.plane.y), __float_as_uint(o.plane.z),
                        __float_as_uint(o.plane.w));
    dst[1] = make_uint4(__float_as_uint(o.tplane.x), __float_as_uint(o.tplane.y), __float_as_uint(o.tplane.z),
                        __float_as_uint(o.tplane.w));
    const uint32_t w0 = (uint32_t)o.status | ((uint32_t)o.rounds << 8) | ((uint32_t)o.flags << 16) | ((uint32_t)o.nv << 24);
    const uint32_t w1 = (uint32_t)o.n_inl | ((uint32_t)o.t_rounds << 8) | ((uint32_t)o.t_inl << 16) |
                        ((uint32_t)o.t_status << 24);
    dst[2] = make_uint4(o.kref, o.amask, w0, w1);
    dst[3] = make_uint4(o.acnt[0], o.acnt[1], o.acnt[2], o.acnt[3]);
}

__device__ __forceinline__ RecOut read_rec(const TileRec *src_rec) {
    const uint4 *src = reinterpret_cast<const uint4 *>(src_rec);
    const uint4 q0 = src[0], q1 = src[1], q2 = src[2];
    RecOut o;
    o.plane = make_float4(__uint_as_float(q0.x), __uint_as_float(q0.y), __uint_as_float(q0.z), __uint_as_float(q0.w));
    o.tplane = make_float4(__uint_as_float(q1.x), __uint_as_float(q1.y), __uint_as_float(q1.z), __uint_as_float(q1.w));
    o.kref = q2.x;
    o.amask = 0;
    o.status = q2.z & 0xff; o.rounds = (q2.z >> 8) & 0xff; o.flags = (q2.z >> 16) & 0xff; o.nv = q2.z >> 24;
    o.n_inl = q2.w & 0xff; o.t_rounds = (q2.w >> 8) & 0xff; o.t_inl = (q2.w >> 16) & 0xff; o.t_status = q2.w >> 24;
    o.acnt[0] = o.acnt[1] = o.acnt[2] = o.acnt[3] = 0;
    o.coef = make_float4(0.f, 0.f, 0.f, 0.f);
    return o;
}

// Warp-aggregated push of (frame, tile) onto a work queue.
__device__ __forceinline__ void queue_push(bool push, uint32_t item, uint32_t *queue, uint32_t *count) {
    const unsigned mask = __ballot_sync(__activemask(), push);
    if (!push) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    queue[base + __popc(mask & ((1u << lane) - 1u))] = item;
}

// Spatial rounds of one tile from its current state (o.rounds fits done, the
// last plane in o.plane).  Runs at most `max_rounds` more fits; returns true
// if the tile is finished (o fully updated), false if it needs more rounds.
//
// With a proposal (logit, v, d_rel) for the tile, the first round starts from
// the pixels within the threshold of the proposed plane instead of all valid
// pixels (fewer than 3 of them: all valid pixels), and a logit below the skip
// threshold leaves the tile unfitted (flag 8).  The proposed plane is formed by
// fixed fp32 operations: n = v / sqrtf(fma sum of squares), d = d_rel + n.anchor
// (fma chain), both negated when d < 0.
template <class TV>
__device__ __forceinline__ bool spatial_rounds(const TV &tv, RecOut &o, int max_rounds,
                                               const float *prop = nullptr, float skip_logit = 0.f) {
    const Geometry &g = tv.g;
    Mask S, I;
    int nS;
    bool border = false;
    if (o.rounds == 0) {
        nS = 0;
        if (prop) {
            const float lg = prop[0], v0 = prop[1], v1 = prop[2], v2 = prop[3], drel = prop[4];
            if (lg < skip_logit) {
                o.flags |= 8;
                return true;
            }
            const float nn = sqrtf(fmaf(v0, v0, fmaf(v1, v1, __fmul_rn(v2, v2))));
            if (nn > 0.0f && isfinite(nn)) {
                float4 pl = make_float4(__fdiv_rn(v0, nn), __fdiv_rn(v1, nn), __fdiv_rn(v2, nn), 0.f);
                pl.w = __fadd_rn(drel, fmaf(pl.x, tv.ax, fmaf(pl.y, tv.ay, __fmul_rn(pl.z, tv.az))));
                if (pl.w < 0.0f) pl = make_float4(-pl.x, -pl.y, -pl.z, -pl.w);
                nS = tv.inliers(pl, S, border);
            }
        }
        if (nS < 3) {
            S = tv.V;
            nS = tv.nv;
        }
    } else {
        nS = tv.inliers(o.plane, S, border);   // the set the previous plane kept
    }
    bool done = false;
    for (int r = 0; r < max_rounds; r++) {
        float ratio = 0.f;
        const bool degen = tv.fit(S, nS, o.plane, o.coef, ratio);
        if (ratio >= 0.999e-12f && ratio <= 1.001e-12f) o.flags |= 1;
        o.rounds++;
        const int nI = degen ? 0 : tv.inliers(o.plane, I, border);
        done = degen || nI < 3 || o.rounds == g.R + 1 || (nI == nS && I == S);
        if (done) {
            o.n_inl = (uint8_t)nI;
            if (degen) o.flags |= 2;
            if (!degen && nI >= need_inliers(g.fmin, tv.nv)) o.status = S_FIT;
            break;
        }
        S = I;
        nS = nI;
    }
    if (border) o.flags |= 1;
    return done;
}

// Lanes per tile of the lane-parallel temporal test (k_temporal): lane l of a
// tile's group owns pixels k = l, l + L, l + 2L, ... (PX / L of them).
template <int TH_, int TW_>
struct TLanes {
    static constexpr int PX = TH_ * TW_;
    static constexpr int L = PX <= 16 ? 4 : (PX <= 64 ? 8 : 16);
    static constexpr int PPL = PX / L;
};

// n'.p of pixel k in float-float (the terms of the temporal offset's mean).
__device__ __forceinline__ ff dot_term(const float n[3], float rr, float ux, float uy, float uz) {
    return ff_add(ff_add(two_prod(n[0], __fmul_rn(rr, ux)), two_prod(n[1], __fmul_rn(rr, uy))),
                  two_prod(n[2], __fmul_rn(rr, uz)));
}

// Sum over the pixels of set S of a tile in the order the L lanes of k_temporal form it:
// pixel class l = k mod L summed in increasing k, then the class sums pairwise,
// ((0+1)+(2+3))+..., which is the order of an xor-butterfly over the lanes (float-float
// addition is commutative bit for bit, so both halves of every butterfly step agree).
template <int TH_, int TW_>
__device__ __forceinline__ ff class_tree_sum(const TileView<TH_, TW_> &tv, const Mask &S, const float n[3]) {
    constexpr int PX = TH_ * TW_, L = TLanes<TH_, TW_>::L;
    ff stk[6];   // pending class sums of the pairwise tree (rolled loop: one code copy)
    int depth = 0;
#pragma unroll 1
    for (int l = 0; l < L; l++) {
        ff p = {0.f, 0.f};
#pragma unroll 2
        for (int k = l; k < PX; k += L) {
            if (!S.get(k)) continue;
            float ux, uy, uz;
            tv.u(k, ux, uy, uz);
            p = ff_add(p, dot_term(n, tv.r(k), ux, uy, uz));
        }
        for (int cnt = l + 1; (cnt & 1) == 0; cnt >>= 1) p = ff_add(stk[--depth], p);
        stk[depth++] = p;
    }
    return stk[0];
}

// Temporal test of a P tile (Sec. III-D): anchor to key-frame coordinates,
// K tile lookup, rotated normal, offset refit rounds.  Updates o.  One thread
// per tile; k_temporal runs the same test with a group of lanes per tile and
// sums in the same order (class_tree_sum), so both give the same bits.
template <int TH_, int TW_>
__device__ __forceinline__ void temporal_test(const TileView<TH_, TW_> &tv, const double *M, const float4 *kf,
                                              RecOut &o) {
    const Geometry &g = tv.g;
    // candidate K tiles: those the valid pixels fall in, distinct, raster order from the
    // anchor's (one candidate: the anchor's K tile only); the first that passes is kept
    const int ncand_max = g.tcand > 1 ? g.tcand : 1;
    int cand[4];
    int ncand = 0;
    bool tested = false, border_all = false;
    for (int k = tv.first; k < TileView<TH_, TW_>::PX && ncand < ncand_max; k++) {
        if (!tv.V.get(k)) continue;
        float px = tv.ax, py = tv.ay, pz = tv.az;
        if (k != tv.first) {
            float ux, uy, uz;
            tv.u(k, ux, uy, uz);
            const float rr = tv.r(k);
            px = __fmul_rn(rr, ux);
            py = __fmul_rn(rr, uy);
            pz = __fmul_rn(rr, uz);
        }
        float aK[3];
        transform_point(M, px, py, pz, aK);
        float rK;
        int pixK;
        if (bin_point(g, aK[0], aK[1], aK[2], rK, pixK) != 0) {
            if (k == tv.first) break;
            continue;
        }
        const int kti = (pixK / g.W / g.th) * g.TC + (pixK % g.W) / g.tw;
        bool seen = false;
        for (int q = 0; q < ncand; q++) seen |= cand[q] == kti;
        if (seen) continue;
        cand[ncand++] = kti;
        const float4 kp = __ldg(kf + kti);
        if (kp.x == 0.f && kp.y == 0.f && kp.z == 0.f) continue;
        float n[3];
        rotate_normal(M, kp.x, kp.y, kp.z, n);
        o.kref = (uint32_t)kti;
        o.t_rounds = 0;
        Mask S = tv.V, I;
        int nS = tv.nv, nI = 0;
        float c = 0.f;
        bool border = false;
        for (;;) {
            const ff acc = class_tree_sum<TH_, TW_>(tv, S, n);
            c = ffm::mul({acc.hi, acc.lo}, ffm::rcp(ffm::mk((float)nS))).hi;   // mean of n'.p
            o.t_rounds++;
            nI = tv.inliers(make_float4(n[0], n[1], n[2], c), I, border);
            if ((nI == nS && I == S) || o.t_rounds == g.R + 1 || nI < 3) break;
            S = I;
            nS = nI;
        }
        tested = true;
        border_all |= border;
        o.tplane = make_float4(n[0], n[1], n[2], c);
        o.t_inl = (uint8_t)nI;
        o.t_status = (tv.nv >= 3 && nI >= need_inliers(g.fmin, tv.nv)) ? 2 : 1;
        if (o.t_status == 2) break;
    }
    if (!tested) return;
    if (border_all) o.flags |= 1;
    o.flags |= 4;
    if (o.t_status == 2) {
        o.status = S_TEMPORAL;
        o.plane = o.tplane;
        o.n_inl = o.t_inl;
    }
}

// First pass over every tile: temporal test (P frames), then the spatial fit.
// Schedule 0 runs all of a tile's rounds in its thread; schedules 1 and 2 run
// at most that many spatial rounds here and queue the tile for dense round
// kernels (k_fit_round, one launch per round), schedule 3 runs one round here
// and the queued tiles' remaining rounds in a single dense launch, so that the
// few tiles needing more rounds do not hold whole warps.
template <int TH_, int TW_, bool kQueue>
__global__ void __launch_bounds__(kFitThreads) k_fit_first(Geometry g, Scratch s, Batch b, Poses ps) {
    using TV = TileView<TH_, TW_>;
    const int f = blockIdx.y;
    const int t = blockIdx.x * kFitThreads + threadIdx.x;
    if (t >= g.NT) return;
    const uint32_t *rimg = s.rimg + (size_t)b.slot[f] * g.H * g.W;
    TileRec *recs = s.tiles + (size_t)b.slot[f] * g.NT;
    const TV tv(g, rimg, t);
    RecOut o;
    o.plane = o.tplane = o.coef = make_float4(0.f, 0.f, 0.f, 0.f);
    o.kref = 0xFFFFFFFFu;
    o.amask = 0;
    o.acnt[0] = o.acnt[1] = o.acnt[2] = o.acnt[3] = 0;
    o.status = tv.nv == 0 ? S_EMPTY : S_FAIL;
    o.rounds = o.flags = o.n_inl = o.t_rounds = o.t_inl = o.t_status = 0;
    o.nv = (uint8_t)tv.nv;
    if (b.kind == 1 && tv.nv > 0 && b.kf[f]) temporal_test<TH_, TW_>(tv, ps.m[f], b.kf[f], o);
    bool queued = false;
    if (o.status != S_TEMPORAL && tv.nv >= 3) {
        const float *prop = b.prop[f] ? b.prop[f] + 5 * (size_t)t : nullptr;
        if (!kQueue) {
            spatial_rounds(tv, o, g.R + 1, prop, b.skip_logit);
        } else if (b.kind == 1 && b.kf[f]) {
            queued = true;   // P-frame spatial fallback after its temporal test: from its first round, dense
        } else if (g.first_rounds == 0) {
            // every round on a lane group (schedule 5): only the proposal's skip is decided here
            if (prop && prop[0] < b.skip_logit) o.flags |= 8;
            else queued = true;
        } else {
            queued = !spatial_rounds(tv, o, g.first_rounds, prop, b.skip_logit);
        }
    }
    if (kQueue)
        queue_push(queued, ((uint32_t)f << 26) | (uint32_t)t, s.queue + (size_t)b.qset * 2 * s.qcap,
                   s.qcount + 8 * b.qset);
    write_rec(recs + t, o);
    if (g.plane3) s.coef[(size_t)b.slot[f] * g.NT + t] = o.coef;
}

// Further spatial rounds (at most max_rounds) for every queued tile, a group of
// FitLanes::L lanes per tile (the few tiles that need them are latency-bound:
// the group splits each round's pixel work); tiles that still need a round are
// pushed onto the next queue.  Under schedule 5 every tile that can be fitted
// arrives here before its first round: a lane group per tile for all rounds.
template <int TH_, int TW_>
__global__ void __launch_bounds__(kFitThreads) k_fit_round(Geometry g, Scratch s, Batch b, int in_q, int out_q,
                                                             int max_rounds) {
    using TV = TileLanes<TH_, TW_>;
    constexpr int L = FitLanes<TH_, TW_>::L;
    static_assert(kFitThreads % L == 0 && 32 % L == 0, "lane groups");
    uint32_t *queue = s.queue + (size_t)b.qset * 2 * s.qcap;
    uint32_t *qcount = s.qcount + 8 * b.qset;
    const uint32_t n_in = qcount[in_q];
    const uint32_t *qin = queue + (size_t)(in_q & 1) * s.qcap;
    uint32_t *qout = queue + (size_t)(out_q & 1) * s.qcap;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * (kFitThreads / L);
    for (uint32_t idx = (blockIdx.x * kFitThreads + threadIdx.x) / L; idx < n_in; idx += stride) {
        const uint32_t item = qin[idx];
        const int f = (int)(item >> 26), t = (int)(item & 0x3FFFFFFu);
        const uint32_t *rimg = s.rimg + (size_t)b.slot[f] * g.H * g.W;
        TileRec *recs = s.tiles + (size_t)b.slot[f] * g.NT;
        const TV tv(g, rimg, t, lane);
        RecOut o = read_rec(recs + t);
        // a tile queued before its first round starts from its proposal's inliers, as in the first pass
        const float *prop = o.rounds == 0 && b.prop[f] ? b.prop[f] + 5 * (size_t)t : nullptr;
        const bool done = spatial_rounds(tv, o, max_rounds, prop, b.skip_logit);
        const bool leader = tv.l == 0;
        queue_push(!done && leader, item, qout, qcount + out_q);
        if (leader) write_rec(recs + t, o);
        if (leader && g.plane3) s.coef[(size_t)b.slot[f] * g.NT + t] = o.coef;
    }
}

// The same rounds for the queued tiles with one thread per tile (schedule 6): the per-thread fit
// of the first pass, so each round's solve runs once per tile instead of on every lane of a group.
template <int TH_, int TW_>
__global__ void __launch_bounds__(kFitThreads) k_fit_round_thr(Geometry g, Scratch s, Batch b, int in_q, int out_q,
                                                                 int max_rounds) {
    using TV = TileView<TH_, TW_>;
    uint32_t *queue = s.queue + (size_t)b.qset * 2 * s.qcap;
    uint32_t *qcount = s.qcount + 8 * b.qset;
    const uint32_t n_in = qcount[in_q];
    const uint32_t *qin = queue + (size_t)(in_q & 1) * s.qcap;
    uint32_t *qout = queue + (size_t)(out_q & 1) * s.qcap;
    const uint32_t stride = gridDim.x * kFitThreads;
    for (uint32_t idx = blockIdx.x * kFitThreads + threadIdx.x; idx < n_in; idx += stride) {
        const uint32_t item = qin[idx];
        const int f = (int)(item >> 26), t = (int)(item & 0x3FFFFFFu);
        const uint32_t *rimg = s.rimg + (size_t)b.slot[f] * g.H * g.W;
        TileRec *recs = s.tiles + (size_t)b.slot[f] * g.NT;
        const TV tv(g, rimg, t);
        RecOut o = read_rec(recs + t);
        const float *prop = o.rounds == 0 && b.prop[f] ? b.prop[f] + 5 * (size_t)t : nullptr;
        const bool done = spatial_rounds(tv, o, max_rounds, prop, b.skip_logit);
        queue_push(!done, item, qout, qcount + out_q);
        write_rec(recs + t, o);
        if (g.plane3) s.coef[(size_t)b.slot[f] * g.NT + t] = o.coef;
    }
}

// Temporal test of the P frames after their spatial fits (lcc_encode_sequence), with the
// same per-tile decision as the fused pass (a tile that passes becomes temporal exactly as
// if its spatial fit had never run):
// a group of L lanes per tile (TLanes), each lane holding its PX / L pixels in
// registers; sums and inlier sets are combined by xor-butterflies inside the
// group.  A tile that passes becomes temporal; otherwise only the temporal
// fields and flags of its record change (its spatial fit and run pre-test stay).
// kCand bounds the candidate K tiles (1: the anchor's only, the default path's registers).  Eight
// blocks per SM (at most 64 registers a thread) measured faster than the unconstrained 94.
template <int TH_, int TW_, int kCand>
__global__ void __launch_bounds__(kFitThreads, 8) k_temporal(Geometry g, Scratch s, Batch b, Poses ps) {
    constexpr int PX = TH_ * TW_, L = TLanes<TH_, TW_>::L, PPL = TLanes<TH_, TW_>::PPL;
    static_assert(PX % L == 0 && kFitThreads % L == 0 && 32 % L == 0, "lane groups");
    const int f = blockIdx.y;
    const int lane = threadIdx.x & 31, l = lane % L;
    const int t = (blockIdx.x * kFitThreads + (int)threadIdx.x) / L;
    const unsigned gmask = ((1u << L) - 1u) << (lane - l);
    if (t >= g.NT || !b.kf[f]) return;   // whole groups leave together
    const uint32_t *rimg = s.rimg + (size_t)b.slot[f] * g.H * g.W;
    TileRec *recs = s.tiles + (size_t)b.slot[f] * g.NT;
    const int i0 = (t / g.TC) * TH_, j0 = (t % g.TC) * TW_;
    // this lane's pixels: range (0 if empty) and unit ray
    float pr[PPL], pux[PPL], puy[PPL], puz[PPL];
    Mask V;
    V.w0 = V.w1 = 0ull;
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        const int k = l + L * m, i = i0 + k / TW_, j = j0 + k % TW_;
        const bool in = i < g.H && j < g.W;
        const uint32_t bits = in ? __ldg(rimg + (size_t)i * g.W + j) : kEmptyBits;
        beam(g, in ? i : 0, in ? j : 0, pux[m], puy[m], puz[m]);   // issued beside the range load
        pr[m] = 0.f;
        if (bits_valid(bits)) {
            pr[m] = __uint_as_float(bits);
            V.set(k);
        }
    }
#pragma unroll
    for (int off = 1; off < L; off <<= 1) {
        V.w0 |= __shfl_xor_sync(gmask, V.w0, off);
        V.w1 |= __shfl_xor_sync(gmask, V.w1, off);
    }
    const int nv = __popcll(V.w0) + __popcll(V.w1);
    if (nv == 0) return;
    const int first = V.w0 ? __ffsll((long long)V.w0) - 1 : 64 + __ffsll((long long)V.w1) - 1;
    float ax, ay, az;
    {
        const int i = i0 + first / TW_, j = j0 + first % TW_;
        float ux, uy, uz;
        beam(g, i, j, ux, uy, uz);
        const float r0 = __uint_as_float(__ldg(rimg + (size_t)i * g.W + j));
        ax = __fmul_rn(r0, ux);
        ay = __fmul_rn(r0, uy);
        az = __fmul_rn(r0, uz);
    }
    RecOut o = read_rec(recs + t);
    {   // keep the run pre-test results when it ran first (they refer to other tiles' spatial planes)
        const uint4 *src = reinterpret_cast<const uint4 *>(recs + t);
        const uint4 q3 = src[3];
        o.amask = src[2].y;
        o.acnt[0] = q3.x; o.acnt[1] = q3.y; o.acnt[2] = q3.z; o.acnt[3] = q3.w;
    }
    // candidate K tiles (the distinct K tiles the valid pixels fall in, raster order from the
    // anchor's; the first that passes is kept).  Per candidate pixel: its point in key-frame
    // coordinates, K tile and rotated normal, the FP64 products of transform_point and
    // rotate_normal (same operations, same order) one output coordinate per lane (GB300's FP64
    // rate is low), gathered by shuffles
    const double *M = ps.m[f];
    const int cl = l < 3 ? l : 2, g0 = lane - l;
    int kti = 0, nI = 0;
    bool tested = false, border = false, pass = false;
    float n[3] = {0.f, 0.f, 0.f}, c = 0.f;
    uint8_t t_rounds = 0;
    // the K tile a point falls in after Eq. 6 (-1 outside the key frame's image)
    auto key_tile = [&](float px, float py, float pz) -> int {
        float aK[3];
        double tt = __dmul_rn(M[cl * 4 + 0], (double)px);
        tt = fma(M[cl * 4 + 1], (double)py, tt);
        tt = fma(M[cl * 4 + 2], (double)pz, tt);
        const float v = (float)__dadd_rn(tt, M[cl * 4 + 3]);
#pragma unroll
        for (int q = 0; q < 3; q++) aK[q] = __shfl_sync(gmask, v, g0 + q);
        float rK;
        int pixK;
        if (bin_point(g, aK[0], aK[1], aK[2], rK, pixK) != 0) return -1;
        return (pixK / g.W / g.th) * g.TC + (pixK % g.W) / g.tw;
    };
    // the relaxed-plane test against K plane kp (rotated normal, offset refit rounds)
    auto relaxed = [&](const float4 kp) {
        double tt = __dmul_rn(M[0 * 4 + cl], (double)kp.x);
        tt = fma(M[1 * 4 + cl], (double)kp.y, tt);
        tt = fma(M[2 * 4 + cl], (double)kp.z, tt);
        const float v = (float)tt;
#pragma unroll
        for (int q = 0; q < 3; q++) n[q] = __shfl_sync(gmask, v, g0 + q);
        Mask S = V, I;
        int nS = nv;
        t_rounds = 0;
        for (;;) {
            ff acc = {0.f, 0.f};
#pragma unroll
            for (int m = 0; m < PPL; m++)
                if (S.get(l + L * m)) acc = ff_add(acc, dot_term(n, pr[m], pux[m], puy[m], puz[m]));
#pragma unroll
            for (int off = 1; off < L; off <<= 1) acc = ff_add(acc, shfl_xor_ff_m(gmask, acc, off));
            c = ffm::mul({acc.hi, acc.lo}, ffm::rcp(ffm::mk((float)nS))).hi;   // mean of n'.p
            t_rounds++;
            const float4 pl = make_float4(n[0], n[1], n[2], c);
            I.w0 = I.w1 = 0ull;
#pragma unroll
            for (int m = 0; m < PPL; m++)
                if (pr[m] > 0.0f && inlier_screened(pl, pux[m], puy[m], puz[m], pr[m], g.thr, border))
                    I.set(l + L * m);
#pragma unroll
            for (int off = 1; off < L; off <<= 1) {
                I.w0 |= __shfl_xor_sync(gmask, I.w0, off);
                I.w1 |= __shfl_xor_sync(gmask, I.w1, off);
            }
            nI = __popcll(I.w0) + __popcll(I.w1);
            if ((nI == nS && I == S) || t_rounds == g.R + 1 || nI < 3) break;
            S = I;
            nS = nI;
        }
        tested = true;
        pass = nv >= 3 && nI >= need_inliers(g.fmin, nv);
    };
    if constexpr (kCand == 1) {
        kti = key_tile(ax, ay, az);
        if (kti < 0) return;
        const float4 kp = __ldg(b.kf[f] + kti);
        if (kp.x == 0.f && kp.y == 0.f && kp.z == 0.f) return;
        relaxed(kp);
    } else {
        const int ncand_max = min(kCand, g.tcand > 1 ? g.tcand : 1);
        int cand[kCand];
        int ncand = 0;
        for (int k = first; k < PX && ncand < ncand_max; k++) {   // group-uniform
            if (!V.get(k)) continue;
            float px = ax, py = ay, pz = az;
            if (k != first) {   // pixel k's point, from the lane that holds it
                const int mk = k / L;
                float rr = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
                for (int m = 0; m < PPL; m++)
                    if (m == mk) {
                        rr = pr[m];
                        ux = pux[m];
                        uy = puy[m];
                        uz = puz[m];
                    }
                const int src = g0 + k % L;
                rr = __shfl_sync(gmask, rr, src);
                ux = __shfl_sync(gmask, ux, src);
                uy = __shfl_sync(gmask, uy, src);
                uz = __shfl_sync(gmask, uz, src);
                px = __fmul_rn(rr, ux);
                py = __fmul_rn(rr, uy);
                pz = __fmul_rn(rr, uz);
            }
            const int kt = key_tile(px, py, pz);
            if (kt < 0) {
                if (k == first) break;
                continue;
            }
            bool seen = false;
            for (int q = 0; q < ncand; q++) seen |= cand[q] == kt;
            if (seen) continue;
            cand[ncand++] = kt;
            const float4 kp = __ldg(b.kf[f] + kt);
            if (kp.x == 0.f && kp.y == 0.f && kp.z == 0.f) continue;
            kti = kt;
            relaxed(kp);
            if (pass) break;
        }
    }
    if (!tested) return;
    border = __any_sync(gmask, border);   // any lane, any candidate tested
    if (l != 0) return;
    o.kref = (uint32_t)kti;
    const uint8_t tflags = (uint8_t)((border ? 1 : 0) | 4);
    o.tplane = make_float4(n[0], n[1], n[2], c);
    o.t_rounds = t_rounds;
    o.t_inl = (uint8_t)nI;
    o.t_status = pass ? 2 : 1;
    if (o.t_status == 2) {
        o.status = S_TEMPORAL;
        o.plane = o.tplane;
        o.n_inl = (uint8_t)nI;
        o.rounds = 0;
        o.flags = tflags;
    } else {
        o.flags |= tflags;
    }
    write_rec(recs + t, o);
}

// Run pre-test, after every tile's own fit is final: tile t tests its own
// pixels against the planes of the (up to `lookahead`) tiles to its left in
// the row whose fit succeeded (and, with temporal runs, that passed the
// temporal test: their plane is the relaxed one).  Bit j of the result (and count byte j) says
// whether tile t would join a run started at tile t-1-j, i.e. passes that
// plane under the acceptance rule (Sec. III-C run growth).
//
// LPT lanes per tile (16 for horizons up to 16, else 32).  Lane l holds the
// tile's pixels k = l, l + LPT, ... (range and unit ray in registers).  The
// group first marks which of the tiles to its left were fitted (lane j reads
// the status of tile t-1-j, a ballot gathers them), then tests the fitted
// planes one after another, every lane its own pixels, and adds the inlier
// counts by ballots: every lane of the group works on every test, whatever
// share of the candidate tiles holds a plane.
//
// kTOnly: the update after the temporal test of P frames whose spatial fits
// (and full pre-test) ran first: only the candidates that became temporal are
// tested, against their relaxed planes, and only their bits and counts are
// rewritten; a tile with no temporal candidate does nothing.
template <int TH_, int TW_, int LPT, bool kTOnly>
__global__ void __launch_bounds__(kFitThreads) k_lookbehind(Geometry g, Scratch s, Batch b) {
    constexpr int PX = TH_ * TW_;
    constexpr int PPL = (PX + LPT - 1) / LPT;
    constexpr int TPB = kFitThreads / LPT;
    const unsigned FULL = 0xffffffffu;
    const int f = blockIdx.y;
    const int lt = threadIdx.x / LPT, l = threadIdx.x % LPT;
    const int lane = threadIdx.x & 31;
    const int gbase = lane & ~(LPT - 1);
    const unsigned gmask = LPT == 32 ? FULL : (((1u << LPT) - 1u) << gbase);
    const int t = blockIdx.x * TPB + lt;
    const bool live = t < g.NT;
    const uint32_t *rimg = s.rimg + (size_t)b.slot[f] * g.H * g.W;
    TileRec *recs = s.tiles + (size_t)b.slot[f] * g.NT;
    const int tc = live ? t % g.TC : 0;
    const int i0 = live ? (t / g.TC) * TH_ : 0, j0 = tc * TW_;
    float pr[PPL], pux[PPL], puy[PPL], puz[PPL];
    int nv = 0;
#pragma unroll
    for (int m = 0; m < PPL; m++) {
        const int k = l + LPT * m;
        const int i = i0 + k / TW_, jj = j0 + k % TW_;
        const bool in = live && k < PX && i < g.H && jj < g.W;
        const uint32_t bits = in ? __ldg(rimg + (size_t)i * g.W + jj) : kEmptyBits;
        beam(g, in ? i : 0, in ? jj : 0, pux[m], puy[m], puz[m]);   // issued beside the range load
        pr[m] = bits_valid(bits) ? __uint_as_float(bits) : 0.0f;
        nv += bits_valid(bits) ? 1 : 0;
    }
#pragma unroll
    for (int off = LPT / 2; off; off >>= 1) nv += __shfl_xor_sync(gmask, nv, off);
    // the fitted tiles among the candidates (group-uniform mask, bit j = tile t-1-j)
    const int ncand = live && nv >= 3 ? min(g.lookahead, tc) : 0;
    bool fitted = false;
    if (l < ncand) {
        const TileRec *src = recs + (t - 1 - l);
        const uint32_t w0 = *reinterpret_cast<const uint32_t *>(reinterpret_cast<const uint8_t *>(src) + 40);
        fitted = kTOnly ? (w0 & 0xff) == S_TEMPORAL
                        : ((w0 & 0xff) == S_FIT || (g.truns && (w0 & 0xff) == S_TEMPORAL));
    }
    const unsigned fmask = (__ballot_sync(gmask, fitted) & gmask) >> gbase;
    if (kTOnly && !fmask) return;   // group-uniform: no candidate became temporal
    const int need = need_inliers(g.fmin, nv);
    int my_nin = 0;
    uint32_t pass_mask = 0;
    bool border = false;
    for (unsigned m = fmask; m; m &= m - 1) {
        const int j = __ffs(m) - 1;
        const float4 pl = recs[t - 1 - j].plane;
        int c = 0;
#pragma unroll
        for (int q = 0; q < PPL; q++) {
            const bool in = pr[q] > 0.0f && inlier_screened(pl, pux[q], puy[q], puz[q], pr[q], g.thr, border);
            c += __popc(__ballot_sync(gmask, in) & gmask);
        }
        if (l == j) my_nin = c;
        if (c >= need) pass_mask |= 1u << j;
    }
    if (live) {
        uint8_t *lb = s.lbcnt + ((size_t)b.slot[f] * g.NT + t) * 32;
        uint8_t *base = reinterpret_cast<uint8_t *>(recs + t);
        if (!kTOnly || ((fmask >> l) & 1u)) {
            lb[l] = (uint8_t)my_nin;
            if (l < 16) base[48 + l] = (uint8_t)my_nin;
        }
        if (!kTOnly && LPT == 16) lb[l + 16] = 0;
        if (l == 0) {
            uint32_t *mw = reinterpret_cast<uint32_t *>(base + 36);
            *mw = kTOnly ? ((*mw & ~fmask) | pass_mask) : pass_mask;
        }
    }
}

template <int TH_, int TW_>
static cudaError_t launch_fit_first_t(const Geometry &g, const Scratch &s, const Batch &b, const Poses &p,
                                     cudaStream_t st) {
    dim3 grid((g.NT + kFitThreads - 1) / kFitThreads, b.nframes);
    if (g.schedule >= 1) {
        cudaError_t e = cudaMemsetAsync(s.qcount + 8 * b.qset, 0, sizeof(uint32_t) * 8, st);
        if (e != cudaSuccess) return e;
        k_fit_first<TH_, TW_, true><<<grid, kFitThreads, 0, st>>>(g, s, b, p);
    } else {
        k_fit_first<TH_, TW_, false><<<grid, kFitThreads, 0, st>>>(g, s, b, p);
    }
    return cudaGetLastError();
}

template <int TH_, int TW_, bool kTOnly>
static cudaError_t launch_lookbehind_t(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st) {
    if (!g.merge || g.lookahead <= 0) return cudaSuccess;
    if (g.lookahead <= 16) {
        constexpr int TPB = kFitThreads / 16;
        k_lookbehind<TH_, TW_, 16, kTOnly><<<dim3((g.NT + TPB - 1) / TPB, b.nframes), kFitThreads, 0, st>>>(g, s, b);
    } else {
        constexpr int TPB = kFitThreads / 32;
        k_lookbehind<TH_, TW_, 32, kTOnly><<<dim3((g.NT + TPB - 1) / TPB, b.nframes), kFitThreads, 0, st>>>(g, s, b);
    }
    return cudaGetLastError();
}

template <int TH_, int TW_>
static cudaError_t launch_queued_rounds_t(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st) {
    if (g.schedule >= 1) {
        // the first pass ran the first rounds, except for P frames whose first pass was their
        // temporal test: their spatial rounds all run here
        const int rounds_left = queued_rounds_left(g, b);
        const long long worst = (long long)g.NT * b.nframes;
        constexpr int L = FitLanes<TH_, TW_>::L;   // lanes per queued tile
        const int blocks = (int)std::min<long long>((worst * L + kFitThreads - 1) / kFitThreads, 152 * 8);
        if (g.schedule == 6) {   // one dense launch, a thread per queued tile
            const int tblocks = (int)std::min<long long>((worst + kFitThreads - 1) / kFitThreads, 152 * 8);
            k_fit_round_thr<TH_, TW_><<<tblocks, kFitThreads, 0, st>>>(g, s, b, 0, 1, rounds_left);
            return cudaGetLastError();
        }
        if (g.schedule >= 3) {   // the queued tiles run all their remaining rounds in one dense launch
            k_fit_round<TH_, TW_><<<blocks, kFitThreads, 0, st>>>(g, s, b, 0, 1, rounds_left);
            return cudaGetLastError();
        }
        for (int r = 0; r < rounds_left; r++) {
            k_fit_round<TH_, TW_><<<blocks, kFitThreads, 0, st>>>(g, s, b, r, r + 1, 1);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template <int TH_, int TW_>
static cudaError_t launch_temporal_t(const Geometry &g, const Scratch &s, const Batch &b, const Poses &p,
                                     cudaStream_t st) {
    constexpr int TPB = kFitThreads / TLanes<TH_, TW_>::L;   // tiles per block
    if (g.tcand > 1)
        k_temporal<TH_, TW_, 4><<<dim3((g.NT + TPB - 1) / TPB, b.nframes), kFitThreads, 0, st>>>(g, s, b, p);
    else
        k_temporal<TH_, TW_, 1><<<dim3((g.NT + TPB - 1) / TPB, b.nframes), kFitThreads, 0, st>>>(g, s, b, p);
    return cudaGetLastError();
}

cudaError_t launch_temporal(const Geometry &g, const Scratch &s, const Batch &b, const Poses &p, cudaStream_t st) {
    if (b.nframes <= 0) return cudaSuccess;
    if (g.th == 4 && g.tw == 4) return launch_temporal_t<4, 4>(g, s, b, p, st);
    if (g.th == 4 && g.tw == 8) return launch_temporal_t<4, 8>(g, s, b, p, st);
    if (g.th == 8 && g.tw == 8) return launch_temporal_t<8, 8>(g, s, b, p, st);
    if (g.th == 8 && g.tw == 16) return launch_temporal_t<8, 16>(g, s, b, p, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fit(const Geometry &g, const Scratch &s, const Batch &b, const Poses &p, cudaStream_t st) {
    if (b.nframes <= 0) return cudaSuccess;
    if (g.th == 4 && g.tw == 4) return launch_fit_first_t<4, 4>(g, s, b, p, st);
    if (g.th == 4 && g.tw == 8) return launch_fit_first_t<4, 8>(g, s, b, p, st);
    if (g.th == 8 && g.tw == 8) return launch_fit_first_t<8, 8>(g, s, b, p, st);
    if (g.th == 8 && g.tw == 16) return launch_fit_first_t<8, 16>(g, s, b, p, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_queued_rounds(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st) {
    if (b.nframes <= 0) return cudaSuccess;
    if (g.th == 4 && g.tw == 4) return launch_queued_rounds_t<4, 4>(g, s, b, st);
    if (g.th == 4 && g.tw == 8) return launch_queued_rounds_t<4, 8>(g, s, b, st);
    if (g.th == 8 && g.tw == 8) return launch_queued_rounds_t<8, 8>(g, s, b, st);
    if (g.th == 8 && g.tw == 16) return launch_queued_rounds_t<8, 16>(g, s, b, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_lookbehind(const Geometry &g, const Scratch &s, const Batch &b, cudaStream_t st, bool temporal_only) {
    if (b.nframes <= 0) return cudaSuccess;
    if (temporal_only) {
        if (g.th == 4 && g.tw == 4) return launch_lookbehind_t<4, 4, true>(g, s, b, st);
        if (g.th == 4 && g.tw == 8) return launch_lookbehind_t<4, 8, true>(g, s, b, st);
        if (g.th == 8 && g.tw == 8) return launch_lookbehind_t<8, 8, true>(g, s, b, st);
        if (g.th == 8 && g.tw == 16) return launch_lookbehind_t<8, 16, true>(g, s, b, st);
        return cudaErrorInvalidValue;
    }
    if (g.th == 4 && g.tw == 4) return launch_lookbehind_t<4, 4, false>(g, s, b, st);
    if (g.th == 4 && g.tw == 8) return launch_lookbehind_t<4, 8, false>(g, s, b, st);
    if (g.th == 8 && g.tw == 8) return launch_lookbehind_t<8, 8, false>(g, s, b, st);
    if (g.th == 8 && g.tw == 16) return launch_lookbehind_t<8, 16, false>(g, s, b, st);
    return cudaErrorInvalidValue;
}

}  // namespace lcc
