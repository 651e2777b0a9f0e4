// Float-float ("double-single") arithmetic and the 3x3 plane solve built on it.
//
// A value is an unevaluated sum hi + lo of two fp32 numbers with
// |lo| <= ulp(hi)/2, giving ~48 bits of significand.  Every operation runs on
// the FP32 pipes, whose dependent-operation latency on GB300 is ~4.7 cycles
// against ~64 cycles for an FP64 FMA and 430-680 cycles for an FP64 division
// or square root (measured), so the per-tile plane solve is both far shorter
// in latency and not limited by GB300's FP64 throughput.
//
// All functions are host+device so the solver can be checked on the CPU.  The
// code relies on IEEE round-to-nearest fp32 operations and a correctly rounded
// fused multiply-add (fmaf), with no contraction of separate operations (the
// library is built with -fmad=false / -ffp-contract=off).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define FF_FN __host__ __device__ __forceinline__
#define FF_OUTLINE __host__ __device__ __noinline__
#else
#define FF_FN inline
#define FF_OUTLINE inline
#endif

namespace lcc {
namespace ffm {

struct f2 {
    float hi, lo;
};

FF_FN f2 mk(float a) { return {a, 0.0f}; }

// Knuth's TwoSum: s + e == a + b exactly.
FF_FN f2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

// Dekker's FastTwoSum, valid for |a| >= |b|.
FF_FN f2 quick_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}

// Exact product p + e == a * b.
FF_FN f2 two_prod(float a, float b) {
    const float p = a * b;
    return {p, fmaf(a, b, -p)};
}

FF_FN f2 add(f2 a, f2 b) {
    f2 s = two_sum(a.hi, b.hi);
    const f2 t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}

FF_FN f2 neg(f2 a) { return {-a.hi, -a.lo}; }
FF_FN f2 sub(f2 a, f2 b) { return add(a, neg(b)); }

FF_FN f2 mul(f2 a, f2 b) {
    f2 p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return quick_two_sum(p.hi, p.lo);
}

FF_FN f2 mulf(f2 a, float b) {
    f2 p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return quick_two_sum(p.hi, p.lo);
}

FF_FN f2 sqr(f2 a) {
    f2 p = two_prod(a.hi, a.hi);
    p.lo += 2.0f * a.hi * a.lo;
    return quick_two_sum(p.hi, p.lo);
}

// a*b - c*d
FF_FN f2 msub(f2 a, f2 b, f2 c, f2 d) { return sub(mul(a, b), mul(c, d)); }

// 1 / a: fp32 estimate refined by one Newton step in float-float.
FF_FN f2 rcp(f2 a) {
    const float y = 1.0f / a.hi;
    const f2 e = sub(mk(1.0f), mulf(a, y));   // 1 - a y
    return add(mk(y), mk(y * e.hi));
}

// 1 / sqrt(a) for a > 0: fp32 estimate refined by one Newton step.
FF_FN f2 rsqrt(f2 a) {
    const float y = 1.0f / sqrtf(a.hi);
    const f2 e = sub(mk(1.0f), mulf(mulf(a, y), y));   // 1 - a y^2
    return add(mk(y), mk(0.5f * y * e.hi));
}

FF_FN float fabs_hi(f2 a) { return fabsf(a.hi); }

// Dot product of two float-float 3-vectors.
FF_FN f2 dot3(f2 ax, f2 ay, f2 az, f2 bx, f2 by, f2 bz) { return add(add(mul(ax, bx), mul(ay, by)), mul(az, bz)); }

// Out-of-line pieces of the solve: one copy each, called several times, so the solve's code
// stays small (the fit kernels run few warps per SM and stall on instruction fetch otherwise).
FF_OUTLINE f2 dot3o(f2 ax, f2 ay, f2 az, f2 bx, f2 by, f2 bz) { return dot3(ax, ay, az, bx, by, bz); }

// r x s of two 3-vectors (each component a*b - c*d by msub)
FF_OUTLINE void cross3(f2 rx, f2 ry, f2 rz, f2 sx, f2 sy, f2 sz, f2 &x, f2 &y, f2 &z) {
    x = msub(ry, sz, rz, sy);
    y = msub(rz, sx, rx, sz);
    z = msub(rx, sy, ry, sx);
}

// C v for the symmetric C = (xx, xy, xz, yy, yz, zz)
FF_OUTLINE void symmv(f2 cxx, f2 cxy, f2 cxz, f2 cyy, f2 cyz, f2 czz, f2 vx, f2 vy, f2 vz, f2 &ox, f2 &oy, f2 &oz) {
    ox = dot3(cxx, cxy, cxz, vx, vy, vz);
    oy = dot3(cxy, cyy, cyz, vx, vy, vz);
    oz = dot3(cxz, cyz, czz, vx, vy, vz);
}

// v / |v| (one Newton-refined reciprocal square root)
FF_OUTLINE void normalize3(f2 &x, f2 &y, f2 &z) {
    const f2 in = rsqrt(dot3(x, y, z, x, y, z));
    x = mul(x, in);
    y = mul(y, in);
    z = mul(z, in);
}

// Plane of the moments of a point set: s1 = sum of q, s2 = sum of q q^T
// (xx, xy, xz, yy, yz, zz) with q = p - a for the anchor a, over n points.
// Writes the fp32 plane (unit normal, offset; n.p = d, canonical sign) and
// lambda_mid / lambda_max; returns true if the scatter matrix is degenerate
// (lambda_mid <= 1e-12 lambda_max).
//
// Method (accuracy ~eps * lambda_max in absolute terms, like a Jacobi sweep):
// lambda_max by Newton on det(C - l I) from an fp32 trigonometric seed (the
// largest root is well conditioned); its eigenvector from the largest cross
// product of two rows of C - lambda_max I; C projected onto the orthogonal
// plane; one exact 2x2 Jacobi rotation there gives the smallest eigenvector.
FF_FN bool solve_plane_ff(const f2 s1[3], const f2 s2[6], int n, float ax, float ay, float az, float out[4],
                          float *ratio) {
    out[0] = out[1] = out[2] = out[3] = 0.0f;
    *ratio = 0.0f;
    const f2 inv = rcp(mk((float)n));
    const f2 mx = mul(s1[0], inv), my = mul(s1[1], inv), mz = mul(s1[2], inv);
    const f2 cxx = sub(mul(s2[0], inv), sqr(mx)), cxy = sub(mul(s2[1], inv), mul(mx, my));
    const f2 cxz = sub(mul(s2[2], inv), mul(mx, mz)), cyy = sub(mul(s2[3], inv), sqr(my));
    const f2 cyz = sub(mul(s2[4], inv), mul(my, mz)), czz = sub(mul(s2[5], inv), sqr(mz));
    const f2 tr = add(add(cxx, cyy), czz);
    if (!(tr.hi > 1e-30f)) return true;

    // fp32 seed of the largest eigenvalue (trigonometric closed form)
    const float fxx = cxx.hi, fyy = cyy.hi, fzz = czz.hi, fxy = cxy.hi, fxz = cxz.hi, fyz = cyz.hi;
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
    // decreasing there, so the iterates fall onto the root.
    f2 lam = add(mk(seed), mk(3e-5f * spread));
#pragma unroll 1
    for (int it = 0; it < 3; it++) {
        const f2 a = sub(cxx, lam), b = sub(cyy, lam), c = sub(czz, lam);
        const f2 myz = msub(b, c, cyz, cyz), mxz = msub(a, c, cxz, cxz), mxy = msub(a, b, cxy, cxy);
        const f2 det = add(sub(mul(a, myz), mul(cxy, msub(cxy, c, cyz, cxz))), mul(cxz, msub(cxy, cyz, b, cxz)));
        const f2 dsum = add(add(myz, mxz), mxy);   // -f'(l) > 0 above the largest root
        if (dsum.hi > 0.0f) lam = add(lam, mulf(det, 1.0f / dsum.hi));
    }
    // eigenvector of lambda_max: largest cross product of two rows of C - lam I
    f2 vx, vy, vz;
    {
        const f2 a = sub(cxx, lam), b = sub(cyy, lam), c = sub(czz, lam);
        f2 x0, y0, z0, x1, y1, z1, x2, y2, z2;
        cross3(a, cxy, cxz, cxy, b, cyz, x0, y0, z0);     // r0 x r1
        cross3(a, cxy, cxz, cxz, cyz, c, x1, y1, z1);     // r0 x r2
        cross3(cxy, b, cyz, cxz, cyz, c, x2, y2, z2);     // r1 x r2
        const float n0 = x0.hi * x0.hi + y0.hi * y0.hi + z0.hi * z0.hi;
        const float n1 = x1.hi * x1.hi + y1.hi * y1.hi + z1.hi * z1.hi;
        const float n2 = x2.hi * x2.hi + y2.hi * y2.hi + z2.hi * z2.hi;
        vx = x2; vy = y2; vz = z2;
        float nn = n2;
        if (n1 > nn) { vx = x1; vy = y1; vz = z1; nn = n1; }
        if (n0 > nn) { vx = x0; vy = y0; vz = z0; nn = n0; }
        const float t2 = tr.hi * tr.hi;
        if (!(nn > 1e-24f * t2 * t2)) {
            // C - lam I has rank <= 1 (lambda_mid ~ lambda_max): its largest row
            // is the normal direction; take any unit vector orthogonal to it.
            const float r0 = a.hi * a.hi + cxy.hi * cxy.hi + cxz.hi * cxz.hi;
            const float r1 = cxy.hi * cxy.hi + b.hi * b.hi + cyz.hi * cyz.hi;
            const float r2 = cxz.hi * cxz.hi + cyz.hi * cyz.hi + c.hi * c.hi;
            f2 wx = a, wy = cxy, wz = cxz;
            if (r1 > r0 && r1 >= r2) { wx = cxy; wy = b; wz = cyz; }
            else if (r2 > r0 && r2 > r1) { wx = cxz; wy = cyz; wz = c; }
            const float aw = fabs_hi(wx), bw = fabs_hi(wy), cw = fabs_hi(wz);
            if (aw <= bw && aw <= cw) { vx = mk(0.0f); vy = wz; vz = neg(wy); }
            else if (bw <= cw) { vx = neg(wz); vy = mk(0.0f); vz = wx; }
            else { vx = wy; vy = neg(wx); vz = mk(0.0f); }
        }
        const float m = fmaxf(fabs_hi(vx), fmaxf(fabs_hi(vy), fabs_hi(vz)));
        if (!(m > 1e-30f)) return true;
        const float sc = 1.0f / m;   // any scale works before normalising
        vx = mulf(vx, sc); vy = mulf(vy, sc); vz = mulf(vz, sc);
        normalize3(vx, vy, vz);
    }
    // orthonormal basis (u, w) of the plane orthogonal to v
    f2 ux, uy, uz;
    {
        const float a2 = fabs_hi(vx), b2 = fabs_hi(vy), c2 = fabs_hi(vz);
        if (a2 <= b2 && a2 <= c2) { ux = mk(0.0f); uy = vz; uz = neg(vy); }
        else if (b2 <= c2) { ux = neg(vz); uy = mk(0.0f); uz = vx; }
        else { ux = vy; uy = neg(vx); uz = mk(0.0f); }
        normalize3(ux, uy, uz);   // the scale is in [1/2, 1]
    }
    f2 wx, wy, wz;
    cross3(vx, vy, vz, ux, uy, uz, wx, wy, wz);
    // B = [u w]^T C [u w]
    f2 cux, cuy, cuz, cwx, cwy, cwz;
    symmv(cxx, cxy, cxz, cyy, cyz, czz, ux, uy, uz, cux, cuy, cuz);
    symmv(cxx, cxy, cxz, cyy, cyz, czz, wx, wy, wz, cwx, cwy, cwz);
    const f2 b00 = dot3o(ux, uy, uz, cux, cuy, cuz);
    const f2 b01 = dot3o(ux, uy, uz, cwx, cwy, cwz);
    const f2 b11 = dot3o(wx, wy, wz, cwx, cwy, cwz);
    // one Jacobi rotation diagonalises the 2x2 block
    f2 e0 = b00, e1 = b11, c0 = mk(1.0f), s0 = mk(0.0f);
    if (fabs_hi(b01) > 1e-30f * tr.hi) {
        const f2 tau = mulf(mul(sub(b11, b00), rcp(b01)), 0.5f);
        const f2 at = tau.hi < 0.0f ? neg(tau) : tau;
        f2 t;
        if (at.hi > 1e3f) {
            // t = 1 / (|tau| + sqrt(tau^2 + 1)) = (1 - 1/(4 tau^2) + O(tau^-4)) / (2 |tau|)
            const f2 r = rcp(at);
            t = mulf(mul(r, sub(mk(1.0f), mulf(sqr(r), 0.25f))), 0.5f);
        } else {
            const f2 x = add(sqr(at), mk(1.0f));
            t = rcp(add(at, mul(x, rsqrt(x))));
        }
        if (tau.hi < 0.0f) t = neg(t);
        c0 = rsqrt(add(sqr(t), mk(1.0f)));
        s0 = mul(t, c0);
        e0 = sub(b00, mul(t, b01));
        e1 = add(b11, mul(t, b01));
    }
    // eigenvectors in the (u, w) basis: (c, -s) for e0 and (s, c) for e1
    f2 nx, ny, nz, lmid;
    if (e0.hi <= e1.hi) {
        nx = msub(c0, ux, s0, wx); ny = msub(c0, uy, s0, wy); nz = msub(c0, uz, s0, wz);
        lmid = e1;
    } else {
        nx = add(mul(s0, ux), mul(c0, wx)); ny = add(mul(s0, uy), mul(c0, wy)); nz = add(mul(s0, uz), mul(c0, wz));
        lmid = e0;
    }
    const bool degenerate = !(lmid.hi > 1e-12f * lam.hi);
    *ratio = lam.hi > 0.0f ? lmid.hi / lam.hi : 0.0f;
    normalize3(nx, ny, nz);   // ~1 already
    const f2 d = dot3(nx, ny, nz, add(mk(ax), mx), add(mk(ay), my), add(mk(az), mz));
    bool flip;
    if (fabsf(d.hi) < 1e-9f) {
        const float ux3 = fabs_hi(nx), uy3 = fabs_hi(ny), uz3 = fabs_hi(nz);
        const float big = (ux3 >= uy3 && ux3 >= uz3) ? nx.hi : ((uy3 >= uz3) ? ny.hi : nz.hi);
        flip = big < 0.0f;
    } else {
        flip = d.hi < 0.0f;
    }
    const float sgn = flip ? -1.0f : 1.0f;
    // a normalised float-float rounds to fp32 as its hi part (except exact ties)
    out[0] = sgn * nx.hi;
    out[1] = sgn * ny.hi;
    out[2] = sgn * nz.hi;
    out[3] = sgn * d.hi;
    return degenerate;
}

}  // namespace ffm
}  // namespace lcc
