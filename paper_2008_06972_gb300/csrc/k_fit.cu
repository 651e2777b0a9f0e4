// Per-tile plane fitting (Sec. III-C) and the relaxed-plane temporal test
// (Sec. III-D).
//
// One thread owns one tile: it reads the tile's pixels from the range image
// (L2/L1), forms the points p = r * u_ij in fp32, and runs the whole iterative
// fit itself, so every FP64 instruction of the plane solve carries up to 32
// tiles (GB300's FP64 pipe is the scarce resource of this kernel).
//
// Spatial fit, per round: anchor-shifted moments q = p - a (a = the tile's
// first valid point) are accumulated in float-float (TwoSum / exact products),
// then the covariance is formed in FP64 and the smallest eigenvector found
// (largest eigenpair by Newton + cross products, then an exact 2x2 Jacobi
// rotation in its orthogonal complement; see solve_plane).  The fp32 plane is
// tested on every valid pixel with the along-ray residual to give the next
// inlier set.
//
// Temporal test (P frames, before the spatial fit): the anchor is moved to
// key-frame coordinates (Eq. 6), binned (Eq. 1-2) into the key frame's grid,
// and the K tile's coding plane normal is rotated into P coordinates; the
// offset c' = mean(n'.p) is refit over the current set with the same rounds.
//
// Look-ahead: a tile whose own fit succeeded also tests the next `lookahead`
// tiles of its row against its plane, so the run-growth walker rarely has to
// touch pixels.
#include "lcc_internal.cuh"

namespace lcc {

constexpr int kFitThreads = 128;

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
// accuracy ~eps*lambda_max, like a full Jacobi sweep.
__device__ __noinline__ bool solve_plane(const double m1[3], const double m2[6], int n, float ax, float ay,
                                         float az, float4 &pl, float &ratio) {
    const double inv = 1.0 / (double)n;
    const double mx = m1[0] * inv, my = m1[1] * inv, mz = m1[2] * inv;
    const double cxx = m2[0] * inv - mx * mx, cxy = m2[1] * inv - mx * my, cxz = m2[2] * inv - mx * mz;
    const double cyy = m2[3] * inv - my * my, cyz = m2[4] * inv - my * mz, czz = m2[5] * inv - mz * mz;
    const double tr = cxx + cyy + czz;
    pl = make_float4(0.f, 0.f, 0.f, 0.f);
    ratio = 0.f;
    if (!(tr > 0.0)) return true;
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
    // decreasing there, so the iterates fall monotonically onto the root.
    const double scale = (double)spread + 1e-30 * tr;
    double lam = (double)seed + 3e-5 * scale;
    for (int it = 0; it < 6; it++) {
        const double a = cxx - lam, b = cyy - lam, c = czz - lam;
        const double myz = b * c - cyz * cyz, mxz = a * c - cxz * cxz, mxy = a * b - cxy * cxy;
        const double det = a * myz - cxy * (cxy * c - cyz * cxz) + cxz * (cxy * cyz - b * cxz);
        const double dsum = myz + mxz + mxy;  // -f'(l) > 0 above the largest root
        if (!(dsum > 0.0)) break;
        const double step = det * (double)__frcp_rn((float)dsum);
        lam += step;
        if (fabs(step) <= 1e-17 * scale) break;
    }
    // eigenvector of lambda_max: largest cross product of two rows of C - lam I
    double v2x, v2y, v2z;
    {
        const double a = cxx - lam, b = cyy - lam, c = czz - lam;
        const double x0 = cxy * cyz - b * cxz, y0 = cxz * cxy - cyz * a, z0 = b * a - cxy * cxy;   // r0 x r1
        const double x1 = cxy * c - cxz * cyz, y1 = cxz * cxz - a * c, z1 = a * cyz - cxy * cxz;   // r0 x r2
        const double x2 = b * c - cyz * cyz, y2 = cyz * cxz - cxy * c, z2 = cxy * cyz - b * cxz;   // r1 x r2
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
            // w x e_k with e_k the axis least aligned with w
            if (aw <= bw && aw <= cw) { v2x = 0.0; v2y = wz; v2z = -wy; }
            else if (bw <= cw) { v2x = -wz; v2y = 0.0; v2z = wx; }
            else { v2x = wy; v2y = -wx; v2z = 0.0; }
            nn = v2x * v2x + v2y * v2y + v2z * v2z;
            if (!(nn > 0.0)) return true;
        }
        const double in = rsqrt(nn);
        v2x *= in; v2y *= in; v2z *= in;
    }
    // orthonormal basis (u, w) of the plane orthogonal to v2
    double ux, uy, uz;
    {
        const double ax2 = fabs(v2x), ay2 = fabs(v2y), az2 = fabs(v2z);
        if (ax2 <= ay2 && ax2 <= az2) { ux = 0.0; uy = v2z; uz = -v2y; }
        else if (ay2 <= az2) { ux = -v2z; uy = 0.0; uz = v2x; }
        else { ux = v2y; uy = -v2x; uz = 0.0; }
        const double in = rsqrt(ux * ux + uy * uy + uz * uz);
        ux *= in; uy *= in; uz *= in;
    }
    const double wx = v2y * uz - v2z * uy, wy = v2z * ux - v2x * uz, wz = v2x * uy - v2y * ux;
    // B = [u w]^T C [u w]
    const double cux = cxx * ux + cxy * uy + cxz * uz, cuy = cxy * ux + cyy * uy + cyz * uz,
                 cuz = cxz * ux + cyz * uy + czz * uz;
    const double cwx = cxx * wx + cxy * wy + cxz * wz, cwy = cxy * wx + cyy * wy + cyz * wz,
                 cwz = cxz * wx + cyz * wy + czz * wz;
    const double b00 = ux * cux + uy * cuy + uz * cuz;
    const double b01 = ux * cwx + uy * cwy + uz * cwz;
    const double b11 = wx * cwx + wy * cwy + wz * cwz;
    // one Jacobi rotation diagonalises the 2x2 block
    double e0, e1, c0 = 1.0, s0 = 0.0;
    if (b01 != 0.0) {
        const double tau = (b11 - b00) / (2.0 * b01);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(tau * tau + 1.0));
        c0 = rsqrt(t * t + 1.0);
        s0 = t * c0;
        e0 = b00 - t * b01;
        e1 = b11 + t * b01;
    } else {
        e0 = b00;
        e1 = b11;
    }
    // eigenvectors in the (u, w) basis: (c, -s) for e0 and (s, c) for e1
    double nx, ny, nz, lmin, lmid;
    if (e0 <= e1) {
        nx = c0 * ux - s0 * wx; ny = c0 * uy - s0 * wy; nz = c0 * uz - s0 * wz;
        lmin = e0; lmid = e1;
    } else {
        nx = s0 * ux + c0 * wx; ny = s0 * uy + c0 * wy; nz = s0 * uz + c0 * wz;
        lmin = e1; lmid = e0;
    }
    (void)lmin;
    const double lmax = lam;
    const bool degenerate = !(lmid > 1e-12 * lmax);   // lambda_mid <= 1e-12 lambda_max
    ratio = lmax > 0.0 ? (float)(lmid / lmax) : 0.0f;
    const double in = rsqrt(nx * nx + ny * ny + nz * nz);
    nx *= in; ny *= in; nz *= in;
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

template <int TH_, int TW_>
__global__ void __launch_bounds__(kFitThreads) k_fit(Geometry g, Scratch s, Batch b, Poses ps) {
    constexpr int PX = TH_ * TW_;
    constexpr int MW = (PX + 63) / 64;   // mask words
    const int f = blockIdx.y;
    const int t = blockIdx.x * kFitThreads + threadIdx.x;
    if (t >= g.NT) return;
    const int tr = t / g.TC, tc = t % g.TC;
    const int i0 = tr * TH_, j0 = tc * TW_;
    const uint32_t *rimg = s.rimg + (size_t)b.slot[f] * g.H * g.W;
    TileRec *recs = s.tiles + (size_t)b.slot[f] * g.NT;
    const float thr = g.thr;

    // range of pixel k of this tile (0 if empty or outside the image)
    auto rng = [&](int k) -> float {
        const int i = i0 + k / TW_, j = j0 + k % TW_;
        if (i >= g.H || j >= g.W) return 0.0f;
        const uint32_t bits = __ldg(rimg + (size_t)i * g.W + j);
        return bits_valid(bits) ? __uint_as_float(bits) : 0.0f;
    };
    auto ubeam = [&](int k, float &ux, float &uy, float &uz) {
        beam(g, i0 + k / TW_, j0 + k % TW_, ux, uy, uz);
    };

    // valid mask and anchor (first valid pixel in raster order)
    unsigned long long V[MW];
    int nv = 0, first = -1;
#pragma unroll
    for (int w = 0; w < MW; w++) V[w] = 0ull;
#pragma unroll 4
    for (int k = 0; k < PX; k++) {
        if (rng(k) > 0.0f) {
            V[k >> 6] |= 1ull << (k & 63);
            nv++;
            if (first < 0) first = k;
        }
    }
    float ax = 0.f, ay = 0.f, az = 0.f;
    if (first >= 0) {
        float ux, uy, uz;
        ubeam(first, ux, uy, uz);
        const float r0 = rng(first);
        ax = __fmul_rn(r0, ux);
        ay = __fmul_rn(r0, uy);
        az = __fmul_rn(r0, uz);
    }

    uint8_t status = nv == 0 ? S_EMPTY : S_FAIL;
    uint8_t flags = 0, t_status = 0, t_rounds = 0, t_inl = 0, rounds = 0, n_inl = 0;
    uint32_t kref = 0xFFFFFFFFu;
    float4 tpl = make_float4(0.f, 0.f, 0.f, 0.f), pl = tpl;
    unsigned long long Sm[MW], Im[MW];

    // inlier set of a plane over the valid pixels; returns its size
    auto inliers = [&](const float4 &q4, unsigned long long (&I)[MW], bool &border) -> int {
        int cnt = 0;
#pragma unroll
        for (int w = 0; w < MW; w++) I[w] = 0ull;
#pragma unroll 4
        for (int k = 0; k < PX; k++) {
            if (!((V[k >> 6] >> (k & 63)) & 1ull)) continue;
            float ux, uy, uz, e;
            ubeam(k, ux, uy, uz);
            if (residual(q4, ux, uy, uz, rng(k), thr, e)) {
                I[k >> 6] |= 1ull << (k & 63);
                cnt++;
            }
            if (isfinite(e) && fabsf(fabsf(e) - thr) <= 1e-6f) border = true;
        }
        return cnt;
    };

    // ---- temporal test (P frames) ----
    if (b.kind == 1 && nv > 0) {
        float aK[3];
        transform_point(ps.m[f], ax, ay, az, aK);
        float rK;
        int pixK;
        if (bin_point(g, aK[0], aK[1], aK[2], rK, pixK) == 0) {
            const int kti = (pixK / g.W / g.th) * g.TC + (pixK % g.W) / g.tw;
            const float4 kp = __ldg(b.kf + kti);
            if (!(kp.x == 0.f && kp.y == 0.f && kp.z == 0.f)) {
                float o[3];
                rotate_normal(ps.m[f], kp.x, kp.y, kp.z, o);
                kref = (uint32_t)kti;
#pragma unroll
                for (int w = 0; w < MW; w++) Sm[w] = V[w];
                int nS = nv, nI = 0;
                float c = 0.f;
                bool border = false;
                for (;;) {
                    ff acc = {0.f, 0.f};
#pragma unroll 4
                    for (int k = 0; k < PX; k++) {
                        if (!((Sm[k >> 6] >> (k & 63)) & 1ull)) continue;
                        float ux, uy, uz;
                        ubeam(k, ux, uy, uz);
                        const float r = rng(k);
                        const ff dp = ff_add(ff_add(two_prod(o[0], __fmul_rn(r, ux)), two_prod(o[1], __fmul_rn(r, uy))),
                                             two_prod(o[2], __fmul_rn(r, uz)));
                        acc = ff_add(acc, dp);
                    }
                    c = (float)(ff_to_d(acc) / (double)nS);
                    t_rounds++;
                    nI = inliers(make_float4(o[0], o[1], o[2], c), Im, border);
                    bool same = nI == nS;
#pragma unroll
                    for (int w = 0; w < MW; w++) same = same && Im[w] == Sm[w];
                    if (same || t_rounds == g.R + 1 || nI < 3) break;
#pragma unroll
                    for (int w = 0; w < MW; w++) Sm[w] = Im[w];
                    nS = nI;
                }
                if (border) flags |= 1;
                flags |= 4;
                tpl = make_float4(o[0], o[1], o[2], c);
                t_inl = (uint8_t)nI;
                t_status = (nv >= 3 && nI >= need_inliers(g.fmin, nv)) ? 2 : 1;
                if (t_status == 2) {
                    status = S_TEMPORAL;
                    pl = tpl;
                    n_inl = (uint8_t)nI;
                }
            }
        }
    }

    // ---- spatial fit with drop-and-refit rounds ----
    if (status != S_TEMPORAL && nv >= 3) {
#pragma unroll
        for (int w = 0; w < MW; w++) Sm[w] = V[w];
        int nS = nv, nI = 0;
        bool degen = false, border = false;
        float4 cur = make_float4(0.f, 0.f, 0.f, 0.f);
        for (;;) {
            ff s1x = {0.f, 0.f}, s1y = s1x, s1z = s1x, sxx = s1x, sxy = s1x, sxz = s1x, syy = s1x, syz = s1x, szz = s1x;
#pragma unroll 4
            for (int k = 0; k < PX; k++) {
                if (!((Sm[k >> 6] >> (k & 63)) & 1ull)) continue;
                float ux, uy, uz;
                ubeam(k, ux, uy, uz);
                const float r = rng(k);
                const ff qx = two_sum(__fmul_rn(r, ux), -ax), qy = two_sum(__fmul_rn(r, uy), -ay),
                         qz = two_sum(__fmul_rn(r, uz), -az);
                s1x = ff_add(s1x, qx);
                s1y = ff_add(s1y, qy);
                s1z = ff_add(s1z, qz);
                sxx = ff_add(sxx, ff_mul(qx, qx));
                sxy = ff_add(sxy, ff_mul(qx, qy));
                sxz = ff_add(sxz, ff_mul(qx, qz));
                syy = ff_add(syy, ff_mul(qy, qy));
                syz = ff_add(syz, ff_mul(qy, qz));
                szz = ff_add(szz, ff_mul(qz, qz));
            }
            const double m1[3] = {ff_to_d(s1x), ff_to_d(s1y), ff_to_d(s1z)};
            const double m2[6] = {ff_to_d(sxx), ff_to_d(sxy), ff_to_d(sxz), ff_to_d(syy), ff_to_d(syz), ff_to_d(szz)};
            float ratio = 0.f;
            degen = solve_plane(m1, m2, nS, ax, ay, az, cur, ratio);
            if (ratio >= 0.999e-12f && ratio <= 1.001e-12f) flags |= 1;
            rounds++;
            if (degen) {
                nI = 0;
                break;
            }
            nI = inliers(cur, Im, border);
            bool same = nI == nS;
#pragma unroll
            for (int w = 0; w < MW; w++) same = same && Im[w] == Sm[w];
            if (same || rounds == g.R + 1 || nI < 3) break;
#pragma unroll
            for (int w = 0; w < MW; w++) Sm[w] = Im[w];
            nS = nI;
        }
        if (border) flags |= 1;
        pl = cur;
        n_inl = (uint8_t)nI;
        if (degen) flags |= 2;
        if (!degen && nI >= need_inliers(g.fmin, nv)) status = S_FIT;
    }

    // ---- look-ahead tests of the next tiles of the row against this plane ----
    uint32_t amask = 0, acnt[4] = {0u, 0u, 0u, 0u};
    if (status == S_FIT && g.merge) {
        for (int k = 1; k <= g.lookahead && tc + k < g.TC; k++) {
            const int jn = j0 + k * TW_;
            int nvn = 0, nin = 0;
#pragma unroll 4
            for (int q = 0; q < PX; q++) {
                const int i = i0 + q / TW_, j = jn + q % TW_;
                if (i >= g.H || j >= g.W) continue;
                const uint32_t bits = __ldg(rimg + (size_t)i * g.W + j);
                if (!bits_valid(bits)) continue;
                nvn++;
                float ux, uy, uz, e;
                beam(g, i, j, ux, uy, uz);
                nin += residual(pl, ux, uy, uz, __uint_as_float(bits), thr, e) ? 1 : 0;
            }
            if (nvn >= 3 && nin >= need_inliers(g.fmin, nvn)) amask |= 1u << (k - 1);
            acnt[(k - 1) >> 2] |= (uint32_t)nin << (8 * ((k - 1) & 3));
        }
    }

    uint4 *dst = reinterpret_cast<uint4 *>(recs + t);
    dst[0] = make_uint4(__float_as_uint(pl.x), __float_as_uint(pl.y), __float_as_uint(pl.z), __float_as_uint(pl.w));
    dst[1] = make_uint4(__float_as_uint(tpl.x), __float_as_uint(tpl.y), __float_as_uint(tpl.z), __float_as_uint(tpl.w));
    const uint32_t w0 = (uint32_t)status | ((uint32_t)rounds << 8) | ((uint32_t)flags << 16) | ((uint32_t)nv << 24);
    const uint32_t w1 = (uint32_t)n_inl | ((uint32_t)t_rounds << 8) | ((uint32_t)t_inl << 16) | ((uint32_t)t_status << 24);
    dst[2] = make_uint4(kref, amask, w0, w1);
    dst[3] = make_uint4(acnt[0], acnt[1], acnt[2], acnt[3]);
}

template <int TH_, int TW_>
static cudaError_t launch_fit_t(const Geometry &g, const Scratch &s, const Batch &b, const Poses &p, cudaStream_t st) {
    dim3 grid((g.NT + kFitThreads - 1) / kFitThreads, b.nframes);
    k_fit<TH_, TW_><<<grid, kFitThreads, 0, st>>>(g, s, b, p);
    return cudaGetLastError();
}

cudaError_t launch_fit(const Geometry &g, const Scratch &s, const Batch &b, const Poses &p, cudaStream_t st) {
    if (b.nframes <= 0) return cudaSuccess;
    if (g.th == 4 && g.tw == 4) return launch_fit_t<4, 4>(g, s, b, p, st);
    if (g.th == 4 && g.tw == 8) return launch_fit_t<4, 8>(g, s, b, p, st);
    if (g.th == 8 && g.tw == 8) return launch_fit_t<8, 8>(g, s, b, p, st);
    if (g.th == 8 && g.tw == 16) return launch_fit_t<8, 16>(g, s, b, p, st);
    return cudaErrorInvalidValue;
}

}  // namespace lcc
