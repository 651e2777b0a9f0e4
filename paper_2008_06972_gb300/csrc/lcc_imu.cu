// Frame pose from IMU samples (Sec. III-D, the transformation paragraph before
// Eq. 6): translational displacements T and the product R of three single-axis
// rotations by the rotational displacements, both integrated from the
// acceleration and rotation rate with the first-order Runge-Kutta (explicit
// Euler) method.  Host code: a handful of floating-point operations per
// sample, done once per frame.
//
// Readings fixed by this implementation (the paper gives no frames or limits):
// samples hold their value until the next sample (the first one also before its
// time, the last one after); integration starts at the key frame's time t_K with
// the key frame's velocity and zero position and angle, in the key frame's axes,
// and runs forward or backward to the P frame's time t_P, one Euler step per
// (partial) sample interval, position updated before velocity; T is the position
// reached; the rotational displacements are the negated angles (about z, about y,
// about x) entered into the printed matrices in the printed order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "lcc.h"

namespace {

// index of the sample holding on an interval that starts at s going forward, or that
// ends at s going backward
int hold_index(const double *t, int n, double s, bool forward) {
    // last k with t[k] <= s (forward) or t[k] < s (backward); 0 if none
    int lo = 0, hi = n - 1, k = 0;
    while (lo <= hi) {
        const int mid = (lo + hi) / 2;
        const bool before = forward ? t[mid] <= s : t[mid] < s;
        if (before) {
            k = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    return k;
}

}  // namespace

extern "C" {

lcc_status lcc_imu_pose(const double *t, const double *acc, const double *gyro, int32_t n, const double v_key[3],
                        double t_key, double t_p, double pose[16]) {
    if (!t || !acc || !gyro || !v_key || !pose || n < 1 || !std::isfinite(t_key) || !std::isfinite(t_p))
        return LCC_ERR_INVALID_ARG;
    for (int k = 1; k < n; k++)
        if (!(t[k] > t[k - 1])) return LCC_ERR_INVALID_ARG;
    double x[3] = {0.0, 0.0, 0.0}, v[3] = {v_key[0], v_key[1], v_key[2]}, th[3] = {0.0, 0.0, 0.0};
    if (t_p != t_key) {
        const bool fwd = t_p > t_key;
        const double lo = std::min(t_key, t_p), hi = std::max(t_key, t_p);
        std::vector<double> cuts;
        cuts.push_back(t_key);
        std::vector<double> inner;
        for (int k = 0; k < n; k++)
            if (t[k] > lo && t[k] < hi) inner.push_back(t[k]);
        if (!fwd) std::reverse(inner.begin(), inner.end());
        cuts.insert(cuts.end(), inner.begin(), inner.end());
        cuts.push_back(t_p);
        for (size_t c = 0; c + 1 < cuts.size(); c++) {
            const double s = cuts[c], h = std::fabs(cuts[c + 1] - s);
            const int k = hold_index(t, n, s, fwd);
            const double *a = acc + 3 * (size_t)k, *w = gyro + 3 * (size_t)k;
            const double sg = fwd ? 1.0 : -1.0;
            for (int i = 0; i < 3; i++) x[i] = x[i] + sg * (v[i] * h);
            for (int i = 0; i < 3; i++) {
                v[i] = v[i] + sg * (a[i] * h);
                th[i] = th[i] + sg * (w[i] * h);
            }
        }
    }
    // R = Rz(alpha) Ry(beta) Rx(gamma) with the printed matrices, alpha = -theta_z,
    // beta = -theta_y, gamma = -theta_x
    const double al = -th[2], be = -th[1], ga = -th[0];
    const double ca = std::cos(al), sa = std::sin(al), cb = std::cos(be), sb = std::sin(be);
    const double cg = std::cos(ga), sgm = std::sin(ga);
    const double Rz[3][3] = {{ca, sa, 0.0}, {-sa, ca, 0.0}, {0.0, 0.0, 1.0}};
    const double Ry[3][3] = {{cb, 0.0, -sb}, {0.0, 1.0, 0.0}, {sb, 0.0, cb}};
    const double Rx[3][3] = {{1.0, 0.0, 0.0}, {0.0, cg, sgm}, {0.0, -sgm, cg}};
    double A[3][3], R[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            A[i][j] = 0.0;
            for (int k = 0; k < 3; k++) A[i][j] += Rz[i][k] * Ry[k][j];
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            R[i][j] = 0.0;
            for (int k = 0; k < 3; k++) R[i][j] += A[i][k] * Rx[k][j];
        }
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) pose[4 * i + j] = R[i][j];
        pose[4 * i + 3] = x[i];
    }
    pose[12] = pose[13] = pose[14] = 0.0;
    pose[15] = 1.0;
    return LCC_OK;
}

}  // extern "C"
