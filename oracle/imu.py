"""CPU oracle of the IMU-derived frame pose — TEST INFRASTRUCTURE ONLY.

Plain Python floats (fp64), one sample interval at a time.  Only the test-suite and the
bench's CPU legs may import it; the GPU library never does and shares no code with it.

Sec. III-D (the transformation paragraph) moves a P frame into the K frame's coordinates with
p' = R p + T (Eq. 6).  T holds the translational displacements and R is the product of three
single-axis matrices of the rotational displacements (the two equations before Eq. 6), all
integrated from the IMU's acceleration and rotation rate with the first-order Runge-Kutta
(explicit Euler) method.

Readings (the paper gives neither the frames nor the integration limits):
  - The samples are a zero-order hold: sample k (acceleration a_k, rate w_k, both 3-vectors in
    the sensor's axes at the key frame, gravity removed) holds on [t_k, t_{k+1}); the last
    sample holds after its time, the first before its time.
  - Integration runs from the key frame's time t_K, with the key frame's velocity v_K given, to
    the P frame's time t_P: forward in time when t_P > t_K, backward when t_P < t_K, one Euler
    step per (partial) sample interval, position before velocity:
        forward over [s, s + h]:   x += v h;  v += a(s) h;  theta += w(s) h
        backward over [s - h, s]:  x -= v h;  v -= a(s - h) h;  theta -= w(s - h) h
    with x = 0, theta = 0 at t_K.  x(t_P) is where the P frame's sensor origin lies in the key
    frame's axes, so T = x(t_P).
  - The rotational displacements carry the P frame's axes back onto the key frame's:
    (alpha, beta, gamma) = -theta(t_P), theta = (about x, about y, about z) integrated from
    w = (w_x, w_y, w_z), with alpha the angle about z, beta about y and gamma about x, entered
    into the printed matrices in the printed order.  For a yaw rate w_z this gives
    R = [[cos psi, -sin psi, 0], [sin psi, cos psi, 0], [0, 0, 1]] with psi = theta_z(t_P), the
    rotation that takes P coordinates of a static point to K coordinates.
"""
from __future__ import annotations

import math

import numpy as np


def _hold(t, vals, s, forward):
    """The sample that holds on the interval starting (forward) or ending (backward) at s."""
    k = 0
    if forward:
        while k + 1 < len(t) and t[k + 1] <= s:
            k += 1
    else:
        while k + 1 < len(t) and t[k + 1] < s:
            k += 1
    return vals[k]


def integrate(t, acc, gyro, v_k, t_k, t_p):
    """(x, theta) at t_p by the Euler steps of the module docstring (x, v, theta from t_k)."""
    t = [float(x) for x in t]
    acc = [[float(c) for c in a] for a in acc]
    gyro = [[float(c) for c in w] for w in gyro]
    x = [0.0, 0.0, 0.0]
    v = [float(c) for c in v_k]
    th = [0.0, 0.0, 0.0]
    if t_p == t_k:
        return x, th
    forward = t_p > t_k
    # breakpoints strictly between t_k and t_p: the sample times
    inner = sorted(s for s in t if min(t_k, t_p) < s < max(t_k, t_p))
    cuts = [t_k] + (inner if forward else inner[::-1]) + [t_p]
    for s0, s1 in zip(cuts[:-1], cuts[1:]):
        h = abs(s1 - s0)
        if forward:
            a = _hold(t, acc, s0, True)
            w = _hold(t, gyro, s0, True)
            for i in range(3):
                x[i] = x[i] + v[i] * h
            for i in range(3):
                v[i] = v[i] + a[i] * h
                th[i] = th[i] + w[i] * h
        else:
            a = _hold(t, acc, s0, False)
            w = _hold(t, gyro, s0, False)
            for i in range(3):
                x[i] = x[i] - v[i] * h
            for i in range(3):
                v[i] = v[i] - a[i] * h
                th[i] = th[i] - w[i] * h
    return x, th


def rotation(alpha, beta, gamma):
    """The product of the three printed single-axis matrices (about z, about y, about x)."""
    ca, sa = math.cos(alpha), math.sin(alpha)
    cb, sb = math.cos(beta), math.sin(beta)
    cg, sg = math.cos(gamma), math.sin(gamma)
    Rz = np.array([[ca, sa, 0.0], [-sa, ca, 0.0], [0.0, 0.0, 1.0]])
    Ry = np.array([[cb, 0.0, -sb], [0.0, 1.0, 0.0], [sb, 0.0, cb]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, cg, sg], [0.0, -sg, cg]])
    return Rz @ Ry @ Rx


def pose_from_imu(t, acc, gyro, v_k, t_k, t_p) -> np.ndarray:
    """4x4 row-major M with p_K = R p_P + T (Eq. 6) for the P frame taken at t_p."""
    x, th = integrate(t, acc, gyro, v_k, t_k, t_p)
    M = np.eye(4)
    M[:3, :3] = rotation(-th[2], -th[1], -th[0])
    M[:3, 3] = x
    return M
