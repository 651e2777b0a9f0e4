"""IMU-derived frame pose (Sec. III-D, the equations of T and R before Eq. 6): the oracle pinned
to closed forms, a library rotation routine and the exact motion it integrates; the C-ABI host
routine checked against the oracle.  No GPU needed."""
import math

import numpy as np
import pytest

import synth
from oracle import imu


def _pose(t, acc, gyro, v, tk, tp):
    return imu.pose_from_imu(t, acc, gyro, v, tk, tp)


def test_same_time_is_the_identity():
    M = _pose([0.0, 0.01], [[1, 2, 3], [4, 5, 6]], [[0.1, 0.2, 0.3]] * 2, [7, 8, 9], 0.004, 0.004)
    assert np.array_equal(M, np.eye(4))


@pytest.mark.parametrize("tp", [0.73, -0.41])
def test_constant_velocity_translates_by_v_dt(tp):
    t = np.arange(-60, 90) * 0.01
    z = np.zeros((len(t), 3))
    v = np.array([10.0, -1.5, 0.25])
    M = _pose(t, z, z, v, 0.0, tp)
    assert np.allclose(M[:3, 3], v * tp, atol=1e-12, rtol=0)
    assert np.array_equal(M[:3, :3], np.eye(3))


@pytest.mark.parametrize("n,sign", [(1, 1), (7, 1), (7, -1), (50, 1), (50, -1)])
def test_constant_acceleration_matches_the_euler_closed_form(n, sign):
    """n equal steps s = +-h of x += v s; v += a s give x_n = v0 n s + a s^2 n (n - 1) / 2: position
    before velocity (velocity first would give n (n + 1) / 2)."""
    h = 0.01
    t = np.arange(-100, 101) * h
    a = np.array([0.8, -0.3, 2.0])
    acc = np.tile(a, (len(t), 1))
    v0 = np.array([3.0, 1.0, -2.0])
    s = sign * h
    M = _pose(t, acc, np.zeros_like(acc), v0, 0.0, sign * n * h)
    want = v0 * n * s + a * s * s * n * (n - 1) / 2.0
    assert np.allclose(M[:3, 3], want, atol=1e-12, rtol=0)


def test_samples_hold_until_the_next_sample():
    """An acceleration step at t = 0.25 s acts only after its time (zero-order hold)."""
    t = np.array([0.0, 0.25, 0.5])
    acc = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    M = _pose(t, acc, np.zeros_like(acc), [0.0, 0.0, 0.0], 0.0, 0.5)
    # one step over [0, 0.25] with a = 0, then one over [0.25, 0.5] with a = 2 (x before v): x = 0
    assert M[0, 3] == 0.0
    M = _pose(t, acc, np.zeros_like(acc), [0.0, 0.0, 0.0], 0.0, 0.75)
    # third step, held by the last sample: x = v(0.5) * 0.25 = 0.5 * 0.25
    assert abs(M[0, 3] - 0.125) < 1e-15
    M = _pose(t, acc, np.zeros_like(acc), [0.0, 0.0, 0.0], 0.0, 1.0)
    # the last sample holds after its time: one step over [0.5, 1.0], x = 0.5 * 0.5
    assert abs(M[0, 3] - 0.25) < 1e-15


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_a_single_rate_gives_the_textbook_rotation(axis):
    """A rate w about one axis for tau seconds gives the right-handed rotation by +w tau about it
    (P coordinates of a static point to K coordinates)."""
    w, tau = 0.3, 0.9
    gyro = np.zeros((1, 3))
    gyro[0, axis] = w
    M = _pose([0.0], np.zeros((1, 3)), gyro, [0.0, 0.0, 0.0], 0.0, tau)
    c, s = math.cos(w * tau), math.sin(w * tau)
    R = {0: [[1, 0, 0], [0, c, -s], [0, s, c]],
         1: [[c, 0, s], [0, 1, 0], [-s, 0, c]],
         2: [[c, -s, 0], [s, c, 0], [0, 0, 1]]}[axis]
    assert np.allclose(M[:3, :3], R, atol=1e-15, rtol=0)


def test_combined_rates_follow_the_z_y_x_product():
    """Rotations about z, y and x in that order, each by its integrated angle: the intrinsic
    z-y-x Euler rotation of a library routine; R orthonormal with det +1."""
    Rotation = pytest.importorskip("scipy.spatial.transform").Rotation
    th = np.array([0.31, -0.22, 0.57])      # about x, y, z
    M = _pose([0.0], np.zeros((1, 3)), th[None, :], [0.0, 0.0, 0.0], 0.0, 1.0)
    R = M[:3, :3]
    assert np.allclose(R, Rotation.from_euler("ZYX", th[::-1]).as_matrix(), atol=1e-15, rtol=0)
    assert np.allclose(R.T @ R, np.eye(3), atol=1e-15, rtol=0)
    assert abs(np.linalg.det(R) - 1.0) < 1e-14
    assert np.array_equal(M[3], [0.0, 0.0, 0.0, 1.0])


def test_arc_motion_converges_to_the_exact_relative_pose_at_first_order():
    """Samples of a constant-speed, constant-yaw-rate drive integrate to the exact relative poses
    of the frames (independent closed form of the arc); the translation error falls tenfold with a
    tenfold sample rate (first-order Runge-Kutta) and the rotation is exact (constant rate)."""
    n, k, v, w = 10, 5, 10.0, math.radians(5.0)
    world = synth.arc_poses(n, v, w)
    errs = []
    for rate in (100.0, 1000.0):
        s = synth.imu_samples(0.0, 0.9, v, w, k * synth.FRAME_DT, rate_hz=rate)
        et = 0.0
        for f in range(n):
            M = _pose(s.t, s.acc, s.gyro, s.v_key, k * synth.FRAME_DT, f * synth.FRAME_DT)
            E = synth.relative_pose(world[f], world[k])
            et = max(et, float(np.abs(M[:3, 3] - E[:3, 3]).max()))
            assert np.allclose(M[:3, :3], E[:3, :3], atol=1e-14, rtol=0)
        errs.append(et)
    # Euler bound for |a| = v w over 0.5 s: v w h (0.5 s) / 2 per axis plus the hold's lag
    assert errs[0] < v * w * 0.01 * 0.5
    assert 7.0 < errs[0] / errs[1] < 13.0


@pytest.fixture(scope="module")
def lib():
    from paper_2008_06972_gb300 import build, lcc
    build.build()
    return lcc.load()


@pytest.mark.parametrize("seed", range(6))
def test_c_abi_matches_the_oracle(lib, seed):
    from paper_2008_06972_gb300 import lcc
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 200))
    t = np.cumsum(rng.uniform(0.002, 0.02, n)) - 0.3
    acc = rng.normal(0.0, 2.0, (n, 3))
    gyro = rng.normal(0.0, 0.2, (n, 3))
    v = rng.normal(0.0, 5.0, 3)
    for tk, tp in ((0.1, 0.55), (0.1, -0.4), (t[0] - 0.05, t[-1] + 0.05), (t[n // 2], t[n // 2]),
                   (t[n // 2], t[0])):
        got = lcc.imu_pose(t, acc, gyro, v, tk, tp)
        want = imu.pose_from_imu(t, acc, gyro, v, tk, tp)
        assert np.abs(got - want).max() <= 1e-12


def test_c_abi_rejects_bad_samples(lib):
    from paper_2008_06972_gb300 import lcc
    z = np.zeros((3, 3))
    with pytest.raises(lcc.LccError) as e:
        lcc.imu_pose([0.0, 0.1, 0.1], z, z, [0, 0, 0], 0.0, 0.5)
    assert e.value.status == lcc.ERR_INVALID_ARG
    with pytest.raises(lcc.LccError) as e:
        lcc.imu_pose(np.zeros(0), np.zeros((0, 3)), np.zeros((0, 3)), [0, 0, 0], 0.0, 0.5)
    assert e.value.status == lcc.ERR_INVALID_ARG
    with pytest.raises(lcc.LccError) as e:
        lcc.imu_pose([0.0], z[:1], z[:1], [0, 0, 0], 0.0, float("nan"))
    assert e.value.status == lcc.ERR_INVALID_ARG
