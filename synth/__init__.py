"""Seeded synthetic LiDAR inputs shared by the oracle tests, the GPU tests and the bench.

The ray caster lives in ``lidar_synth.c`` (compiled on first use with gcc).  It
holds none of the compression method's arithmetic: it only produces point
clouds shaped like HDL-64E / KITTI scans and the exact sensor poses of a
sequence.  Workload presets mirror the five benchmark configurations:

* ``frame_cfg1``  16x512 key frame, elevation -15..+15 deg, 4 walls closing a
  courtyard 10-40 m away, 6 boxes, 10 poles, sigma 2 cm, 5 % dropout, max
  range 80 m.
* ``sequence_cfg2``  64x2048 frames (elevation -24.8..+2 deg), 20 walls,
  40 boxes, 60 poles, 2 % clutter, sigma 2 cm, 1 m/frame forward, 0.5 deg/frame
  yaw, 10 frames with the key frame in the middle.
* ``sequence_cfg5``  128x4096 frames, twice the frame-1 density, 5% clutter,
  1.5 m and 1 deg per frame, noisy poses.
* ``batch_cfg3``  64 sequences of U{5..40} frames, each at one of the
  resolutions 16x1024, 32x1024, 64x2048, 128x2048 (elevation -15..+15 deg),
  the frame-1 scene family and noise, the cfg2 ego motion, key-frame groups of
  10 frames with the key frame in the middle of each group.
* ``batch_cfg5``  32 sequences of 100 frames of 128x4096 with the
  ``sequence_cfg5`` scene family, motion and pose noise, key-frame groups of
  10 frames; frames are rendered straight into one caller-owned buffer.

Seeds follow ``seed = 1000003*config + 1009*sequence + frame``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lidar_synth.c")
_LIB_PATH = os.path.join(_HERE, "liblidar_synth.so")
_lock = threading.Lock()
_lib = None


class _Obj(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("p", ctypes.c_double * 6)]


def build(force: bool = False) -> str:
    """Compile the generator shared library (gcc, OpenMP not needed)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.syn_make_scene.restype = ctypes.c_int
            lib.syn_make_scene.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_int]
            lib.syn_render.restype = ctypes.c_int64
            lib.syn_render.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                       ctypes.c_void_p, ctypes.c_int64]
            _lib = lib
    return _lib


@dataclass(frozen=True)
class Sensor:
    rows: int
    cols: int
    elev_min_deg: float
    elev_max_deg: float
    max_range_m: float


CFG1_SENSOR = Sensor(16, 512, -15.0, 15.0, 80.0)
HDL64_SENSOR = Sensor(64, 2048, -24.8, 2.0, 80.0)


def config_seed(config: int, sequence: int, frame: int) -> int:
    return 1000003 * config + 1009 * sequence + frame


class Scene:
    def __init__(self, seed: int, n_walls: int, n_boxes: int, n_poles: int,
                 ground_z: float = -1.7, path_len: float = 0.0, enclose: bool = False):
        lib = _load()
        cap = 1 + n_walls + n_boxes + n_poles
        self._objs = (_Obj * cap)()
        n = lib.syn_make_scene(seed, n_walls, n_boxes, n_poles, ground_z, path_len, int(enclose),
                               ctypes.cast(self._objs, ctypes.c_void_p), cap)
        if n < 0:
            raise RuntimeError("scene generation failed")
        self.n = n

    def objects(self):
        return [(o.kind, tuple(o.p)) for o in self._objs[: self.n]]

    def render(self, sensor: Sensor, R=None, t=None, sigma=0.02, dropout=0.0, clutter=0.0,
               seed=0) -> np.ndarray:
        """One frame as float32 (n, 4) = (x, y, z, 0) in sensor coordinates."""
        lib = _load()
        R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
        t = np.zeros(3) if t is None else np.asarray(t, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64).reshape(9)
        t = np.ascontiguousarray(t, dtype=np.float64).reshape(3)
        cap = sensor.rows * sensor.cols
        out = np.empty((cap, 4), dtype=np.float32)
        n = lib.syn_render(ctypes.cast(self._objs, ctypes.c_void_p), self.n, sensor.rows, sensor.cols,
                           sensor.elev_min_deg, sensor.elev_max_deg, sensor.max_range_m,
                           R.ctypes.data, t.ctypes.data, sigma, dropout, clutter, seed,
                           out.ctypes.data, cap)
        if n < 0:
            raise RuntimeError("render failed")
        return out[:n].copy()

    def render_into(self, sensor: Sensor, out: np.ndarray, R=None, t=None, sigma=0.02, dropout=0.0, clutter=0.0,
                    seed=0) -> int:
        """The same frame as render(), written into out (float32, C-contiguous, at least
        rows*cols x 4); returns the number of points."""
        lib = _load()
        R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
        t = np.zeros(3) if t is None else np.asarray(t, dtype=np.float64)
        R = np.ascontiguousarray(R, dtype=np.float64).reshape(9)
        t = np.ascontiguousarray(t, dtype=np.float64).reshape(3)
        cap = sensor.rows * sensor.cols
        if out.dtype != np.float32 or not out.flags.c_contiguous or out.size < 4 * cap:
            raise ValueError("out must be a contiguous float32 array of at least rows*cols x 4")
        n = lib.syn_render(ctypes.cast(self._objs, ctypes.c_void_p), self.n, sensor.rows, sensor.cols,
                           sensor.elev_min_deg, sensor.elev_max_deg, sensor.max_range_m,
                           R.ctypes.data, t.ctypes.data, sigma, dropout, clutter, seed,
                           out.ctypes.data, cap)
        if n < 0:
            raise RuntimeError("render failed")
        return int(n)


def yaw_matrix(psi: float) -> np.ndarray:
    c, s = math.cos(psi), math.sin(psi)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def ego_poses(n_frames: int, step_m: float, yaw_deg_per_frame: float):
    """World poses (R, t) of a sensor that drives forward along its heading and yaws
    by a fixed angle per frame (frame 0 at the origin, heading +x)."""
    poses = []
    pos = np.zeros(3)
    for f in range(n_frames):
        psi = math.radians(yaw_deg_per_frame * f)
        poses.append((yaw_matrix(psi), pos.copy()))
        pos = pos + step_m * np.array([math.cos(psi), math.sin(psi), 0.0])
    return poses


FRAME_DT = 0.1   # a 10 Hz spinning sensor


def arc_poses(n_frames: int, speed: float, yaw_rate: float, frame_dt: float = FRAME_DT):
    """World poses (R, t) at times f * frame_dt of a sensor that drives at a constant speed (m/s)
    along its heading while yawing at a constant rate (rad/s): frame 0 at the origin, heading +x."""
    poses = []
    for f in range(n_frames):
        tau = f * frame_dt
        psi = yaw_rate * tau
        if yaw_rate == 0.0:
            pos = np.array([speed * tau, 0.0, 0.0])
        else:
            r = speed / yaw_rate
            pos = np.array([r * math.sin(psi), r * (1.0 - math.cos(psi)), 0.0])
        poses.append((yaw_matrix(psi), pos))
    return poses


@dataclass
class ImuSamples:
    t: np.ndarray        # (n,) sample times, s
    acc: np.ndarray      # (n, 3) acceleration, m/s^2, gravity removed, key frame's axes
    gyro: np.ndarray     # (n, 3) rotation rate about x, y, z, rad/s
    v_key: np.ndarray    # (3,) velocity at the key frame's time, key frame's axes


def imu_samples(t0: float, t1: float, speed: float, yaw_rate: float, t_key: float, rate_hz: float = 100.0,
                offset: float = 0.0037, acc_sigma: float = 0.0, gyro_sigma: float = 0.0,
                acc_bias=(0.0, 0.0, 0.0), gyro_bias=(0.0, 0.0, 0.0), seed: int = 0) -> ImuSamples:
    """IMU samples of the arc_poses motion on [t0 - 1/rate, t1 + 1/rate], expressed in the axes of the
    frame taken at t_key: velocity speed * (cos phi, sin phi, 0) with phi = yaw_rate * (t - t_key), so
    acceleration speed * yaw_rate * (-sin phi, cos phi, 0) and rate (0, 0, yaw_rate).  The sample
    clock is offset from the frame clock; white noise (per-sample sigma) and a constant bias model
    the sensor."""
    h = 1.0 / rate_hz
    k0 = math.floor((t0 - offset) / h) - 1
    k1 = math.ceil((t1 - offset) / h) + 1
    t = offset + np.arange(k0, k1 + 1) * h
    phi = yaw_rate * (t - t_key)
    acc = speed * yaw_rate * np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=1)
    gyro = np.zeros((len(t), 3))
    gyro[:, 2] = yaw_rate
    rng = np.random.default_rng(seed)
    acc = acc + rng.normal(0.0, 1.0, acc.shape) * acc_sigma + np.asarray(acc_bias, dtype=np.float64)
    gyro = gyro + rng.normal(0.0, 1.0, gyro.shape) * gyro_sigma + np.asarray(gyro_bias, dtype=np.float64)
    return ImuSamples(t, acc, gyro, np.array([speed, 0.0, 0.0]))


def relative_pose(pose_f, pose_k) -> np.ndarray:
    """4x4 row-major matrix M with p_K = R p_f + T (frame f coordinates to frame k)."""
    Rf, tf = pose_f
    Rk, tk = pose_k
    M = np.eye(4)
    M[:3, :3] = Rk.T @ Rf
    M[:3, 3] = Rk.T @ (tf - tk)
    return M


def perturb_pose(M: np.ndarray, sigma_t: float, sigma_rot_deg: float, seed: int) -> np.ndarray:
    """Add Gaussian noise (translation sigma_t metres, small rotation sigma_rot_deg about
    each axis) to a 4x4 pose; models an IMU-derived pose."""
    rng = np.random.default_rng(seed)
    a = np.radians(rng.normal(0.0, sigma_rot_deg, 3))
    cx, sx, cy, sy, cz, sz = math.cos(a[0]), math.sin(a[0]), math.cos(a[1]), math.sin(a[1]), \
        math.cos(a[2]), math.sin(a[2])
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    out = M.copy()
    out[:3, :3] = Rz @ Ry @ Rx @ M[:3, :3]
    out[:3, 3] = M[:3, 3] + rng.normal(0.0, sigma_t, 3)
    return out


def frame_cfg1(sequence: int = 0) -> tuple[Sensor, np.ndarray]:
    """Single 16x512 key frame of the small workload."""
    seed = config_seed(1, sequence, 0)
    scene = Scene(seed, n_walls=4, n_boxes=6, n_poles=10, enclose=True)
    pts = scene.render(CFG1_SENSOR, sigma=0.02, dropout=0.05, clutter=0.0, seed=seed)
    return CFG1_SENSOR, pts


@dataclass
class Sequence:
    sensor: Sensor
    frames: list          # list of float32 (n_i, 4)
    key_index: int
    poses: np.ndarray     # (n_frames, 4, 4): frame i coordinates -> key frame coordinates


def sequence(sensor: Sensor, n_frames: int, seed: int, n_walls: int, n_boxes: int, n_poles: int,
             step_m: float, yaw_deg: float, sigma: float = 0.02, dropout: float = 0.0,
             clutter: float = 0.0, pose_noise=None, key_index=None, world=None) -> Sequence:
    """A sequence in one scene; the key frame is the middle one (floor(n/2)).  The sensor moves by
    ego_poses(step_m, yaw_deg) unless world poses are given."""
    world = ego_poses(n_frames, step_m, yaw_deg) if world is None else world
    path_len = step_m * max(n_frames - 1, 0)
    scene = Scene(seed, n_walls, n_boxes, n_poles, path_len=path_len)
    k = n_frames // 2 if key_index is None else key_index
    frames, poses = [], []
    for f in range(n_frames):
        Rw, tw = world[f]
        frames.append(scene.render(sensor, Rw, tw, sigma=sigma, dropout=dropout, clutter=clutter,
                                   seed=seed * 131 + f))
        M = relative_pose(world[f], world[k])
        if pose_noise is not None and f != k:
            M = perturb_pose(M, pose_noise[0], pose_noise[1], seed * 7 + f)
        poses.append(M)
    return Sequence(sensor, frames, k, np.stack(poses))


def sequence_cfg2(sequence_id: int = 0, n_frames: int = 10) -> Sequence:
    """HDL-64E-shaped urban sequence: 1 key frame (the middle one) + 9 P-frames."""
    seed = config_seed(2, sequence_id, 0)
    return sequence(HDL64_SENSOR, n_frames, seed, n_walls=20, n_boxes=40, n_poles=60,
                    step_m=1.0, yaw_deg=0.5, sigma=0.02, dropout=0.0, clutter=0.02)


def sequence_arc(sequence_id: int = 0, n_frames: int = 10, speed: float = 10.0,
                 yaw_rate: float = math.radians(5.0)) -> Sequence:
    """The HDL-64E urban scene driven on a constant-speed, constant-yaw-rate arc (10 m/s and
    5 deg/s: 1 m and 0.5 deg per 10 Hz frame), exact poses; the IMU workload."""
    seed = config_seed(2, sequence_id, 0)
    return sequence(HDL64_SENSOR, n_frames, seed, n_walls=20, n_boxes=40, n_poles=60, step_m=speed * FRAME_DT,
                    yaw_deg=0.0, sigma=0.02, dropout=0.0, clutter=0.02,
                    world=arc_poses(n_frames, speed, yaw_rate))


CFG5_SENSOR = Sensor(128, 4096, -15.0, 15.0, 80.0)


def sequence_cfg5(sequence_id: int = 0, n_frames: int = 10) -> Sequence:
    """128x4096 frames (524,288 beams): twice the frame-1 scene density (8 walls, 12 boxes, 20 poles),
    5% clutter, sigma 2 cm, 1.5 m/frame forward and 1 deg/frame yaw, the given poses perturbed
    by 1 cm / 0.05 deg (an IMU-like pose); the key frame is the middle one."""
    seed = config_seed(5, sequence_id, 0)
    return sequence(CFG5_SENSOR, n_frames, seed, n_walls=8, n_boxes=12, n_poles=20, step_m=1.5, yaw_deg=1.0,
                    sigma=0.02, dropout=0.0, clutter=0.05, pose_noise=(0.01, 0.05))


def offgrid_points(n: int, seed: int, r_lo=0.5, r_hi=90.0, elev_lo_deg=-40.0, elev_hi_deg=40.0):
    """Random points anywhere (not on beam centres): binning and collision tests."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(r_lo, r_hi, n)
    az = rng.uniform(-math.pi, math.pi, n)
    el = np.radians(rng.uniform(elev_lo_deg, elev_hi_deg, n))
    pts = np.zeros((n, 4), dtype=np.float32)
    pts[:, 0] = r * np.cos(el) * np.cos(az)
    pts[:, 1] = r * np.cos(el) * np.sin(az)
    pts[:, 2] = r * np.sin(el)
    return pts


CFG3_SENSORS = (Sensor(16, 1024, -15.0, 15.0, 80.0), Sensor(32, 1024, -15.0, 15.0, 80.0),
                Sensor(64, 2048, -15.0, 15.0, 80.0), Sensor(128, 2048, -15.0, 15.0, 80.0))


def group_key(frame: int, n_frames: int, interval: int) -> int:
    """Key frame of the group holding `frame`: groups are [g*I, min((g+1)*I, n)), the key is the
    group's middle frame (start + floor(len/2))."""
    start = (frame // interval) * interval
    return start + min(interval, n_frames - start) // 2


@dataclass
class GroupedSequence:
    sensor: Sensor
    sensor_class: int
    frames: list          # list of float32 (n_i, 4)
    key_interval: int
    poses: np.ndarray     # (n_frames, 4, 4): frame i coordinates -> its group's key frame coordinates


def grouped_sequence(sensor: Sensor, sensor_class: int, n_frames: int, seed: int, key_interval: int,
                     n_walls=4, n_boxes=6, n_poles=10, step_m=1.0, yaw_deg=0.5, sigma=0.02, dropout=0.05,
                     clutter=0.0, pool=None, enclose=True, pose_noise=None, out=None, only=None) -> GroupedSequence:
    """A sequence in key-frame groups of key_interval frames (key = each group's middle frame).
    pose_noise (sigma_t m, sigma_rot deg) perturbs every P frame's pose as perturb_pose does.
    With `out` (float32, n_frames x rows*cols x 4) frame f is rendered into out[f] and the
    sequence's frames are views of it.  With `only` (frame indices) just those frames are
    rendered (the others are empty); poses are given for every frame."""
    world = ego_poses(n_frames, step_m, yaw_deg)
    scene = Scene(seed, n_walls, n_boxes, n_poles, path_len=step_m * max(n_frames - 1, 0), enclose=enclose)

    def one(f):
        Rw, tw = world[f]
        if only is not None and f not in only:
            return np.zeros((0, 4), np.float32)
        if out is None:
            return scene.render(sensor, Rw, tw, sigma=sigma, dropout=dropout, clutter=clutter, seed=seed * 131 + f)
        n = scene.render_into(sensor, out[f], Rw, tw, sigma=sigma, dropout=dropout, clutter=clutter,
                              seed=seed * 131 + f)
        return out[f, :n]

    frames = list(pool.map(one, range(n_frames))) if pool else [one(f) for f in range(n_frames)]
    poses = []
    for f in range(n_frames):
        k = group_key(f, n_frames, key_interval)
        M = relative_pose(world[f], world[k])
        if pose_noise is not None and f != k:
            M = perturb_pose(M, pose_noise[0], pose_noise[1], seed * 7 + f)
        poses.append(M)
    return GroupedSequence(sensor, sensor_class, frames, key_interval, np.stack(poses))


def batch_cfg3(n_seq: int = 64, min_len: int = 5, max_len: int = 40, key_interval: int = 10,
               classes=None, threads: int = 0) -> list:
    """Uneven batch: per sequence a length U{min_len..max_len} and a resolution class drawn with a
    generator seeded by config 3; frames rendered in parallel threads (the ray caster releases
    the GIL)."""
    import concurrent.futures as cf
    rng = np.random.default_rng(config_seed(3, 0, 0))
    lens = rng.integers(min_len, max_len + 1, n_seq)
    cls = rng.integers(0, len(CFG3_SENSORS), n_seq)
    if classes is not None:
        cls = np.asarray([classes[i % len(classes)] for i in range(n_seq)])
    threads = threads or min(16, os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(threads) as pool:
        return [grouped_sequence(CFG3_SENSORS[int(c)], int(c), int(L), config_seed(3, i, 0), key_interval,
                                 pool=pool) for i, (L, c) in enumerate(zip(lens, cls))]


CFG5_FRAMES, CFG5_SEQUENCES, CFG5_KEY_INTERVAL = 100, 32, 10


def sequence_cfg5_grouped(sequence_id: int, n_frames: int = CFG5_FRAMES, key_interval: int = CFG5_KEY_INTERVAL,
                          out=None, pool=None, only=None) -> GroupedSequence:
    """One sequence of the large batched workload: 128x4096 frames, the sequence_cfg5 scene family
    (8 walls, 12 boxes, 20 poles along the path, 5% clutter, sigma 2 cm), 1.5 m and 1 deg per frame,
    poses perturbed by 1 cm / 0.05 deg, key-frame groups of key_interval frames."""
    return grouped_sequence(CFG5_SENSOR, 0, n_frames, config_seed(5, sequence_id, 0), key_interval, n_walls=8,
                            n_boxes=12, n_poles=20, step_m=1.5, yaw_deg=1.0, sigma=0.02, dropout=0.0, clutter=0.05,
                            pool=pool, enclose=False, pose_noise=(0.01, 0.05), out=out, only=only)


def batch_cfg5(out: np.ndarray, n_seq: int = CFG5_SEQUENCES, n_frames: int = CFG5_FRAMES,
               key_interval: int = CFG5_KEY_INTERVAL, first: int = 0, threads: int = 0) -> list:
    """The large batched workload: n_seq sequences (ids first..first+n_seq-1) of n_frames 128x4096
    frames each, rendered in parallel threads into out, a float32 array of shape
    (n_seq * n_frames, 128 * 4096, 4) (sequence i's frame f in out[i * n_frames + f])."""
    import concurrent.futures as cf
    npx = CFG5_SENSOR.rows * CFG5_SENSOR.cols
    if out.shape != (n_seq * n_frames, npx, 4) or out.dtype != np.float32:
        raise ValueError("out must be float32 of shape (n_seq * n_frames, rows * cols, 4)")
    threads = threads or min(32, os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(threads) as pool:
        return [sequence_cfg5_grouped(first + i, n_frames, key_interval, out=out[i * n_frames:(i + 1) * n_frames],
                                      pool=pool) for i in range(n_seq)]
