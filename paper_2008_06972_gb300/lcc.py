"""ctypes binding of the lcc C ABI (include/lcc.h) — argument marshalling only.

Function names mirror the C entry points.  Device buffers are passed as torch
CUDA tensors (their ``data_ptr()``) or raw integer addresses; every step of the
encoder and decoder runs in the CUDA kernels of ``liblcc.so``.  There is no CPU
fallback: loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblcc.so")

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_CORRUPT, ERR_UNSUPPORTED, ERR_NO_DEVICE = range(8)
T_EMPTY, T_RAW, T_RUN_START, T_RUN_CONT, T_TEMPORAL, T_TEMPORAL_CONT = range(6)
T_RUN_START3 = 6   # .. 8: a three-coefficient run start along axis x, y, z
S_EMPTY, S_FAIL, S_FIT, S_TEMPORAL = range(4)


class LccError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


class lcc_sensor(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32), ("elev_min_deg", ctypes.c_double),
                ("elev_max_deg", ctypes.c_double), ("max_range_m", ctypes.c_double)]


class lcc_params(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("fit_thr_m", ctypes.c_float),
                ("quant_m", ctypes.c_float), ("max_refits", ctypes.c_int32), ("min_inlier_frac", ctypes.c_float),
                ("merge_runs", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("lookahead", ctypes.c_int32),
                ("solver", ctypes.c_int32), ("fit_schedule", ctypes.c_int32), ("no_delta", ctypes.c_int32),
                ("raw_exact", ctypes.c_int32), ("temporal_candidates", ctypes.c_int32),
                ("temporal_runs", ctypes.c_int32), ("plane3", ctypes.c_int32)]


class lcc_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("points_in", "points_invalid", "points_fov", "points_binned",
                                               "pixels_valid", "tiles_empty", "tiles_raw", "tiles_run_start",
                                               "tiles_run_cont", "tiles_temporal")] + \
               [("fit_rounds", ctypes.c_int64 * 8), ("tiles_borderline", ctypes.c_int64),
                ("cand", ctypes.c_int64), ("fitted", ctypes.c_int64), ("raw", ctypes.c_int64),
                ("bytes", ctypes.c_uint64), ("tiles_temporal_cont", ctypes.c_int64), ("tiles_net", ctypes.c_int64)]


class lcc_seq_desc(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_int32), ("nframes", ctypes.c_int32), ("key_interval", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("poses", ctypes.c_void_p), ("d_pts", ctypes.c_void_p),
                ("n", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("cap", ctypes.c_void_p),
                ("d_nbytes", ctypes.c_void_p)]


class lcc_plan_info(ctypes.Structure):
    _fields_ = [("frames", ctypes.c_int64), ("key_frames", ctypes.c_int64), ("points", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("graph_nodes", ctypes.c_int64), ("classes", ctypes.c_int32),
                ("captured", ctypes.c_int32), ("seeded_key_frames", ctypes.c_int64)]


class lcc_tune_result(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32), ("lookahead", ctypes.c_int32),
                ("fit_schedule", ctypes.c_int32), ("status", ctypes.c_int32), ("chosen", ctypes.c_int32),
                ("ms", ctypes.c_double), ("mpts_per_s", ctypes.c_double), ("bytes", ctypes.c_uint64),
                ("max_err_m", ctypes.c_float), ("reserved", ctypes.c_float)]


TILE_INFO_DTYPE = np.dtype([("plane", "<f4", 4), ("tplane", "<f4", 4), ("kref", "<u4"), ("ahead_mask", "<u4"),
                            ("status", "u1"), ("rounds", "u1"), ("flags", "u1"), ("n_valid", "u1"),
                            ("n_inlier", "u1"), ("t_rounds", "u1"), ("t_inlier", "u1"), ("t_status", "u1"),
                            ("ahead_cnt", "u1", 16)])
assert TILE_INFO_DTYPE.itemsize == 64

_lib = None
KERNEL_NAMES = ("bin", "fit", "merge", "rounds", "pack", "decode_prep", "decode_px", "range_export", "lookbehind",
                "temporal", "ent_build", "ent_layout", "ent_write", "ent_decode", "net_inputs", "net_fwd")


def load(path: str = LIB_PATH):
    """Load liblcc.so (built by paper_2008_06972_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (__graft_entry__.build())")
    L = ctypes.CDLL(path)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "lcc_status_string": (ctypes.c_char_p, [i32]),
        "lcc_default_params": (None, [vp]),
        "lcc_create": (i32, [vp, vp, vp, vp]),
        "lcc_destroy": (i32, [vp]),
        "lcc_max_encoded_bytes": (u64, [vp]),
        "lcc_num_tiles": (i64, [vp]),
        "lcc_tables": (i32, [vp] * 9),
        "lcc_range_image": (i32, [vp, vp, i64, vp, vp]),
        "lcc_keyframe_create": (i32, [vp, vp]),
        "lcc_keyframe_free": (None, [vp]),
        "lcc_encode_keyframe": (i32, [vp, vp, i64, vp, vp, u64, vp]),
        "lcc_encode_pframe": (i32, [vp, vp, vp, vp, i64, vp, u64, vp]),
        "lcc_encode_pframes": (i32, [vp, vp, i32, vp, vp, vp, vp, vp, vp]),
        "lcc_encode_keyframe_seeded": (i32, [vp, vp, i64, vp, ctypes.c_float, vp, vp, u64, vp]),
        "lcc_encode_keyframes": (i32, [vp, i32, vp, vp, vp, ctypes.c_float, vp, vp, vp]),
        "lcc_encode_sequence": (i32, [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp]),
        "lcc_encode_sequence_host": (i32, [vp, i32, i32, vp, vp, vp, vp, vp, vp]),
        "lcc_keyframe_from_stream": (i32, [vp, vp, u64, vp]),
        "lcc_decode": (i32, [vp, vp, u64, vp, vp, vp, vp, vp]),
        "lcc_decode_sequence": (i32, [vp, i32, i32, vp, vp, vp, vp, vp, vp]),
        "lcc_imu_pose": (i32, [vp, vp, vp, i32, vp, ctypes.c_double, ctypes.c_double, vp]),
        "lcc_entropy_encode": (i32, [vp, i32, vp, vp, vp, vp, vp]),
        "lcc_entropy_decode": (i32, [vp, i32, vp, vp, vp, vp, vp]),
        "lcc_sync": (i32, [vp]),
        "lcc_last_stats": (i32, [vp, i32, vp]),
        "lcc_tile_records": (i32, [vp, i32, vp, i64]),
        "lcc_tile_coefficients": (i32, [vp, i32, vp, i64]),
        "lcc_set_profiling": (i32, [vp, i32]),
        "lcc_kernel_times": (i32, [vp, vp, vp, vp, i32]),
        "lcc_kernel_timeline": (i32, [vp, vp, vp, vp, i32]),
        "lcc_range_image_static": (i32, [vp, vp, i64, vp, vp, vp]),
        "lcc_net_num_params": (i64, []),
        "lcc_net_create": (i32, [vp, vp, i64, vp]),
        "lcc_net_destroy": (None, [vp]),
        "lcc_net_get_params": (i32, [vp, vp]),
        "lcc_net_set_params": (i32, [vp, vp]),
        "lcc_net_tile_inputs": (i32, [vp, vp, i64, vp, vp]),
        "lcc_net_tile_inputs_batch": (i32, [vp, i32, vp, vp, vp, vp]),
        "lcc_net_tile_labels": (i32, [vp, i32, vp, vp]),
        "lcc_net_forward": (i32, [vp, vp, i64, vp]),
        "lcc_net_sync": (i32, [vp]),
        "lcc_selftest_bounded_wait": (i32, [i64, vp]),
        "lcc_net_gradient": (i32, [vp, vp, vp, i64, vp, vp]),
        "lcc_net_train_step": (i32, [vp, vp, vp, i64, ctypes.c_float, i32, vp]),
        "lcc_plan_create": (i32, [vp, i32, vp, i32, vp]),
        "lcc_plan_update": (i32, [vp, i32, vp]),
        "lcc_plan_set_proposals": (i32, [vp, vp, ctypes.c_float]),
        "lcc_plan_set_staging": (i32, [vp, i32]),
        "lcc_plan_encode": (i32, [vp]),
        "lcc_plan_capture": (i32, [vp]),
        "lcc_plan_replay": (i32, [vp]),
        "lcc_plan_sync": (i32, [vp]),
        "lcc_plan_encode_host": (i32, [vp, vp, vp]),
        "lcc_plan_get_info": (i32, [vp, vp]),
        "lcc_plan_stats": (i32, [vp, i32, i32, vp]),
        "lcc_plan_destroy": (None, [vp]),
        "lcc_autotune": (i32, [vp, vp, i32, i32, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_uint32,
                               vp, vp, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def exported_symbols() -> list[str]:
    """Entry points this binding expects liblcc.so to export."""
    return ["lcc_status_string", "lcc_default_params", "lcc_create", "lcc_destroy", "lcc_max_encoded_bytes",
            "lcc_num_tiles", "lcc_tables", "lcc_range_image", "lcc_keyframe_create", "lcc_keyframe_free",
            "lcc_encode_keyframe", "lcc_encode_keyframe_seeded", "lcc_encode_keyframes", "lcc_encode_pframe", "lcc_encode_pframes", "lcc_encode_sequence",
            "lcc_encode_sequence_host", "lcc_keyframe_from_stream", "lcc_decode", "lcc_decode_sequence", "lcc_imu_pose", "lcc_entropy_encode", "lcc_entropy_decode", "lcc_sync", "lcc_last_stats",
            "lcc_tile_records", "lcc_tile_coefficients", "lcc_set_profiling", "lcc_kernel_times", "lcc_kernel_timeline", "lcc_range_image_static", "lcc_net_num_params", "lcc_net_create", "lcc_net_destroy",
            "lcc_net_get_params", "lcc_net_set_params", "lcc_net_tile_inputs", "lcc_net_tile_inputs_batch", "lcc_net_tile_labels", "lcc_net_forward", "lcc_net_sync", "lcc_net_gradient",
            "lcc_net_train_step", "lcc_selftest_bounded_wait", "lcc_plan_create", "lcc_plan_update",
            "lcc_plan_set_proposals", "lcc_plan_set_staging", "lcc_plan_encode", "lcc_plan_capture", "lcc_plan_replay", "lcc_plan_sync", "lcc_plan_encode_host", "lcc_plan_get_info", "lcc_plan_stats",
            "lcc_plan_destroy", "lcc_autotune"]


def status_string(s: int) -> str:
    try:
        return load().lcc_status_string(s).decode()
    except Exception:
        return str(s)


def _check(st: int, what: str):
    if st != OK:
        raise LccError(st, what)


def _ptr(x) -> int | None:
    """Device address of a torch tensor, or an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_cuda") and not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        return x.data_ptr()
    raise TypeError(f"cannot take a device address of {type(x)}")


def _arr(ctype, values):
    return (ctype * len(values))(*values)


def default_params(**kw) -> lcc_params:
    p = lcc_params()
    load().lcc_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def imu_pose(t, acc, gyro, v_key, t_key: float, t_p: float) -> np.ndarray:
    """4x4 pose of the frame taken at t_p in the key frame's coordinates (lcc_imu_pose)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    acc = np.ascontiguousarray(acc, dtype=np.float64).reshape(-1, 3)
    gyro = np.ascontiguousarray(gyro, dtype=np.float64).reshape(-1, 3)
    v = np.ascontiguousarray(v_key, dtype=np.float64).reshape(3)
    out = np.zeros(16, np.float64)
    _check(load().lcc_imu_pose(t.ctypes.data, acc.ctypes.data, gyro.ctypes.data, len(t), v.ctypes.data,
                               float(t_key), float(t_p), out.ctypes.data), "lcc_imu_pose")
    return out.reshape(4, 4)


def sensor(s) -> lcc_sensor:
    return lcc_sensor(s.rows, s.cols, s.elev_min_deg, s.elev_max_deg, s.max_range_m)


class Keyframe:
    def __init__(self, ctx: "Context"):
        self.ctx = ctx
        h = ctypes.c_void_p()
        _check(load().lcc_keyframe_create(ctx.h, ctypes.byref(h)), "lcc_keyframe_create")
        self.h = h

    def free(self):
        if self.h:
            load().lcc_keyframe_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """An lcc context bound to a CUDA stream (torch stream or raw handle)."""

    def __init__(self, sensor_, params: lcc_params | None = None, stream=None):
        self.lib = load()
        self.sensor = sensor(sensor_) if not isinstance(sensor_, lcc_sensor) else sensor_
        self.params = params or default_params()
        if stream is None:
            handle = None
        elif isinstance(stream, int):
            handle = stream
        else:
            handle = stream.cuda_stream
        self.stream_handle = handle
        h = ctypes.c_void_p()
        _check(self.lib.lcc_create(ctypes.byref(h), ctypes.byref(self.sensor), ctypes.byref(self.params), handle),
               "lcc_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.lcc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- queries ---
    @property
    def max_encoded_bytes(self) -> int:
        return int(self.lib.lcc_max_encoded_bytes(self.h))

    @property
    def num_tiles(self) -> int:
        return int(self.lib.lcc_num_tiles(self.h))

    def tables(self) -> dict:
        H, W = self.sensor.rows, self.sensor.cols
        out = {k: np.zeros(n, np.float32) for k, n in
               [("ce", H), ("se", H), ("ct", W), ("st", W), ("rbc", H + 1), ("rbs", H + 1), ("cbc", W), ("cbs", W)]}
        _check(self.lib.lcc_tables(self.h, *[out[k].ctypes.data for k in
                                             ("ce", "se", "ct", "st", "rbc", "rbs", "cbc", "cbs")]), "lcc_tables")
        return out

    # --- calls (async on the context stream) ---
    def lcc_range_image(self, d_pts, n: int, d_range=None, d_valid=None):
        _check(self.lib.lcc_range_image(self.h, _ptr(d_pts), n, _ptr(d_range), _ptr(d_valid)), "lcc_range_image")

    def lcc_encode_keyframe(self, d_pts, n: int, kf: Keyframe | None, d_out, cap: int, out_bytes):
        _check(self.lib.lcc_encode_keyframe(self.h, _ptr(d_pts), n, kf.h if kf else None, _ptr(d_out), cap,
                                            _ptr(out_bytes)), "lcc_encode_keyframe")

    def lcc_encode_keyframe_seeded(self, d_pts, n: int, d_prop, skip_logit: float, kf: Keyframe | None, d_out,
                                   cap: int, out_bytes):
        _check(self.lib.lcc_encode_keyframe_seeded(self.h, _ptr(d_pts), n, _ptr(d_prop), skip_logit,
                                                   kf.h if kf else None, _ptr(d_out), cap, _ptr(out_bytes)),
               "lcc_encode_keyframe_seeded")

    def lcc_encode_keyframes(self, d_pts: list, n: list, d_prop: list | None, skip_logit: float, d_out: list,
                             cap: list, out_bytes):
        nf = len(d_pts)
        props = _arr(ctypes.c_void_p, [_ptr(x) for x in d_prop]) if d_prop is not None else None
        _check(self.lib.lcc_encode_keyframes(self.h, nf, _arr(ctypes.c_void_p, [_ptr(x) for x in d_pts]),
                                             _arr(ctypes.c_int64, n), props, skip_logit,
                                             _arr(ctypes.c_void_p, [_ptr(x) for x in d_out]),
                                             _arr(ctypes.c_uint64, cap), _ptr(out_bytes)), "lcc_encode_keyframes")

    def lcc_encode_pframe(self, kf: Keyframe, pose: np.ndarray, d_pts, n: int, d_out, cap: int, out_bytes):
        pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
        _check(self.lib.lcc_encode_pframe(self.h, kf.h, pose.ctypes.data, _ptr(d_pts), n, _ptr(d_out), cap,
                                          _ptr(out_bytes)), "lcc_encode_pframe")

    def lcc_encode_pframes(self, kf: Keyframe, poses, d_pts: list, n: list, d_out: list, cap: list, out_bytes):
        poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1)
        nf = len(d_pts)
        _check(self.lib.lcc_encode_pframes(self.h, kf.h, nf, poses.ctypes.data,
                                           _arr(ctypes.c_void_p, [_ptr(x) for x in d_pts]),
                                           _arr(ctypes.c_int64, n), _arr(ctypes.c_void_p, [_ptr(x) for x in d_out]),
                                           _arr(ctypes.c_uint64, cap), _ptr(out_bytes)), "lcc_encode_pframes")

    def lcc_encode_sequence(self, key_index: int, poses, d_pts: list, n: list, d_out: list, cap: list, out_bytes,
                            kf: Keyframe | None = None):
        poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1)
        nf = len(d_pts)
        _check(self.lib.lcc_encode_sequence(self.h, nf, key_index, poses.ctypes.data,
                                            _arr(ctypes.c_void_p, [_ptr(x) for x in d_pts]),
                                            _arr(ctypes.c_int64, n), _arr(ctypes.c_void_p, [_ptr(x) for x in d_out]),
                                            _arr(ctypes.c_uint64, cap), _ptr(out_bytes), kf.h if kf else None),
               "lcc_encode_sequence")

    def lcc_encode_sequence_host(self, key_index: int, poses, h_pts: list, h_out: list, cap: list) -> np.ndarray:
        """HOST buffers: h_pts numpy float32 (n,4) arrays, h_out numpy uint8 arrays.  Synchronous."""
        poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1)
        nf = len(h_pts)
        nbytes = np.zeros(nf, np.uint64)
        _check(self.lib.lcc_encode_sequence_host(self.h, nf, key_index, poses.ctypes.data,
                                                 _arr(ctypes.c_void_p, [_host_ptr(a) for a in h_pts]),
                                                 _arr(ctypes.c_int64, [len(a) for a in h_pts]),
                                                 _arr(ctypes.c_void_p, [_host_ptr(a) for a in h_out]),
                                                 _arr(ctypes.c_uint64, cap), nbytes.ctypes.data),
               "lcc_encode_sequence_host")
        return nbytes

    def lcc_keyframe_from_stream(self, d_bits, nbytes: int, kf: Keyframe):
        _check(self.lib.lcc_keyframe_from_stream(self.h, _ptr(d_bits), nbytes, kf.h), "lcc_keyframe_from_stream")

    def lcc_decode(self, d_bits, nbytes: int, kf: Keyframe | None, pose, d_range=None, d_xyz4=None, d_valid=None):
        pose_p = None
        if pose is not None:
            pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
            pose_p = pose.ctypes.data
        _check(self.lib.lcc_decode(self.h, _ptr(d_bits), nbytes, kf.h if kf else None, pose_p, _ptr(d_range),
                                   _ptr(d_xyz4), _ptr(d_valid)), "lcc_decode")

    def lcc_decode_sequence(self, key_index: int, poses, d_bits, nbytes, d_range=None, d_xyz4=None, d_valid=None):
        """Decode the frames of one sequence (device buffers; optional lists of outputs)."""
        n = len(d_bits)
        P = ctypes.c_void_p * n
        pz = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(n, 16))
        nb = np.ascontiguousarray(np.asarray(nbytes, dtype=np.uint64))

        def arr(xs):
            return None if xs is None else P(*[_ptr(x) for x in xs])

        bits_a, rng_a, xyz_a, val_a = arr(d_bits), arr(d_range), arr(d_xyz4), arr(d_valid)
        _check(self.lib.lcc_decode_sequence(self.h, n, key_index, pz.ctypes.data, bits_a, nb.ctypes.data, rng_a,
                                            xyz_a, val_a), "lcc_decode_sequence")

    def _entropy(self, fn, name, d_in, in_size, d_out, out_cap, out_bytes):
        n = len(d_in)
        P = ctypes.c_void_p * n
        isz = np.ascontiguousarray(np.asarray(in_size, dtype=np.uint64))
        cap = np.ascontiguousarray(np.asarray(out_cap, dtype=np.uint64))
        _check(fn(self.h, n, P(*[_ptr(x) for x in d_in]), isz.ctypes.data, P(*[_ptr(x) for x in d_out]),
                  cap.ctypes.data, _ptr(out_bytes)), name)

    def lcc_entropy_encode(self, d_in, in_size, d_out, out_cap, out_bytes):
        """Entropy streams of fixed-width streams (device buffers; out_bytes a device uint64/int64 array)."""
        self._entropy(self.lib.lcc_entropy_encode, "lcc_entropy_encode", d_in, in_size, d_out, out_cap, out_bytes)

    def lcc_entropy_decode(self, d_in, in_bytes, d_out, out_cap, out_bytes):
        """Fixed-width streams back from entropy streams (device buffers)."""
        self._entropy(self.lib.lcc_entropy_decode, "lcc_entropy_decode", d_in, in_bytes, d_out, out_cap, out_bytes)

    def lcc_sync(self) -> int:
        return int(self.lib.lcc_sync(self.h))

    def lcc_last_stats(self, frame: int = 0) -> dict:
        st = lcc_stats()
        _check(self.lib.lcc_last_stats(self.h, frame, ctypes.byref(st)), "lcc_last_stats")
        out = {n: getattr(st, n) for n, _ in lcc_stats._fields_}
        out["fit_rounds"] = list(st.fit_rounds)
        return out

    def lcc_tile_records(self, frame: int = 0) -> np.ndarray:
        out = np.zeros(self.num_tiles, TILE_INFO_DTYPE)
        _check(self.lib.lcc_tile_records(self.h, frame, out.ctypes.data, len(out)), "lcc_tile_records")
        return out

    def lcc_tile_coefficients(self, frame: int = 0) -> np.ndarray:
        """(T, 4) float32: a, b, c and the axis of each tile's last fit (plane3 contexts)."""
        out = np.zeros((self.num_tiles, 4), np.float32)
        _check(self.lib.lcc_tile_coefficients(self.h, frame, out.ctypes.data, self.num_tiles), "lcc_tile_coefficients")
        return out

    def lcc_set_profiling(self, enable: bool):
        _check(self.lib.lcc_set_profiling(self.h, 1 if enable else 0), "lcc_set_profiling")

    def lcc_kernel_times(self) -> dict:
        names = (ctypes.c_char * 16 * 16)()
        launches = np.zeros(16, np.int64)
        ms = np.zeros(16, np.float64)
        n = self.lib.lcc_kernel_times(self.h, names, launches.ctypes.data, ms.ctypes.data, 16)
        return {bytes(names[i]).split(b"\0")[0].decode(): (int(launches[i]), float(ms[i])) for i in range(n)}

    def lcc_kernel_timeline(self, cap: int = 4096) -> list:
        """[(name, start_ms, end_ms)] of the launches timed since profiling was enabled."""
        names = (ctypes.c_char * 16 * cap)()
        t0 = np.zeros(cap, np.float32)
        t1 = np.zeros(cap, np.float32)
        n = self.lib.lcc_kernel_timeline(self.h, names, t0.ctypes.data, t1.ctypes.data, cap)
        return [(bytes(names[i]).split(b"\0")[0].decode(), float(t0[i]), float(t1[i])) for i in range(n)]


def _host_ptr(a) -> int:
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("host arrays must be contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(type(a))


def lcc_range_image_static(sensor_, d_pts, n: int, d_range=None, d_valid=None, stream=None):
    """Range image with the library's fixed scratch (no context, no allocation).  Asynchronous on
    `stream` (torch stream, raw handle or None for the default stream); returns the status."""
    sn = sensor(sensor_) if not isinstance(sensor_, lcc_sensor) else sensor_
    sp = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
    return int(load().lcc_range_image_static(ctypes.byref(sn), _ptr(d_pts), n, _ptr(d_range), _ptr(d_valid), sp))


class Plan:
    """A table of sequences encoded together (lcc_plan_*).

    ``seqs`` is a list of dicts with keys ``ctx`` (index into ``contexts``),
    ``key_interval``, ``poses`` ((nframes, 4, 4) float64, frame -> its group's key frame),
    ``d_pts`` (list of CUDA float4 tensors), ``n``, ``d_out`` (list of CUDA uint8 tensors),
    ``cap`` and ``d_nbytes`` (CUDA int64 tensor of nframes)."""

    def __init__(self, contexts: list, seqs: list):
        self.lib = load()
        self.contexts = contexts
        self._keep = []
        descs = self._descs(seqs)
        h = ctypes.c_void_p()
        ctxs = _arr(ctypes.c_void_p, [c.h for c in contexts])
        _check(self.lib.lcc_plan_create(ctypes.byref(h), len(contexts), ctxs, len(seqs), descs), "lcc_plan_create")
        self.h = h

    def _descs(self, seqs):
        keep = []
        descs = (lcc_seq_desc * len(seqs))()
        for i, q in enumerate(seqs):
            nf = len(q["d_pts"])
            poses = np.ascontiguousarray(q["poses"], dtype=np.float64).reshape(-1)
            arrs = (poses, _arr(ctypes.c_void_p, [_ptr(x) for x in q["d_pts"]]), _arr(ctypes.c_int64, q["n"]),
                    _arr(ctypes.c_void_p, [_ptr(x) for x in q["d_out"]]), _arr(ctypes.c_uint64, q["cap"]))
            keep.append(arrs)
            descs[i] = lcc_seq_desc(q["ctx"], nf, q["key_interval"], 0, poses.ctypes.data,
                                    ctypes.addressof(arrs[1]), ctypes.addressof(arrs[2]), ctypes.addressof(arrs[3]),
                                    ctypes.addressof(arrs[4]), _ptr(q["d_nbytes"]))
        self._keep = keep
        return descs

    def update(self, seqs: list):
        _check(self.lib.lcc_plan_update(self.h, len(seqs), self._descs(seqs)), "lcc_plan_update")

    def set_proposals(self, net: "Net | None", skip_logit: float = 0.0):
        """Seed the key frames of 8x8-tile classes with the net's proposals (None: plain)."""
        self.net = net
        _check(self.lib.lcc_plan_set_proposals(self.h, net.h if net is not None else None, skip_logit),
               "lcc_plan_set_proposals")

    def set_staging(self, enable: bool):
        """Host points copied by the copy engines ahead of each chunk (lcc_plan_set_staging)."""
        _check(self.lib.lcc_plan_set_staging(self.h, int(enable)), "lcc_plan_set_staging")

    def encode(self):
        _check(self.lib.lcc_plan_encode(self.h), "lcc_plan_encode")

    def capture(self):
        _check(self.lib.lcc_plan_capture(self.h), "lcc_plan_capture")

    def replay(self):
        _check(self.lib.lcc_plan_replay(self.h), "lcc_plan_replay")

    def sync(self) -> int:
        return int(self.lib.lcc_plan_sync(self.h))

    def encode_host(self, h_out) -> np.ndarray:
        """lcc_plan_encode_host: h_out is a list of page-locked host buffers (numpy arrays or CPU
        tensors), one per frame in table order; returns the stream sizes.  Synchronous."""
        n = len(h_out)
        sizes = np.zeros(n, np.uint64)
        ptrs = _arr(ctypes.c_void_p, [_host_ptr(a) for a in h_out])
        _check(self.lib.lcc_plan_encode_host(self.h, ptrs, sizes.ctypes.data), "lcc_plan_encode_host")
        return sizes

    def info(self) -> dict:
        i = lcc_plan_info()
        _check(self.lib.lcc_plan_get_info(self.h, ctypes.byref(i)), "lcc_plan_get_info")
        return {n: getattr(i, n) for n, _ in lcc_plan_info._fields_}

    def stats(self, seq: int = -1, frame: int = 0) -> dict:
        """lcc_plan_stats: one frame's statistics of the last encode, or (seq=-1) their sum."""
        st = lcc_stats()
        _check(self.lib.lcc_plan_stats(self.h, seq, frame, ctypes.byref(st)), "lcc_plan_stats")
        out = {n: getattr(st, n) for n, _ in lcc_stats._fields_}
        out["fit_rounds"] = list(st.fit_rounds)
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.lcc_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TUNE_SHAPES = ((4, 4), (4, 8), (8, 8), (8, 16))


def autotune(sensor_, base: lcc_params, key_index: int, poses, d_pts: list, n: list, reps: int = 3,
             max_err_m: float = 0.02, bytes_slack: float = 0.05, stream=None, shapes=None):
    """lcc_autotune: returns (best lcc_params, list of candidate dicts).  shapes: the tile shapes
    to search (a subset of TUNE_SHAPES; None = all)."""
    lib = load()
    sn = sensor(sensor_) if not isinstance(sensor_, lcc_sensor) else sensor_
    poses = np.ascontiguousarray(poses, dtype=np.float64).reshape(-1)
    res = (lcc_tune_result * 64)()
    nres = ctypes.c_int32()
    best = lcc_params()
    sp = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
    mask = 0 if shapes is None else sum(1 << TUNE_SHAPES.index(tuple(t)) for t in shapes)
    st = lib.lcc_autotune(ctypes.byref(sn), ctypes.byref(base), len(d_pts), key_index, poses.ctypes.data,
                          _arr(ctypes.c_void_p, [_ptr(x) for x in d_pts]), _arr(ctypes.c_int64, n), reps,
                          max_err_m, bytes_slack, mask, sp, res, 64, ctypes.byref(nres), ctypes.byref(best))
    _check(st, "lcc_autotune")
    rows = [{k: getattr(res[i], k) for k, _ in lcc_tune_result._fields_ if k != "reserved"}
            for i in range(min(nres.value, 64))]
    return best, rows


class Net:
    """The learned tile proposal net (lcc_net_*): fp32 master parameters on the device."""

    def __init__(self, params: np.ndarray, max_tiles: int, stream=None):
        self.lib = load()
        params = np.ascontiguousarray(params, dtype=np.float32)
        assert params.size == self.lib.lcc_net_num_params()
        sp = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
        h = ctypes.c_void_p()
        _check(self.lib.lcc_net_create(ctypes.byref(h), params.ctypes.data, max_tiles, sp), "lcc_net_create")
        self.h = h
        self.max_tiles = max_tiles

    @staticmethod
    def num_params() -> int:
        return int(load().lcc_net_num_params())

    def params(self) -> np.ndarray:
        out = np.zeros(self.num_params(), np.float32)
        _check(self.lib.lcc_net_get_params(self.h, out.ctypes.data), "lcc_net_get_params")
        return out

    def set_params(self, params: np.ndarray):
        params = np.ascontiguousarray(params, dtype=np.float32)
        _check(self.lib.lcc_net_set_params(self.h, params.ctypes.data), "lcc_net_set_params")

    def forward(self, d_x, ntiles: int, d_out):
        _check(self.lib.lcc_net_forward(self.h, _ptr(d_x), ntiles, _ptr(d_out)), "lcc_net_forward")

    def sync(self) -> int:
        return int(self.lib.lcc_net_sync(self.h))

    def gradient(self, d_x, d_labels, ntiles: int, d_grad=None, d_loss=None):
        _check(self.lib.lcc_net_gradient(self.h, _ptr(d_x), _ptr(d_labels), ntiles, _ptr(d_grad), _ptr(d_loss)),
               "lcc_net_gradient")

    def train_step(self, d_x, d_labels, ntiles: int, lr: float, step: int, d_loss=None):
        _check(self.lib.lcc_net_train_step(self.h, _ptr(d_x), _ptr(d_labels), ntiles, lr, step, _ptr(d_loss)),
               "lcc_net_train_step")

    def close(self):
        if getattr(self, "h", None):
            self.lib.lcc_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def net_tile_inputs(ctx: "Context", d_pts, n: int, d_x, d_anchor):
    _check(load().lcc_net_tile_inputs(ctx.h, _ptr(d_pts), n, _ptr(d_x), _ptr(d_anchor)), "lcc_net_tile_inputs")


def net_tile_labels(ctx: "Context", frame: int, d_anchor, d_labels):
    """Training labels (fit, n, d - n.anchor) of frame `frame` of the context's last encode."""
    _check(load().lcc_net_tile_labels(ctx.h, frame, _ptr(d_anchor), _ptr(d_labels)), "lcc_net_tile_labels")


def net_tile_inputs_batch(ctx: "Context", d_pts: list, n: list, d_x, d_anchor):
    _check(load().lcc_net_tile_inputs_batch(ctx.h, len(d_pts), _arr(ctypes.c_void_p, [_ptr(x) for x in d_pts]),
                                            _arr(ctypes.c_int64, n), _ptr(d_x), _ptr(d_anchor)),
           "lcc_net_tile_inputs_batch")
