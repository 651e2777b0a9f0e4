"""CPU oracle of the spatio-temporal LiDAR encoder — TEST INFRASTRUCTURE ONLY.

Thin ctypes wrapper around ``lcc_oracle.c`` (plain single-threaded C).  Only the
test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package; the GPU library never does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lcc_oracle.c")
_HDR = os.path.join(_HERE, "lcc_oracle.h")
_LIB_PATH = os.path.join(_HERE, "liblcc_oracle.so")
_lock = threading.Lock()
_lib = None

T_EMPTY, T_RAW, T_RUN_START, T_RUN_CONT, T_TEMPORAL, T_TEMPORAL_CONT = range(6)
T_RUN_START3 = 6   # .. 8: a three-coefficient run start along axis x, y, z
FIT_EMPTY, FIT_FAIL, FIT_OK = range(3)
OK, ERR_ARG, ERR_CORRUPT, ERR_CAPACITY, ERR_INCONSISTENT = 0, -1, -2, -3, -4


class Sensor(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("cols", ctypes.c_int32),
                ("elev_min_deg", ctypes.c_double), ("elev_max_deg", ctypes.c_double),
                ("max_range_m", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("tile_h", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("fit_thr_m", ctypes.c_float), ("quant_m", ctypes.c_float),
                ("max_refits", ctypes.c_int32), ("min_inlier_frac", ctypes.c_float),
                ("merge_runs", ctypes.c_int32), ("no_delta", ctypes.c_int32), ("raw_exact", ctypes.c_int32),
                ("temporal_candidates", ctypes.c_int32), ("temporal_runs", ctypes.c_int32),
                ("plane3", ctypes.c_int32)]


class TileFit(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("n_valid", ctypes.c_int32), ("n_inlier", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("borderline", ctypes.c_int32), ("degenerate", ctypes.c_int32),
                ("plane", ctypes.c_float * 4), ("plane64", ctypes.c_double * 4), ("lam", ctypes.c_double * 3),
                ("coef", ctypes.c_float * 3), ("axis", ctypes.c_int32)]


class TileTemporal(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("kref", ctypes.c_int32), ("n_valid", ctypes.c_int32),
                ("n_inlier", ctypes.c_int32), ("rounds", ctypes.c_int32), ("borderline", ctypes.c_int32),
                ("plane", ctypes.c_float * 4)]


FIT_DTYPE = np.dtype([("status", "<i4"), ("n_valid", "<i4"), ("n_inlier", "<i4"), ("rounds", "<i4"),
                      ("borderline", "<i4"), ("degenerate", "<i4"), ("plane", "<f4", 4),
                      ("plane64", "<f8", 4), ("lam", "<f8", 3), ("coef", "<f4", 3), ("axis", "<i4")], align=True)
TEMPORAL_DTYPE = np.dtype([("status", "<i4"), ("kref", "<i4"), ("n_valid", "<i4"), ("n_inlier", "<i4"),
                           ("rounds", "<i4"), ("borderline", "<i4"), ("plane", "<f4", 4)], align=True)
assert FIT_DTYPE.itemsize == ctypes.sizeof(TileFit)
assert TEMPORAL_DTYPE.itemsize == ctypes.sizeof(TileTemporal)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -ffp-contract=off so no multiply-add is fused)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            vp, i64, u64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
            L.orc_tables.restype = i32
            L.orc_tables.argtypes = [vp] * 9
            L.orc_range_image.restype = i64
            L.orc_range_image.argtypes = [vp, vp, i64, vp, vp, vp]
            L.orc_tls_fit.restype = i32
            L.orc_tls_fit.argtypes = [vp, i32, vp, vp, vp]
            L.orc_fit_tiles.restype = i32
            L.orc_fit_tiles.argtypes = [vp, vp, vp, vp]
            L.orc_fit_tiles_seeded.restype = i32
            L.orc_fit_tiles_seeded.argtypes = [vp, vp, vp, vp, ctypes.c_float, vp]
            L.orc_temporal_tiles.restype = i32
            L.orc_temporal_tiles.argtypes = [vp, vp, vp, vp, vp, vp]
            L.orc_pack3.restype = i64
            L.orc_pack3.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, u64, vp, vp]
            L.orc_plane_to3.restype = None
            L.orc_plane_to3.argtypes = [vp, vp, vp]
            L.orc_plane_from3.restype = None
            L.orc_plane_from3.argtypes = [i32, vp, vp]
            L.orc_pack.restype = i64
            L.orc_pack.argtypes = [vp, vp, i32, vp, vp, vp, vp, vp, vp, u64, vp, vp]
            L.orc_encode_keyframe.restype = i64
            L.orc_encode_keyframe.argtypes = [vp, vp, vp, i64, vp, u64, vp, vp, vp]
            L.orc_encode_pframe.restype = i64
            L.orc_encode_pframe.argtypes = [vp, vp, vp, vp, vp, i64, vp, u64, vp, vp, vp]
            L.orc_decode.restype = i32
            L.orc_decode.argtypes = [vp, vp, u64, vp, vp, vp, vp, vp]
            L.orc_kf_table_from_stream.restype = i32
            L.orc_kf_table_from_stream.argtypes = [vp, vp, u64, vp]
            _lib = L
    return _lib


def sensor(s) -> Sensor:
    """Convert any object with rows/cols/elev_min_deg/elev_max_deg/max_range_m."""
    return Sensor(s.rows, s.cols, s.elev_min_deg, s.elev_max_deg, s.max_range_m)


def params(tile_h=4, tile_w=4, fit_thr_m=0.05, quant_m=0.02, max_refits=3, min_inlier_frac=0.75,
           merge_runs=1, no_delta=0, raw_exact=0, temporal_candidates=1, temporal_runs=1, plane3=0) -> Params:
    return Params(tile_h, tile_w, fit_thr_m, quant_m, max_refits, min_inlier_frac, merge_runs, no_delta, raw_exact,
                  temporal_candidates, temporal_runs, plane3)


def n_tiles(s: Sensor, p: Params) -> int:
    return ((s.rows + p.tile_h - 1) // p.tile_h) * ((s.cols + p.tile_w - 1) // p.tile_w)


def tables(s: Sensor) -> dict:
    H, W = s.rows, s.cols
    out = {k: np.zeros(n, np.float32) for k, n in
           [("ce", H), ("se", H), ("ct", W), ("st", W), ("rbc", H + 1), ("rbs", H + 1), ("cbc", W), ("cbs", W)]}
    rc = lib().orc_tables(ctypes.byref(s), *[_p(out[k]) for k in ("ce", "se", "ct", "st", "rbc", "rbs", "cbc", "cbs")])
    if rc != OK:
        raise ValueError(f"orc_tables: {rc}")
    return out


def beams(s: Sensor) -> np.ndarray:
    """(H, W, 3) fp32 pixel-centre beam directions as the oracle forms them."""
    t = tables(s)
    u = np.empty((s.rows, s.cols, 3), np.float32)
    u[..., 0] = t["ce"][:, None] * t["ct"][None, :]
    u[..., 1] = t["ce"][:, None] * t["st"][None, :]
    u[..., 2] = np.broadcast_to(t["se"][:, None], (s.rows, s.cols))
    return u


def range_image(s: Sensor, pts: np.ndarray):
    pts = np.ascontiguousarray(pts, dtype=np.float32)
    rng = np.zeros(s.rows * s.cols, np.float32)
    pix = np.zeros(len(pts), np.int32)
    st = np.zeros(4, np.int64)
    lib().orc_range_image(ctypes.byref(s), _p(pts), len(pts), _p(rng), _p(pix), _p(st))
    return rng.reshape(s.rows, s.cols), pix, st


def tls_fit(p: np.ndarray):
    p = np.ascontiguousarray(p, dtype=np.float64)
    nrm = np.zeros(3)
    d = np.zeros(1)
    lam = np.zeros(3)
    rc = lib().orc_tls_fit(_p(p), len(p), _p(nrm), _p(d), _p(lam))
    if rc != OK:
        raise ValueError(f"orc_tls_fit: {rc}")
    return nrm, float(d[0]), lam


def fit_tiles(s: Sensor, p: Params, rng: np.ndarray) -> np.ndarray:
    rng = np.ascontiguousarray(rng, dtype=np.float32)
    out = np.zeros(n_tiles(s, p), FIT_DTYPE)
    rc = lib().orc_fit_tiles(ctypes.byref(s), ctypes.byref(p), _p(rng), _p(out))
    if rc != OK:
        raise ValueError(f"orc_fit_tiles: {rc}")
    return out


def fit_tiles_seeded(s: Sensor, p: Params, rng: np.ndarray, prop: np.ndarray, skip_logit: float) -> np.ndarray:
    """Fit of every tile seeded by a proposal (T, 5) float32 per tile: (logit, v0, v1, v2, d_rel)."""
    rng = np.ascontiguousarray(rng, dtype=np.float32)
    prop = np.ascontiguousarray(prop, dtype=np.float32)
    out = np.zeros(n_tiles(s, p), FIT_DTYPE)
    assert prop.shape == (len(out), 5)
    rc = lib().orc_fit_tiles_seeded(ctypes.byref(s), ctypes.byref(p), _p(rng), _p(prop), skip_logit, _p(out))
    if rc != OK:
        raise ValueError(f"orc_fit_tiles_seeded: {rc}")
    return out


def temporal_tiles(s: Sensor, p: Params, rng: np.ndarray, kf_table: np.ndarray, pose: np.ndarray):
    rng = np.ascontiguousarray(rng, dtype=np.float32)
    kf_table = np.ascontiguousarray(kf_table, dtype=np.float32)
    pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
    out = np.zeros(n_tiles(s, p), TEMPORAL_DTYPE)
    rc = lib().orc_temporal_tiles(ctypes.byref(s), ctypes.byref(p), _p(rng), _p(kf_table), _p(pose), _p(out))
    if rc != OK:
        raise ValueError(f"orc_temporal_tiles: {rc}")
    return out


def max_stream_bytes(s: Sensor, p: Params) -> int:
    npx = s.rows * s.cols
    nt = n_tiles(s, p)
    return 64 + 4 * (npx // 32 + 1 + nt // 8 + 1 + 4 * nt + 2 * nt + npx // 32 + 1) + 4 * (npx * 40 // 32 + 2)


def pack(s: Sensor, p: Params, kind: int, rng, fit_plane, fit_ok, temporal_plane=None, temporal_kref=None,
         fit_coef=None):
    """Merge + code + pack given per-tile results (fit_coef: (T, 4) a, b, c, axis for plane3
    streams).  Returns (bytes, kf_table, modes)."""
    rng = np.ascontiguousarray(rng, dtype=np.float32)
    fit_plane = np.ascontiguousarray(fit_plane, dtype=np.float32)
    fit_ok = np.ascontiguousarray(fit_ok, dtype=np.uint8)
    if temporal_plane is not None:
        temporal_plane = np.ascontiguousarray(temporal_plane, dtype=np.float32)
        temporal_kref = np.ascontiguousarray(temporal_kref, dtype=np.int32)
    nt = n_tiles(s, p)
    cap = max_stream_bytes(s, p)
    out = np.zeros(cap, np.uint8)
    kft = np.zeros((nt, 4), np.float32)
    modes = np.zeros(nt, np.uint8)
    if fit_coef is not None:
        fit_coef = np.ascontiguousarray(fit_coef, dtype=np.float32)
    n = lib().orc_pack3(ctypes.byref(s), ctypes.byref(p), kind, _p(rng), _p(fit_plane), _p(fit_coef), _p(fit_ok),
                        _p(temporal_plane), _p(temporal_kref), _p(out), cap, _p(kft), _p(modes))
    if n < 0:
        raise ValueError(f"orc_pack: {n}")
    if n > cap:
        raise ValueError("orc_pack: capacity")
    return out[:n].copy(), kft, modes


def encode_keyframe(s: Sensor, p: Params, pts: np.ndarray):
    """Returns (bytes, kf_table (ntiles,4), fits, modes)."""
    pts = np.ascontiguousarray(pts, dtype=np.float32)
    nt = n_tiles(s, p)
    cap = max_stream_bytes(s, p)
    out = np.zeros(cap, np.uint8)
    kft = np.zeros((nt, 4), np.float32)
    fits = np.zeros(nt, FIT_DTYPE)
    modes = np.zeros(nt, np.uint8)
    n = lib().orc_encode_keyframe(ctypes.byref(s), ctypes.byref(p), _p(pts), len(pts), _p(out), cap,
                                  _p(kft), _p(fits), _p(modes))
    if n < 0 or n > cap:
        raise ValueError(f"orc_encode_keyframe: {n}")
    return out[:n].copy(), kft, fits, modes


def encode_pframe(s: Sensor, p: Params, kf_table: np.ndarray, pose: np.ndarray, pts: np.ndarray):
    """Returns (bytes, fits, temporal, modes)."""
    pts = np.ascontiguousarray(pts, dtype=np.float32)
    kf_table = np.ascontiguousarray(kf_table, dtype=np.float32)
    pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
    nt = n_tiles(s, p)
    cap = max_stream_bytes(s, p)
    out = np.zeros(cap, np.uint8)
    fits = np.zeros(nt, FIT_DTYPE)
    tmp = np.zeros(nt, TEMPORAL_DTYPE)
    modes = np.zeros(nt, np.uint8)
    n = lib().orc_encode_pframe(ctypes.byref(s), ctypes.byref(p), _p(kf_table), _p(pose), _p(pts), len(pts),
                                _p(out), cap, _p(fits), _p(tmp), _p(modes))
    if n < 0 or n > cap:
        raise ValueError(f"orc_encode_pframe: {n}")
    return out[:n].copy(), fits, tmp, modes


def decode(s: Sensor, bits: np.ndarray, kf_table=None, pose=None):
    """Returns (range (H,W), xyz4 (H,W,4), valid words) or raises on a corrupt stream."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    npx = s.rows * s.cols
    rng = np.zeros(npx, np.float32)
    xyz = np.zeros((npx, 4), np.float32)
    valid = np.zeros((npx + 31) // 32, np.uint32)
    if kf_table is not None:
        kf_table = np.ascontiguousarray(kf_table, dtype=np.float32)
    if pose is not None:
        pose = np.ascontiguousarray(pose, dtype=np.float64).reshape(16)
    rc = lib().orc_decode(ctypes.byref(s), _p(bits), len(bits), _p(kf_table), _p(pose), _p(rng), _p(xyz),
                          _p(valid))
    if rc != OK:
        raise ValueError(f"orc_decode: {rc}")
    return rng.reshape(s.rows, s.cols), xyz.reshape(s.rows, s.cols, 4), valid


def decode_status(s: Sensor, bits: np.ndarray, kf_table=None, pose=None) -> int:
    try:
        decode(s, bits, kf_table, pose)
        return OK
    except ValueError as e:
        return int(str(e).split(":")[1])


def kf_table_from_stream(s: Sensor, bits: np.ndarray, n_tiles_: int) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    kft = np.zeros((n_tiles_, 4), np.float32)
    rc = lib().orc_kf_table_from_stream(ctypes.byref(s), _p(bits), len(bits), _p(kft))
    if rc != OK:
        raise ValueError(f"orc_kf_table_from_stream: {rc}")
    return kft


def plane_to3(pl) -> tuple:
    """(axis, (a, b, c)) of a unit-normal fp32 plane (Eq. 3's form with the dominant axis)."""
    pl = np.ascontiguousarray(pl, dtype=np.float32)
    axis = ctypes.c_int32()
    abc = np.zeros(3, np.float32)
    lib().orc_plane_to3(_p(pl), ctypes.byref(axis), _p(abc))
    return int(axis.value), abc


def plane_from3(axis: int, abc) -> np.ndarray:
    abc = np.ascontiguousarray(abc, dtype=np.float32)
    pl = np.zeros(4, np.float32)
    lib().orc_plane_from3(int(axis), _p(abc), _p(pl))
    return pl
