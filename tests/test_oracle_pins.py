"""Pins of the CPU oracle against things other than itself.

Every test here checks the oracle against a closed form, a library routine, a
brute-force search or an invariant that the paper's definitions fix, so that a
dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.  No GPU is needed.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import synth
from tests import streamfmt

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sensor(rows=16, cols=64, lo=-15.0, hi=15.0, rmax=80.0):
    return O.Sensor(rows, cols, lo, hi, rmax)


def _centre_dirs(s):
    """fp64 pixel-centre beam directions from the grid definition (Sec. III-B)."""
    de = (s.elev_max_deg - s.elev_min_deg) / s.rows
    el = np.radians(s.elev_max_deg - (np.arange(s.rows) + 0.5) * de)
    az = -math.pi + (np.arange(s.cols) + 0.5) * 2 * math.pi / s.cols
    E, A = np.meshgrid(el, az, indexing="ij")
    return np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], -1)


# ---------------------------------------------------------------- Eq. 1-2 --

def test_beam_table_is_unit_and_matches_pixel_centres():
    s = _sensor(32, 1024, -24.8, 2.0)
    u = O.beams(s).astype(np.float64)
    ref = _centre_dirs(s)
    assert np.abs(np.linalg.norm(u, axis=-1) - 1).max() < 3e-7
    assert np.abs(u - ref).max() < 2e-7


def test_pixel_centre_points_land_in_their_pixel():
    s = _sensor(16, 512)
    d = _centre_dirs(s).reshape(-1, 3)
    r = np.random.default_rng(1).uniform(0.5, 79.0, len(d))
    pts = np.zeros((len(d), 4), np.float32)
    pts[:, :3] = (d * r[:, None]).astype(np.float32)
    img, pix, st = O.range_image(s, pts)
    assert (pix == np.arange(len(d))).all()
    assert st[3] == len(d)
    # Eq. 1: the stored value is the point's range
    r32 = np.sqrt((pts[:, :3].astype(np.float64) ** 2).sum(1))
    assert np.abs(img.reshape(-1) - r32).max() < 1e-5


def test_binning_matches_eq2_in_fp64_away_from_boundaries():
    s = _sensor(64, 2048, -24.8, 2.0)
    pts = synth.offgrid_points(60000, seed=3, r_hi=79.0, elev_lo_deg=-30, elev_hi_deg=8)
    img, pix, st = O.range_image(s, pts)
    p = pts[:, :3].astype(np.float64)
    az = np.arctan2(p[:, 1], p[:, 0])
    el = np.degrees(np.arctan2(p[:, 2], np.hypot(p[:, 0], p[:, 1])))
    de = (s.elev_max_deg - s.elev_min_deg) / s.rows
    rowf = (s.elev_max_deg - el) / de
    colf = (az + math.pi) / (2 * math.pi / s.cols)
    infov = (el < s.elev_max_deg) & (el > s.elev_min_deg)
    far_row = np.abs(rowf - np.round(rowf)) * de > 1e-4      # > 1e-4 deg from a row edge
    far_col = np.abs(colf - np.round(colf)) * 360 / s.cols > 1e-4
    sel = far_row & far_col
    exp = np.where(infov, np.floor(rowf).astype(np.int64) * s.cols + np.floor(colf).astype(np.int64) % s.cols, -1)
    assert sel.sum() > 50000
    assert (pix[sel] == exp[sel]).all()


def test_boundary_convention_and_azimuth_wrap():
    s = _sensor(8, 16, -10.0, 10.0)
    de = 20.0 / 8
    eps = 1e-4
    pts, want = [], []
    for k in range(1, 8):                 # row boundaries b_k between rows k-1 and k
        b = math.radians(10.0 - k * de)
        for sgn, row in ((+1, k - 1), (-1, k)):
            e = b + sgn * math.radians(eps)
            a = math.radians(-180 + 360 / 16 * 3.5)
            pts.append([10 * math.cos(e) * math.cos(a), 10 * math.cos(e) * math.sin(a), 10 * math.sin(e), 0])
            want.append(row * 16 + 3)
    for j in range(16):                   # column boundaries a_j between cols j-1 and j
        a = -math.pi + j * 2 * math.pi / 16
        for sgn, col in ((+1, j), (-1, (j - 1) % 16)):
            aa = a + sgn * math.radians(eps)
            e = math.radians(10.0 - 4.5 * de)
            pts.append([10 * math.cos(e) * math.cos(aa), 10 * math.cos(e) * math.sin(aa), 10 * math.sin(e), 0])
            want.append(4 * 16 + col)
    # outside the vertical field of view
    for e in (10.0 + eps, -10.0 - eps, 45.0, -60.0):
        er = math.radians(e)
        pts.append([10 * math.cos(er), 0, 10 * math.sin(er), 0])
        want.append(-1)
    _, pix, st = O.range_image(s, np.array(pts, np.float32))
    assert pix.tolist() == want
    assert st[2] == 4


def test_collision_keeps_nearest_and_drops_invalid():
    s = _sensor(16, 64)
    d = _centre_dirs(s).reshape(-1, 3)
    rng = np.random.default_rng(5)
    sel = rng.choice(len(d), 200, replace=False)
    ranges = rng.uniform(1, 70, (200, 4))
    pts = []
    for i, k in enumerate(sel):
        for r in ranges[i]:
            pts.append(np.append(d[k] * r, 0))
    pts = np.array(pts, np.float32)
    perm = rng.permutation(len(pts))
    img, pix, st = O.range_image(s, pts[perm])
    got = img.reshape(-1)[sel]
    want = np.sqrt((pts[:, :3].astype(np.float64) ** 2).sum(1)).reshape(200, 4).min(1)
    assert np.abs(got - want).max() < 1e-5
    assert st[0] == 800 and st[3] == 200
    bad = np.array([[np.nan, 1, 1, 0], [np.inf, 0, 0, 0], [0, 0, 0, 0], [100, 0, 0, 0]], np.float32)
    _, pix, st = O.range_image(s, bad)
    assert (pix == -1).all() and st[1] == 4


# --------------------------------------------------------- TLS plane fit --

def _cov(p):
    c = p.mean(0)
    q = p - c
    return q.T @ q / len(p), c


def test_tls_matches_numpy_eigh():
    rng = np.random.default_rng(7)
    for trial in range(300):
        n = int(rng.integers(3, 40))
        p = rng.normal(0, 1, (n, 3)) * rng.uniform(0.01, 3, 3) + rng.uniform(-40, 40, 3)
        nrm, d, lam = O.tls_fit(p)
        C, c = _cov(p)
        w, V = np.linalg.eigh(C)
        assert np.allclose(lam, w, rtol=1e-9, atol=1e-12 * w.max())
        if w[1] - w[0] > 1e-6 * w[2]:
            assert abs(abs(nrm @ V[:, 0]) - 1) < 1e-10
        assert abs(d - nrm @ c) < 1e-9 * max(1, abs(d))
        assert d >= 0 or abs(d) < 1e-9
        assert abs(np.linalg.norm(nrm) - 1) < 1e-12


def test_tls_matches_brute_force_search():
    from scipy.optimize import minimize
    rng = np.random.default_rng(11)
    th, ph = np.meshgrid(np.linspace(0, math.pi, 181), np.linspace(0, 2 * math.pi, 361), indexing="ij")
    grid = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1).reshape(-1, 3)
    for trial in range(12):
        n = int(rng.integers(3, 7))
        p = rng.normal(0, 1, (n, 3)) * np.array([2.0, 1.0, 0.2]) + rng.uniform(-5, 5, 3)
        q = p - p.mean(0)
        cost = ((q @ grid.T) ** 2).sum(0)
        g = grid[np.argmin(cost)]
        t0, p0 = math.acos(np.clip(g[2], -1, 1)), math.atan2(g[1], g[0])

        def f(x):
            v = np.array([math.sin(x[0]) * math.cos(x[1]), math.sin(x[0]) * math.sin(x[1]), math.cos(x[0])])
            return ((q @ v) ** 2).sum()

        res = minimize(f, [t0, p0], method="Nelder-Mead", options={"xatol": 1e-12, "fatol": 1e-20,
                                                                   "maxiter": 20000})
        v = np.array([math.sin(res.x[0]) * math.cos(res.x[1]), math.sin(res.x[0]) * math.sin(res.x[1]),
                      math.cos(res.x[0])])
        nrm, d, lam = O.tls_fit(p)
        assert abs(abs(nrm @ v) - 1) < 1e-10
        assert f([math.acos(np.clip(nrm[2], -1, 1)), math.atan2(nrm[1], nrm[0])]) <= res.fun * (1 + 1e-9) + 1e-18


def test_tls_recovers_exact_planes_with_canonical_sign():
    rng = np.random.default_rng(13)
    for trial in range(100):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        d = rng.uniform(-30, 30)
        a = np.cross(n, [1, 0, 0] if abs(n[0]) < 0.9 else [0, 1, 0])
        a /= np.linalg.norm(a)
        b = np.cross(n, a)
        uv = rng.uniform(-1, 1, (10, 2))
        p = d * n + uv[:, :1] * a + uv[:, 1:] * b
        nrm, dd, lam = O.tls_fit(p)
        s = 1 if d >= 0 else -1
        assert np.abs(nrm - s * n).max() < 1e-10
        assert abs(dd - abs(d)) < 1e-10
        assert lam[0] <= 1e-14 * lam[2]


def test_tile_golden_examples():
    """Hand-built tiles (tests/golden/tile_examples.json) with closed-form planes (Eq. 3)."""
    with open(os.path.join(GOLDEN, "tile_examples.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        p = np.array(case["points"], np.float64)
        nrm, d, lam = O.tls_fit(p)
        want = np.array(case["normal"], np.float64)
        assert np.abs(nrm - want).max() < 1e-9, case["name"]
        assert abs(d - case["d"]) < 1e-9, case["name"]


# -------------------------------------------------- iterative tile fit --

def test_noise_free_ground_tiles_fit_exactly_in_one_round():
    sen = synth.Sensor(64, 2048, -24.8, 2.0, 80.0)
    s = O.sensor(sen)
    p = O.params()
    pts = synth.Scene(5, 0, 0, 0).render(sen, sigma=0.0)
    bits, kft, fits, modes = O.encode_keyframe(s, p, pts)
    has = fits["n_valid"] >= 3
    assert (fits["status"][has] == O.FIT_OK).all()
    assert (fits["rounds"][has] == 1).all()
    assert np.abs(fits["plane"][has] - np.array([0, 0, -1, 1.7], np.float32)).max() < 1e-5
    rng, _, _ = O.range_image(s, pts)
    dec, _, _ = O.decode(s, bits)
    m = rng > 0
    # every point is fitted with residual code 0: the decoded range is the ray-cast plane range
    h = streamfmt.header(bits)
    assert h["n_fitted"] == m.sum() and h["n_raw"] == 0
    assert (streamfmt.residual_codes(bits) == 0).all()
    assert np.abs(dec[m] - rng[m]).max() < 0.01


def test_planted_outlier_is_dropped_and_plane_refit():
    """One pixel of a noise-free planar tile moved 0.5 m along its ray: the
    rounds must drop it, refit on the 15 others and recover the exact plane."""
    s = O.Sensor(4, 256, -10.0, 10.0, 80.0)
    p = O.params(min_inlier_frac=0.75)
    u = O.beams(s).astype(np.float64)
    n = np.array([0.9, 0.3, 0.1])
    n /= np.linalg.norm(n)
    d = 12.0
    dots = u @ n
    rng_img = np.where(dots > 0.1, d / np.where(dots > 0.1, dots, 1), 0).astype(np.float32)
    tc = int(np.argmax(dots[1])) // 4
    rng_img[1, 4 * tc + 2] -= 0.5
    fits = O.fit_tiles(s, p, rng_img)
    tile = fits[tc]
    assert tile["status"] == O.FIT_OK
    assert tile["n_valid"] == 16 and tile["n_inlier"] == 15
    assert tile["rounds"] in (2, 3)
    assert np.abs(tile["plane"] - np.array([*n, d], np.float32)).max() < 2e-5
    # the moved pixel is raw-coded, the others are fitted
    bits, kft, modes = O.pack(s, p, 0, rng_img, fits["plane"], fits["status"] == O.FIT_OK)
    dec, _, _ = O.decode(s, bits)
    assert abs(dec[1, 4 * tc + 2] - rng_img[1, 4 * tc + 2]) <= 0.01 + 1e-5
    # its neighbours (no outlier) fit in one round
    assert fits[tc - 2]["rounds"] == 1 and fits[tc - 2]["n_inlier"] == 16


def test_all_points_reading_rejects_tile_with_outlier():
    s = O.Sensor(4, 256, -10.0, 10.0, 80.0)
    u = O.beams(s).astype(np.float64)
    n = np.array([1.0, 0.0, 0.0])
    rng_img = (10.0 / (u @ n)).astype(np.float32)
    rng_img[rng_img < 0] = 0
    rng_img[2, 129] += 0.3
    fits_all = O.fit_tiles(s, O.params(min_inlier_frac=1.0), rng_img)
    fits_75 = O.fit_tiles(s, O.params(min_inlier_frac=0.75), rng_img)
    t = 128 // 4  # the tile covering azimuth 0 (x axis)
    assert fits_all[t]["status"] == O.FIT_FAIL
    assert fits_75[t]["status"] == O.FIT_OK


# ------------------------------------------------------- coding, decode --

@pytest.mark.parametrize("tile,thr", [((4, 4), 0.05), ((8, 8), 0.05), ((4, 4), 0.02), ((4, 8), 0.10),
                                      ((8, 16), 0.05)])
def test_decode_error_within_half_step(cfg1, tile, thr):
    sen, pts = cfg1
    s = O.sensor(sen)
    p = O.params(tile[0], tile[1], fit_thr_m=thr)
    bits, kft, fits, modes = O.encode_keyframe(s, p, pts)
    rng, _, _ = O.range_image(s, pts)
    dec, xyz, valid = O.decode(s, bits)
    m = rng > 0
    assert ((dec > 0) == m).all()
    assert np.abs(dec[m] - rng[m]).max() <= 0.01 + 1e-5
    # Eq. 1-2 inverted: the decoded point lies on the pixel's beam at the decoded range
    u = O.beams(s)
    assert np.abs(xyz[..., :3] - dec[..., None] * u).max() == 0


def test_partial_edge_tiles_round_trip():
    sen = synth.Sensor(18, 515, -15.0, 15.0, 80.0)
    pts = synth.Scene(9, 4, 6, 10, enclose=True).render(sen, sigma=0.02, dropout=0.05, seed=9)
    s = O.sensor(sen)
    for tile in ((4, 4), (8, 16)):
        p = O.params(*tile)
        bits, kft, fits, modes = O.encode_keyframe(s, p, pts)
        rng, _, _ = O.range_image(s, pts)
        dec, _, _ = O.decode(s, bits)
        m = rng > 0
        assert np.abs(dec[m] - rng[m]).max() <= 0.01 + 1e-5


def test_raw_round_trip_and_reencode_identity(cfg1):
    sen, pts = cfg1
    s = O.sensor(sen)
    p = O.params(min_inlier_frac=2.0)       # no plane can qualify: every tile is raw
    bits, kft, fits, modes = O.encode_keyframe(s, p, pts)
    assert set(np.unique(modes)) <= {O.T_RAW, O.T_EMPTY}
    rng, _, _ = O.range_image(s, pts)
    dec, xyz, _ = O.decode(s, bits)
    m = rng > 0
    q = np.float32(0.02)
    want = (np.floor(rng[m] / q + np.float32(0.5)) * q).astype(np.float32)
    assert (dec[m] == want).all()
    pts2 = xyz.reshape(-1, 4)[m.reshape(-1)]
    bits2, _, _, _ = O.encode_keyframe(s, p, pts2)
    assert bits2.tobytes() == bits.tobytes()


def test_greedy_run_invariants(cfg2_seq):
    seq = cfg2_seq
    s = O.sensor(seq.sensor)
    p = O.params()
    pts = seq.frames[seq.key_index]
    bits, kft, fits, modes = O.encode_keyframe(s, p, pts)
    rng, _, _ = O.range_image(s, pts)
    u = O.beams(s).astype(np.float64)
    TW = s.cols // p.tile_w

    def passes(t, plane):
        tr, tc = divmod(t, TW)
        r = rng[tr * 4:(tr + 1) * 4, tc * 4:(tc + 1) * 4].astype(np.float64).reshape(-1)
        uu = u[tr * 4:(tr + 1) * 4, tc * 4:(tc + 1) * 4].reshape(-1, 3)
        v = r > 0
        if v.sum() < 3:
            return False, False
        dot = uu[v] @ plane[:3].astype(np.float64)
        e = np.where(dot > 1e-3, r[v] - plane[3] / np.where(dot > 1e-3, dot, 1), np.inf)
        near = np.any(np.abs(np.abs(e) - 0.05) < 1e-4)
        need = max(3, math.ceil(0.75 * v.sum()))
        return (np.abs(e) <= 0.05).sum() >= need, near

    ok = fits["status"] == O.FIT_OK
    assert ((modes == O.T_RUN_START) <= ok).all()          # a run starts at an own-fit tile
    assert ((modes == O.T_RAW) <= ~ok).all()               # raw tiles failed their own fit
    checked = 0
    for t in range(len(modes)):
        if modes[t] == O.T_RUN_START:
            plane = kft[t]
            k = t + 1
            while k % TW and modes[k] == O.T_RUN_CONT:
                assert (kft[k] == plane).all()
                good, near = passes(k, plane)
                assert good or near
                k += 1
            if k % TW:
                good, near = passes(k, plane)
                assert (not good) or near
                checked += 1
    assert checked > 500


def test_corrupt_streams_are_rejected(cfg1):
    sen, pts = cfg1
    s = O.sensor(sen)
    p = O.params()
    bits, kft, fits, modes = O.encode_keyframe(s, p, pts)
    assert O.decode_status(s, bits[:-4]) == O.ERR_CORRUPT
    bad = bits.copy()
    bad[0] ^= 1
    assert O.decode_status(s, bad) == O.ERR_CORRUPT
    bad = bits.copy()
    bad[64 + (16 * 512 // 8) + 0] = 0x33       # first tile codes: RUN_CONT at the row start
    assert O.decode_status(s, bad) == O.ERR_CORRUPT
    assert O.decode_status(s, bits[:40]) == O.ERR_CORRUPT


def test_empty_frame():
    s = _sensor(16, 512)
    p = O.params()
    bits, kft, fits, modes = O.encode_keyframe(s, p, np.zeros((0, 4), np.float32))
    assert (modes == O.T_EMPTY).all()
    assert len(bits) == 64 + 4 * (16 * 512 // 32 + 512 // 8)
    dec, _, valid = O.decode(s, bits)
    assert (dec == 0).all() and (valid == 0).all()


# ----------------------------------------------------------- temporal --

def _pitch(deg):
    a = math.radians(deg)
    return np.array([[math.cos(a), 0, math.sin(a)], [0, 1, 0], [-math.sin(a), 0, math.cos(a)]])


@pytest.mark.parametrize("R", [np.eye(3), synth.yaw_matrix(math.radians(3.0)) @ _pitch(1.5)])
def test_temporal_offset_is_exact_under_known_motion(R):
    """Ground plane only: every P tile whose anchor lands in the K image is
    temporally coded with n' = R^T n and c' = d - n.T."""
    sen = synth.HDL64_SENSOR
    s = O.sensor(sen)
    p = O.params()
    scene = synth.Scene(5, 0, 0, 0)
    kpts = scene.render(sen, sigma=0.0)
    T = np.array([1.0, 0.4, 0.05])
    ppts = scene.render(sen, R=R, t=T, sigma=0.0)
    M = np.eye(4)
    M[:3, :3] = R
    M[:3, 3] = T
    _, kft, _, _ = O.encode_keyframe(s, p, kpts)
    bits, fits, tmp, modes = O.encode_pframe(s, p, kft, M, ppts)
    found = tmp["kref"] >= 0
    assert (tmp["status"][found & (tmp["n_valid"] >= 3)] == 2).all()
    assert found.sum() > 0.9 * (tmp["n_valid"] > 0).sum()
    sel = tmp["status"] == 2
    assert np.isin(modes[sel], [O.T_TEMPORAL, O.T_TEMPORAL_CONT]).all()   # a temporal run start or continuation
    n = np.array([0, 0, -1.0])
    assert np.abs(tmp["plane"][sel][:, :3] - (R.T @ n).astype(np.float32)).max() < 1e-6
    assert np.abs(tmp["plane"][sel][:, 3] - (1.7 - n @ T)).max() < 2e-5
    rng, _, _ = O.range_image(s, ppts)
    dec, _, _ = O.decode(s, bits, kft, M)
    m = rng > 0
    assert np.abs(dec[m] - rng[m]).max() <= 0.01 + 1e-5


def test_identity_pose_makes_every_plane_tile_temporal():
    sen = synth.HDL64_SENSOR
    s = O.sensor(sen)
    p = O.params()
    pts = synth.Scene(7, 4, 0, 0, enclose=True).render(sen, sigma=0.0)
    _, kft, kfits, kmodes = O.encode_keyframe(s, p, pts)
    bits, fits, tmp, modes = O.encode_pframe(s, p, kft, np.eye(4), pts)
    plane = (kmodes == O.T_RUN_START) | (kmodes == O.T_RUN_CONT)
    assert (tmp["kref"][plane] == np.nonzero(plane)[0]).all()
    assert np.isin(modes[plane], [O.T_TEMPORAL, O.T_TEMPORAL_CONT]).mean() > 0.99


def test_pframe_decode_error_and_kf_table_from_stream(cfg2_seq):
    seq = cfg2_seq
    s = O.sensor(seq.sensor)
    p = O.params()
    kbits, kft, _, _ = O.encode_keyframe(s, p, seq.frames[seq.key_index])
    kft2 = O.kf_table_from_stream(s, kbits, len(kft))
    assert (kft2 == kft).all()
    for f in (0, seq.key_index + 1, len(seq.frames) - 1):
        bits, fits, tmp, modes = O.encode_pframe(s, p, kft, seq.poses[f], seq.frames[f])
        assert np.isin(modes, [O.T_TEMPORAL, O.T_TEMPORAL_CONT]).sum() > 1000
        rng, _, _ = O.range_image(s, seq.frames[f])
        dec, _, _ = O.decode(s, bits, kft2, seq.poses[f])
        m = rng > 0
        assert np.abs(dec[m] - rng[m]).max() <= 0.01 + 1e-5


# ------------------------------------------------------------------ seeded fit (learned proposal) --

def _planar_tile_with_outlier():
    s = O.Sensor(8, 256, -10.0, 10.0, 80.0)
    p = O.params(tile_h=8, tile_w=8, min_inlier_frac=0.75)
    u = O.beams(s).astype(np.float64)
    n = np.array([0.9, 0.3, 0.1])
    n /= np.linalg.norm(n)
    d = 12.0
    dots = u @ n
    rng_img = np.where(dots > 0.1, d / np.where(dots > 0.1, dots, 1), 0).astype(np.float32)
    tc = int(np.argmax(dots[3])) // 8
    rng_img[3, 8 * tc + 2] -= 0.5
    return s, p, rng_img, tc, n, d


def _prop_for(s, p, rng_img, n, d, logit=3.0):
    """Proposal rows for every tile: the true plane relative to each tile's anchor."""
    u = O.beams(s)
    nt = O.n_tiles(s, p)
    TC = (s.cols + p.tile_w - 1) // p.tile_w
    prop = np.zeros((nt, 5), np.float32)
    for t in range(nt):
        tr, tc = divmod(t, TC)
        r = rng_img[tr * 8:(tr + 1) * 8, tc * 8:(tc + 1) * 8]
        idx = np.flatnonzero(r.reshape(-1) > 0)
        if len(idx) == 0:
            continue
        k = idx[0]
        pa = (r.reshape(-1)[k] * u[tr * 8:(tr + 1) * 8, tc * 8:(tc + 1) * 8].reshape(-1, 3)[k]).astype(np.float32)
        prop[t] = [logit, n[0], n[1], n[2], d - float(np.dot(n, pa))]
    return prop


def test_seeded_fit_starts_from_the_proposal_inliers():
    """A proposal equal to the true plane puts the moved pixel out of the first set, so the
    seeded fit reaches the plain fit's final plane in one round (the plain fit needs two)."""
    s, p, rng_img, tc, n, d = _planar_tile_with_outlier()
    plain = O.fit_tiles(s, p, rng_img)
    prop = _prop_for(s, p, rng_img, n, d)
    seeded = O.fit_tiles_seeded(s, p, rng_img, prop, -2.944)
    assert plain[tc]["rounds"] >= 2 and seeded[tc]["rounds"] == 1
    assert seeded[tc]["status"] == O.FIT_OK and seeded[tc]["n_inlier"] == plain[tc]["n_inlier"] == 63
    assert np.abs(seeded[tc]["plane"] - np.array([*n, d], np.float32)).max() < 2e-5
    # the proposal's sign does not matter (the plane is made canonical, d >= 0)
    neg = prop.copy()
    neg[:, 1:] = -neg[:, 1:]
    seeded2 = O.fit_tiles_seeded(s, p, rng_img, neg, -2.944)
    assert seeded2.tobytes() == seeded.tobytes()


def test_seeded_fit_skip_and_fallbacks():
    s, p, rng_img, tc, n, d = _planar_tile_with_outlier()
    plain = O.fit_tiles(s, p, rng_img)
    has = plain["n_valid"] >= 3
    # below the skip logit: no fit at all
    prop = _prop_for(s, p, rng_img, n, d, logit=-5.0)
    skipped = O.fit_tiles_seeded(s, p, rng_img, prop, -2.944)
    assert (skipped["status"][has] == O.FIT_FAIL).all() and (skipped["rounds"] == 0).all()
    # a zero normal, or a plane with fewer than 3 pixels near it, falls back to the plain fit
    zero = np.zeros((O.n_tiles(s, p), 5), np.float32)
    zero[:, 0] = 3.0
    assert O.fit_tiles_seeded(s, p, rng_img, zero, -2.944).tobytes() == plain.tobytes()
    far = _prop_for(s, p, rng_img, n, d)
    far[:, 4] += 5.0
    assert O.fit_tiles_seeded(s, p, rng_img, far, -2.944).tobytes() == plain.tobytes()


# ------------------------------------------------------------- no-delta mode --

def _no_delta_pair(s, p_kw, pts):
    pd = O.params(**p_kw)
    pn = O.params(no_delta=1, **p_kw)
    bd, kd, fd, md = O.encode_keyframe(s, pd, pts)
    bn, kn, fn, mn = O.encode_keyframe(s, pn, pts)
    return bd, bn, kd, kn, md, mn


@pytest.mark.parametrize("tile,thr", [((4, 4), 0.05), ((8, 8), 0.02)])
def test_no_delta_stream_is_the_delta_stream_without_residual_codes(cfg1, tile, thr):
    """Sec. III-C drops the deltas of plane-coded points: the no-delta stream holds every section
    of the delta stream except the residual codes, flags bit 1 set, and the same planes."""
    sen, pts = cfg1
    s = O.sensor(sen)
    bd, bn, kd, kn, md, mn = _no_delta_pair(s, dict(tile_h=tile[0], tile_w=tile[1], fit_thr_m=thr), pts)
    sd, sn = streamfmt.sections(bd), streamfmt.sections(bn)
    hd, hn = sd["header"], sn["header"]
    assert hn["flags"] == hd["flags"] | 2 and hd["flags"] & 2 == 0
    for k in ("n_tiles", "n_valid", "n_runs", "n_temporal", "n_cand", "n_fitted", "n_raw", "w_res", "w_raw", "k_max"):
        assert hn[k] == hd[k], k
    for name in ("bitmap", "tiles", "runs", "temporal", "fitted", "raw"):
        assert np.array_equal(sn[name], sd[name]), name
    assert len(sn["res"]) == 0 and len(sd["res"]) > 0
    assert hn["total_bytes"] == hd["total_bytes"] - 4 * len(sd["res"]) == len(bn)
    assert np.array_equal(kn, kd) and np.array_equal(mn, md)


def test_no_delta_decode_lies_on_the_plane_within_the_threshold(cfg1):
    """Decoded without deltas, a plane-coded point is the plane's intersection with its ray: it
    differs from the delta decode by exactly its residual code times q, so it is within the
    threshold of the input range; raw points decode as with deltas."""
    sen, pts = cfg1
    s = O.sensor(sen)
    thr = 0.05
    bd, bn, *_ = _no_delta_pair(s, dict(fit_thr_m=thr), pts)
    rng, _, _ = O.range_image(s, pts)
    dd, xd, _ = O.decode(s, bd)
    dn, xn, _ = O.decode(s, bn)
    m = rng > 0
    assert ((dn > 0) == m).all()
    assert np.abs(dn[m] - rng[m]).max() <= thr + 1e-5
    # the pixels whose decode differs are plane-coded; the difference is k q with |k| <= k_max
    k = streamfmt.residual_codes(bd)
    diff = (dd - dn)[m]
    q = np.float32(0.02)
    assert np.abs(diff).max() <= (np.abs(k).max() + 0.5) * q + 1e-5
    assert np.count_nonzero(diff) <= np.count_nonzero(k)
    u = O.beams(s)
    assert np.abs(xn[..., :3] - dn[..., None] * u).max() == 0


@pytest.mark.parametrize("tile", [(4, 4), (8, 8)])
def test_raw_exact_keeps_raw_points_losslessly(cfg1, tile):
    """The lossless raw option: header flags bit 2 and 32-bit raw codes holding each raw pixel's
    fp32 range; every other section equals the quantised mode's, the raw codes quantise to the
    quantised mode's raw codes in the same order, and raw pixels decode to their range exactly."""
    sensor, pts = cfg1
    s = O.sensor(sensor)
    pq, pe = O.params(*tile), O.params(*tile, raw_exact=1)
    bq, _, _, _ = O.encode_keyframe(s, pq, pts)
    be, _, _, _ = O.encode_keyframe(s, pe, pts)
    hq, he = streamfmt.header(bq), streamfmt.header(be)
    assert he["flags"] & 4 and not hq["flags"] & 4 and he["w_raw"] == 32 and hq["w_raw"] < 32
    assert he["n_raw"] == hq["n_raw"] > 0
    sq, se = streamfmt.sections(bq), streamfmt.sections(be)
    for k in ("bitmap", "tiles", "runs", "temporal", "fitted", "res"):
        assert np.array_equal(sq[k], se[k]), k
    assert len(se["raw"]) == he["n_raw"]
    raw_e = streamfmt.raw_codes(be).astype(np.uint32).view(np.float32)
    q = np.float32(pq.quant_m)
    assert np.array_equal(np.floor(raw_e / q + np.float32(0.5)).astype(np.int64), streamfmt.raw_codes(bq))
    rng, _, _ = O.range_image(s, pts)
    drng, dxyz, _ = O.decode(s, be)
    m = rng > 0
    exact = m & (drng.view(np.uint32) == rng.view(np.uint32))
    assert exact.sum() >= he["n_raw"]
    assert np.isin(raw_e, rng[m]).all()
    assert np.abs(drng[m] - rng[m]).max() <= q / 2 + 1e-5
    # the raw pixels of the quantised mode are the exact ones here
    dq, _, _ = O.decode(s, bq)
    raw_px = m & (np.abs(dq - rng) > 0) & ~np.isclose(dq, drng, rtol=0, atol=0)
    assert (drng[raw_px] == rng[raw_px]).all()


def test_raw_exact_flag_needs_32_bit_raw_codes(cfg1):
    sensor, pts = cfg1
    s = O.sensor(sensor)
    b, _, _, _ = O.encode_keyframe(s, O.params(raw_exact=1), pts)
    bad = b.copy()
    bad[15] = 12   # w_raw
    with pytest.raises(ValueError):
        O.decode(s, bad)
    bad = b.copy()
    bad[7] |= 8    # an unknown flag
    with pytest.raises(ValueError):
        O.decode(s, bad)


def test_temporal_candidates_extend_the_anchor_test():
    """Several candidate K tiles: every tile that passes against its anchor's K tile keeps the
    same record; the other passes name a K tile that one of the tile's own valid pixels falls in
    after Eq. 6 (binned here through the range-image conversion of the moved points)."""
    seq = synth.sequence_cfg2(0, 10)
    s = O.sensor(seq.sensor)
    k, f = seq.key_index, 0
    p1, p4 = O.params(), O.params(temporal_candidates=4)
    _, kft, _, _ = O.encode_keyframe(s, p1, seq.frames[k])
    rng, _, _ = O.range_image(s, seq.frames[f])
    t1 = O.temporal_tiles(s, p1, rng, kft, seq.poses[f])
    t4 = O.temporal_tiles(s, p4, rng, kft, seq.poses[f])
    pass1, pass4 = t1["status"] == 2, t4["status"] == 2
    assert (pass4 >= pass1).all() and pass4.sum() > pass1.sum()
    for name in ("kref", "plane", "n_inlier", "rounds"):
        assert np.array_equal(t1[name][pass1], t4[name][pass1]), name
    # tiles untouched by the extra candidates: no anchor bin, or the anchor's K tile only
    H, W, th, tw = seq.sensor.rows, seq.sensor.cols, p1.tile_h, p1.tile_w
    TC = (W + tw - 1) // tw
    beams = O.beams(s).reshape(H, W, 3)
    M = seq.poses[f]
    new = np.nonzero(pass4 & ~pass1)[0]
    assert len(new) > 0
    for t in new[:200]:
        i0, j0 = (t // TC) * th, (t % TC) * tw
        r = rng[i0:i0 + th, j0:j0 + tw]
        u = beams[i0:i0 + th, j0:j0 + tw]
        m = r > 0
        pts = (r[m][:, None] * u[m]).astype(np.float32)
        moved = (pts.astype(np.float64) @ M[:3, :3].T + M[:3, 3]).astype(np.float32)
        img, _, _ = O.range_image(s, np.concatenate([moved, np.zeros((len(moved), 1), np.float32)], 1))
        hit = np.argwhere(img > 0)
        ktiles = {(a // th) * TC + b // tw for a, b in hit}
        assert int(t4["kref"][t]) in ktiles
        assert int(t4["kref"][t]) != int(t1["kref"][t])


# ----------------------------------------------------- temporal run growth (Sec. III-D) --

def _tile_passes(s, p, rng, u, t, plane):
    """fp64 acceptance rule of a tile against a plane (independent of the oracle's fp32 test);
    returns (passes, near the threshold)."""
    TW = (s.cols + p.tile_w - 1) // p.tile_w
    tr, tc = divmod(t, TW)
    r = rng[tr * p.tile_h:(tr + 1) * p.tile_h, tc * p.tile_w:(tc + 1) * p.tile_w].astype(np.float64).reshape(-1)
    uu = u[tr * p.tile_h:(tr + 1) * p.tile_h, tc * p.tile_w:(tc + 1) * p.tile_w].reshape(-1, 3)
    v = r > 0
    if v.sum() < 3:
        return False, False
    dot = uu[v] @ plane[:3].astype(np.float64)
    e = np.where(dot > 1e-3, r[v] - plane[3] / np.where(dot > 1e-3, dot, 1), np.inf)
    near = bool(np.any(np.abs(np.abs(e) - p.fit_thr_m) < 1e-4))
    need = max(3, math.ceil(p.min_inlier_frac * v.sum()))
    return bool((np.abs(e) <= p.fit_thr_m).sum() >= need), near


@pytest.mark.parametrize("tile", [(4, 4), (8, 8)])
def test_temporal_run_invariants(cfg2_seq, tile):
    """Temporal runs: a run starts at a tile that passed the relaxed-plane test; every tile coded
    TEMPORAL_CONT passes the acceptance rule against the run start's relaxed plane (n', c'), and the
    tile after a run fails it (or the row ends); every tile that passed its own relaxed-plane test is
    coded temporally (a run start or inside a temporal run: spatial runs never cross it); spatial
    runs keep their rule.  The stream carries one temporal record per temporal run."""
    seq = cfg2_seq
    s = O.sensor(seq.sensor)
    p = O.params(tile[0], tile[1], temporal_runs=1)
    _, kft, _, _ = O.encode_keyframe(s, p, seq.frames[seq.key_index])
    u = O.beams(s).astype(np.float64)
    TW = (s.cols + p.tile_w - 1) // p.tile_w
    checked = conts = 0
    for f in (seq.key_index - 1, seq.key_index + 2):
        bits, fits, tmp, modes = O.encode_pframe(s, p, kft, seq.poses[f], seq.frames[f])
        rng, _, _ = O.range_image(s, seq.frames[f])
        passed = tmp["status"] == 2
        temporal = (modes == O.T_TEMPORAL) | (modes == O.T_TEMPORAL_CONT)
        assert ((modes == O.T_TEMPORAL) <= passed).all()
        assert (passed <= temporal).all()
        h = streamfmt.header(bits)
        assert h["flags"] & 8 and h["n_temporal"] == int((modes == O.T_TEMPORAL).sum())
        for t in np.nonzero(modes == O.T_TEMPORAL)[0]:
            plane = tmp["plane"][t]
            k = t + 1
            while k % TW and modes[k] == O.T_TEMPORAL_CONT:
                good, near = _tile_passes(s, p, rng, u, k, plane)
                assert good or near
                conts += 1
                k += 1
            if k % TW:
                good, near = _tile_passes(s, p, rng, u, k, plane)
                assert (not good) or near
                checked += 1
        # spatial runs: a continuation follows a run start or continuation, never a temporal tile
        cont = np.nonzero(modes == O.T_RUN_CONT)[0]
        assert (cont % TW > 0).all()
        assert np.isin(modes[cont - 1], [O.T_RUN_START, O.T_RUN_CONT]).all()
        tc = np.nonzero(modes == O.T_TEMPORAL_CONT)[0]
        assert (tc % TW > 0).all()
        assert np.isin(modes[tc - 1], [O.T_TEMPORAL, O.T_TEMPORAL_CONT]).all()
    assert conts > 100 and checked > 100


def test_temporal_runs_cut_records_and_decode_within_half_step(cfg2_seq):
    """Growing temporal runs codes the same tiles with fewer records than one record per temporal
    tile (the reading without growth), every pixel still decodes within q/2, and without growth no
    stream holds a TEMPORAL_CONT tile or flags bit 3."""
    seq = cfg2_seq
    s = O.sensor(seq.sensor)
    f = seq.key_index + 1
    rng, _, _ = O.range_image(s, seq.frames[f])
    m = rng > 0
    out = {}
    for tr in (0, 1):
        p = O.params(temporal_runs=tr)
        kbits, kft, _, _ = O.encode_keyframe(s, p, seq.frames[seq.key_index])
        bits, _, tmp, modes = O.encode_pframe(s, p, kft, seq.poses[f], seq.frames[f])
        kft2 = O.kf_table_from_stream(s, kbits, O.n_tiles(s, p))
        drng, _, _ = O.decode(s, bits, kft2, seq.poses[f])
        assert ((drng > 0) == m).all()
        assert np.abs(drng[m] - rng[m]).max() <= p.quant_m / 2 + 1e-5
        out[tr] = (bits, tmp, modes)
    (b0, t0, m0), (b1, t1, m1) = out[0], out[1]
    assert not (m0 == O.T_TEMPORAL_CONT).any() and not (streamfmt.header(b0)["flags"] & 8)
    assert (m0 == O.T_TEMPORAL).sum() == (t0["status"] == 2).sum()
    h0, h1 = streamfmt.header(b0), streamfmt.header(b1)
    assert h1["n_temporal"] < h0["n_temporal"]
    assert ((m1 == O.T_TEMPORAL) | (m1 == O.T_TEMPORAL_CONT)).sum() >= (m0 == O.T_TEMPORAL).sum()
    assert len(b1) < len(b0)


def test_temporal_cont_without_flag_or_after_a_spatial_tile_is_corrupt(cfg2_seq):
    """The decoder accepts a TEMPORAL_CONT tile only in a stream flagged for temporal runs and only
    right after a temporal tile of the same row."""
    seq = cfg2_seq
    s = O.sensor(seq.sensor)
    p = O.params(temporal_runs=1)
    f = seq.key_index + 1
    kbits, kft, _, _ = O.encode_keyframe(s, p, seq.frames[seq.key_index])
    bits, _, _, modes = O.encode_pframe(s, p, kft, seq.poses[f], seq.frames[f])
    assert O.decode_status(s, bits, kft, seq.poses[f]) == O.OK
    bad = bits.copy()
    bad[7] &= ~np.uint8(8)                       # clear flags bit 3
    assert O.decode_status(s, bad, kft, seq.poses[f]) == O.ERR_CORRUPT
    # turn the first spatial continuation into a temporal continuation
    t = int(np.nonzero(modes == O.T_RUN_CONT)[0][0])
    sec = streamfmt.sections(bits)
    off = 64 + 4 * (len(sec["bitmap"]))
    word = off + 4 * (t // 8)
    v = int.from_bytes(bits[word:word + 4].tobytes(), "little")
    v = (v & ~(0xF << (4 * (t % 8)))) | (O.T_TEMPORAL_CONT << (4 * (t % 8)))
    bad = bits.copy()
    bad[word:word + 4] = np.frombuffer(v.to_bytes(4, "little"), np.uint8)
    assert O.decode_status(s, bad, kft, seq.poses[f]) == O.ERR_CORRUPT


# ------------------------------------------------- Eq. 3's three-coefficient plane form --

def test_three_coefficient_form_closed_forms():
    """The dominant-axis form of Eq. 3: axis-aligned planes (the ground z = -1.7 m, walls x = 12 m,
    y = -30 m), which x + a y + b z = c cannot hold when n_x = 0, convert and come back exactly;
    a general plane's coefficients satisfy Eq. 3 along its dominant axis for points on it, and it
    comes back within fp32 rounding with the canonical sign (d >= 0)."""
    for pl, axis, abc in (((0.0, 0.0, -1.0, 1.7), 2, (0.0, 0.0, -1.7)), ((1.0, 0.0, 0.0, 12.0), 0, (0.0, 0.0, 12.0)),
                          ((0.0, -1.0, 0.0, 30.0), 1, (0.0, 0.0, -30.0))):
        k, c = O.plane_to3(np.array(pl, np.float32))
        assert k == axis and np.array_equal(c, np.array(abc, np.float32))
        assert np.array_equal(O.plane_from3(k, c), np.array(pl, np.float32))
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        d = rng.uniform(0.5, 60.0)
        pl = np.array([*n, d], np.float32)
        k, abc = O.plane_to3(pl)
        assert k == int(np.argmax(np.abs(pl[:3])))
        i, j = (k + 1) % 3, (k + 2) % 3
        # Eq. 3 along axis k: p_k + a p_i + b p_j = c for a point on the plane (fp64)
        p = d * n.astype(np.float64) + np.cross(n, rng.normal(size=3))
        lhs = p[k] + float(abc[0]) * p[i] + float(abc[1]) * p[j]
        assert abs(lhs - float(abc[2])) <= 1e-5 * max(1.0, abs(float(abc[2])))
        back = O.plane_from3(k, abc)
        assert back[3] >= 0 and np.abs(back - pl).max() <= 2e-6 * max(1.0, d)


@pytest.mark.parametrize("tile", [(4, 4), (8, 8)])
def test_three_coefficient_streams(cfg2_seq, tile):
    """With plane3 every fitted plane is the plane of its stored coefficients (bit for bit), fits
    agree with the unit-normal ones except near the threshold, each run record shrinks from 4 words
    to 3 (the axis in the run start's tile code), and key and P streams decode within q/2 (the P frames' temporal test
    against the key frame's reconstructed planes)."""
    seq = cfg2_seq
    s = O.sensor(seq.sensor)
    p3 = O.params(tile[0], tile[1], plane3=1)
    p4 = O.params(tile[0], tile[1])
    kpts = seq.frames[seq.key_index]
    b3, kft3, f3, m3 = O.encode_keyframe(s, p3, kpts)
    b4, kft4, f4, m4 = O.encode_keyframe(s, p4, kpts)
    ok = f3["status"] == O.FIT_OK
    for t in np.nonzero(ok)[0]:
        assert np.array_equal(O.plane_from3(int(f3["axis"][t]), f3["coef"][t]), f3["plane"][t])
    same = (f3["status"] == f4["status"])
    assert same.mean() > 0.995
    both = ok & (f4["status"] == O.FIT_OK)
    assert np.abs(f3["plane"][both] - f4["plane"][both]).max() < 1e-4
    h3, h4 = streamfmt.header(b3), streamfmt.header(b4)
    assert h3["flags"] & 16 and not (h4["flags"] & 16)
    runs = h3["n_runs"]
    assert len(streamfmt.sections(b3)["runs"]) == 3 * runs
    codes = streamfmt.tile_codes(b3)
    assert not (codes == O.T_RUN_START).any()
    starts = np.nonzero(m3 == O.T_RUN_START)[0]
    assert np.array_equal(codes[starts], O.T_RUN_START3 + f3["axis"][starts])
    assert len(b4) - len(b3) == 4 * runs
    rng, _, _ = O.range_image(s, kpts)
    m = rng > 0
    dec, _, _ = O.decode(s, b3)
    assert np.abs(dec[m] - rng[m]).max() <= p3.quant_m / 2 + 1e-5
    assert np.array_equal(O.kf_table_from_stream(s, b3, len(kft3)), kft3)
    for f in (seq.key_index - 2, seq.key_index + 1):
        bits, _, _, _ = O.encode_pframe(s, p3, kft3, seq.poses[f], seq.frames[f])
        rng, _, _ = O.range_image(s, seq.frames[f])
        m = rng > 0
        dec, _, _ = O.decode(s, bits, kft3, seq.poses[f])
        assert streamfmt.header(bits)["flags"] & 16
        assert np.abs(dec[m] - rng[m]).max() <= p3.quant_m / 2 + 1e-5
    # a unit-normal run start code in a three-coefficient stream is corrupt
    sec = streamfmt.sections(b3)
    t = int(starts[0])
    word = 64 + 4 * (len(sec["bitmap"]) + t // 8)
    v = int.from_bytes(b3[word:word + 4].tobytes(), "little")
    v = (v & ~(0xF << (4 * (t % 8)))) | (O.T_RUN_START << (4 * (t % 8)))
    bad = b3.copy()
    bad[word:word + 4] = np.frombuffer(v.to_bytes(4, "little"), np.uint8)
    assert O.decode_status(s, bad) == O.ERR_CORRUPT
