"""GPU path vs the CPU oracle, through the C ABI.

Layered parity (the contract):
* bit-exact: range-image binning, tile membership and occupancy, the K-tile
  lookup of the temporal test, and — given the GPU's own fp32 planes and fit
  decisions — the whole packed stream (modes, runs, fitted bits, residual and
  raw codes);  decoding is bit-exact on both sides;
* tolerance: independently fitted planes agree within 1e-5 relative; a tile's
  fit decision or inlier count may differ only where a residual lies within
  1e-6 m of the threshold (the borderline tiles, counted and reported).
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from tests import harness as H
from tests import streamfmt

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06972_gb300 import lcc
    lcc.load()


def _oparams(tile=(4, 4), thr=0.05, q=0.02, R=3, fmin=0.75, merge=1, no_delta=0, raw_exact=0, tcand=1, plane3=0):
    return O.params(tile[0], tile[1], thr, q, R, fmin, merge, no_delta, raw_exact, tcand, plane3=plane3)


def _gparams(tile=(4, 4), thr=0.05, q=0.02, R=3, fmin=0.75, merge=1, solver=0, **kw):
    return dict(tile_h=tile[0], tile_w=tile[1], fit_thr_m=thr, quant_m=q, max_refits=R, min_inlier_frac=fmin,
                merge_runs=merge, solver=solver, **kw)


def _compare_spatial(s, p, rng, recs, ofits, thr, skip=None):
    """Layer-2 comparison of own spatial fits.  Returns (n_compared, n_borderline)."""
    from paper_2008_06972_gb300 import lcc
    assert (recs["n_valid"] == ofits["n_valid"]).all(), "tile membership differs"
    g_ok = recs["status"] == lcc.S_FIT
    o_ok = ofits["status"] == O.FIT_OK
    border = 0
    compared = 0
    for t in range(len(recs)):
        if skip is not None and skip[t]:
            continue
        if ofits["n_valid"][t] < 3:
            assert recs["status"][t] in (lcc.S_EMPTY, lcc.S_FAIL)
            continue
        compared += 1
        same = (g_ok[t] == o_ok[t]) and (recs["n_inlier"][t] == ofits["n_inlier"][t] or not (g_ok[t] or o_ok[t]))
        close = True
        if g_ok[t] and o_ok[t]:
            close = H.plane_close(recs["plane"][t], ofits["plane"][t])
        if same and close and (not g_ok[t] or recs["rounds"][t] == ofits["rounds"][t]):
            continue
        is_border = bool(ofits["borderline"][t]) or bool(recs["flags"][t] & 1) or \
            H.borderline_tile(s, p, rng, recs["plane"][t], ofits["plane"][t], t, thr)
        assert is_border, f"tile {t}: gpu status {recs['status'][t]} inl {recs['n_inlier'][t]} " \
                          f"plane {recs['plane'][t]} rounds {recs['rounds'][t]} | oracle status " \
                          f"{ofits['status'][t]} inl {ofits['n_inlier'][t]} plane {ofits['plane'][t]} " \
                          f"rounds {ofits['rounds'][t]}"
        border += 1
    return compared, border


def _check_decode(c, s, bits, rng, q, kf_gpu=None, kft=None, pose=None, bound=None):
    st, drng, dxyz, dvalid = H.decode(c, bits, kf_gpu, pose)
    assert st == 0
    orng, oxyz, ovalid = O.decode(s, bits, kft, pose)
    assert np.array_equal(drng.view(np.uint32), orng.view(np.uint32))
    assert np.array_equal(dxyz.view(np.uint32), oxyz.view(np.uint32))
    assert np.array_equal(dvalid, ovalid)
    m = rng > 0
    assert ((drng > 0) == m).all()
    err = np.abs(drng[m] - rng[m]).max() if m.any() else 0.0
    assert err <= (q / 2 if bound is None else bound) + 1e-5
    return err


def _keyframe_case(sensor_, pts, **kw):
    from paper_2008_06972_gb300 import lcc
    s = O.sensor(sensor_)
    p = _oparams(**{k: v for k, v in kw.items() if k not in ("solver", "fit_schedule")})
    c = H.ctx(sensor_, **_gparams(**kw))
    gbits, recs = H.encode_keyframe(c, pts)
    rng, _, _ = O.range_image(s, pts)
    ofits = O.fit_tiles(s, p, rng)
    compared, border = _compare_spatial(s, p, rng, recs, ofits, p.fit_thr_m)
    assert border <= max(2, 0.005 * compared), f"{border} borderline tiles of {compared}"
    # Layer 1: the oracle's merge + code + pack on the GPU's planes reproduces the GPU stream
    planes, ok = H.gpu_planes(recs)
    coef = c.lcc_tile_coefficients(0) if p.plane3 else None
    cbits, _, _ = O.pack(s, p, 0, rng, planes, ok, fit_coef=coef)
    assert cbits.tobytes() == gbits.tobytes()
    # with identical planes the streams are identical outright
    obits, _, _, _ = O.encode_keyframe(s, p, pts)
    same_planes = np.array_equal(recs["plane"][ok.astype(bool)].view(np.uint32),
                                 ofits["plane"][ok.astype(bool)].view(np.uint32)) and \
        np.array_equal(ok, (ofits["status"] == O.FIT_OK).astype(np.uint8))
    if same_planes:
        assert obits.tobytes() == gbits.tobytes()
    err = _check_decode(c, s, gbits, rng, p.quant_m, bound=p.fit_thr_m if p.no_delta else None)
    return dict(bytes=len(gbits), border=border, compared=compared, err=err, same_planes=same_planes, ctx=c,
                recs=recs, bits=gbits)


# ------------------------------------------------------------------ tables, binning --

def test_sensor_tables_match_oracle():
    for sen in (synth.CFG1_SENSOR, synth.HDL64_SENSOR, synth.Sensor(18, 515, -15, 15, 80.0)):
        c = H.ctx(sen)
        g = c.tables()
        o = O.tables(O.sensor(sen))
        for k in g:
            assert np.array_equal(g[k].view(np.uint32), o[k].view(np.uint32)), k


@pytest.mark.parametrize("case", ["cfg1", "cfg2", "offgrid", "ragged"])
def test_range_image_bit_exact(case, cfg1, cfg2_seq):
    if case == "cfg1":
        sen, pts = cfg1
    elif case == "cfg2":
        sen, pts = cfg2_seq.sensor, cfg2_seq.frames[0]
    elif case == "offgrid":
        sen = synth.HDL64_SENSOR
        pts = synth.offgrid_points(300000, seed=17, r_hi=95.0, elev_lo_deg=-40, elev_hi_deg=10)
        pts[::997, 0] = np.nan
        pts[::1009, :3] = 0.0
        pts[::1013, 1] = np.inf
    else:
        sen = synth.Sensor(18, 515, -15.0, 15.0, 80.0)
        pts = synth.Scene(9, 4, 6, 10, enclose=True).render(sen, sigma=0.02, dropout=0.05, seed=9)
        pts = np.concatenate([pts, pts[::3] * np.float32(1.01), pts[::5]])   # collisions, exact duplicates
    s = O.sensor(sen)
    c = H.ctx(sen)
    d = H.to_dev(pts)
    npx = sen.rows * sen.cols
    rng = torch.empty(npx, dtype=torch.float32, device="cuda")
    valid = torch.empty((npx + 31) // 32, dtype=torch.int32, device="cuda")
    c.lcc_range_image(d, len(pts), rng, valid)
    assert c.lcc_sync() == 0
    orng, _, ost = O.range_image(s, pts)
    assert np.array_equal(rng.cpu().numpy().view(np.uint32), orng.reshape(-1).view(np.uint32))
    obits = np.packbits((orng.reshape(-1) > 0).astype(np.uint8), bitorder="little")
    obits = np.concatenate([obits, np.zeros((-len(obits)) % 4, np.uint8)]).view(np.uint32)
    assert np.array_equal(valid.cpu().numpy().view(np.uint32), obits)
    st = c.lcc_last_stats(0)
    assert st["points_in"] == len(pts)
    assert (st["points_binned"], st["points_invalid"], st["points_fov"]) == (ost[0], ost[1], ost[2])


# -------------------------------------------------------------------- key frames --

@pytest.mark.parametrize("tile,thr", [((4, 4), 0.05), ((4, 8), 0.05), ((8, 8), 0.05), ((8, 16), 0.05),
                                      ((4, 4), 0.02), ((8, 8), 0.10)])
def test_keyframe_parity_cfg1(cfg1, tile, thr):
    sen, pts = cfg1
    r = _keyframe_case(sen, pts, tile=tile, thr=thr)
    assert r["err"] <= 0.01 + 1e-5


@pytest.mark.parametrize("merge,fmin,R", [(0, 0.75, 3), (1, 1.0, 3), (1, 0.75, 0), (1, 0.5, 6)])
def test_keyframe_parity_variants(cfg1, merge, fmin, R):
    sen, pts = cfg1
    _keyframe_case(sen, pts, merge=merge, fmin=fmin, R=R)


@pytest.mark.parametrize("solver,schedule", [(0, 0), (1, 0), (0, 1), (1, 1), (0, 3)])
def test_keyframe_parity_solvers_and_schedules(cfg2_seq, solver, schedule):
    """Both plane solvers (float-float, FP64) and both fit schedules meet the parity contract."""
    seq = cfg2_seq
    _keyframe_case(seq.sensor, seq.frames[seq.key_index], solver=solver, fit_schedule=schedule)


@pytest.mark.parametrize("tile", [(4, 4), (8, 16)])
def test_keyframe_parity_ragged_sensor(tile):
    sen = synth.Sensor(18, 515, -15.0, 15.0, 80.0)   # partial edge tiles in both directions
    pts = synth.Scene(21, 4, 6, 10, enclose=True).render(sen, sigma=0.02, dropout=0.05, seed=21)
    _keyframe_case(sen, pts, tile=tile)


def test_keyframe_parity_full_size_hdl64(cfg2_seq):
    """The bench's workload size: a 64x2048 key frame."""
    seq = cfg2_seq
    r = _keyframe_case(seq.sensor, seq.frames[seq.key_index])
    recs = r["recs"]
    assert (recs["status"] == 2).sum() > 4000


def test_empty_and_tiny_frames():
    sen = synth.CFG1_SENSOR
    for pts in (np.zeros((0, 4), np.float32), np.array([[10, 0, 0, 0]], np.float32)):
        r = _keyframe_case(sen, pts)
        assert r["bytes"] == len(O.encode_keyframe(O.sensor(sen), _oparams(), pts)[0])


def test_schedule_invariance_and_determinism(cfg1):
    sen, pts = cfg1
    ref = None
    ref_recs = None
    for la, sched in ((0, 0), (1, 0), (8, 0), (16, 0), (32, 0), (16, 1), (16, 2), (0, 2), (16, 3), (16, 4),
                      (16, 5), (0, 5), (16, 6)):
        c = H.ctx(sen, lookahead=la, fit_schedule=sched)
        b1, r1 = H.encode_keyframe(c, pts)
        b2, _ = H.encode_keyframe(c, pts)
        assert b1.tobytes() == b2.tobytes()
        ref = b1 if ref is None else ref
        assert b1.tobytes() == ref.tobytes()
        fields = ("plane", "status", "rounds", "n_inlier", "n_valid")
        if ref_recs is None:
            ref_recs = r1
        for k in fields:   # every fit schedule runs the same rounds on every tile
            assert np.array_equal(r1[k], ref_recs[k]), (la, sched, k)


# ------------------------------------------------------------------- P frames --

def _pframe_case(seq, frames, tile=(4, 4), thr=0.05, poses=None, schedule=0, tcand=1, plane3=0):
    from paper_2008_06972_gb300 import lcc
    s = O.sensor(seq.sensor)
    p = _oparams(tile=tile, thr=thr, tcand=tcand, plane3=plane3)
    c = H.ctx(seq.sensor, **_gparams(tile=tile, thr=thr, max_batch=max(16, len(frames)), fit_schedule=schedule,
                                     temporal_candidates=tcand, plane3=plane3))
    kf = lcc.Keyframe(c)
    kbits, krecs = H.encode_keyframe(c, seq.frames[seq.key_index], kf)
    okft = O.kf_table_from_stream(s, kbits, c.num_tiles)
    poses = [seq.poses[f] for f in frames] if poses is None else poses
    pbits, precs = H.encode_pframes(c, kf, poses, [seq.frames[f] for f in frames])
    kf2 = lcc.Keyframe(c)
    c.lcc_keyframe_from_stream(torch.from_numpy(kbits).cuda(), len(kbits), kf2)
    assert c.lcc_sync() == 0
    total_border = 0
    for i, f in enumerate(frames):
        pts = seq.frames[f]
        rng, _, _ = O.range_image(s, pts)
        recs = precs[i]
        otmp = O.temporal_tiles(s, p, rng, okft, poses[i])
        # the K tile of every anchor is found identically (FP64 transform + exact binning); with
        # several candidates the K tile tested last depends on the earlier tests' outcomes, so it
        # may differ only where a test was borderline
        found = otmp["status"] > 0
        assert np.array_equal(recs["t_status"] > 0, found)
        same_k = recs["kref"].astype(np.int64) == otmp["kref"].astype(np.int64)
        excused = (otmp["borderline"] != 0) | ((recs["flags"] & 1) != 0) if tcand > 1 else np.zeros_like(found)
        assert (same_k | ~found | excused).all()
        keep = found & same_k
        assert np.array_equal(recs["tplane"][keep][:, :3].view(np.uint32),
                              otmp["plane"][keep][:, :3].view(np.uint32))
        border = 0
        for t in np.nonzero(found)[0]:
            same = recs["t_status"][t] == otmp["status"][t] and recs["t_inlier"][t] == otmp["n_inlier"][t] and \
                same_k[t]
            cg, co = float(recs["tplane"][t][3]), float(otmp["plane"][t][3])
            close = abs(cg - co) <= H.PLANE_TOL * max(abs(co), 1.0)
            if same and close:
                continue
            assert otmp["borderline"][t] or (recs["flags"][t] & 1) or \
                H.borderline_tile(s, p, rng, recs["tplane"][t], otmp["plane"][t], t, p.fit_thr_m), \
                f"frame {f} tile {t}: gpu {recs['t_status'][t]} {recs['t_inlier'][t]} {cg} | " \
                f"oracle {otmp['status'][t]} {otmp['n_inlier'][t]} {co}"
            border += 1
        ofits = O.fit_tiles(s, p, rng)
        temporal = recs["status"] == lcc.S_TEMPORAL
        _, b2 = _compare_spatial(s, p, rng, recs, ofits, p.fit_thr_m,
                                 skip=temporal | (otmp["status"] == 2))
        total_border += border + b2
        planes, ok = H.gpu_planes(recs)
        tplanes, kref = H.gpu_temporal(recs)
        coef = c.lcc_tile_coefficients(i) if plane3 else None
        cbits, _, _ = O.pack(s, p, 1, rng, planes, ok, tplanes, kref, fit_coef=coef)
        assert cbits.tobytes() == pbits[i].tobytes(), f"frame {f}: stream differs from the oracle's packing"
        codes = streamfmt.tile_codes(pbits[i])
        assert np.isin(codes[temporal], [4, 5]).all()            # temporal run start or continuation
        assert (codes == 4).sum() == streamfmt.header(pbits[i])["n_temporal"] <= temporal.sum()
        _check_decode(c, s, pbits[i], rng, p.quant_m, kf_gpu=kf2, kft=okft, pose=poses[i])
    return total_border


def test_pframe_parity_cfg2(cfg2_seq):
    seq = cfg2_seq
    frames = [f for f in range(len(seq.frames)) if f != seq.key_index]
    border = _pframe_case(seq, frames)
    assert border <= 20


@pytest.mark.parametrize("tile,thr", [((8, 8), 0.05), ((4, 4), 0.10), ((8, 16), 0.02)])
def test_pframe_parity_tiles(cfg2_seq, tile, thr):
    seq = cfg2_seq
    _pframe_case(seq, [0, seq.key_index + 1], tile=tile, thr=thr)


@pytest.mark.parametrize("schedule", [1, 4, 5, 6])
def test_pframe_parity_queued_schedule(cfg2_seq, schedule):
    """Queued rounds (1); spatial fits first and the temporal test after them (4)."""
    seq = cfg2_seq
    _pframe_case(seq, [1, 7], schedule=schedule)


def test_pframe_noisy_pose(cfg2_seq):
    seq = cfg2_seq
    poses = [synth.perturb_pose(seq.poses[f], 0.01, 0.05, 100 + f) for f in (2, 8)]
    _pframe_case(seq, [2, 8], poses=poses)


def _canonical_ahead(recs, tc):
    """Tile records with the run pre-test entries that refer to a tile whose own fit did not
    succeed cleared (the merge reads pre-test results only against run starts, which are
    fitted tiles; the sequence call runs the P frames' pre-test before their temporal test, so
    its entries against tiles that then become temporal are set where the fused order has 0)."""
    r = recs.copy()
    status = r["status"]
    col = np.arange(len(r)) % tc
    for j in range(32):
        src = np.arange(len(r)) - 1 - j
        stale = (col > j) & (status[np.maximum(src, 0)] != 2)
        stale |= col <= j
        r["ahead_mask"][stale] &= np.uint32(~(1 << j) & 0xFFFFFFFF)
        if j < 16:
            r["ahead_cnt"][stale, j] = 0
    return r


def test_sequence_call_matches_separate_calls(cfg2_seq):
    from paper_2008_06972_gb300 import lcc
    seq = cfg2_seq
    n = len(seq.frames)
    c = H.ctx(seq.sensor, max_batch=16)
    ds = [H.to_dev(p) for p in seq.frames]
    outs = [H.out_buf(c) for _ in range(n)]
    nb = torch.zeros(n, dtype=torch.int64, device="cuda")
    kf = lcc.Keyframe(c)
    c.lcc_encode_sequence(seq.key_index, seq.poses, ds, [len(p) for p in seq.frames], outs,
                          [o.numel() for o in outs], nb, kf)
    assert c.lcc_sync() == 0
    nbs = nb.cpu().numpy()
    seq_bits = [outs[i][:nbs[i]].cpu().numpy() for i in range(n)]
    seq_recs = [c.lcc_tile_records(i) for i in range(n)]
    c2 = H.ctx(seq.sensor, max_batch=16)
    kf2 = lcc.Keyframe(c2)
    kbits, krecs = H.encode_keyframe(c2, seq.frames[seq.key_index], kf2)
    assert kbits.tobytes() == seq_bits[seq.key_index].tobytes()
    assert krecs.tobytes() == seq_recs[seq.key_index].tobytes()
    others = [f for f in range(n) if f != seq.key_index]
    pb, precs = H.encode_pframes(c2, kf2, [seq.poses[f] for f in others], [seq.frames[f] for f in others])
    for i, f in enumerate(others):
        assert pb[i].tobytes() == seq_bits[f].tobytes()
        # the sequence call fits P tiles spatially (and runs their run pre-test) while the key
        # frame is encoded and tests them temporally afterwards; every tile record (rounds and
        # flags included) is as if fused, up to pre-test entries against tiles that are not fitted
        tc = seq.sensor.cols // 4
        assert _canonical_ahead(precs[i], tc).tobytes() == _canonical_ahead(seq_recs[f], tc).tobytes(), \
            f"frame {f}: tile records differ"
    # the same with the queued fit schedules (their P rounds also run beside the key frame)
    for sched in (1, 2, 3, 5, 6):
        cq = H.ctx(seq.sensor, max_batch=16, fit_schedule=sched)
        outs_q = [H.out_buf(cq) for _ in range(n)]
        cq.lcc_encode_sequence(seq.key_index, seq.poses, ds, [len(p) for p in seq.frames], outs_q,
                               [o.numel() for o in outs_q], nb, None)
        assert cq.lcc_sync() == 0
        nbq = nb.cpu().numpy()
        for f in range(n):
            assert outs_q[f][:nbq[f]].cpu().numpy().tobytes() == seq_bits[f].tobytes(), (sched, f)
    # host-buffer variant (end-to-end path of the bench)
    h_out = [np.zeros(c.max_encoded_bytes, np.uint8) for _ in range(n)]
    nbh = c.lcc_encode_sequence_host(seq.key_index, seq.poses, [np.ascontiguousarray(p) for p in seq.frames], h_out,
                                     [len(h) for h in h_out])
    for f in range(n):
        assert h_out[f][:nbh[f]].tobytes() == seq_bits[f].tobytes()
    # page-locked host buffers: points read in place over the host link, streams written by the
    # copy-out kernel
    hp = [torch.from_numpy(np.ascontiguousarray(p)).pin_memory() for p in seq.frames]
    ho = [torch.zeros(c.max_encoded_bytes, dtype=torch.uint8).pin_memory() for _ in range(n)]
    nbp = c.lcc_encode_sequence_host(seq.key_index, seq.poses, hp, ho, [o.numel() for o in ho])
    for f in range(n):
        assert ho[f][:int(nbp[f])].numpy().tobytes() == seq_bits[f].tobytes()


# ------------------------------------------------------------------ errors --

def test_capacity_error_reports_needed_size(cfg1):
    from paper_2008_06972_gb300 import lcc
    sen, pts = cfg1
    c = H.ctx(sen)
    need = len(H.encode_keyframe(c, pts)[0])
    out = torch.zeros(256, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    c.lcc_encode_keyframe(H.to_dev(pts), len(pts), None, out, 256, nb)
    assert c.lcc_sync() == lcc.ERR_CAPACITY
    assert int(nb.item()) == need
    assert c.lcc_sync() == lcc.OK     # the error is cleared once reported
    b, _ = H.encode_keyframe(c, pts)  # the context stays usable
    assert len(b) == need


def test_corrupt_streams_are_rejected(cfg1):
    from paper_2008_06972_gb300 import lcc
    sen, pts = cfg1
    c = H.ctx(sen)
    bits, _ = H.encode_keyframe(c, pts)
    cases = [bits[:-4], bits[:40]]
    bad = bits.copy()
    bad[0] ^= 1
    cases.append(bad)
    bad = bits.copy()
    bad[64 + (16 * 512 // 8)] = 0x33     # first tile codes: a run continuation at the row start
    cases.append(bad)
    bad = bits.copy()
    bad[44] ^= 0x10                       # fitted count no longer matches the fitted bits
    cases.append(bad)
    for b in cases:
        padded = np.concatenate([b, np.zeros(64, np.uint8)])
        st, _, _, _ = H.decode(c, padded[:max(len(b), 1)] if len(b) >= 64 else padded[:len(b)])
        assert st == lcc.ERR_CORRUPT
        assert O.decode_status(O.sensor(sen), b) == O.ERR_CORRUPT
    st, _, _, _ = H.decode(c, bits)
    assert st == lcc.OK


def test_invalid_arguments_fail_fast(cfg1):
    from paper_2008_06972_gb300 import lcc
    sen, pts = cfg1
    with pytest.raises(lcc.LccError) as e:
        H.ctx(sen, tile_h=3, tile_w=5)
    assert e.value.status == lcc.ERR_UNSUPPORTED
    c = H.ctx(sen)
    d = H.to_dev(pts)
    out = H.out_buf(c)
    with pytest.raises(lcc.LccError) as e:
        c.lcc_encode_keyframe(d, len(pts), None, out[1:], out.numel() - 1, None)   # misaligned output
    assert e.value.status == lcc.ERR_INVALID_ARG


def test_bounded_wait_expires_and_reports_timeout(cfg1):
    """Failure detection without a fault: a device wait on a barrier nothing arrives on gives up
    after its limit, the host sees LCC_ERR_TIMEOUT, and the GPU keeps working."""
    from paper_2008_06972_gb300 import lcc
    assert lcc.load().lcc_selftest_bounded_wait(1 << 12, None) == lcc.ERR_TIMEOUT
    sensor, pts = cfg1
    c = H.ctx(sensor)
    bits, _ = H.encode_keyframe(c, pts)
    assert len(bits) > 64


def test_largest_resolution_sequence_with_noisy_poses():
    """128x4096 frames (the largest configuration's resolution, 524k beams, 32,768 4x4 tiles per
    frame) with IMU-like pose noise: key-frame and P-frame parity with the oracle, tile by tile."""
    seq = synth.sequence_cfg5(0, 3)
    info = _keyframe_case(seq.sensor, seq.frames[seq.key_index])
    assert info["border"] <= max(2, 0.005 * info["compared"])
    border = _pframe_case(seq, [f for f in range(3) if f != seq.key_index])
    assert border <= 40


def test_profiler_counts_every_kernel_and_orders_the_timeline(cfg2_seq):
    """The profiler's launch counts (what bench.py reports as gpu_launches) are the kernels a
    sequence call launches: per call, two binnings, two first fit passes, two queued-round
    launches (fit schedule 3), three run pre-tests, two merges, two packs and one temporal test;
    the timeline lists the same launches, each ending after it starts."""
    from paper_2008_06972_gb300 import lcc
    seq = cfg2_seq
    n = len(seq.frames)
    c = H.ctx(seq.sensor, max_batch=16, fit_schedule=3)
    ds = [H.to_dev(p) for p in seq.frames]
    outs = [H.out_buf(c) for _ in range(n)]
    nb = torch.zeros(n, dtype=torch.int64, device="cuda")
    call = lambda: c.lcc_encode_sequence(seq.key_index, seq.poses, ds, [len(p) for p in seq.frames], outs,
                                         [o.numel() for o in outs], nb, None)
    call()
    assert c.lcc_sync() == 0
    c.lcc_set_profiling(True)
    for _ in range(3):
        call()
    assert c.lcc_sync() == 0
    times = c.lcc_kernel_times()
    tl = c.lcc_kernel_timeline()
    c.lcc_set_profiling(False)
    # run pre-tests: the key frame's, the P frames' beside it, and (temporal runs) the P frames' update
    # against the tiles that became temporal
    per_call = {"bin": 2, "fit": 2, "rounds": 2, "lookbehind": 3, "merge": 2, "pack": 2, "temporal": 1}
    assert {k: v[0] for k, v in times.items()} == {k: 3 * v for k, v in per_call.items()}
    assert len(tl) == 3 * sum(per_call.values())
    assert all(t1 >= t0 >= 0.0 for _, t0, t1 in tl)
    # in issue order per call; the P frames' run pre-test (which, with temporal runs, also tests
    # against the temporal tiles' planes), merge and pack follow their temporal test on one stream
    k = sum(per_call.values())
    for i in range(3):
        chunk = tl[i * k:(i + 1) * k]
        names = [nm for nm, _, _ in chunk]
        assert names[0] == "bin" and names.count("temporal") == 1
        it = names.index("temporal")
        assert names[it + 1:] == ["lookbehind", "merge", "pack"]
        for q in range(it, it + 3):
            assert chunk[q + 1][1] >= chunk[q][2] - 1e-3


@pytest.mark.parametrize("plane3", [0, 1])
def test_sequence_decode_matches_per_frame_decode(cfg2_seq, plane3):
    """lcc_decode_sequence (key stream first, all P streams in one launch) gives the ranges, points
    and occupancy of the per-frame decoder bit for bit, with four-word and with three-coefficient
    run records; a corrupt P stream in the batch is reported."""
    from paper_2008_06972_gb300 import lcc
    seq = cfg2_seq
    n = len(seq.frames)
    c = H.ctx(seq.sensor, max_batch=16, plane3=plane3)
    ds = [H.to_dev(p) for p in seq.frames]
    outs = [H.out_buf(c) for _ in range(n)]
    nb = torch.zeros(n, dtype=torch.int64, device="cuda")
    c.lcc_encode_sequence(seq.key_index, seq.poses, ds, [len(p) for p in seq.frames], outs,
                          [o.numel() for o in outs], nb, None)
    assert c.lcc_sync() == 0
    sizes = [int(x) for x in nb.cpu().numpy()]
    npx = seq.sensor.rows * seq.sensor.cols
    new = lambda *shape, dt=torch.float32: [torch.full(shape, -1, dtype=dt, device="cuda") for _ in range(n)]
    r1, x1, v1 = new(npx), new(npx * 4), new((npx + 31) // 32, dt=torch.int32)
    kf = lcc.Keyframe(c)
    c.lcc_keyframe_from_stream(outs[seq.key_index], sizes[seq.key_index], kf)
    for f in range(n):
        isk = f == seq.key_index
        c.lcc_decode(outs[f], sizes[f], None if isk else kf, None if isk else seq.poses[f], r1[f], x1[f], v1[f])
    assert c.lcc_sync() == 0
    r2, x2, v2 = new(npx), new(npx * 4), new((npx + 31) // 32, dt=torch.int32)
    c.lcc_decode_sequence(seq.key_index, seq.poses, outs, sizes, r2, x2, v2)
    assert c.lcc_sync() == 0
    for f in range(n):
        assert torch.equal(r1[f], r2[f]) and torch.equal(x1[f], x2[f]) and torch.equal(v1[f], v2[f]), f
    bad = outs[(seq.key_index + 1) % n].clone()
    bad[:4] = 0   # magic number
    outs2 = list(outs)
    outs2[(seq.key_index + 1) % n] = bad
    c.lcc_decode_sequence(seq.key_index, seq.poses, outs2, sizes, r2, None, None)
    assert c.lcc_sync() == lcc.ERR_CORRUPT


@pytest.mark.parametrize("tile,thr", [((4, 4), 0.05), ((8, 8), 0.02)])
def test_no_delta_keyframe_parity(cfg2_seq, tile, thr):
    """The no-delta mode (Sec. III-C drops the deltas): the GPU stream is the oracle's on the GPU's
    planes, both decoders agree bit for bit, and the decode error stays within the threshold."""
    seq = cfg2_seq
    r = _keyframe_case(seq.sensor, seq.frames[seq.key_index], tile=tile, thr=thr, no_delta=1)
    h = streamfmt.header(r["bits"])
    assert h["flags"] & 2 and r["err"] <= thr + 1e-5
    d = _keyframe_case(seq.sensor, seq.frames[seq.key_index], tile=tile, thr=thr)
    assert r["bytes"] < d["bytes"]


def test_no_delta_sequence_decodes_within_threshold(cfg2_seq):
    """A whole sequence in the no-delta mode: every frame decodes with the oracle's decoder to the
    GPU decoder's ranges, within the threshold of its range image."""
    from paper_2008_06972_gb300 import lcc
    seq = cfg2_seq
    n = len(seq.frames)
    thr = 0.05
    c = H.ctx(seq.sensor, max_batch=16, no_delta=1, fit_thr_m=thr)
    ds = [H.to_dev(p) for p in seq.frames]
    outs = [H.out_buf(c) for _ in range(n)]
    nb = torch.zeros(n, dtype=torch.int64, device="cuda")
    kf = lcc.Keyframe(c)
    c.lcc_encode_sequence(seq.key_index, seq.poses, ds, [len(p) for p in seq.frames], outs,
                          [o.numel() for o in outs], nb, kf)
    assert c.lcc_sync() == 0
    sizes = [int(x) for x in nb.cpu().numpy()]
    s = O.sensor(seq.sensor)
    bits = [outs[f][:sizes[f]].cpu().numpy() for f in range(n)]
    kft = O.kf_table_from_stream(s, bits[seq.key_index], c.num_tiles)
    kfd = lcc.Keyframe(c)
    c.lcc_keyframe_from_stream(outs[seq.key_index], sizes[seq.key_index], kfd)
    for f in range(n):
        isk = f == seq.key_index
        rng, _, _ = O.range_image(s, seq.frames[f])
        _check_decode(c, s, bits[f], rng, 0.02, None if isk else kfd, None if isk else kft,
                      None if isk else seq.poses[f], bound=thr)


def test_imu_poses_parity_and_decode():
    """P frames moved into the key frame's coordinates by poses integrated from 100 Hz IMU samples
    (Sec. III-D; automotive-grade noise and bias): the C-ABI poses agree with the oracle's within
    1e-12, the P frames encoded with the oracle's IMU poses match the oracle tile by tile, and the
    whole sequence encoded with the C-ABI's poses decodes (GPU decoder) within the quantisation
    bound of the oracle's range images."""
    from paper_2008_06972_gb300 import lcc
    from oracle import imu
    seq = synth.sequence_arc(0, 5)
    t_key = seq.key_index * synth.FRAME_DT
    smp = synth.imu_samples(0.0, 0.4, 10.0, math.radians(5.0), t_key, acc_sigma=0.05, gyro_sigma=math.radians(0.05),
                            acc_bias=(0.02, -0.02, 0.02), gyro_bias=(math.radians(0.05),) * 3, seed=17)
    n = len(seq.frames)
    pc = np.stack([lcc.imu_pose(smp.t, smp.acc, smp.gyro, smp.v_key, t_key, f * synth.FRAME_DT) for f in range(n)])
    po = np.stack([imu.pose_from_imu(smp.t, smp.acc, smp.gyro, smp.v_key, t_key, f * synth.FRAME_DT)
                   for f in range(n)])
    assert np.abs(pc - po).max() <= 1e-12
    assert np.abs(po[:, :3, 3] - seq.poses[:, :3, 3]).max() < 0.01   # the IMU pose is close to the arc
    frames = [f for f in range(n) if f != seq.key_index]
    border = _pframe_case(seq, frames, poses=[po[f] for f in frames])
    assert border <= 20
    c = H.ctx(seq.sensor, max_batch=16)
    ds = [H.to_dev(p) for p in seq.frames]
    outs = [H.out_buf(c) for _ in range(n)]
    nb = torch.zeros(n, dtype=torch.int64, device="cuda")
    kf = lcc.Keyframe(c)
    c.lcc_encode_sequence(seq.key_index, pc, ds, [len(p) for p in seq.frames], outs, [o.numel() for o in outs], nb, kf)
    assert c.lcc_sync() == 0
    assert sum(c.lcc_last_stats(f)["tiles_temporal"] for f in frames) > 0
    sizes = [int(x) for x in nb.cpu().numpy()]
    s = O.sensor(seq.sensor)
    kfd = lcc.Keyframe(c)
    c.lcc_keyframe_from_stream(outs[seq.key_index], sizes[seq.key_index], kfd)
    for f in range(n):
        isk = f == seq.key_index
        rng, _, _ = O.range_image(s, seq.frames[f])
        st, drng, _, _ = H.decode(c, outs[f][:sizes[f]].cpu().numpy(), None if isk else kfd, None if isk else pc[f])
        assert st == 0
        m = rng > 0
        assert ((drng > 0) == m).all()
        assert np.abs(drng[m] - rng[m]).max() <= 0.01 + 1e-5


@pytest.mark.parametrize("tile", [(4, 4), (4, 8), (8, 8), (8, 16)])
def test_raw_exact_keyframe_parity(cfg2_seq, tile):
    """The lossless raw option: the GPU stream is the oracle's on the GPU's planes, both decoders
    agree bit for bit, raw pixels decode to their range exactly and the raw section holds 32 bits
    per raw pixel."""
    seq = cfg2_seq
    r = _keyframe_case(seq.sensor, seq.frames[seq.key_index], tile=tile, raw_exact=1)
    h = streamfmt.header(r["bits"])
    assert h["flags"] & 4 and h["w_raw"] == 32 and h["n_raw"] > 0
    raw = streamfmt.raw_codes(r["bits"]).astype(np.uint32).view(np.float32)
    s = O.sensor(seq.sensor)
    rng, _, _ = O.range_image(s, seq.frames[seq.key_index])
    assert np.isin(raw, rng[rng > 0]).all()


def test_raw_exact_sequence_round_trip(cfg2_seq):
    """A whole sequence with raw_exact: every frame decodes (GPU) within q/2 and at least the raw
    pixels' count of pixels decode to their range bit for bit."""
    from paper_2008_06972_gb300 import lcc
    seq = cfg2_seq
    n = len(seq.frames)
    c = H.ctx(seq.sensor, max_batch=16, raw_exact=1)
    ds = [H.to_dev(p) for p in seq.frames]
    outs = [H.out_buf(c) for _ in range(n)]
    nb = torch.zeros(n, dtype=torch.int64, device="cuda")
    kf = lcc.Keyframe(c)
    c.lcc_encode_sequence(seq.key_index, seq.poses, ds, [len(p) for p in seq.frames], outs,
                          [o.numel() for o in outs], nb, kf)
    assert c.lcc_sync() == 0
    sizes = [int(x) for x in nb.cpu().numpy()]
    s = O.sensor(seq.sensor)
    kfd = lcc.Keyframe(c)
    c.lcc_keyframe_from_stream(outs[seq.key_index], sizes[seq.key_index], kfd)
    for f in (seq.key_index, 0, n - 1):
        isk = f == seq.key_index
        bits = outs[f][:sizes[f]].cpu().numpy()
        rng, _, _ = O.range_image(s, seq.frames[f])
        st, drng, _, _ = H.decode(c, bits, None if isk else kfd, None if isk else seq.poses[f])
        assert st == 0
        m = rng > 0
        assert np.abs(drng[m] - rng[m]).max() <= 0.01 + 1e-5
        exact = (drng.view(np.uint32) == rng.view(np.uint32)) & m
        assert exact.sum() >= streamfmt.header(bits)["n_raw"]


@pytest.mark.parametrize("tile,tcand", [((4, 4), 4), ((8, 8), 3)])
def test_temporal_candidates_parity(cfg2_seq, tile, tcand):
    """Several candidate K tiles per P tile: the K tile each test settled on, its rotated normal and
    the packed stream match the oracle's; more tiles pass than with the anchor's K tile alone."""
    seq = cfg2_seq
    border = _pframe_case(seq, [0, seq.key_index + 1], tile=tile, tcand=tcand)
    assert border <= 20


def test_temporal_candidates_sequence_matches_separate_calls(cfg2_seq):
    """The sequence call's lane-group temporal test with 4 candidates gives the fused per-thread
    test's streams, and passes more tiles than one candidate."""
    from paper_2008_06972_gb300 import lcc
    seq = cfg2_seq
    n = len(seq.frames)
    ds = [H.to_dev(p) for p in seq.frames]
    nb = torch.zeros(n, dtype=torch.int64, device="cuda")
    temporal = {}
    for tc in (1, 4):
        c = H.ctx(seq.sensor, max_batch=16, temporal_candidates=tc)
        outs = [H.out_buf(c) for _ in range(n)]
        c.lcc_encode_sequence(seq.key_index, seq.poses, ds, [len(p) for p in seq.frames], outs,
                              [o.numel() for o in outs], nb, None)
        assert c.lcc_sync() == 0
        nbs = nb.cpu().numpy()
        seq_bits = [outs[i][:nbs[i]].cpu().numpy() for i in range(n)]
        temporal[tc] = sum(c.lcc_last_stats(f)["tiles_temporal"] for f in range(n))
        c2 = H.ctx(seq.sensor, max_batch=16, temporal_candidates=tc)
        kf2 = lcc.Keyframe(c2)
        H.encode_keyframe(c2, seq.frames[seq.key_index], kf2)
        others = [f for f in range(n) if f != seq.key_index]
        pb, _ = H.encode_pframes(c2, kf2, [seq.poses[f] for f in others], [seq.frames[f] for f in others])
        for i, f in enumerate(others):
            assert pb[i].tobytes() == seq_bits[f].tobytes(), (tc, f)
    assert temporal[4] > temporal[1]


# --------------------------------------------- Eq. 3's three-coefficient plane form (plane3) --

@pytest.mark.parametrize("tile", [(4, 4), (8, 16)])
def test_plane3_keyframe_parity(cfg2_seq, tile):
    """Three-coefficient planes: the GPU's planes are the unit-normal planes of its coefficients (the
    oracle's conversion, bit for bit), its stream is the oracle's packing of its planes and
    coefficients, the fits agree with the oracle's plane3 fits (Layer 2), both decoders agree and
    every pixel decodes within q/2."""
    seq = cfg2_seq
    r = _keyframe_case(seq.sensor, seq.frames[seq.key_index], tile=tile, plane3=1)
    assert streamfmt.header(r["bits"])["flags"] & 16
    coef = r["ctx"].lcc_tile_coefficients(0)
    ok = r["recs"]["status"] == 2
    for t in np.nonzero(ok)[0]:
        back = O.plane_from3(int(coef[t, 3]), coef[t, :3])
        assert np.array_equal(back.view(np.uint32), r["recs"]["plane"][t].view(np.uint32))
    codes = streamfmt.tile_codes(r["bits"])
    assert not (codes == 2).any() and np.isin(codes, [6, 7, 8]).sum() == streamfmt.header(r["bits"])["n_runs"]


def test_plane3_pframe_parity(cfg2_seq):
    """P frames of a three-coefficient key frame: temporal test against its reconstructed planes,
    spatial fallback in the three-coefficient form, streams equal to the oracle's packing."""
    seq = cfg2_seq
    border = _pframe_case(seq, [1, seq.key_index + 2], plane3=1)
    assert border <= 20
