"""Batched encode of a table of sequences (lcc_plan_*), its CUDA-graph replay, and the autotuner.

Every stream a plan writes must be byte-identical to what the single-sequence entry point
(lcc_encode_sequence, itself checked against the oracle in test_gpu_parity.py) writes for the
same key-frame group, and must decode with the oracle's independent decoder to the same
ranges as the GPU decoder, within q/2 of the binned input (Sec. III-C: groups of frames with
the middle frame as key frame)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
import synth
from tests import harness as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06972_gb300 import lcc
    lcc.load()


# (sensor class, frames) per sequence: uneven lengths, two resolutions, groups of 10 with a
# short last group, one sequence shorter than a group
SEQS = [(0, 5), (2, 12), (0, 23), (2, 7), (0, 3), (2, 10)]
PARAMS = {0: dict(tile_h=4, tile_w=4, max_batch=4), 2: dict(tile_h=8, tile_w=8, max_batch=3)}
INTERVAL = 10


@pytest.fixture(scope="module")
def batch():
    out = []
    for i, (cls, n) in enumerate(SEQS):
        out.append(synth.grouped_sequence(synth.CFG3_SENSORS[cls], cls, n, synth.config_seed(3, 100 + i, 0),
                                          INTERVAL))
    return out


def _setup(batch, poses=None):
    from paper_2008_06972_gb300 import lcc
    stream = torch.cuda.current_stream()
    classes = sorted({s.sensor_class for s in batch})
    ctxs = [H.ctx(synth.CFG3_SENSORS[c], stream=stream, **PARAMS[c]) for c in classes]
    descs, bufs = [], []
    for i, s in enumerate(batch):
        c = ctxs[classes.index(s.sensor_class)]
        d_pts = [H.to_dev(f) for f in s.frames]
        d_out = [H.out_buf(c) for _ in s.frames]
        nb = torch.zeros(len(s.frames), dtype=torch.int64, device="cuda")
        descs.append(dict(ctx=classes.index(s.sensor_class), key_interval=s.key_interval,
                          poses=s.poses if poses is None else poses[i], d_pts=d_pts,
                          n=[len(f) for f in s.frames], d_out=d_out, cap=[o.numel() for o in d_out], d_nbytes=nb))
        bufs.append((d_pts, d_out, nb))
    return lcc, classes, ctxs, descs


def _streams(descs):
    out = []
    for d in descs:
        nb = d["d_nbytes"].cpu().numpy()
        out.append([d["d_out"][f][:nb[f]].cpu().numpy() for f in range(len(nb))])
    return out


def _reference(batch, poses=None):
    """Each key-frame group encoded by lcc_encode_sequence on a context of its own."""
    from paper_2008_06972_gb300 import lcc
    ref = []
    for i, s in enumerate(batch):
        n = len(s.frames)
        P = s.poses if poses is None else poses[i]
        c = H.ctx(s.sensor, **{**PARAMS[s.sensor_class], "max_batch": 16})
        streams = [None] * n
        for g0 in range(0, n, s.key_interval):
            fr = list(range(g0, min(g0 + s.key_interval, n)))
            k = synth.group_key(g0, n, s.key_interval)
            ds = [H.to_dev(s.frames[f]) for f in fr]
            outs = [H.out_buf(c) for _ in fr]
            nb = torch.zeros(len(fr), dtype=torch.int64, device="cuda")
            c.lcc_encode_sequence(k - g0, np.stack([P[f] for f in fr]), ds, [len(s.frames[f]) for f in fr], outs,
                                  [o.numel() for o in outs], nb, None)
            assert c.lcc_sync() == lcc.OK
            nbs = nb.cpu().numpy()
            for j, f in enumerate(fr):
                streams[f] = outs[j][:nbs[j]].cpu().numpy()
        ref.append(streams)
    return ref


def _assert_same(a, b):
    for i, (sa, sb) in enumerate(zip(a, b)):
        for f, (x, y) in enumerate(zip(sa, sb)):
            assert x.tobytes() == y.tobytes(), f"sequence {i} frame {f}: stream differs"


def test_plan_matches_per_sequence_encode(batch):
    lcc, classes, ctxs, descs = _setup(batch)
    plan = lcc.Plan(ctxs, descs)
    plan.encode()
    assert plan.sync() == lcc.OK
    got = _streams(descs)
    _assert_same(got, _reference(batch))
    info = plan.info()
    assert info["frames"] == sum(n for _, n in SEQS)
    assert info["key_frames"] == sum((n + INTERVAL - 1) // INTERVAL for _, n in SEQS)
    assert info["classes"] == 2 and info["launches"] > 0
    # the oracle's decoder reads every stream to the GPU decoder's ranges, within q/2 of the input
    for i, s in enumerate(batch):
        os_ = O.sensor(s.sensor)
        c = ctxs[classes.index(s.sensor_class)]
        n = len(s.frames)
        for g0 in range(0, n, s.key_interval):
            k = synth.group_key(g0, n, s.key_interval)
            kft = O.kf_table_from_stream(os_, got[i][k], c.num_tiles)
            kf = lcc.Keyframe(c)
            c.lcc_keyframe_from_stream(torch.from_numpy(got[i][k]).cuda(), len(got[i][k]), kf)
            assert c.lcc_sync() == lcc.OK
            for f in range(g0, min(g0 + s.key_interval, n)):
                pose = None if f == k else s.poses[f]
                st, drng, _, _ = H.decode(c, got[i][f], None if f == k else kf, pose)
                assert st == lcc.OK
                orng, _, _ = O.decode(os_, got[i][f], None if f == k else kft, pose)
                assert np.array_equal(drng.view(np.uint32), orng.view(np.uint32))
                rng, _, _ = O.range_image(os_, s.frames[f])
                m = rng > 0
                assert ((drng > 0) == m).all()
                assert np.abs(drng[m] - rng[m]).max() <= 0.01 + 1e-5
    plan.close()


def test_plan_graph_replay_and_update(batch):
    lcc, classes, ctxs, descs = _setup(batch)
    plan = lcc.Plan(ctxs, descs)
    plan.capture()
    info = plan.info()
    assert info["captured"] == 1 and info["graph_nodes"] >= info["launches"] > 0
    for d in descs:
        for o in d["d_out"]:
            o.zero_()
    plan.replay()
    assert plan.sync() == lcc.OK
    first = _streams(descs)
    _assert_same(first, _reference(batch))
    plan.replay()
    assert plan.sync() == lcc.OK
    _assert_same(_streams(descs), first)
    # new (noisy) poses: the captured graph is updated in place and replays the new work
    noisy = [np.stack([synth.perturb_pose(s.poses[f], 0.01, 0.05, 500 + 31 * i + f)
                       if f != synth.group_key(f, len(s.frames), s.key_interval) else s.poses[f]
                       for f in range(len(s.frames))]) for i, s in enumerate(batch)]
    for d, p in zip(descs, noisy):
        d["poses"] = p
    plan.update(descs)
    plan.replay()
    assert plan.sync() == lcc.OK
    _assert_same(_streams(descs), _reference(batch, noisy))
    plan.close()


def test_plan_spatial_first_schedule_matches_per_sequence_encode(batch):
    """Fit schedule 4 (P frames fitted spatially first, temporal test after) writes the streams
    of the per-sequence encode."""
    from paper_2008_06972_gb300 import lcc
    stream = torch.cuda.current_stream()
    classes = sorted({s.sensor_class for s in batch})
    ctxs = [H.ctx(synth.CFG3_SENSORS[c], stream=stream, fit_schedule=4, **PARAMS[c]) for c in classes]
    _, _, _, descs = _setup(batch)
    plan = lcc.Plan(ctxs, descs)
    plan.capture()
    plan.replay()
    assert plan.sync() == lcc.OK
    _assert_same(_streams(descs), _reference(batch))
    plan.close()


def test_plan_rejects_bad_tables(batch):
    from paper_2008_06972_gb300 import lcc
    lcc_, classes, ctxs, descs = _setup(batch[:2])
    bad = [dict(d) for d in descs]
    bad[0]["ctx"] = 5
    with pytest.raises(lcc.LccError):
        lcc.Plan(ctxs, bad)
    with pytest.raises(lcc.LccError):
        lcc.Plan([ctxs[0], ctxs[0]], descs)
    other = torch.cuda.Stream()
    c_other = H.ctx(synth.CFG3_SENSORS[2], stream=other, **PARAMS[2])
    with pytest.raises(lcc.LccError):
        lcc.Plan([ctxs[0], c_other], descs)
    plan = lcc.Plan(ctxs, descs)
    changed = [dict(d) for d in descs]
    changed[0]["key_interval"] = 3
    with pytest.raises(lcc.LccError):
        plan.update(changed)
    # a rejected update leaves the plan as it was
    plan.encode()
    assert plan.sync() == lcc.OK
    _assert_same(_streams(descs), _reference(batch[:2]))
    plan.close()


def test_autotune_picks_fastest_within_byte_slack():
    from paper_2008_06972_gb300 import lcc
    s = synth.grouped_sequence(synth.CFG3_SENSORS[1], 1, 6, synth.config_seed(3, 200, 0), 10)
    k = synth.group_key(0, 6, 10)
    ds = [H.to_dev(f) for f in s.frames]
    base = lcc.default_params(max_batch=8)
    best, rows = lcc.autotune(s.sensor, base, k, s.poses, ds, [len(f) for f in s.frames], reps=2,
                              stream=torch.cuda.current_stream())
    assert len(rows) == 4 * 3 * 5   # tile shapes x horizons x fit schedules {0, 3, 4, 5, 6}
    assert sorted({r["fit_schedule"] for r in rows}) == [0, 3, 4, 5, 6]
    # every schedule fits the same planes: per tile shape and horizon one stream size
    for th, tw, la in {(r["tile_h"], r["tile_w"], r["lookahead"]) for r in rows}:
        assert len({r["bytes"] for r in rows if (r["tile_h"], r["tile_w"], r["lookahead"]) == (th, tw, la)}) == 1
    ok = [r for r in rows if r["status"] == lcc.OK]
    assert len(ok) == len(rows)
    assert all(r["max_err_m"] <= 0.01 + 1e-5 for r in ok)
    chosen = [r for r in rows if r["chosen"]]
    assert len(chosen) == 1
    ch = chosen[0]
    mn = min(r["bytes"] for r in ok)
    assert ch["bytes"] <= 1.05 * mn
    assert ch["mpts_per_s"] == max(r["mpts_per_s"] for r in ok if r["bytes"] <= 1.05 * mn)
    assert (best.tile_h, best.tile_w, best.lookahead, best.fit_schedule) == \
        (ch["tile_h"], ch["tile_w"], ch["lookahead"], ch["fit_schedule"])
    assert best.max_batch == 8 and abs(best.fit_thr_m - base.fit_thr_m) < 1e-9
