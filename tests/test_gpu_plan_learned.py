"""The batched plan with learned proposals (lcc_plan_set_proposals) on a subsample of the large
batched workload: 128x4096 frames, noisy poses, key-frame groups of 10 with the middle frame as key
frame (Sec. III-D), tiles autotuned among the shapes the net takes (8x8).

Every key-frame stream the plan writes must equal the oracle's packing of the GPU's planes, and the
GPU's seeded fits must agree with the oracle's seeded fit given the same proposals (Layer 2); every
P-frame stream must equal the oracle's packing of the GPU's temporal and spatial results against the
seeded key frame; every stream must decode with the oracle's decoder to the GPU decoder's ranges,
within q/2 of the binned input."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
import synth
from tests import harness as H
from tests.test_gpu_parity import _compare_spatial

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NSEQ, NFR = 2, 12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2008_06972_gb300 import lcc
    lcc.load()


@pytest.fixture(scope="module")
def trained_net():
    """A net trained on the GPU on two frames of other sequences of the same workload family."""
    from paper_2008_06972_gb300 import lcc
    from paper_2008_06972_gb300 import train as TR
    ctx = H.ctx(synth.CFG5_SENSOR, tile_h=8, tile_w=8)
    X, Y = [], []
    for sid in (1000, 1001):
        q = synth.sequence_cfg5_grouped(sid, n_frames=1)
        x, _, y, _ = TR.frame_examples(ctx, H.to_dev(q.frames[0]), len(q.frames[0]))
        X.append(x)
        Y.append(y)
    X, Y = torch.cat(X), torch.cat(Y)
    net = lcc.Net(TR.he_uniform_params(5), max_tiles=2048)
    losses = TR.train(net, X, Y, 200, 2048, 2e-3, seed=2, lr_final=2e-4)
    assert losses[-10:].mean() < 0.7 * losses[0]
    assert net.sync() == lcc.OK
    return net


@pytest.fixture(scope="module")
def batch():
    out = np.empty((NSEQ * NFR, synth.CFG5_SENSOR.rows * synth.CFG5_SENSOR.cols, 4), np.float32)
    return synth.batch_cfg5(out, n_seq=NSEQ, n_frames=NFR), out


def test_seeded_plan_matches_oracle_on_large_frames(trained_net, batch):
    from paper_2008_06972_gb300 import lcc
    from paper_2008_06972_gb300 import train as TR
    seqs, _ = batch
    net = trained_net
    stream = torch.cuda.current_stream()
    sensor = synth.CFG5_SENSOR
    s = O.sensor(sensor)
    d_pts = [[H.to_dev(f) for f in q.frames] for q in seqs]
    # autotuned among the net's tile shape: horizon and fit schedule on the first group
    k0 = synth.group_key(0, NFR, 10)
    best, rows = lcc.autotune(sensor, lcc.default_params(max_batch=10), k0, seqs[0].poses[:10], d_pts[0][:10],
                              [len(f) for f in seqs[0].frames[:10]], reps=1, stream=stream, shapes=[(8, 8)])
    assert (best.tile_h, best.tile_w) == (8, 8) and len(rows) == 3 * 5   # horizons x fit schedules
    best.max_batch = 3            # several chunks of key and P frames
    ctx = lcc.Context(sensor, best, stream=stream)
    descs = []
    for i, q in enumerate(seqs):
        outs = [H.out_buf(ctx) for _ in q.frames]
        descs.append(dict(ctx=0, key_interval=10, poses=q.poses, d_pts=d_pts[i], n=[len(f) for f in q.frames],
                          d_out=outs, cap=[o.numel() for o in outs],
                          d_nbytes=torch.zeros(NFR, dtype=torch.int64, device="cuda")))
    plan = lcc.Plan([ctx], descs)
    plan.set_proposals(net, TR.SKIP_LOGIT)
    plan.encode()
    assert plan.sync() == lcc.OK
    info = plan.info()
    assert info["seeded_key_frames"] == info["key_frames"] == NSEQ * 2
    # per-frame statistics of the plan: stream sizes and point counts of every frame, and their sum
    total = plan.stats()
    sizes = [d["d_nbytes"].cpu().numpy() for d in descs]
    assert total["bytes"] == sum(int(x.sum()) for x in sizes)
    assert total["points_in"] == sum(len(f) for q in seqs for f in q.frames)
    for i, q in enumerate(seqs):
        for f in (0, 5, 11):
            st_f = plan.stats(i, f)
            assert st_f["bytes"] == int(sizes[i][f]) and st_f["points_in"] == len(q.frames[f])
    got = [[d["d_out"][f][:int(n)].cpu().numpy() for f, n in enumerate(d["d_nbytes"].cpu().numpy())] for d in descs]
    # the captured graph replays the same streams
    plan.capture()
    for d in descs:
        for o in d["d_out"]:
            o.zero_()
    plan.replay()
    assert plan.sync() == lcc.OK
    again = [[d["d_out"][f][:int(n)].cpu().numpy() for f, n in enumerate(d["d_nbytes"].cpu().numpy())]
             for d in descs]
    assert all(a.tobytes() == b.tobytes() for x, y in zip(got, again) for a, b in zip(x, y))

    p = O.params(8, 8, best.fit_thr_m, best.quant_m, best.max_refits, best.min_inlier_frac, best.merge_runs)
    ref = H.ctx(sensor, **{k: getattr(best, k) for k in ("tile_h", "tile_w", "lookahead", "fit_schedule")},
                max_batch=16)
    nt = ref.num_tiles
    x = torch.zeros((nt, 64, 4), dtype=torch.int16, device="cuda")
    anc = torch.zeros((nt, 4), dtype=torch.float32, device="cuda")
    prop = torch.zeros((nt, 5), dtype=torch.float32, device="cuda")
    border_total = compared_total = 0
    for i, q in enumerate(seqs):
        for g0 in range(0, NFR, 10):
            fr = list(range(g0, min(g0 + 10, NFR)))
            k = synth.group_key(g0, NFR, 10)
            # key frame: the proposals recomputed through the public calls
            lcc.net_tile_inputs(ref, d_pts[i][k], len(q.frames[k]), x, anc)
            net.forward(x, nt, prop)
            assert net.sync() == lcc.OK and ref.lcc_sync() == lcc.OK
            pr = prop.cpu().numpy()
            one = H.out_buf(ref)
            nb1 = torch.zeros(1, dtype=torch.int64, device="cuda")
            ref.lcc_encode_keyframe_seeded(d_pts[i][k], len(q.frames[k]), prop, TR.SKIP_LOGIT, None, one,
                                           one.numel(), nb1)
            assert ref.lcc_sync() == lcc.OK
            assert one[:int(nb1.item())].cpu().numpy().tobytes() == got[i][k].tobytes(), f"seq {i} key {k}"
            recs = ref.lcc_tile_records(0)
            rng, _, _ = O.range_image(s, q.frames[k])
            ofits = O.fit_tiles_seeded(s, p, rng, pr, TR.SKIP_LOGIT)
            compared, border = _compare_spatial(s, p, rng, recs, ofits, p.fit_thr_m)
            border_total += border
            compared_total += compared
            planes, ok = H.gpu_planes(recs)
            cbits, _, _ = O.pack(s, p, 0, rng, planes, ok)
            assert cbits.tobytes() == got[i][k].tobytes(), f"seq {i} key {k}: oracle packing differs"
            skipped = (pr[:, 0] < TR.SKIP_LOGIT) & (ofits["n_valid"] >= 3)
            assert np.array_equal((recs["flags"] & 8) != 0, skipped)
            st, drng, _, _ = H.decode(ref, got[i][k])
            orng, _, _ = O.decode(s, got[i][k])
            assert st == lcc.OK and np.array_equal(drng.view(np.uint32), orng.view(np.uint32))
            m = rng > 0
            assert np.abs(drng[m] - rng[m]).max() <= p.quant_m / 2 + 1e-5
            # P frames of the group: against the seeded key frame's planes from its stream
            kf = lcc.Keyframe(ref)
            ref.lcc_keyframe_from_stream(torch.from_numpy(got[i][k]).cuda(), len(got[i][k]), kf)
            okft = O.kf_table_from_stream(s, got[i][k], nt)
            pf = [f for f in fr if f != k]
            pbits, precs = H.encode_pframes(ref, kf, [q.poses[f] for f in pf], [q.frames[f] for f in pf])
            for j, f in enumerate(pf):
                assert pbits[j].tobytes() == got[i][f].tobytes(), f"seq {i} frame {f}"
                r = precs[j]
                rng, _, _ = O.range_image(s, q.frames[f])
                otmp = O.temporal_tiles(s, p, rng, okft, q.poses[f])
                found = otmp["status"] > 0
                assert np.array_equal(r["t_status"] > 0, found)
                assert np.array_equal(r["kref"][found].astype(np.int64), otmp["kref"][found].astype(np.int64))
                planes, ok = H.gpu_planes(r)
                tplanes, kref = H.gpu_temporal(r)
                cbits, _, _ = O.pack(s, p, 1, rng, planes, ok, tplanes, kref)
                assert cbits.tobytes() == got[i][f].tobytes(), f"seq {i} frame {f}: oracle packing differs"
                st, drng, _, _ = H.decode(ref, got[i][f], kf, q.poses[f])
                orng, _, _ = O.decode(s, got[i][f], okft, q.poses[f])
                assert st == lcc.OK and np.array_equal(drng.view(np.uint32), orng.view(np.uint32))
                m = rng > 0
                assert np.abs(drng[m] - rng[m]).max() <= p.quant_m / 2 + 1e-5
            kf.free()
    assert border_total <= max(2, 0.005 * compared_total), (border_total, compared_total)
    plan.close()


def test_plan_host_outputs_match_device_outputs(batch):
    """lcc_plan_encode_host (page-locked points read in place or staged by the copy engines,
    streams copied to page-locked host buffers by one kernel) writes the streams the device-buffer
    plan writes."""
    from paper_2008_06972_gb300 import lcc
    seqs, host = batch
    stream = torch.cuda.current_stream()
    ctx = H.ctx(synth.CFG5_SENSOR, tile_h=8, tile_w=16, max_batch=4, stream=stream)
    cap = ctx.max_encoded_bytes
    pinned = torch.from_numpy(host).pin_memory()
    dev_descs, host_descs, h_out = [], [], []
    for i, q in enumerate(seqs):
        n = [len(f) for f in q.frames]
        outs = [H.out_buf(ctx) for _ in q.frames]
        dev_descs.append(dict(ctx=0, key_interval=10, poses=q.poses, d_pts=[H.to_dev(f) for f in q.frames], n=n,
                              d_out=outs, cap=[cap] * NFR, d_nbytes=torch.zeros(NFR, dtype=torch.int64,
                                                                                  device="cuda")))
        houts = [H.out_buf(ctx) for _ in q.frames]
        host_descs.append(dict(ctx=0, key_interval=10, poses=q.poses,
                               d_pts=[pinned[i * NFR + f].data_ptr() for f in range(NFR)], n=n, d_out=houts,
                               cap=[cap] * NFR, d_nbytes=torch.zeros(NFR, dtype=torch.int64, device="cuda")))
        h_out += [torch.zeros(cap, dtype=torch.uint8).pin_memory() for _ in range(NFR)]
    p_dev = lcc.Plan([ctx], dev_descs)
    p_dev.encode()
    assert p_dev.sync() == lcc.OK
    p_host = lcc.Plan([ctx], host_descs)
    p_host.capture()
    sizes = p_host.encode_host(h_out)
    for i, d in enumerate(dev_descs):
        nb = d["d_nbytes"].cpu().numpy()
        for f in range(NFR):
            assert int(sizes[i * NFR + f]) == int(nb[f])
            assert h_out[i * NFR + f][:int(nb[f])].numpy().tobytes() == \
                d["d_out"][f][:int(nb[f])].cpu().numpy().tobytes(), f"seq {i} frame {f}"
    # the points staged by the copy engines (two chunk buffers, one copy per frame) instead of read
    # in place: the same streams; then spread over two contexts of the same parameters, whose
    # classes run on two streams, each with its own staging
    p_host.set_staging(True)
    for ho in h_out:
        ho.zero_()
    sizes = p_host.encode_host(h_out)
    ctx2 = H.ctx(synth.CFG5_SENSOR, tile_h=8, tile_w=16, max_batch=4, stream=stream)
    for k, d in enumerate(host_descs):
        d["ctx"] = k % 2
    p_two = lcc.Plan([ctx, ctx2], host_descs)
    p_two.set_staging(True)
    p_two.capture()
    sizes2 = p_two.encode_host(h_out)
    assert np.array_equal(sizes, sizes2)
    for i, d in enumerate(dev_descs):
        nb = d["d_nbytes"].cpu().numpy()
        for f in range(NFR):
            assert int(sizes[i * NFR + f]) == int(nb[f])
            assert h_out[i * NFR + f][:int(nb[f])].numpy().tobytes() == \
                d["d_out"][f][:int(nb[f])].cpu().numpy().tobytes(), f"staged: seq {i} frame {f}"
    p_two.close()
    # pageable host outputs are rejected before anything runs
    with pytest.raises(lcc.LccError):
        p_host.encode_host([np.zeros(cap, np.uint8) for _ in range(NSEQ * NFR)])
    with pytest.raises(lcc.LccError):
        p_host.set_staging(2)
    p_dev.close()
    p_host.close()
