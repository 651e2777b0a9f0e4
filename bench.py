"""Throughput of the spatio-temporal LiDAR encoder on the large batched workload.

Headline workload (one step): 32 sequences of 100 frames of 128x4096 range images (about 1.07 G
points, 17 GB of float4 input resident in HBM), key-frame groups of 10 frames with the middle
frame as key frame (Sec. III-D), 1.5 m and 1 deg of ego motion per frame, poses perturbed by
1 cm / 0.05 deg, twice the frame-1 scene density with 5% clutter.  One batched plan over the whole
table is recorded as a CUDA graph and replayed once per step; its tiles are autotuned among the
shapes the proposal net takes (8x8), and the net (trained on the GPU beforehand on frames of other
sequences, labelled by the plain encoder) seeds the key frames' fits.  The plain plan (tiles
autotuned over every shape, no net) is timed on the same inputs in the same run.  Threshold
0.05 m, quantisation 0.02 m: max decode error 0.01 m <= 2 cm, checked on every frame.

The JSON line also carries: the oracle on the host cores over a sample of the same workload
(cpu_baseline), the end-to-end figure through lcc_plan_encode_host (page-locked host inputs read
in place, streams copied to page-locked host buffers), the dominant kernel's roofline, and
sections: "hdl64_sequence" (one 10-frame 64x2048 sequence per call, with decode, entropy, sweep
and IMU rows), "batched" (64 uneven sequences of four resolutions), "learned" (the proposal net on
64x2048 key frames).  --impl reference times the oracle on the headline workload.
Multi-GPU: one process per GPU (torchrun); each rank encodes its own 32 sequences (no data-path
collective; weak scaling); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpoints/s encoded at ≤2 cm max error: plain vs batched+learned, % HBM roofline"
WORKLOAD = "HDL-64E sequence: 10 frames of 64x2048 (1 key frame + 9 P-frames), tiles 4x4, thr 0.05 m, q 0.02 m"
CFG5_WORKLOAD = ("large batched + learned: 32 sequences x 100 frames of 128x4096, key-frame groups of 10, "
                 "1.5 m + 1 deg/frame, poses perturbed 1 cm / 0.05 deg, 2x frame-1 scene density, 5% clutter; "
                 "one plan replayed as a CUDA graph, tiles autotuned among 8x8 + learned proposal on the key frames")
UNIT = "Mpoints/s"


def cfg5_config(args) -> dict:
    return {"workload": CFG5_WORKLOAD, "sequences": args.cfg5_seqs, "frames_per_sequence": args.cfg5_frames,
            "key_interval": 10, "sensor": "128x4096, elevation -15..+15 deg, 80 m", "thr_m": args.thr, "q_m": 0.02,
            "l2": "inputs (about 17 GB) larger than L2: no flush"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lcc", choices=["lcc", "reference"])
    ap.add_argument("--tile", default="4x4")
    ap.add_argument("--thr", type=float, default=0.05)
    ap.add_argument("--lookahead", type=int, default=16)
    ap.add_argument("--refits", type=int, default=3)
    ap.add_argument("--solver", default="ff", choices=["ff", "fp64"])
    ap.add_argument("--schedule", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="bounded oracle sample length")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the uneven multi-sequence batch")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal section")
    ap.add_argument("--no-sweep", action="store_true", help="skip the tile / threshold sweep")
    ap.add_argument("--no-imu", action="store_true", help="skip the IMU-pose section")
    ap.add_argument("--no-entropy", action="store_true", help="skip the entropy-stage section")
    ap.add_argument("--clocks-csv", default="", help="where the SM-clock samples of the timed region go "
                    "({rank} is replaced by the rank); default: a file under /tmp")
    ap.add_argument("--train-steps", type=int, default=0, help="training steps of the learned section "
                    "(0: one epoch over the training tiles, at least 300)")
    ap.add_argument("--train-frames", type=int, default=512, help="64x2048 frames the learned section trains on "
                    "(the configuration's full scale is 20000)")
    ap.add_argument("--cfg5-seqs", type=int, default=32, help="sequences of the headline workload (per rank)")
    ap.add_argument("--cfg5-frames", type=int, default=100, help="frames per sequence of the headline workload")
    ap.add_argument("--cfg5-train-frames", type=int, default=64,
                    help="128x4096 frames (of other sequences) the headline's net is trained on")
    ap.add_argument("--cfg5-train-steps", type=int, default=600)
    ap.add_argument("--cpu-steps", type=int, default=10, help="oracle frames per core for cpu_baseline")
    ap.add_argument("--no-hdl64", action="store_true", help="skip the single-sequence HDL-64E section")
    ap.add_argument("--profile-plan", action="store_true",
                    help="profiling case: --cfg5-seqs x --cfg5-frames of the headline workload encoded --steps times "
                         "by one eager plan with fixed parameters (--tile, --lookahead, --schedule, --max-batch), "
                         "no autotuning, training or other sections (for ncu)")
    ap.add_argument("--max-batch", type=int, default=64, help="frames per launch of the profiling case")
    ap.add_argument("--profile-net", action="store_true",
                    help="profiling case: the proposal net's forward over --net-tiles seeded tiles, --steps calls after "
                         "one warm-up call, nothing else (for ncu)")
    ap.add_argument("--net-tiles", type=int, default=98304)
    ap.add_argument("--profile-sequence", action="store_true",
                    help="profiling case: the HDL-64E sequence encoded by lcc_encode_sequence --steps times after one "
                         "warm-up call (--tile, --thr, --lookahead, --schedule), nothing else (for ncu)")
    ap.add_argument("--profile-train", action="store_true",
                    help="profiling case: --steps training steps of the proposal net on 4096 seeded tiles after one "
                         "warm-up step, nothing else (for ncu)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_workload(rank: int):
    """Each rank encodes its own sequence (weak scaling): sequence id = rank."""
    import synth
    seq = synth.sequence_cfg2(sequence_id=rank)
    return seq


def oracle_sample(seq, th, tw, thr, seconds):
    """Time the oracle (as it stands) on whole sequences until `seconds` pass."""
    import oracle as O
    s = O.sensor(seq.sensor)
    p = O.params(th, tw, thr, 0.02)
    pts_per_seq = sum(len(f) for f in seq.frames)
    t0 = time.perf_counter()
    nseq = 0
    while True:
        _, kft, _, _ = O.encode_keyframe(s, p, seq.frames[seq.key_index])
        for f in range(len(seq.frames)):
            if f != seq.key_index:
                O.encode_pframe(s, p, kft, seq.poses[f], seq.frames[f])
        nseq += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return pts_per_seq * nseq / el / 1e6, nseq, el


def _oracle_worker(job):
    seq, th, tw, thr, seconds = job
    return oracle_sample(seq, th, tw, thr, seconds)


def oracle_all_cores(seq, th, tw, thr, seconds, pool=None):
    """The oracle as it stands, one process per host core, each on whole sequences for `seconds`
    (the CPU analogue of one thread per cloud).  Processes are spawned, not forked; `pool` (a
    spawned pool of one process per core) may be passed to reuse it across calls."""
    import multiprocessing as mp
    import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    if pool is None:
        with mp.get_context("spawn").Pool(cores) as own:
            res = own.map(_oracle_worker, [(seq, th, tw, thr, seconds)] * cores)
    else:
        res = pool.map(_oracle_worker, [(seq, th, tw, thr, seconds)] * cores)
    pts = sum(len(f) for f in seq.frames)
    wall = max(el for _, _, el in res)
    nseq = sum(n for _, n, _ in res)
    return pts * nseq / wall / 1e6, nseq, wall, cores


TRAFFIC_FILE_CFG5 = os.path.join(ROOT, "profiles", "dram_traffic_cfg5_plan.txt")


def measured_traffic_cfg5(kernel: str):
    """DRAM bytes per frame of a headline-plan kernel from the committed ncu summary (to be scaled
    by the frames of a launch), or None when the kernel's sources changed since."""
    if kernel not in KERNEL_SOURCES:
        return None
    try:
        for line in open(TRAFFIC_FILE_CFG5):
            f = line.split()
            if len(f) == 3 and f[0] == kernel and not line.startswith("#"):
                return float(f[1]) if f[2] == source_digest(kernel) else None
    except OSError:
        pass
    return None


KERNEL_SOURCES = {"bin": ("k_bin.cu",), "fit": ("k_fit.cu",), "rounds": ("k_fit.cu",), "lookbehind": ("k_fit.cu",),
                  "temporal": ("k_fit.cu",),
                  "merge": ("k_merge.cu", "scan_frame.cuh"), "pack": ("k_pack.cu",), "net_inputs": ("k_net.cu",),
                  "net_fwd": ("k_net.cu",)}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic_hdl64_sequence.txt")


def source_digest(kernel: str) -> str:
    """Digest of the sources a kernel is compiled from (its .cu plus the shared headers)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2008_06972_gb300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kernel] + ("lcc_internal.cuh", "ffmath.cuh"):
        with open(os.path.join(csrc, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, averaged over one
    step's launches) from the committed ncu summary, or None when the kernel's sources changed
    after the counters were taken."""
    if kernel not in KERNEL_SOURCES:
        return None
    try:
        for line in open(TRAFFIC_FILE):
            f = line.split()
            if len(f) == 3 and f[0] == kernel and not line.startswith("#"):
                return float(f[1]) if f[2] == source_digest(kernel) else None
    except OSError:
        pass
    return None


class Clocks:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "10", "-i", str(int(os.environ.get("LOCAL_RANK", "0")))],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            # enter the timed region only once the sampler is producing samples
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 10.0:
                self.fh.flush()
                if os.path.getsize(self.path) > 0:
                    break
                time.sleep(0.01)
            self.skip = 0
            try:
                self.skip = len(open(self.path).read().strip().splitlines())   # samples before the region
            except Exception:
                pass
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines()]
            rows = rows[getattr(self, "skip", 0):] or rows[-1:]
            rows = [[c.strip() for c in r] for r in rows if len(r) >= 9]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _oracle_core(conn, seq_id, learned, thr, n_frames, key_interval):
    """One host core: the oracle (as it stands) encodes the frames of its own key-frame groups of
    the large batched workload (sequence seq_id), one frame per request, key frame first.  The key
    frame takes the learned path when `learned` (the oracle net's forward on every 8x8 tile, with
    its own seeded initial weights, then the seeded fit) and the plain fit otherwise; P frames are
    encoded against it.  Replies (points, seconds of oracle work, stream bytes).  Rendering the
    next group happens between requests and is not part of the reported seconds."""
    import oracle as O
    from oracle import net as N
    import synth
    O.build()
    s = O.sensor(synth.CFG5_SENSOR)
    p = O.params(8, 8, thr, 0.02)
    theta = N.init_params(7)
    beams = O.beams(s)
    skip = math.log(0.05 / 0.95)
    ngroups = (n_frames + key_interval - 1) // key_interval

    def load(g):
        f0 = g * key_interval
        f1 = min(f0 + key_interval, n_frames)
        q = synth.sequence_cfg5_grouped(seq_id, n_frames, key_interval, only=set(range(f0, f1)))
        k = synth.group_key(f0, n_frames, key_interval)
        return q, [k] + [f for f in range(f0, f1) if f != k]

    g, j = 0, 0
    q, order = load(0)
    kft = None
    while True:
        msg = conn.recv()
        if msg is None:
            break
        f = order[j]
        pts = q.frames[f]
        t0 = time.perf_counter()
        if j == 0:
            rng, _, _ = O.range_image(s, pts)
            if learned:
                X, _, _ = N.tile_inputs(rng, beams)
                prop = np.concatenate([N.forward(theta, X[a:a + 1024])[0] for a in range(0, len(X), 1024)])
                fits = O.fit_tiles_seeded(s, p, rng, prop.astype(np.float32), skip)
            else:
                fits = O.fit_tiles(s, p, rng)
            bits, kft, _ = O.pack(s, p, 0, rng, fits["plane"], (fits["status"] == O.FIT_OK).astype(np.uint8))
        else:
            bits = O.encode_pframe(s, p, kft, q.poses[f], pts)[0]
        conn.send((len(pts), time.perf_counter() - t0, len(bits)))
        j += 1
        if j == len(order):
            g = (g + 1) % ngroups
            q, order = load(g)
            j = 0


class OracleCores:
    """One spawned process per host core (_oracle_core), each on its own sequence of the large
    batched workload; step() has every core encode its next frame (the cores work side by side)
    and returns (points, seconds: the slowest core's oracle time, stream bytes)."""

    def __init__(self, cores, learned=True, thr=0.05, first_seq=0, n_frames=100, key_interval=10):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.cores = cores
        self.conns, self.procs = [], []
        for c in range(cores):
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_core, args=(b, first_seq + c, learned, thr, n_frames, key_interval),
                             daemon=True)
            pr.start()
            self.conns.append(a)
            self.procs.append(pr)

    def step(self):
        for c in self.conns:
            c.send(1)
        res = [c.recv() for c in self.conns]
        return sum(r[0] for r in res), max(r[1] for r in res), sum(r[2] for r in res)

    def close(self):
        for c in self.conns:
            try:
                c.send(None)
            except Exception:
                pass
        for pr in self.procs:
            pr.join(timeout=10)
            if pr.is_alive():
                pr.terminate()


def oracle_cfg5(steps, thr=0.05, cores=None, warmup=0):
    """The oracle on all host cores over `steps` frames per core (one key-frame group = 10
    steps, key frame first): Mpoints/s over the summed step times, and what was sampled."""
    cores = cores or os.cpu_count() or 1
    oc = OracleCores(cores, learned=True, thr=thr)
    try:
        for _ in range(warmup):
            oc.step()
        pts = sec = 0.0
        for _ in range(steps):
            a, b, _ = oc.step()
            pts += a
            sec += b
    finally:
        oc.close()
    return pts / sec / 1e6, pts, sec, cores


def run_reference(args, rank, world):
    """The reference arm: the oracle (plain C and numpy, as it stands) on the headline workload,
    one process per host core, each step every core encoding the next frame of its own key-frame
    group (key frame first: the oracle net's forward on every tile, then the seeded fit)."""
    if world > 1 and rank != 0:
        return
    cores = os.cpu_count() or 1
    oc = OracleCores(cores, learned=True, thr=args.thr)
    try:
        for _ in range(args.warmup):
            oc.step()
        pts = sec = 0.0
        for _ in range(args.steps):
            a, b, _ = oc.step()
            pts += a
            sec += b
    finally:
        oc.close()
    value = pts / sec / 1e6
    groups = args.steps / 10.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg5_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} steps of one frame per core ({groups:g} key-frame groups of "
                                       f"10 frames of 128x4096 per core, key frame first: oracle net forward on "
                                       f"every 8x8 tile + seeded fit; P frames plain), {pts / 1e6:.1f} M points"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args, stream, hbm):
    """Uneven batch of 64 sequences (lengths U{5..40}, four resolutions, key-frame groups of 10):
    one plan over four autotuned class contexts, captured once as a CUDA graph and replayed,
    against the plain path (one lcc_encode_sequence call per key-frame group, default params)
    on the same inputs.  Inputs (about 2.3 GB) are larger than L2."""
    import torch
    import synth
    from paper_2008_06972_gb300 import lcc
    t0 = time.perf_counter()
    seqs = synth.batch_cfg3()
    gen_s = time.perf_counter() - t0
    classes = sorted({s.sensor_class for s in seqs})
    d_pts = [[torch.from_numpy(f).cuda() for f in s.frames] for s in seqs]
    npts = [[len(f) for f in s.frames] for s in seqs]
    total_pts = sum(sum(n) for n in npts)
    # autotune every resolution class on its first sequence's first key-frame group
    tuned, tune_rows = {}, {}
    t0 = time.perf_counter()
    for c in classes:
        s = next(q for q in seqs if q.sensor_class == c)
        m = min(len(s.frames), s.key_interval)
        k = synth.group_key(0, len(s.frames), s.key_interval)
        best, rows = lcc.autotune(s.sensor, lcc.default_params(max_batch=64, fit_thr_m=args.thr), k, s.poses[:m],
                                  d_pts[seqs.index(s)][:m], npts[seqs.index(s)][:m], reps=3, stream=stream)
        tuned[c] = best
        ch = next(r for r in rows if r["chosen"])
        tune_rows[c] = {"tile": f"{ch['tile_h']}x{ch['tile_w']}", "lookahead": ch["lookahead"],
                        "fit_schedule": ch["fit_schedule"], "sample_mpts_s": round(ch["mpts_per_s"], 1),
                        "candidates": len(rows)}
    tune_s = time.perf_counter() - t0
    ctxs = [lcc.Context(synth.CFG3_SENSORS[c], tuned[c], stream=stream) for c in classes]
    descs = []
    for i, s in enumerate(seqs):
        cx = ctxs[classes.index(s.sensor_class)]
        outs = [torch.empty(cx.max_encoded_bytes, dtype=torch.uint8, device="cuda") for _ in s.frames]
        descs.append(dict(ctx=classes.index(s.sensor_class), key_interval=s.key_interval, poses=s.poses,
                          d_pts=d_pts[i], n=npts[i], d_out=outs, cap=[o.numel() for o in outs],
                          d_nbytes=torch.zeros(len(s.frames), dtype=torch.int64, device="cuda")))
    plan = lcc.Plan(ctxs, descs)
    plan.capture()
    for _ in range(3):
        plan.replay()
    assert plan.sync() == lcc.OK
    steps = max(3, min(args.steps, 10))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        evs[k][0].record(stream)
        plan.replay()
        evs[k][1].record(stream)
    st = plan.sync()
    assert st == lcc.OK, lcc.status_string(st)
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    info = plan.info()
    bytes_b = int(sum(int(d["d_nbytes"].sum().item()) for d in descs))
    # max decode error over the first key-frame group of every sequence
    max_err = 0.0
    for i, s in enumerate(seqs):
        cx = ctxs[classes.index(s.sensor_class)]
        npx = s.sensor.rows * s.sensor.cols
        ref = torch.empty(npx, dtype=torch.float32, device="cuda")
        dec = torch.empty(npx, dtype=torch.float32, device="cuda")
        nb = descs[i]["d_nbytes"].cpu().numpy()
        k = synth.group_key(0, len(s.frames), s.key_interval)
        kfd = lcc.Keyframe(cx)
        cx.lcc_keyframe_from_stream(descs[i]["d_out"][k], int(nb[k]), kfd)
        for f in range(min(len(s.frames), s.key_interval)):
            cx.lcc_range_image(d_pts[i][f], npts[i][f], ref, None)
            cx.lcc_decode(descs[i]["d_out"][f], int(nb[f]), None if f == k else kfd, None if f == k else s.poses[f],
                          dec, None, None)
            assert cx.lcc_sync() == lcc.OK
            msk = ref > 0
            if bool(msk.any()):
                max_err = max(max_err, float((dec[msk] - ref[msk]).abs().max().item()))
        kfd.free()
    plan.close()
    # plain path: one lcc_encode_sequence per key-frame group, default params, eager launches
    pctx = {c: lcc.Context(synth.CFG3_SENSORS[c], lcc.default_params(max_batch=16, fit_thr_m=args.thr),
                           stream=stream) for c in classes}
    pouts = {c: [torch.empty(pctx[c].max_encoded_bytes, dtype=torch.uint8, device="cuda") for _ in range(10)]
             for c in classes}
    pnb = torch.zeros(10, dtype=torch.int64, device="cuda")
    pbytes = torch.zeros(1, dtype=torch.int64, device="cuda")

    def plain(count=False):
        for i, s in enumerate(seqs):
            cx = pctx[s.sensor_class]
            n = len(s.frames)
            for g0 in range(0, n, s.key_interval):
                fr = list(range(g0, min(g0 + s.key_interval, n)))
                k = synth.group_key(g0, n, s.key_interval)
                cx.lcc_encode_sequence(k - g0, s.poses[g0:g0 + len(fr)], d_pts[i][g0:g0 + len(fr)],
                                       npts[i][g0:g0 + len(fr)], pouts[s.sensor_class][:len(fr)],
                                       [o.numel() for o in pouts[s.sensor_class][:len(fr)]], pnb, None)
                if count:
                    pbytes.add_(pnb[:len(fr)].sum())

    plain(count=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    plain()
    b.record(stream)
    torch.cuda.synchronize()
    for cx in pctx.values():
        assert cx.lcc_sync() == lcc.OK
    plain_ms = a.elapsed_time(b)
    path_bytes = 16.0 * total_pts + bytes_b
    return {
        "workload": "64 sequences, lengths U{5..40}, resolutions {16x1024, 32x1024, 64x2048, 128x2048}, "
                    "key-frame groups of 10, frame-1 scene family",
        "sequences": len(seqs), "frames": info["frames"], "key_frames": info["key_frames"],
        "points": total_pts, "value": total_pts / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
        "steps": steps, "graph_nodes": info["graph_nodes"], "gpu_launches_per_step": info["launches"],
        "bytes_per_step": bytes_b, "compression_ratio": 12.0 * total_pts / bytes_b,
        "max_decode_error_m_sampled": max_err,
        "roofline_path": {"alg_bytes_per_step": path_bytes, "achieved_gbs": path_bytes / (ms * 1e-3) / 1e9,
                          "frac": path_bytes / (ms * 1e-3) / 1e9 / hbm},
        "autotuned": {f"{synth.CFG3_SENSORS[c].rows}x{synth.CFG3_SENSORS[c].cols}": tune_rows[c] for c in classes},
        "plain_per_group": {"value": total_pts / (plain_ms * 1e-3) / 1e6, "ms_per_step": plain_ms,
                            "bytes_per_step": int(pbytes.item()), "params": "tiles 4x4, horizon 16, schedule 0"},
        "speedup_vs_plain": plain_ms / ms,
        "l2": "inputs (2.3 GB) larger than L2", "setup_s": {"generate": gen_s, "autotune": tune_s},
    }


def run_sweep(args, stream, seq, d_pts, flush):
    """The HDL-64E sequence under the swept parameters (tiles 4x4 and 8x8, fit thresholds 0.02,
    0.05 and 0.10 m, q 0.02 m; the no-delta mode at 0.02 m; lossless raw codes; four temporal
    candidates; temporal run growth off; three-coefficient planes; the FP64 plane solver): device
    throughput (CUDA events, L2 flushed between steps), compression ratio, tile modes and the max
    decode error of every frame."""
    import torch
    from paper_2008_06972_gb300 import lcc
    n_frames = len(seq.frames)
    n = [len(f) for f in seq.frames]
    pts = sum(n)
    H, W = seq.sensor.rows, seq.sensor.cols
    steps = max(10, min(args.steps, 50))
    rows = []
    points = [(th, tw, thr, 0, 0, 1, 1, 0, 0) for th, tw in ((4, 4), (8, 8)) for thr in (0.02, 0.05, 0.10)]
    points += [(4, 4, 0.02, 1, 0, 1, 1, 0, 0), (8, 8, 0.02, 1, 0, 1, 1, 0, 0)]   # the paper's no-delta mode at 2 cm
    points += [(4, 4, 0.05, 0, 1, 1, 1, 0, 0)]                      # raw pixels kept losslessly (fp32 raw codes)
    points += [(4, 4, 0.05, 0, 0, 4, 1, 0, 0)]                      # up to 4 candidate K tiles per P tile
    points += [(4, 4, 0.05, 0, 0, 1, 0, 0, 0)]                      # temporal tiles never grow runs
    points += [(4, 4, 0.05, 0, 0, 1, 1, 1, 0), (8, 8, 0.05, 0, 0, 1, 1, 1, 0)]   # Eq. 3's three-coefficient planes
    points += [(4, 4, 0.05, 0, 0, 1, 1, 0, 1), (8, 8, 0.05, 0, 0, 1, 1, 0, 1)]   # FP64 plane solver
    for th, tw, thr, nd, rx, tc, tr, p3, sv in points:
        if True:
            ctx = lcc.Context(seq.sensor, lcc.default_params(tile_h=th, tile_w=tw, fit_thr_m=thr, no_delta=nd,
                                                            raw_exact=rx, temporal_candidates=tc,
                                                            temporal_runs=tr, plane3=p3, solver=sv,
                                                            max_batch=max(16, n_frames)), stream=stream)
            cap = ctx.max_encoded_bytes
            outs = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(n_frames)]
            nb = torch.zeros(n_frames, dtype=torch.int64, device="cuda")
            kf = lcc.Keyframe(ctx)

            def step():
                ctx.lcc_encode_sequence(seq.key_index, seq.poses, d_pts, n, outs, [cap] * n_frames, nb, kf)

            for _ in range(3):
                step()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            torch.cuda.synchronize()
            for k in range(steps):
                flush.zero_()
                evs[k][0].record(stream)
                step()
                evs[k][1].record(stream)
            torch.cuda.synchronize()
            assert ctx.lcc_sync() == lcc.OK
            ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
            sizes = nb.cpu().numpy()
            modes = {"raw": 0, "run": 0, "temporal": 0}
            for f in range(n_frames):
                st_f = ctx.lcc_last_stats(f)
                modes["raw"] += st_f["tiles_raw"]
                modes["run"] += st_f["tiles_run_start"] + st_f["tiles_run_cont"]
                modes["temporal"] += st_f["tiles_temporal"] + st_f["tiles_temporal_cont"]
            ref = torch.empty(H * W, dtype=torch.float32, device="cuda")
            dec = torch.empty(H * W, dtype=torch.float32, device="cuda")
            kfd = lcc.Keyframe(ctx)
            ctx.lcc_keyframe_from_stream(outs[seq.key_index], int(sizes[seq.key_index]), kfd)
            err = 0.0
            for f in range(n_frames):
                ctx.lcc_range_image(d_pts[f], n[f], ref, None)
                isk = f == seq.key_index
                ctx.lcc_decode(outs[f], int(sizes[f]), None if isk else kfd, None if isk else seq.poses[f], dec,
                               None, None)
                assert ctx.lcc_sync() == lcc.OK
                m = ref > 0
                if bool(m.any()):
                    err = max(err, float((dec[m] - ref[m]).abs().max().item()))
            rows.append({"tile": f"{th}x{tw}", "thr_m": thr, "no_delta": nd, "raw_exact": rx,
                         "temporal_candidates": tc, "temporal_runs": tr, "plane3": p3,
                         "solver": "fp64" if sv else "float-float",
                         "bytes": int(sizes.sum()), "mpts_per_s": round(pts / (ms * 1e-3) / 1e6, 1),
                         "ms_per_step": round(ms, 4), "compression_ratio": round(12.0 * pts / float(sizes.sum()), 3),
                         "max_decode_error_m": err, "tile_modes": modes})
            del kf, kfd, ctx
    return {"workload": WORKLOAD.split(",")[0] + ", swept tiles and thresholds, q 0.02 m", "steps": steps,
            "rows": rows}


def run_entropy(args, stream, ctx, d_out, sizes, pts_step, flush, hbm):
    """The lossless entropy stage (Sec. III-A) on the step's 10 fixed-width streams: one
    lcc_entropy_encode call and one lcc_entropy_decode call, each timed with CUDA events (L2
    flushed between steps); sizes per section; the round trip checked byte for byte."""
    import torch
    from paper_2008_06972_gb300 import lcc
    n = len(d_out)
    cap = ctx.max_encoded_bytes + 4096
    ent = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(n)]
    enb = torch.zeros(n, dtype=torch.int64, device="cuda")
    back = [torch.zeros(ctx.max_encoded_bytes, dtype=torch.uint8, device="cuda") for _ in range(n)]
    bnb = torch.zeros(n, dtype=torch.int64, device="cuda")
    in_size = [o.numel() for o in d_out]

    def enc():
        ctx.lcc_entropy_encode(d_out, in_size, ent, [cap] * n, enb)

    enc()
    assert ctx.lcc_sync() == lcc.OK
    ent_sizes = [int(x) for x in enb.cpu().numpy()]

    def dec():
        ctx.lcc_entropy_decode(ent, ent_sizes, back, [b.numel() for b in back], bnb)

    def timed(fn):
        for _ in range(3):
            fn()
        assert ctx.lcc_sync() == lcc.OK
        k_steps = max(5, min(args.steps, 50))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_steps)]
        for k in range(k_steps):
            flush.zero_()
            evs[k][0].record(stream)
            fn()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        assert ctx.lcc_sync() == lcc.OK
        return float(np.mean([a.elapsed_time(b) for a, b in evs])), k_steps

    enc_ms, k_steps = timed(enc)
    dec_ms, _ = timed(dec)
    assert [int(x) for x in bnb.cpu().numpy()] == list(sizes)
    for f in range(n):
        assert torch.equal(back[f][:sizes[f]], d_out[f][:sizes[f]]), f"frame {f}: entropy round trip differs"
    ctx.lcc_set_profiling(True)
    enc()
    dec()
    kt = ctx.lcc_kernel_times()
    ctx.lcc_set_profiling(False)
    names = ("bitmap", "tiles", "runs", "temporal", "fitted", "res", "raw")
    fixed_w = {k: 0 for k in names}
    ent_w = {k: 0 for k in names}
    coded = {k: 0 for k in names}
    for f in range(n):
        h = ent[f][:184].cpu().numpy().view("<u4")
        fx = d_out[f][:64].cpu().numpy().view("<u4")
        for s_, k in enumerate(names):
            mode, count, alph, words = (int(x) for x in h[18 + 4 * s_:22 + 4 * s_])
            ent_w[k] += words
            coded[k] += mode & 1
        # fixed-width section sizes from the fixed header
        rows, cols = int(fx[2] & 0xFFFF), int(fx[2] >> 16)
        w_res, w_raw, flags = int((fx[3] >> 16) & 0xFF), int(fx[3] >> 24), int(fx[1] >> 24)
        nt, nr, ntm, nc, nf, nraw = (int(fx[i]) for i in (6, 8, 9, 10, 11, 12))
        wd = lambda b: (b + 31) // 32
        for k, v in zip(names, (wd(rows * cols), wd(4 * nt), 4 * nr, 2 * ntm, wd(nc),
                                0 if flags & 2 else wd(nf * w_res), wd(nraw * w_raw))):
            fixed_w[k] += v
    fixed_bytes, ent_bytes = int(sum(sizes)), int(sum(ent_sizes))
    alg = fixed_bytes + ent_bytes
    return {"workload": "the step's 10 fixed-width streams through one lcc_entropy_encode and one "
                        "lcc_entropy_decode call (canonical Huffman per section, 1024-symbol chunks)",
            "steps": k_steps, "fixed_bytes": fixed_bytes, "entropy_bytes": ent_bytes,
            "compression_ratio_fixed": 12.0 * pts_step / fixed_bytes,
            "compression_ratio_entropy": 12.0 * pts_step / ent_bytes,
            "encode_ms": enc_ms, "encode_mpts_per_s": pts_step / (enc_ms * 1e-3) / 1e6,
            "decode_ms": dec_ms, "decode_mpts_per_s": pts_step / (dec_ms * 1e-3) / 1e6,
            "encode_hbm_frac": alg / (enc_ms * 1e-3) / 1e9 / hbm,
            "kernel_ms": {k: v[1] for k, v in kt.items()},
            "section_bytes": {k: {"fixed": 4 * fixed_w[k], "entropy": 4 * ent_w[k], "frames_coded": coded[k]}
                              for k in names}}


IMU_LEVELS = (
    # name, acc white sigma (m/s^2), gyro white sigma (deg/s), acc bias (m/s^2), gyro bias (deg/s)
    ("ideal", 0.0, 0.0, 0.0, 0.0),
    ("navigation grade", 0.01, 0.005, 0.002, 0.001),
    ("automotive MEMS", 0.05, 0.05, 0.02, 0.05),
    ("low-cost MEMS", 0.2, 0.3, 0.1, 0.5),
)


def run_imu(args, stream, flush):
    """Frame poses from IMU samples (Sec. III-D): the HDL-64E scene driven on a 10 m/s, 5 deg/s arc,
    10 frames at 10 Hz, key frame the middle one; 100 Hz samples (clock offset from the frames) at
    four noise levels, integrated by lcc_imu_pose into every P frame's pose, then the sequence encoded
    and decoded with those poses.  Rows: pose error against the exact arc, temporal tiles, bytes,
    device time of the encode and the max decode error."""
    import torch
    import synth
    from paper_2008_06972_gb300 import lcc
    seq = synth.sequence_arc(0, 10)
    n_frames = len(seq.frames)
    n = [len(f) for f in seq.frames]
    pts = sum(n)
    H, W = seq.sensor.rows, seq.sensor.cols
    t_key = seq.key_index * synth.FRAME_DT
    d_pts = [torch.from_numpy(f).cuda() for f in seq.frames]
    ctx = lcc.Context(seq.sensor, lcc.default_params(max_batch=max(16, n_frames)), stream=stream)
    cap = ctx.max_encoded_bytes
    outs = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(n_frames)]
    nb = torch.zeros(n_frames, dtype=torch.int64, device="cuda")
    kf = lcc.Keyframe(ctx)
    kfd = lcc.Keyframe(ctx)
    ref = torch.empty(H * W, dtype=torch.float32, device="cuda")
    dec = torch.empty(H * W, dtype=torch.float32, device="cuda")
    steps = max(5, min(args.steps, 30))
    rows = []
    for name, sa, sg, ba, bg in (("exact",) + IMU_LEVELS[0][1:],) + IMU_LEVELS:
        if name == "exact":
            poses, pose_us = seq.poses, 0.0
        else:
            smp = synth.imu_samples(0.0, (n_frames - 1) * synth.FRAME_DT, 10.0, math.radians(5.0), t_key,
                                    acc_sigma=sa, gyro_sigma=math.radians(sg), acc_bias=(ba, -ba, ba),
                                    gyro_bias=(math.radians(bg),) * 3, seed=17)
            t0 = time.perf_counter()
            poses = np.stack([lcc.imu_pose(smp.t, smp.acc, smp.gyro, smp.v_key, t_key, f * synth.FRAME_DT)
                              for f in range(n_frames)])
            pose_us = (time.perf_counter() - t0) / n_frames * 1e6
        et = max(float(np.abs(poses[f][:3, 3] - seq.poses[f][:3, 3]).max()) for f in range(n_frames))
        er = max(math.degrees(math.acos(min(1.0, (np.trace(poses[f][:3, :3].T @ seq.poses[f][:3, :3]) - 1) / 2)))
                 for f in range(n_frames))

        def step():
            ctx.lcc_encode_sequence(seq.key_index, poses, d_pts, n, outs, [cap] * n_frames, nb, kf)

        for _ in range(3):
            step()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        assert ctx.lcc_sync() == lcc.OK
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        sizes = nb.cpu().numpy()
        temporal = sum(ctx.lcc_last_stats(f)["tiles_temporal"] for f in range(n_frames))
        ctx.lcc_keyframe_from_stream(outs[seq.key_index], int(sizes[seq.key_index]), kfd)
        err = 0.0
        for f in range(n_frames):
            ctx.lcc_range_image(d_pts[f], n[f], ref, None)
            isk = f == seq.key_index
            ctx.lcc_decode(outs[f], int(sizes[f]), None if isk else kfd, None if isk else poses[f], dec, None, None)
            assert ctx.lcc_sync() == lcc.OK
            m = ref > 0
            if bool(m.any()):
                err = max(err, float((dec[m] - ref[m]).abs().max().item()))
        assert err <= 0.02, err
        rows.append({"poses": name, "acc_sigma": sa, "gyro_sigma_dps": sg, "acc_bias": ba, "gyro_bias_dps": bg,
                     "max_pose_err_m": et, "max_pose_err_deg": er, "pose_us_per_frame": round(pose_us, 2),
                     "tiles_temporal": temporal, "bytes": int(sizes.sum()),
                     "compression_ratio": round(12.0 * pts / float(sizes.sum()), 3),
                     "ms_per_step": round(ms, 4), "mpts_per_s": round(pts / (ms * 1e-3) / 1e6, 1),
                     "max_decode_error_m": err})
    del kf, kfd, ctx
    return {"workload": "64x2048 HDL-64E-shaped frames, 10 per sequence on a 10 m/s, 5 deg/s arc, "
                        "4x4 tiles, thr 0.05 m, q 0.02 m; 100 Hz IMU samples", "steps": steps, "rows": rows}


def run_learned(args, stream):
    """Learned tile proposal on 64x2048 key frames with 8x8 tiles: the net is trained on the GPU
    (its own forward/backward/Adam kernels) on tiles the plain encoder labels, then the seeded
    encode (net inputs + inference + seeded fit) is compared with the plain encode on held-out
    frames: time, fit rounds, bytes, max decode error."""
    import torch
    import synth
    from paper_2008_06972_gb300 import lcc
    from paper_2008_06972_gb300 import train as TR
    sensor = synth.HDL64_SENSOR

    import concurrent.futures as cf

    def seq_frames(i, n):
        return synth.sequence(sensor, n, synth.config_seed(4, i, 0), n_walls=20, n_boxes=40, n_poles=60,
                              step_m=1.0, yaw_deg=0.5, sigma=0.02, clutter=0.02).frames

    def frames(ids, n, pool):
        return [f for fr in pool.map(lambda i: seq_frames(i, n), ids) for f in fr]

    # training data: sequences of 8 frames (seeds of sequences 0.., disjoint from the evaluation's
    # 1000..), rendered in parallel threads chunk by chunk; only the BF16 tile inputs and the labels
    # of the plain GPU encoder stay (on the device)
    ctx = lcc.Context(sensor, lcc.default_params(tile_h=8, tile_w=8, fit_thr_m=0.05), stream=stream)
    n_train_seq = max(1, args.train_frames // 8)
    X, Y = [], []
    gen_s = label_s = 0.0
    with cf.ThreadPoolExecutor(min(32, os.cpu_count() or 4)) as pool:
        for a in range(0, n_train_seq, 32):
            t0 = time.perf_counter()
            chunk = frames(range(a, min(a + 32, n_train_seq)), 8, pool)
            gen_s += time.perf_counter() - t0
            t0 = time.perf_counter()
            for f in chunk:
                x, _, y, _ = TR.frame_examples(ctx, torch.from_numpy(f).cuda(), len(f))
                X.append(x)
                Y.append(y)
            label_s += time.perf_counter() - t0
        t0 = time.perf_counter()
        eval_f = frames(range(1000, 1002), 8, pool)
        gen_s += time.perf_counter() - t0
    train_f_count = 8 * n_train_seq
    X, Y = torch.cat(X), torch.cat(Y)
    batch = 4096
    net = lcc.Net(TR.he_uniform_params(4), max_tiles=batch, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    train_steps = args.train_steps if args.train_steps > 0 else max(300, int(X.shape[0]) // batch)   # one epoch
    losses = TR.train(net, X, Y, train_steps, batch, 2e-3, seed=1, lr_final=2e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    nt = ctx.num_tiles
    xin = torch.zeros((nt, 64, 4), dtype=torch.int16, device="cuda")
    anc = torch.zeros((nt, 4), dtype=torch.float32, device="cuda")
    prop = torch.zeros((nt, 5), dtype=torch.float32, device="cuda")
    out = torch.empty(ctx.max_encoded_bytes, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    ref = torch.empty(sensor.rows * sensor.cols, dtype=torch.float32, device="cuda")
    dec = torch.empty_like(ref)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    stats = {"plain": dict(ms=0.0, bytes=0, rounds=0, fitted_tiles=0, err=0.0),
             "learned": dict(ms=0.0, net_ms=0.0, bytes=0, rounds=0, fitted_tiles=0, skipped=0, err=0.0)}
    pts_total = 0
    for rep in range(2):      # the first pass warms up; the second is measured
        for f in eval_f:
            d = torch.from_numpy(f).cuda()
            torch.cuda.synchronize()
            ev[0].record(stream)
            ctx.lcc_encode_keyframe(d, len(f), None, out, out.numel(), nb)
            ev[1].record(stream)
            assert ctx.lcc_sync() == lcc.OK
            recs = ctx.lcc_tile_records(0)
            nbytes = int(nb.item())
            ctx.lcc_range_image(d, len(f), ref, None)
            ctx.lcc_decode(out, nbytes, None, None, dec, None, None)
            assert ctx.lcc_sync() == lcc.OK
            m = ref > 0
            err_p = float((dec[m] - ref[m]).abs().max().item())
            torch.cuda.synchronize()
            ev[0].record(stream)
            lcc.net_tile_inputs(ctx, d, len(f), xin, anc)
            net.forward(xin, nt, prop)
            ev[2].record(stream)
            ctx.lcc_encode_keyframe_seeded(d, len(f), prop, TR.SKIP_LOGIT, None, out, out.numel(), nb)
            ev[3].record(stream)
            assert ctx.lcc_sync() == lcc.OK
            srecs = ctx.lcc_tile_records(0)
            sbytes = int(nb.item())
            ctx.lcc_range_image(d, len(f), ref, None)
            ctx.lcc_decode(out, sbytes, None, None, dec, None, None)
            assert ctx.lcc_sync() == lcc.OK
            err_l = float((dec[m] - ref[m]).abs().max().item())
            if rep == 0:
                continue
            pts_total += len(f)
            P, L = stats["plain"], stats["learned"]
            P["bytes"] += nbytes
            P["rounds"] += int(recs["rounds"].sum())
            P["fitted_tiles"] += int((recs["status"] == lcc.S_FIT).sum())
            P["err"] = max(P["err"], err_p)
            L["net_ms"] += ev[0].elapsed_time(ev[2])
            L["ms"] += ev[0].elapsed_time(ev[3])
            L["bytes"] += sbytes
            L["rounds"] += int(srecs["rounds"].sum())
            L["fitted_tiles"] += int((srecs["status"] == lcc.S_FIT).sum())
            L["skipped"] += int(((srecs["flags"] & 8) != 0).sum())
            L["err"] = max(L["err"], err_l)
    # the plain encode timed on its own (same frames, same warm-up)
    plain_ms = 0.0
    for rep in range(2):
        for f in eval_f:
            d = torch.from_numpy(f).cuda()
            torch.cuda.synchronize()
            ev[0].record(stream)
            ctx.lcc_encode_keyframe(d, len(f), None, out, out.numel(), nb)
            ev[1].record(stream)
            torch.cuda.synchronize()
            if rep:
                plain_ms += ev[0].elapsed_time(ev[1])
    stats["plain"]["ms"] = plain_ms
    for k in stats:
        stats[k]["mpts_per_s"] = pts_total / (stats[k]["ms"] * 1e-3) / 1e6
        stats[k]["ms_per_frame"] = stats[k]["ms"] / len(eval_f)
    # the same 16 frames in one batched call each: plain, and learned (inputs + one inference
    # over all frames' tiles + the seeded batched encode)
    nf = len(eval_f)
    d_eval = [torch.from_numpy(f).cuda() for f in eval_f]
    n_eval = [len(f) for f in eval_f]
    outs = [torch.empty(ctx.max_encoded_bytes, dtype=torch.uint8, device="cuda") for _ in range(nf)]
    caps = [o.numel() for o in outs]
    nbs = torch.zeros(nf, dtype=torch.int64, device="cuda")
    xall = torch.zeros((nf * nt, 64, 4), dtype=torch.int16, device="cuda")
    aall = torch.zeros((nf * nt, 4), dtype=torch.float32, device="cuda")
    pall = torch.zeros((nf * nt, 5), dtype=torch.float32, device="cuda")
    props = [pall[i * nt:(i + 1) * nt] for i in range(nf)]

    def batched_plain():
        ctx.lcc_encode_keyframes(d_eval, n_eval, None, 0.0, outs, caps, nbs)

    def batched_learned():
        lcc.net_tile_inputs_batch(ctx, d_eval, n_eval, xall, aall)
        net.forward(xall, nf * nt, pall)
        ctx.lcc_encode_keyframes(d_eval, n_eval, props, TR.SKIP_LOGIT, outs, caps, nbs)

    batched = {}
    for name, fn in (("plain", batched_plain), ("learned", batched_learned)):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev[0].record(stream)
        for _ in range(5):
            fn()
        ev[1].record(stream)
        assert ctx.lcc_sync() == lcc.OK
        ms = ev[0].elapsed_time(ev[1]) / 5
        rounds = sum(int(ctx.lcc_tile_records(i)["rounds"].sum()) for i in range(nf))
        batched[name] = {"ms": ms, "mpts_per_s": sum(n_eval) / (ms * 1e-3) / 1e6,
                         "bytes": int(nbs.sum().item()), "rounds": rounds}
    # inference throughput of the net alone (tcgen05 kernel) on all training tiles at once
    big = X.shape[0]
    pbig = torch.zeros((big, 5), dtype=torch.float32, device="cuda")
    for _ in range(3):
        net.forward(X, big, pbig)
    torch.cuda.synchronize()
    reps = 10
    ev[0].record(stream)
    for _ in range(reps):
        net.forward(X, big, pbig)
    ev[1].record(stream)
    assert net.sync() == lcc.OK
    inf_ms = ev[0].elapsed_time(ev[1]) / reps
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16_peak, bf16_src = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        bf16_peak, bf16_src = 1900.0, "fallback"
    inference = {"tiles": big, "ms": inf_ms, "tflops": 7.2e6 * big / (inf_ms * 1e-3) / 1e12,
                 "peak_tflops": bf16_peak, "peak_source": bf16_src,
                 "frac": 7.2e6 * big / (inf_ms * 1e-3) / 1e12 / bf16_peak, "kernel": "k_net_fwd_tc (tcgen05)"}
    return {
        "workload": "HDL-64E key frames 64x2048, tiles 8x8, thr 0.05 m; net trained on "
                    f"{train_f_count} frames ({X.shape[0]} tiles) of the same scene family, evaluated on "
                    f"{len(eval_f)} held-out frames",
        "train": {"frames": train_f_count, "tiles": int(X.shape[0]), "steps": train_steps, "batch_tiles": batch,
                  "seconds": train_s, "loss_first": float(losses[0]), "loss_last": float(np.mean(losses[-10:])),
                  "tflops": 3 * 7.2e6 * batch * train_steps / train_s / 1e12},
        "net_flops_per_tile": 7.2e6,
        "inference": inference,
        "plain": stats["plain"], "learned": stats["learned"],
        "batched_16_frames": batched,
        "rounds_saved_frac": 1.0 - stats["learned"]["rounds"] / max(stats["plain"]["rounds"], 1),
        "bytes_ratio_learned_vs_plain": stats["learned"]["bytes"] / max(stats["plain"]["bytes"], 1),
        "setup_s": {"generate": gen_s, "label": label_s},
    }


# Algorithmic bytes (or FLOPs) of each kernel per unit, the figures the roofline uses:
#   bin:        20 B per input point (16 B float4 read + 4 B atomic into the range image)
#   fit:        4 B per pixel (range image) + 64 B per tile record written
#   rounds:     128 B per queued tile (its record read and written) + 4 B per pixel per further round
#   lookbehind: 4 B per pixel + 96 B per tile (record read, look-behind counts written)
#   temporal:   (P frames) 4 B per pixel + 128 B per tile (record read and written)
#   merge:      128 B per tile (record read, code and offsets written) + the stream bytes zeroed
#   pack:       8 B per pixel (range read and reset) + the stream bytes written
#   net_inputs: (seeded key frames) 4 B per pixel read + 8 B per pixel of BF16 input + 16 B anchor per tile
#   net_fwd:    7.2 MFLOP per 8x8 tile on the tensor cores
NET_FLOPS_PER_TILE = 7.2e6


def kernel_units(st: dict, frames: int, p_frames: int, key_seeded: int, npx: int, nt: int, tpx: int) -> dict:
    """Per-kernel algorithmic bytes of one encode of `frames` frames from its statistics."""
    hist = st["fit_rounds"]
    queued = sum(hist[r] for r in range(2, 8))
    extra = sum((r - 1) * hist[r] for r in range(2, 8))
    return {
        "bin": 20.0 * st["points_in"],
        "fit": frames * (4.0 * npx + 64.0 * nt),
        "rounds": 128.0 * queued + 4.0 * tpx * extra,
        "lookbehind": frames * (4.0 * npx + 96.0 * nt),
        "temporal": p_frames * (4.0 * npx + 128.0 * nt),
        "merge": frames * 128.0 * nt + st["bytes"],
        "pack": frames * 8.0 * npx + st["bytes"],
        "net_inputs": key_seeded * (12.0 * npx + 16.0 * nt),
        # the net runs on pairs of tiles that hold a tile with the 3 valid pixels a fit needs; the
        # work counted is those tiles' alone (st["tiles_net"]), not their pair partners'
        "net_fwd": st.get("tiles_net", key_seeded * nt) * NET_FLOPS_PER_TILE,
    }


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops_sustained"]), "measured (sustained)"
    except Exception:
        return 1700.0, "fallback (sustained)"


def run_cfg5(args, stream, rank, world, dist):
    """The headline: the large batched workload encoded by one plan with the learned proposal
    (value) and by the plain plan on the same inputs, plus e2e, roofline and the CPU baseline."""
    import concurrent.futures as cf
    import torch
    import synth
    from paper_2008_06972_gb300 import lcc
    from paper_2008_06972_gb300 import multi
    from paper_2008_06972_gb300 import train as TR
    S = synth.CFG5_SENSOR
    npx = S.rows * S.cols
    nseq, nfr, ki = args.cfg5_seqs, args.cfg5_frames, synth.CFG5_KEY_INTERVAL
    nf = nseq * nfr
    setup = {}
    # the inputs in page-locked host memory (the end-to-end plan reads them in place over the host
    # link), rendered straight into it, then one copy into HBM for the device-resident steps
    t0 = time.perf_counter()
    hostt = torch.empty((nf, npx, 4), dtype=torch.float32, pin_memory=True)
    setup["pin_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    host = hostt.numpy()
    seqs = synth.batch_cfg5(host, n_seq=nseq, n_frames=nfr, first=rank * nseq)
    setup["generate_s"] = time.perf_counter() - t0
    npts = [[len(f) for f in q.frames] for q in seqs]
    total_pts = sum(sum(n) for n in npts)
    t0 = time.perf_counter()
    dev = torch.empty((nf, npx, 4), dtype=torch.float32, device="cuda")
    for a in range(0, nf, 64):
        dev[a:a + 64].copy_(hostt[a:a + 64], non_blocking=True)
    torch.cuda.synchronize()
    setup["to_device_s"] = time.perf_counter() - t0

    def pts_dev(i, f):
        return dev[i * nfr + f].data_ptr()

    # ---- the proposal net: trained on the GPU on frames of other sequences of the same family ----
    t0 = time.perf_counter()
    ctx_tr = lcc.Context(S, lcc.default_params(tile_h=8, tile_w=8, fit_thr_m=args.thr), stream=stream)
    per_seq = 8
    tr_ids = [100000 + rank * 1000 + i for i in range(max(1, args.cfg5_train_frames // per_seq))]
    with cf.ThreadPoolExecutor(min(32, os.cpu_count() or 4)) as pool:
        tr_seqs = list(pool.map(lambda sid: synth.sequence_cfg5_grouped(sid, n_frames=per_seq), tr_ids))
    X, Y = [], []
    for q in tr_seqs:
        for f in q.frames:
            x, _, y, _ = TR.frame_examples(ctx_tr, torch.from_numpy(f).cuda(), len(f))
            X.append(x)
            Y.append(y)
    X, Y = torch.cat(X), torch.cat(Y)
    setup["train_data_s"] = time.perf_counter() - t0
    batch = 4096
    net = lcc.Net(TR.he_uniform_params(4), max_tiles=batch, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = TR.train(net, X, Y, args.cfg5_train_steps, batch, 2e-3, seed=1, lr_final=2e-4)
    torch.cuda.synchronize()
    train = {"frames": len(tr_ids) * per_seq, "tiles": int(X.shape[0]), "steps": args.cfg5_train_steps,
             "batch_tiles": batch, "seconds": time.perf_counter() - t0, "loss_first": float(losses[0]),
             "loss_last": float(np.mean(losses[-10:]))}
    assert net.sync() == lcc.OK
    del X, Y

    # ---- autotune: the plain plan over every tile shape, the learned plan among 8x8 ----
    t0 = time.perf_counter()
    k0 = synth.group_key(0, nfr, ki)
    m0 = min(ki, nfr)
    samp = [pts_dev(0, f) for f in range(m0)]
    tuned = {}
    for name, shapes in (("plain", None), ("learned", [(8, 8)]), ("plain_8x8", [(8, 8)])):
        best, rows = lcc.autotune(S, lcc.default_params(max_batch=64, fit_thr_m=args.thr), k0, seqs[0].poses[:m0],
                                  samp, npts[0][:m0], reps=3, stream=stream, shapes=shapes)
        ch = next(r for r in rows if r["chosen"])
        tuned[name] = (best, {"tile": f"{ch['tile_h']}x{ch['tile_w']}", "lookahead": ch["lookahead"],
                              "fit_schedule": ch["fit_schedule"], "sample_mpts_s": round(ch["mpts_per_s"], 1),
                              "candidates": len(rows)})
    setup["autotune_s"] = time.perf_counter() - t0

    cap = (max(lcc.Context(S, tuned[k][0], stream=stream).max_encoded_bytes for k in tuned) + 255) // 256 * 256
    outs = {k: torch.empty((nf, cap), dtype=torch.uint8, device="cuda") for k in tuned}
    nbytes = {k: torch.zeros(nf, dtype=torch.int64, device="cuda") for k in tuned}

    # sequence i goes to context i % lanes: with two lanes the plan runs two classes of the same
    # parameters on two side streams, so one lane's binning (over the host link on the e2e path)
    # overlaps the other lane's fits, merges and packs
    def descs(kind, pts_of, lanes=1):
        return [dict(ctx=i % lanes, key_interval=ki, poses=q.poses, d_pts=[pts_of(i, f) for f in range(nfr)],
                     n=npts[i], d_out=[outs[kind][i * nfr + f].data_ptr() for f in range(nfr)], cap=[cap] * nfr,
                     d_nbytes=nbytes[kind][i * nfr:(i + 1) * nfr]) for i, q in enumerate(seqs)]

    def build_plan(kind, frames_per_launch, lookahead=None, lanes=1, pts_of=pts_dev, capture=True):
        prm = lcc.lcc_params.from_buffer_copy(tuned[kind][0])
        prm.max_batch = frames_per_launch
        if lookahead is not None:
            prm.lookahead = lookahead
        cl = [lcc.Context(S, prm, stream=stream) for _ in range(lanes)]
        plan = lcc.Plan(cl, descs(kind, pts_of, lanes))
        if kind == "learned":
            plan.set_proposals(net, TR.SKIP_LOGIT)
        if capture:
            plan.capture()
        return cl, plan

    # frames per launch (the plan's chunk size), run-test horizon and lanes, on the whole table: the
    # autotuner timed one key-frame group with the per-group calls, while a plan's launches hold up
    # to 64 frames, so the speed knobs are settled here (none changes a stream byte): one timed
    # replay at 16, 32 and 64 frames per launch and horizons 16 and 32 on one lane, and at 32 and 64
    # on two, the fastest kept
    t0 = time.perf_counter()
    ctxs, plans = {}, {}
    for kind in tuned:
        rows = {}
        best = None
        for fpl, la, ln in [(f, h, 1) for f in (16, 32, 64) for h in (16, 32)] + \
                [(f, h, 2) for f in (32, 64) for h in (16, 32)]:
            ctx, plan = build_plan(kind, fpl, la, ln)
            plan.replay()
            assert plan.sync() == lcc.OK
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.replay()
            b.record(stream)
            assert plan.sync() == lcc.OK
            ms = a.elapsed_time(b)
            rows[f"{fpl}/{la}/{ln}"] = round(total_pts / (ms * 1e-3) / 1e6, 1)
            if best is None or ms < best[0]:
                if best is not None:
                    best[3].close()
                best = (ms, (fpl, la, ln), ctx, plan)
            else:
                plan.close()
        # the queued rounds on a thread per tile (schedule 6) at the chosen knobs: the autotuner's
        # one-group sample has too few queued tiles to tell it from schedule 4
        if tuned[kind][0].fit_schedule == 4:
            tuned[kind][0].fit_schedule = 6
            ctx, plan = build_plan(kind, *best[1])
            plan.replay()
            assert plan.sync() == lcc.OK
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            plan.replay()
            b.record(stream)
            assert plan.sync() == lcc.OK
            ms = a.elapsed_time(b)
            rows[f"{best[1][0]}/{best[1][1]}/{best[1][2]}/schedule6"] = round(total_pts / (ms * 1e-3) / 1e6, 1)
            if ms < best[0]:
                best[3].close()
                best = (ms, best[1], ctx, plan)
            else:
                plan.close()
                tuned[kind][0].fit_schedule = 4
        ctxs[kind], plans[kind] = best[2], best[3]
        tuned[kind][1]["fit_schedule"] = tuned[kind][0].fit_schedule
        tuned[kind][1]["frames_per_launch"] = best[1][0]
        tuned[kind][1]["lookahead"] = best[1][1]
        tuned[kind][1]["lanes"] = best[1][2]
        tuned[kind][1]["frames_per_launch_mpts_s"] = rows   # keys: frames per launch / horizon / lanes
    setup["frames_per_launch_s"] = time.perf_counter() - t0
    for k in plans:
        for _ in range(max(args.warmup, 3)):
            plans[k].replay()
        st = plans[k].sync()
        assert st == lcc.OK, lcc.status_string(st)

    def timed(plan, steps, clocks=None):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        if clocks:
            clocks.__enter__()
        try:
            for k in range(steps):
                evs[k][0].record(stream)
                plan.replay()
                evs[k][1].record(stream)
            torch.cuda.synchronize()
        finally:
            if clocks:
                clocks.__exit__()
        t_wall = time.perf_counter() - t_wall
        if dist:
            dist.barrier()
        st = plan.sync()
        assert st == lcc.OK, lcc.status_string(st)
        return float(np.mean([a.elapsed_time(b) for a, b in evs])), t_wall

    # ---- timed region: K replays of the learned plan (the headline), then the plain plan ----
    clocks = Clocks(args.clocks_csv.replace("{rank}", str(rank)) if args.clocks_csv
                    else f"/tmp/lcc_clocks_{os.getpid()}_rank{rank}.csv")
    ms_l, wall_l = timed(plans["learned"], args.steps, clocks)
    value, sec_step, _ = multi.job_value(total_pts, ms_l * 1e-3, dist, "cuda")
    plain_steps = max(3, min(args.steps, 10))
    ms_p, _ = timed(plans["plain"], plain_steps)
    value_p, _, _ = multi.job_value(total_pts, ms_p * 1e-3, dist, "cuda")
    ms_p8, _ = timed(plans["plain_8x8"], plain_steps)
    value_p8, _, _ = multi.job_value(total_pts, ms_p8 * 1e-3, dist, "cuda")

    # ---- correctness of what was timed: every frame decoded, max error against its range image ----
    def check(kind):
        c = ctxs[kind][0]   # every lane's context has the same parameters
        nb = nbytes[kind].cpu().numpy()
        ref = torch.empty(npx, dtype=torch.float32, device="cuda")
        dec = [torch.empty(npx, dtype=torch.float32, device="cuda") for _ in range(ki)]
        err = torch.zeros((), dtype=torch.float32, device="cuda")
        bad = torch.zeros((), dtype=torch.int64, device="cuda")
        for i, q in enumerate(seqs):
            for g0 in range(0, nfr, ki):
                fr = list(range(g0, min(g0 + ki, nfr)))
                k = synth.group_key(g0, nfr, ki)
                c.lcc_decode_sequence(k - g0, q.poses[g0:g0 + len(fr)], [outs[kind][i * nfr + f] for f in fr],
                                      [int(nb[i * nfr + f]) for f in fr], dec[:len(fr)], None, None)
                for j, f in enumerate(fr):
                    c.lcc_range_image(pts_dev(i, f), npts[i][f], ref, None)
                    m = ref > 0
                    bad += ((dec[j] > 0) != m).sum()
                    err = torch.maximum(err, torch.where(m, (dec[j] - ref).abs(), 0.0).max())
        assert c.lcc_sync() == lcc.OK
        return float(err.item()), int(bad.item()), int(nb.sum())

    err_l, bad_l, bytes_l = check("learned")
    err_p, bad_p, bytes_p = check("plain")
    err_p8, bad_p8, bytes_p8 = check("plain_8x8")
    assert max(err_l, err_p, err_p8) <= 0.02 and bad_l == bad_p == bad_p8 == 0, (err_l, err_p, err_p8)

    # ---- per-kernel times: one eager encode of each plan with a CUDA event pair around every launch ----
    hbm, src = peaks()
    tpeak, tsrc = bf16_peak()
    kernels, stats, stats_info = {}, {}, {}
    for kind in ("learned", "plain", "plain_8x8"):
        # one lane, so that no other launch shares the GPU while a launch is timed
        (c,), pplan = build_plan(kind, tuned[kind][1]["frames_per_launch"], tuned[kind][1]["lookahead"], 1,
                                 capture=False)
        c.lcc_set_profiling(True)
        pplan.encode()
        assert pplan.sync() == lcc.OK
        kt = c.lcc_kernel_times()
        c.lcc_set_profiling(False)
        st = pplan.stats()
        pplan.close()
        info = plans[kind].info()
        stats_info[kind] = info
        p_ = tuned[kind][0]
        nt = c.num_tiles
        units = kernel_units(st, nf, nf - info["key_frames"], info["seeded_key_frames"], npx, nt,
                             p_.tile_h * p_.tile_w)
        tot = sum(v[1] for v in kt.values())
        rows = {}
        for name, (launches, ms_k) in kt.items():
            if launches == 0:
                continue
            per_launch = ms_k / launches
            if name == "net_fwd":
                ach = units[name] / launches / (per_launch * 1e-3) / 1e12
                rows[name] = {"launches": launches, "ms": ms_k, "share": ms_k / tot, "bound": "tensor",
                              "achieved": ach, "unit": "TFLOP/s", "frac": ach / tpeak,
                              "alg_per_launch": units[name] / launches}
            else:
                ach = units.get(name, 0.0) / launches / (per_launch * 1e-3) / 1e9
                rows[name] = {"launches": launches, "ms": ms_k, "share": ms_k / tot, "bound": "hbm",
                              "achieved": ach, "unit": "GB/s", "frac": ach / hbm,
                              "alg_per_launch": units.get(name, 0.0) / launches}
        kernels[kind] = rows
        stats[kind] = st
    dname = max(kernels["learned"].items(), key=lambda kv: kv[1]["ms"])[0]
    d = kernels["learned"][dname]
    # measured DRAM bytes per frame x the frames one launch of that kernel processed
    per_frame = measured_traffic_cfg5(dname)
    nfp = nf - stats_info["learned"]["key_frames"]
    frames_done = {"temporal": nfp, "lookbehind": nf + nfp}.get(dname, nf)
    traffic_per_launch = per_frame * frames_done / d["launches"] if per_frame is not None else None
    roof = {"bound": d["bound"], "kernel": dname, "achieved": d["achieved"],
            "peak": tpeak if d["bound"] == "tensor" else hbm, "unit": d["unit"], "frac": d["frac"],
            "traffic": traffic_per_launch, "alg_per_launch": d["alg_per_launch"],
            "peak_source": tsrc if d["bound"] == "tensor" else src,
            "path": {"alg_bytes_per_step": 16.0 * total_pts + bytes_l,
                     "achieved": (16.0 * total_pts + bytes_l) / (ms_l * 1e-3) / 1e9,
                     "frac": (16.0 * total_pts + bytes_l) / (ms_l * 1e-3) / 1e9 / hbm}}

    # ---- end to end through lcc_plan_encode_host: page-locked host points read in place, every
    #      stream copied into page-locked host buffers, sizes back: one host round trip per step ----
    h_out = torch.empty((nf, cap), dtype=torch.uint8, pin_memory=True)
    # the host link is the bound here, so this path's lanes and the way the points cross the link
    # (read in place by the binning kernels, or staged into device buffers by the copy engines one
    # chunk ahead) are chosen on their own: each combination timed alike, the fastest kept
    h_rows = [h_out[f] for f in range(nf)]
    e2e_steps = max(3, min(args.steps, 10))
    e2e_rows, e2e_best = {}, None
    for ln, stg in ((1, 0), (2, 0), (1, 1), (2, 1)):
        _, plan_e = build_plan("learned", tuned["learned"][1]["frames_per_launch"], tuned["learned"][1]["lookahead"],
                               ln, pts_of=lambda i, f: hostt[i * nfr + f].data_ptr())
        plan_e.set_staging(bool(stg))
        for _ in range(3):
            sizes = plan_e.encode_host(h_rows)
        assert np.array_equal(sizes.astype(np.int64), nbytes["learned"].cpu().numpy())
        if dist:
            dist.barrier()
        calls = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            sizes = plan_e.encode_host(h_rows)
            calls.append(time.perf_counter() - t0)
        e2e_s = float(np.mean(calls))   # the mean over the calls, stalls included
        plan_e.close()
        e2e_rows[f"{ln}/{'staged' if stg else 'in_place'}"] = round(total_pts / e2e_s / 1e6, 1)
        if e2e_best is None or e2e_s < e2e_best[0]:
            e2e_best = (e2e_s, ln, stg, calls)
    e2e_value, _, _ = multi.job_value(total_pts, e2e_best[0], dist, "cuda")

    info_l = plans["learned"].info()
    for k in plans:
        plans[k].close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, pts_c, sec_c, cores = oracle_cfg5(args.cpu_steps, args.thr)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_steps} frames per core of the same workload ({args.cpu_steps / 10:g} key-frame "
                         f"groups of 10 per core, key frame first: oracle net forward on every 8x8 tile + seeded "
                         f"fit; P frames plain), {pts_c / 1e6:.1f} M points in {sec_c:.1f} s of oracle time"}
        # the same sample on one core (the oracle's single-thread rate)
        v1, pts1, sec1, _ = oracle_cfg5(args.cpu_steps, args.thr, cores=1)
        cpu["single_core"] = {"value": v1, "unit": UNIT, "cores": 1,
                              "sample": f"{args.cpu_steps} frames, {pts1 / 1e6:.1f} M points in {sec1:.1f} s"}

    def summary(kind, ms, val, err, nbytes_):
        st = stats[kind]
        return {"value": val, "unit": UNIT, "ms_per_step": ms, "params": tuned[kind][1],
                "compression_ratio": 12.0 * total_pts / nbytes_, "bytes_per_step": nbytes_,
                "max_decode_error_m": err,
                "tile_modes": {"empty": st["tiles_empty"], "raw": st["tiles_raw"], "run_start": st["tiles_run_start"],
                               "run_cont": st["tiles_run_cont"], "temporal": st["tiles_temporal"],
                               "temporal_cont": st["tiles_temporal_cont"]},
                "fit_rounds_hist": st["fit_rounds"], "fit_rounds": sum(r * c for r, c in enumerate(st["fit_rounds"])),
                "tiles_borderline": st["tiles_borderline"],
                "hbm_path_frac": (16.0 * total_pts + nbytes_) / (ms * 1e-3) / 1e9 / hbm,
                "kernels": kernels[kind]}

    learned = summary("learned", ms_l, value, err_l, bytes_l)
    plain = summary("plain", ms_p, value_p, err_p, bytes_p)
    plain8 = summary("plain_8x8", ms_p8, value_p8, err_p8, bytes_p8)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sec_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**cfg5_config(args), "points_per_step": total_pts, "frames": nf,
                   "key_frames": info_l["key_frames"], "seeded_key_frames": info_l["seeded_key_frames"],
                   "parallelism": f"replicas x{world}", "tile": tuned["learned"][1]["tile"]},
        "max_decode_error_m": max(err_l, err_p),
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(16 * total_pts),
                "d2h_bytes_per_step": int(bytes_l + 8 * nf), "steps": e2e_steps,
                "lanes": e2e_best[1], "points": "staged" if e2e_best[2] else "in_place",
                "mpts_s_by_lanes_and_points": e2e_rows,
                "call_ms": {"mean": 1e3 * float(np.mean(e2e_best[3])), "median": 1e3 * float(np.median(e2e_best[3])),
                            "min": 1e3 * float(np.min(e2e_best[3])), "max": 1e3 * float(np.max(e2e_best[3]))},
                "how": "lcc_plan_encode_host: page-locked host points either read in place by the binning "
                       "kernels or copied by the copy engines (lcc_plan_set_staging) into device buffers one "
                       "chunk ahead of their binning; streams copied to page-locked host buffers by one kernel, "
                       "sizes back; with two lanes the sequences alternate between two contexts of the same "
                       "parameters, whose classes run on two streams"},
        "gpu_launches": int(info_l["launches"] * args.steps),
        "graph_nodes": info_l["graph_nodes"],
        "clocks": clocks.summary(),
        "wall_s_timed": wall_l,
        "learned_vs_plain": {"throughput_ratio": value / value_p, "bytes_ratio": bytes_l / bytes_p,
                             "fit_rounds_saved_frac": 1.0 - learned["fit_rounds"] / max(plain["fit_rounds"], 1),
                             "same_tiles": {"throughput_ratio": value / value_p8, "bytes_ratio": bytes_l / bytes_p8,
                                            "fit_rounds_saved_frac":
                                                1.0 - learned["fit_rounds"] / max(plain8["fit_rounds"], 1)}},
        "batched_learned": learned,
        "batched_plain": plain,
        "batched_plain_same_tiles": plain8,
        "net_training": train,
        "setup_s": setup,
    }


def run_profile_plan(args, stream):
    """A fixed-parameter plan over a subsample of the headline workload, encoded eagerly --steps
    times after one warm-up encode: the case the ncu summaries under profiles/ are taken on."""
    import torch
    import synth
    from paper_2008_06972_gb300 import lcc
    S = synth.CFG5_SENSOR
    npx = S.rows * S.cols
    nseq, nfr = args.cfg5_seqs, args.cfg5_frames
    host = np.empty((nseq * nfr, npx, 4), np.float32)
    seqs = synth.batch_cfg5(host, n_seq=nseq, n_frames=nfr)
    dev = torch.from_numpy(host).cuda()
    th, tw = (int(x) for x in args.tile.split("x"))
    prm = lcc.default_params(tile_h=th, tile_w=tw, fit_thr_m=args.thr, max_batch=args.max_batch,
                             lookahead=args.lookahead, fit_schedule=args.schedule,
                             solver=0 if args.solver == "ff" else 1)
    ctx = lcc.Context(S, prm, stream=stream)
    cap = (ctx.max_encoded_bytes + 255) // 256 * 256
    outs = torch.empty((nseq * nfr, cap), dtype=torch.uint8, device="cuda")
    nb = torch.zeros(nseq * nfr, dtype=torch.int64, device="cuda")
    descs = [dict(ctx=0, key_interval=synth.CFG5_KEY_INTERVAL, poses=q.poses,
                  d_pts=[dev[i * nfr + f].data_ptr() for f in range(nfr)], n=[len(f) for f in q.frames],
                  d_out=[outs[i * nfr + f].data_ptr() for f in range(nfr)], cap=[cap] * nfr,
                  d_nbytes=nb[i * nfr:(i + 1) * nfr]) for i, q in enumerate(seqs)]
    plan = lcc.Plan([ctx], descs)
    plan.encode()
    assert plan.sync() == lcc.OK
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.encode()
    assert plan.sync() == lcc.OK
    el = time.perf_counter() - t0
    pts = sum(len(f) for q in seqs for f in q.frames)
    info = plan.info()
    plan.close()
    return {"profile_plan": True, "frames": nseq * nfr, "points": pts, "tile": args.tile,
            "schedule": args.schedule, "max_batch": args.max_batch, "launches_per_encode": info["launches"],
            "mpts_per_s_wall": pts * args.steps / el / 1e6, "bytes": int(nb.sum().item())}


def run_profile_net(args, stream):
    """The proposal net's inference alone (k_net_fwd_tc): --net-tiles tiles of seeded BF16 inputs and
    He-initialised weights, one warm-up call and --steps timed calls: the case the net's ncu summary
    under profiles/ is taken on."""
    import torch
    from paper_2008_06972_gb300 import lcc
    from paper_2008_06972_gb300 import train as TR
    T = args.net_tiles
    net = lcc.Net(TR.he_uniform_params(4), max_tiles=4096, stream=stream)
    g = torch.Generator(device="cpu").manual_seed(0)
    x = (torch.randn((T, 64, 4), generator=g) * 0.3).to(torch.bfloat16).view(torch.int16).cuda()
    out = torch.zeros((T, 5), dtype=torch.float32, device="cuda")
    net.forward(x, T, out)
    assert net.sync() == lcc.OK
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        net.forward(x, T, out)
    b.record(stream)
    assert net.sync() == lcc.OK
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    flops = NET_FLOPS_PER_TILE * T
    return {"profile_net": True, "tiles": T, "ms_per_call": ms, "tflops": flops / (ms * 1e-3) / 1e12}


def run_profile_sequence(args, stream):
    """The HDL-64E sequence alone: one warm-up lcc_encode_sequence call and --steps timed calls
    (the case the DRAM traffic of the sequence's kernels is captured on)."""
    import torch
    from paper_2008_06972_gb300 import lcc
    th, tw = (int(v) for v in args.tile.split("x"))
    seq = make_workload(0)
    n = [len(f) for f in seq.frames]
    prm = lcc.default_params(tile_h=th, tile_w=tw, fit_thr_m=args.thr, max_batch=max(16, len(n)),
                             lookahead=args.lookahead, fit_schedule=args.schedule)
    ctx = lcc.Context(seq.sensor, prm, stream=stream)
    kf = lcc.Keyframe(ctx)
    d_pts = [torch.from_numpy(f).cuda() for f in seq.frames]
    cap = ctx.max_encoded_bytes
    outs = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in n]
    nb = torch.zeros(len(n), dtype=torch.int64, device="cuda")
    step = lambda: ctx.lcc_encode_sequence(seq.key_index, seq.poses, d_pts, n, outs, [cap] * len(n), nb, kf)
    step()
    assert ctx.lcc_sync() == lcc.OK
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        step()
    b.record(stream)
    assert ctx.lcc_sync() == lcc.OK
    torch.cuda.synchronize()
    return {"profile_sequence": True, "points": sum(n), "ms_per_step": a.elapsed_time(b) / args.steps,
            "bytes": int(nb.sum().item())}


def run_profile_train(args, stream):
    """Training steps of the proposal net alone (tcgen05 forward with saved activations, head
    backward, input gradients, weight gradients, Adam) on 4096 seeded tiles with random labels:
    one warm-up step and --steps timed steps, the case the training summary under profiles/ is
    taken on."""
    import torch
    from paper_2008_06972_gb300 import lcc
    from paper_2008_06972_gb300 import train as TR
    T = 4096
    net = lcc.Net(TR.he_uniform_params(4), max_tiles=T, stream=stream)
    g = torch.Generator(device="cpu").manual_seed(1)
    x = (torch.randn((T, 64, 4), generator=g) * 0.3).to(torch.bfloat16).view(torch.int16).cuda()
    y = torch.zeros((T, 5), dtype=torch.float32)
    y[:, 0] = (torch.rand(T, generator=g) < 0.5).float()
    n = torch.randn((T, 3), generator=g)
    y[:, 1:4] = n / n.norm(dim=1, keepdim=True) * y[:, :1]
    y = y.cuda()
    net.train_step(x, y, T, 1e-3, 1)
    assert net.sync() == lcc.OK
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(args.steps):
        net.train_step(x, y, T, 1e-3, k + 2)
    b.record(stream)
    assert net.sync() == lcc.OK
    torch.cuda.synchronize()
    return {"profile_train": True, "tiles": T, "ms_per_step": a.elapsed_time(b) / args.steps}


def run_hdl64(args, stream):
    """One synthetic HDL-64E sequence (10 frames of 64x2048, the middle one the key frame) encoded
    per call by lcc_encode_sequence: throughput (L2 flushed between steps), kernel times, decode,
    the entropy stage, the end-to-end host-buffer call, the dominant kernel's roofline, and the
    tile / threshold sweep and IMU rows."""
    import torch
    from paper_2008_06972_gb300 import lcc
    th, tw = (int(x) for x in args.tile.split("x"))
    seq = make_workload(0)
    n_frames = len(seq.frames)
    stream = torch.cuda.current_stream()
    params = lcc.default_params(tile_h=th, tile_w=tw, fit_thr_m=args.thr, max_batch=max(16, n_frames),
                                lookahead=args.lookahead, max_refits=args.refits,
                                solver=0 if args.solver == "ff" else 1, fit_schedule=args.schedule)
    ctx = lcc.Context(seq.sensor, params, stream=stream)
    kf = lcc.Keyframe(ctx)
    d_pts = [torch.from_numpy(f).cuda() for f in seq.frames]
    n = [len(f) for f in seq.frames]
    cap = ctx.max_encoded_bytes
    d_out = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(n_frames)]
    nbytes = torch.zeros(n_frames, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    pts_step = sum(n)

    def step():
        ctx.lcc_encode_sequence(seq.key_index, seq.poses, d_pts, n, d_out, [cap] * n_frames, nbytes, kf)

    for _ in range(max(args.warmup, 3)):
        step()
    assert ctx.lcc_sync() == lcc.OK
    # ---- timed region: K steps, each bracketed by CUDA events on the context stream ----
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(f"/tmp/lcc_clocks_{os.getpid()}_hdl64.csv")
    torch.cuda.synchronize()
    with clocks:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    st = ctx.lcc_sync()
    assert st == lcc.OK, lcc.status_string(st)
    ms = np.array([a.elapsed_time(b) for a, b in evs])
    value = pts_step / (float(ms.mean()) * 1e-3) / 1e6
    ms_step = float(ms.mean())

    # ---- per-kernel times (same workload, profiling events around each launch) ----
    ctx.lcc_set_profiling(True)
    for k in range(args.steps):
        flush.zero_()
        step()
    ktimes = ctx.lcc_kernel_times()
    ctx.lcc_set_profiling(False)
    launches_per_step = sum(v[0] for v in ktimes.values()) / args.steps
    # tile-mode split and fit rounds of the last step (library statistics, all frames)
    modes = {"empty": 0, "raw": 0, "run_start": 0, "run_cont": 0, "temporal": 0, "temporal_cont": 0}
    rounds_hist = [0] * 8
    border = 0
    for f in range(n_frames):
        st_f = ctx.lcc_last_stats(f)
        modes["empty"] += st_f["tiles_empty"]
        modes["raw"] += st_f["tiles_raw"]
        modes["run_start"] += st_f["tiles_run_start"]
        modes["run_cont"] += st_f["tiles_run_cont"]
        modes["temporal"] += st_f["tiles_temporal"]
        modes["temporal_cont"] += st_f["tiles_temporal_cont"]
        rounds_hist = [a + b for a, b in zip(rounds_hist, st_f["fit_rounds"])]
        border += st_f["tiles_borderline"]

    # ---- correctness of what was timed: decode every frame, max error vs the range image ----
    out_sizes = nbytes.cpu().numpy()
    H, W = seq.sensor.rows, seq.sensor.cols
    max_err = 0.0
    ref = torch.empty(H * W, dtype=torch.float32, device="cuda")
    dec = torch.empty(H * W, dtype=torch.float32, device="cuda")
    kfd = lcc.Keyframe(ctx)
    ctx.lcc_keyframe_from_stream(d_out[seq.key_index], int(out_sizes[seq.key_index]), kfd)
    for f in range(n_frames):
        ctx.lcc_range_image(d_pts[f], n[f], ref, None)
        isk = f == seq.key_index
        ctx.lcc_decode(d_out[f], int(out_sizes[f]), None if isk else kfd, None if isk else seq.poses[f], dec,
                       None, None)
        assert ctx.lcc_sync() == lcc.OK
        m = ref > 0
        if bool(m.any()):
            max_err = max(max_err, float((dec[m] - ref[m]).abs().max().item()))
    total_bytes = int(out_sizes.sum())

    # ---- decode throughput: the step's streams back to ranges, points and occupancy bitmaps ----
    xyz = torch.empty(H * W * 4, dtype=torch.float32, device="cuda")
    valid = torch.empty((H * W + 31) // 32, dtype=torch.int32, device="cuda")
    sizes = [int(x) for x in out_sizes]

    dec_r = [torch.empty(H * W, dtype=torch.float32, device="cuda") for _ in range(n_frames)]
    dec_x = [torch.empty(H * W * 4, dtype=torch.float32, device="cuda") for _ in range(n_frames)]
    dec_v = [torch.empty((H * W + 31) // 32, dtype=torch.int32, device="cuda") for _ in range(n_frames)]

    def decode_sequence():
        ctx.lcc_decode_sequence(seq.key_index, seq.poses, d_out, sizes, dec_r, dec_x, dec_v)

    def decode_frames():
        ctx.lcc_keyframe_from_stream(d_out[seq.key_index], sizes[seq.key_index], kfd)
        for f in range(n_frames):
            isk = f == seq.key_index
            ctx.lcc_decode(d_out[f], sizes[f], None if isk else kfd, None if isk else seq.poses[f], dec, xyz, valid)

    def time_decode(fn):
        for _ in range(3):
            fn()
        assert ctx.lcc_sync() == lcc.OK
        k_steps = max(5, min(args.steps, 50))
        dev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k_steps)]
        for k in range(k_steps):
            flush.zero_()
            dev[k][0].record(stream)
            fn()
            dev[k][1].record(stream)
        torch.cuda.synchronize()
        assert ctx.lcc_sync() == lcc.OK
        return float(np.mean([a.elapsed_time(b) for a, b in dev])), k_steps

    dec_ms, dec_steps = time_decode(decode_sequence)
    dec1_ms, _ = time_decode(decode_frames)
    decode = {"workload": "the step's 10 streams decoded to range, xyz and occupancy bitmap by one "
                          "lcc_decode_sequence call (key stream, then all P streams in one launch)",
              "steps": dec_steps, "ms_per_step": dec_ms, "mpts_per_s": pts_step / (dec_ms * 1e-3) / 1e6,
              "per_frame_calls": {"ms_per_step": dec1_ms, "mpts_per_s": pts_step / (dec1_ms * 1e-3) / 1e6}}

    hbm_peak, _ = peaks()
    entropy = None if args.no_entropy else run_entropy(args, stream, ctx, d_out, sizes, pts_step, flush, hbm_peak)

    # ---- end to end through the C ABI with HOST buffers (pinned) ----
    h_pts = [torch.from_numpy(f).pin_memory() for f in seq.frames]
    h_out = [torch.zeros(cap, dtype=torch.uint8).pin_memory() for _ in range(n_frames)]
    for _ in range(2):
        ctx.lcc_encode_sequence_host(seq.key_index, seq.poses, h_pts, h_out, [cap] * n_frames)
    torch.cuda.synchronize()
    e2e_steps = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        nb = ctx.lcc_encode_sequence_host(seq.key_index, seq.poses, h_pts, h_out, [cap] * n_frames)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = pts_step / e2e_s / 1e6

    # ---- roofline of the dominant kernel ----
    hbm, src = peaks()
    dom = max(ktimes.items(), key=lambda kv: kv[1][1])
    dname, (dl, dms) = dom
    per_launch_ms = dms / dl
    # algorithmic bytes per launch (per-unit figures):
    #   bin:   16 B per input point (float4 read) + 4 B per point atomic into the range image
    #   fit:   4 B per pixel (range image read) + 64 B per tile record written
    #   merge: 64 B per tile record read + 32 B tile code and 32 B tile offsets written per tile
    #          + the stream bytes zeroed by the frame's layout step
    #   pack:  4 B per pixel read + 4 B per pixel reset + stream bytes written
    #   temporal: (P frames) 4 B per pixel + 64 B per tile record read and written
    #   lookbehind: 4 B per pixel (range image read) + 64 B per tile record read + 32 B per tile
    #          of look-behind counts written
    #   rounds: per queued tile its record read and written (128 B), and 4 B per pixel per
    #          further round (the fit rounds after the first pass, from the rounds histogram)
    npx = H * W
    nt = ctx.num_tiles
    queued_tiles = sum(rounds_hist[r] for r in range(2, 8))
    extra_rounds = sum((r - 1) * rounds_hist[r] for r in range(2, 8))
    per_step_units = {
        "bin": 20.0 * pts_step,
        "fit": n_frames * (4.0 * npx + 64.0 * nt),
        "rounds": 128.0 * queued_tiles + 4.0 * th * tw * extra_rounds,
        "lookbehind": n_frames * (4.0 * npx + 96.0 * nt),
        "temporal": (n_frames - 1) * (4.0 * npx + 128.0 * nt),
        "merge": n_frames * (64.0 * nt + 32.0 * nt + 32.0 * nt) + total_bytes,
        "pack": n_frames * 8.0 * npx + total_bytes,
    }
    launches_of = {k: v[0] / args.steps for k, v in ktimes.items()}
    alg_bytes = per_step_units.get(dname, 0.0) / max(launches_of.get(dname, 1.0), 1e-9)
    achieved = alg_bytes / (per_launch_ms * 1e-3) / 1e9
    path_bytes = 16.0 * pts_step + total_bytes
    traffic = measured_traffic(dname) if (args.tile, args.thr, args.lookahead, args.schedule) == (
        "4x4", 0.05, 16, 3) else None
    roof = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "alg_bytes_per_launch": alg_bytes,
            "peak_source": src,
            "path": {"alg_bytes_per_step": path_bytes, "achieved": path_bytes / (ms_step * 1e-3) / 1e9,
                     "frac": path_bytes / (ms_step * 1e-3) / 1e9 / hbm}}

    sweep = None if args.no_sweep else run_sweep(args, stream, seq, d_pts, flush)
    imu_rows = None if args.no_imu else run_imu(args, stream, flush)
    assert max_err <= 0.02, max_err
    return {
        "workload": WORKLOAD, "value": value, "unit": UNIT, "ms_per_step": ms_step, "steps": args.steps,
        "config": {"frames": n_frames, "points_per_step": pts_step, "tile": args.tile, "thr_m": args.thr, "q_m": 0.02,
                   "lookahead": args.lookahead, "max_refits": args.refits,
                   "plane_solver": "float-float" if args.solver == "ff" else "fp64", "fit_schedule": args.schedule,
                   "l2": "flushed between steps (256 MiB write, untimed)"},
        "max_decode_error_m": max_err, "tile_modes": modes, "fit_rounds_hist": rounds_hist,
        "tiles_borderline": border, "compression_ratio": 12.0 * pts_step / total_bytes,
        "bytes_per_step": total_bytes, "kernel_ms_per_step": {k: v[1] / args.steps for k, v in ktimes.items()},
        "gpu_launches_per_step": launches_per_step, "roofline": roof, "decode": decode, "entropy": entropy,
        "sweep": sweep, "imu": imu_rows, "clocks": clocks.summary(),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(16 * pts_step),
                "d2h_bytes_per_step": int(total_bytes + 8 * n_frames)},
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2008_06972_gb300 import build as B
    B.build()
    stream = torch.cuda.current_stream()
    hbm, _ = peaks()
    if args.profile_plan:
        print(json.dumps(run_profile_plan(args, stream)), flush=True)
        return
    if args.profile_net:
        print(json.dumps(run_profile_net(args, stream)), flush=True)
        return
    if args.profile_train:
        print(json.dumps(run_profile_train(args, stream)), flush=True)
        return
    if args.profile_sequence:
        print(json.dumps(run_profile_sequence(args, stream)), flush=True)
        return
    line = run_cfg5(args, stream, rank, world, dist)
    if world == 1:
        line["hdl64_sequence"] = None if args.no_hdl64 else run_hdl64(args, stream)
        line["batched"] = None if args.no_batched else run_batched(args, stream, hbm)
        line["learned"] = None if args.no_learned else run_learned(args, stream)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
