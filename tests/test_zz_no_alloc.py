"""lcc_range_image_static (fixed device scratch, no allocation) against lcc_range_image.

Collected last so that it also runs after every other GPU test in the same process; it must
pass alone as well.  The range image is integer/bit work (Sec. III-B binning, nearest point
per pixel), so the two entry points must agree bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import synth
from tests import harness as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _dense(sensor, pts):
    from paper_2008_06972_gb300 import lcc
    npx = sensor.rows * sensor.cols
    c = H.ctx(sensor)
    d = H.to_dev(pts)
    rng = torch.full((npx,), -1.0, dtype=torch.float32, device="cuda")
    valid = torch.full(((npx + 31) // 32,), -1, dtype=torch.int32, device="cuda")
    c.lcc_range_image(d, len(pts), rng, valid)
    assert c.lcc_sync() == lcc.OK
    return rng.cpu().numpy(), valid.cpu().numpy()


def _alloc_state():
    """Free device memory and the torch allocator's counters: neither may move across a call."""
    free, _ = torch.cuda.mem_get_info()
    st = torch.cuda.memory_stats()
    keys = ("allocation.all.allocated", "reserved_bytes.all.current", "segment.all.allocated")
    return free, {k: st.get(k, 0) for k in keys}


def test_static_scratch_range_image_matches_context_path():
    """Two calls in a row per sensor, then a change of sensor back to the first one: each call's
    outputs equal the context path's, and no call allocates (free device memory and torch's
    allocator counters unchanged across the calls, after the first call's set-up)."""
    from paper_2008_06972_gb300 import lcc
    cases = []
    sensor, pts = synth.frame_cfg1()
    cases.append((sensor, pts))
    s3 = synth.CFG3_SENSORS[3]   # 128 x 2048: the largest size the fixed scratch holds
    scene = synth.Scene(synth.config_seed(3, 900, 0), 4, 6, 10, enclose=True)
    cases.append((s3, scene.render(s3, sigma=0.02, dropout=0.05, seed=7)))
    cases.append(cases[0])       # back to the first sensor: its tables are copied again
    stream = torch.cuda.current_stream()
    prepared = []
    for sensor, pts in cases:
        ref_rng, ref_valid = _dense(sensor, pts)
        npx = sensor.rows * sensor.cols
        bufs = [(torch.full((npx,), -1.0, dtype=torch.float32, device="cuda"),
                 torch.full(((npx + 31) // 32,), -1, dtype=torch.int32, device="cuda")) for _ in range(2)]
        prepared.append((sensor, H.to_dev(pts), len(pts), ref_rng, ref_valid, bufs))
    # set-up call (looks the array's address up; may load the library's kernels)
    sensor, d, n, _, _, bufs = prepared[0]
    assert lcc.lcc_range_image_static(sensor, d, n, bufs[0][0], bufs[0][1], stream) == lcc.OK
    torch.cuda.synchronize()
    before = _alloc_state()
    for k, (sensor, d, n, ref_rng, ref_valid, bufs) in enumerate(prepared):
        for call in range(2):   # two calls in a row: the scratch is cleared by each call
            rng, valid = bufs[call]
            rng.fill_(-1.0)
            valid.fill_(-1)
            st = lcc.lcc_range_image_static(sensor, d, n, rng, valid, stream)
            assert st == lcc.OK, lcc.status_string(st)
            torch.cuda.synchronize()
            got_rng, got_valid = rng.cpu().numpy(), valid.cpu().numpy()
            assert np.array_equal(got_rng.view(np.uint32), ref_rng.view(np.uint32)), f"case {k} call {call}"
            assert np.array_equal(got_valid, ref_valid), f"case {k} call {call}"
    assert _alloc_state() == before
    # beyond the fixed scratch: a clear error, nothing launched
    big = synth.Sensor(256, 2048, -15.0, 15.0, 80.0)
    st = lcc.lcc_range_image_static(big, None, 0, None, None, stream)
    assert st == lcc.ERR_UNSUPPORTED
