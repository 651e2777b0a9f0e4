"""Launch configurations checked in a fresh process.

A kernel's shared-memory opt-in is a per-process attribute: once an earlier launch (a larger
sensor) has raised it, a later launch that forgot to ask for it still succeeds.  This test runs
every tile shape on a 1024-column sensor in a new interpreter, before anything else launches, so
a launcher that under-counts its shared memory fails here."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SNIPPET = r"""
import sys
sys.path.insert(0, sys.argv[1])
import torch
import synth
from paper_2008_06972_gb300 import lcc
sen = synth.CFG3_SENSORS[1]
s = synth.grouped_sequence(sen, 1, 5, synth.config_seed(3, 201, 0), 10)
k = synth.group_key(0, 5, 10)
d = [torch.from_numpy(f).cuda() for f in s.frames]
n = [len(f) for f in s.frames]
for th, tw in ((4, 4), (4, 8), (8, 8), (8, 16)):
    for sched in (0, 3, 5):
        c = lcc.Context(sen, lcc.default_params(max_batch=5, tile_h=th, tile_w=tw, fit_schedule=sched))
        cap = c.max_encoded_bytes
        outs = [torch.zeros(cap, dtype=torch.uint8, device="cuda") for _ in range(5)]
        nb = torch.zeros(5, dtype=torch.int64, device="cuda")
        c.lcc_encode_sequence(k, s.poses, d, n, outs, [cap] * 5, nb, lcc.Keyframe(c))
        assert c.lcc_sync() == lcc.OK, (th, tw, sched)
        assert int(nb.min()) > 64, (th, tw, sched)
print("ok")
"""


def test_every_tile_shape_launches_in_a_fresh_process():
    res = subprocess.run([sys.executable, "-c", SNIPPET, ROOT], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert res.returncode == 0 and res.stdout.strip().endswith("ok"), res.stdout[-2000:] + res.stderr[-4000:]
