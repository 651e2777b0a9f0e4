"""Training recipe of the learned tile proposal (lcc_net_*), driven through the C ABI.

Labels come from the plain encoder itself: for every 8x8 tile of a key frame, the fit flag
of its own iterative fit and its plane, with the offset expressed relative to the tile's
anchor (the first valid pixel's point), formed on the device (lcc_net_tile_labels).  Every
forward, backward and optimiser step runs in the library's CUDA kernels; this module only
gathers tiles into batches.
"""
from __future__ import annotations

import math

import numpy as np

from . import lcc

SKIP_PROB = 0.05
SKIP_LOGIT = math.log(SKIP_PROB / (1.0 - SKIP_PROB))   # tiles below this logit are not fitted


def he_uniform_params(seed: int) -> np.ndarray:
    """Initial parameters: weights uniform in +-sqrt(6 / fan_in), biases zero (fp32, flat order
    W1, b1, W2, b2, W3, b3, F1, c1, F2, c2)."""
    rng = np.random.default_rng(seed)
    shapes = [(32, 4, 3, 3), (32,), (64, 32, 3, 3), (64,), (64, 64, 3, 3), (64,), (32, 64), (32,), (5, 32), (5,)]
    parts = []
    for shp in shapes:
        if len(shp) > 1:
            bound = math.sqrt(6.0 / int(np.prod(shp[1:])))
            parts.append(rng.uniform(-bound, bound, shp).reshape(-1))
        else:
            parts.append(np.zeros(shp))
    out = np.concatenate(parts).astype(np.float32)
    assert out.size == lcc.Net.num_params()
    return out


def frame_examples(ctx: "lcc.Context", pts_dev, n: int):
    """Net inputs (T, 64, 4) bf16-as-int16 device tensor, anchors and labels of one frame."""
    import torch
    nt = ctx.num_tiles
    x = torch.zeros((nt, 64, 4), dtype=torch.int16, device="cuda")
    anc = torch.zeros((nt, 4), dtype=torch.float32, device="cuda")
    lcc.net_tile_inputs(ctx, pts_dev, n, x, anc)
    out = torch.empty(ctx.max_encoded_bytes, dtype=torch.uint8, device="cuda")
    nb = torch.zeros(1, dtype=torch.int64, device="cuda")
    ctx.lcc_encode_keyframe(pts_dev, n, None, out, out.numel(), nb)
    st = ctx.lcc_sync()
    if st != lcc.OK:
        raise lcc.LccError(st, "frame_examples")
    y = torch.empty((nt, 5), dtype=torch.float32, device="cuda")
    lcc.net_tile_labels(ctx, 0, anc, y)
    recs = ctx.lcc_tile_records(0)
    return x, anc, y, recs


def train(net: "lcc.Net", x, y, steps: int, batch: int, lr: float, seed: int = 0, lr_final: float | None = None):
    """Adam over random batches of tiles (with replacement across steps); returns the loss of
    every step (read back once at the end)."""
    import torch
    T = x.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = torch.zeros(steps, dtype=torch.float32, device="cuda")
    lr_final = lr if lr_final is None else lr_final
    for s in range(steps):
        idx = torch.randint(0, T, (batch,), generator=g).cuda()
        xb = x[idx].contiguous()
        yb = y[idx].contiguous()
        lr_s = lr * (lr_final / lr) ** (s / max(steps - 1, 1))
        net.train_step(xb, yb, batch, lr_s, s + 1, losses[s:s + 1])
    return losses.cpu().numpy()
