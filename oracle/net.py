"""CPU oracle of the learned tile proposal net — TEST INFRASTRUCTURE ONLY.

Plain numpy, fp64 accumulation.  Only the test-suite and the bench's CPU legs may
import it; the GPU library never does and shares no code with it.

The net (a proposal of a tile's planarity and plane, used to seed the iterative fit
of Sec. III-C; not in the paper) takes an 8x8 tile as 4 channels:
  channel 0: r - r_anchor, channels 1-3: p - p_anchor, in metres, where p = r*u is
  the fp32 point of a pixel (three fp32 products) and the anchor is the tile's first
  valid pixel in raster order; empty pixels are 0 in every channel.
Layers: conv3x3 pad 1 (4->32), ReLU, conv3x3 (32->64), ReLU, conv3x3 (64->64), ReLU,
global average pool (64), linear 64->32, ReLU, linear 32->5.  The padding is zero
outside the tile: every tile is its own 8x8 image.  Outputs: planarity logit, normal
(3, unnormalised), plane offset relative to the anchor (d - n.p_anchor).

BF16 rounding points (round to nearest even), when ``rounding`` is on:
  the input, every weight matrix (biases stay fp32), each activation after its ReLU
  (a1, a2, a3), the pooled vector and the hidden head activation; in the backward
  pass the pre-activation gradients dz1..dz3 that feed the convolution products.
With ``rounding`` off the same functions are the plain fp64 net, which the
finite-difference and autograd pins check.

Parameters are one flat float vector in this order: W1[32,4,3,3], b1[32],
W2[64,32,3,3], b2[64], W3[64,64,3,3], b3[64], F1[32,64], c1[32], F2[5,32], c2[5]
(58,853 values).
"""
from __future__ import annotations

import numpy as np

TILE = 8
SHAPES = [("W1", (32, 4, 3, 3)), ("b1", (32,)), ("W2", (64, 32, 3, 3)), ("b2", (64,)),
          ("W3", (64, 64, 3, 3)), ("b3", (64,)), ("F1", (32, 64)), ("c1", (32,)), ("F2", (5, 32)), ("c2", (5,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
SMOOTH_L1_BETA = 0.02   # metres
NORM_EPS = 1e-12


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (8-bit significand), nearest even, returned as float64 values."""
    x = np.asarray(x, dtype=np.float64)
    b = x.view(np.uint64).copy()
    lsb = (b >> np.uint64(45)) & np.uint64(1)
    b = b + np.uint64((1 << 44) - 1) + lsb
    b &= ~np.uint64((1 << 45) - 1)
    return b.view(np.float64)


def _r(x, rounding):
    return bf16(x) if rounding else np.asarray(x, dtype=np.float64)


def unflatten(theta: np.ndarray) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def flatten(P: dict) -> np.ndarray:
    return np.concatenate([np.asarray(P[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, from a seeded generator."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, shp in SHAPES:
        if name[0] in "WF":
            fan_in = int(np.prod(shp[1:]))
            P[name] = rng.uniform(-1.0, 1.0, shp) * np.sqrt(6.0 / fan_in)
        else:
            P[name] = np.zeros(shp)
    return flatten(P).astype(np.float32).astype(np.float64)


# ------------------------------------------------------------------ inputs and labels --

def tile_inputs(rng: np.ndarray, beams: np.ndarray):
    """Net inputs of every 8x8 tile of a range image.

    rng: (H, W) fp32 ranges (0 = empty); beams: (H, W, 3) fp32 unit rays.
    Returns X (T, 4, 8, 8) float64 holding fp32 values (before BF16 rounding), the anchor
    points (T, 3) fp32 and the valid-pixel counts (T,), tiles in row-major order."""
    H, W = rng.shape
    TR, TC = (H + TILE - 1) // TILE, (W + TILE - 1) // TILE
    r = np.zeros((TR * TILE, TC * TILE), np.float32)
    r[:H, :W] = rng
    u = np.zeros((TR * TILE, TC * TILE, 3), np.float32)
    u[:H, :W] = beams
    p = (r[..., None] * u).astype(np.float32)   # fp32 products, one rounding each
    X = np.zeros((TR * TC, 4, TILE, TILE))
    anchors = np.zeros((TR * TC, 3), np.float32)
    nv = np.zeros(TR * TC, np.int64)
    for tr in range(TR):
        for tc in range(TC):
            t = tr * TC + tc
            rt = r[tr * TILE:(tr + 1) * TILE, tc * TILE:(tc + 1) * TILE]
            pt = p[tr * TILE:(tr + 1) * TILE, tc * TILE:(tc + 1) * TILE]
            valid = rt > 0
            nv[t] = int(valid.sum())
            if nv[t] == 0:
                continue
            k = int(np.flatnonzero(valid.reshape(-1))[0])
            ra, pa = rt.reshape(-1)[k], pt.reshape(-1, 3)[k]
            anchors[t] = pa
            X[t, 0] = np.where(valid, (rt - ra).astype(np.float32), 0.0)
            for c in range(3):
                X[t, 1 + c] = np.where(valid, (pt[..., c] - pa[c]).astype(np.float32), 0.0)
    return X, anchors, nv


def labels(status_fit: np.ndarray, planes: np.ndarray, anchors: np.ndarray) -> np.ndarray:
    """Training targets (T, 5): fit flag, unit normal, offset relative to the anchor (fp64)."""
    y = np.zeros((len(status_fit), 5))
    y[:, 0] = status_fit.astype(np.float64)
    n = planes[:, :3].astype(np.float64)
    y[:, 1:4] = n
    y[:, 4] = planes[:, 3].astype(np.float64) - (n * anchors.astype(np.float64)).sum(axis=1)
    y[status_fit == 0, 1:] = 0.0
    return y


# ------------------------------------------------------------------ forward / backward --

def _conv(a, Wt, b):
    """3x3 convolution, zero padding 1, per 8x8 image: z[n,co,y,x] = b[co] +
    sum over ci, ky, kx of W[co,ci,ky,kx] * a[n,ci,y+ky-1,x+kx-1]."""
    n, ci = a.shape[:2]
    ap = np.zeros((n, ci, TILE + 2, TILE + 2))
    ap[:, :, 1:-1, 1:-1] = a
    z = np.zeros((n, Wt.shape[0], TILE, TILE))
    for ky in range(3):
        for kx in range(3):
            z += np.einsum("oc,ncyx->noyx", Wt[:, :, ky, kx], ap[:, :, ky:ky + TILE, kx:kx + TILE])
    return z + b[None, :, None, None]


def _conv_back(dz, a, Wt):
    """Gradients of _conv: dW[co,ci,ky,kx] = sum over n, y, x of dz[n,co,y,x] * a_pad[n,ci,y+ky,x+kx];
    da[n,ci] = the same taps summed the other way (transposed convolution), cropped to the tile."""
    n, ci = a.shape[:2]
    ap = np.zeros((n, ci, TILE + 2, TILE + 2))
    ap[:, :, 1:-1, 1:-1] = a
    dW = np.zeros_like(Wt)
    dap = np.zeros_like(ap)
    for ky in range(3):
        for kx in range(3):
            win = ap[:, :, ky:ky + TILE, kx:kx + TILE]
            dW[:, :, ky, kx] = np.einsum("noyx,ncyx->oc", dz, win)
            dap[:, :, ky:ky + TILE, kx:kx + TILE] += np.einsum("oc,noyx->ncyx", Wt[:, :, ky, kx], dz)
    return dW, dz.sum(axis=(0, 2, 3)), dap[:, :, 1:-1, 1:-1]


def forward(theta: np.ndarray, X: np.ndarray, rounding: bool = True):
    """Outputs (T, 5) and the cache the backward pass needs."""
    P = unflatten(theta)
    Wb = {k: _r(P[k], rounding) for k in ("W1", "W2", "W3", "F1", "F2")}
    a0 = _r(X, rounding)
    a1 = _r(np.maximum(_conv(a0, Wb["W1"], P["b1"]), 0.0), rounding)
    a2 = _r(np.maximum(_conv(a1, Wb["W2"], P["b2"]), 0.0), rounding)
    a3 = _r(np.maximum(_conv(a2, Wb["W3"], P["b3"]), 0.0), rounding)
    g = _r(a3.mean(axis=(2, 3)), rounding)
    h = _r(np.maximum(g @ Wb["F1"].T + P["c1"], 0.0), rounding)
    o = h @ Wb["F2"].T + P["c2"]
    return o, dict(Wb=Wb, a0=a0, a1=a1, a2=a2, a3=a3, g=g, h=h)


def loss_terms(o: np.ndarray, y: np.ndarray):
    """Per-tile loss and its gradient w.r.t. the outputs.

    loss = BCE-with-logits(o0, fit) + fit * (1 - |n_hat . n|) + fit * SmoothL1_beta(o4 - d_rel),
    n_hat = o[1:4] / sqrt(|o[1:4]|^2 + eps)."""
    lg, v, dd = o[:, 0], o[:, 1:4], o[:, 4]
    fit, n, drel = y[:, 0], y[:, 1:4], y[:, 4]
    bce = np.maximum(lg, 0.0) - fit * lg + np.log1p(np.exp(-np.abs(lg)))
    s = np.sqrt((v * v).sum(axis=1) + NORM_EPS)
    vn = (v * n).sum(axis=1)
    cos = vn / s
    x = dd - drel
    ax = np.abs(x)
    sl1 = np.where(ax < SMOOTH_L1_BETA, 0.5 * x * x / SMOOTH_L1_BETA, ax - 0.5 * SMOOTH_L1_BETA)
    loss = bce + fit * (1.0 - np.abs(cos)) + fit * sl1
    do = np.zeros_like(o)
    do[:, 0] = 1.0 / (1.0 + np.exp(-lg)) - fit
    dcos_dv = n / s[:, None] - (vn / s ** 3)[:, None] * v
    do[:, 1:4] = -(fit * np.sign(cos))[:, None] * dcos_dv
    do[:, 4] = fit * np.clip(x / SMOOTH_L1_BETA, -1.0, 1.0)
    return loss, do


def loss_and_grad(theta: np.ndarray, X: np.ndarray, y: np.ndarray, rounding: bool = True):
    """Mean loss over the tiles and its gradient w.r.t. theta (flat, same order)."""
    P = unflatten(theta)
    o, c = forward(theta, X, rounding)
    T = len(X)
    loss, do = loss_terms(o, y)
    do = do / T
    Wb = c["Wb"]
    dF2 = do.T @ c["h"]
    dc2 = do.sum(axis=0)
    dh = do @ Wb["F2"]
    dy1 = dh * (c["h"] > 0)
    dF1 = dy1.T @ c["g"]
    dc1 = dy1.sum(axis=0)
    dg = dy1 @ Wb["F1"]
    da3 = np.broadcast_to((dg / (TILE * TILE))[:, :, None, None], c["a3"].shape)
    dz3 = _r(da3 * (c["a3"] > 0), rounding)
    dW3, db3, da2 = _conv_back(dz3, c["a2"], Wb["W3"])
    dz2 = _r(da2 * (c["a2"] > 0), rounding)
    dW2, db2, da1 = _conv_back(dz2, c["a1"], Wb["W2"])
    dz1 = _r(da1 * (c["a1"] > 0), rounding)
    dW1, db1, _ = _conv_back(dz1, c["a0"], Wb["W1"])
    grads = dict(W1=dW1, b1=db1, W2=dW2, b2=db2, W3=dW3, b3=db3, F1=dF1, c1=dc1, F2=dF2, c2=dc2)
    return float(loss.mean()), flatten(grads), o


def adam(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected, step counted from 1); returns new theta, m, v."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
