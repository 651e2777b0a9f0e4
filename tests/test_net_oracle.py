"""Pins of the proposal-net oracle (oracle/net.py) against things other than itself:
torch's CPU bfloat16 conversion, torch's fp64 convolution / linear / loss functions and
autograd, central finite differences, torch's Adam, and hand-built tiles."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import net as N

torch = pytest.importorskip("torch")
F = torch.nn.functional


def _torch_net(theta, X, y):
    """The same net and loss written with torch fp64 ops (no BF16 rounding)."""
    P = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in N.unflatten(theta).items()}
    x = torch.tensor(X, dtype=torch.float64)
    a1 = F.relu(F.conv2d(x, P["W1"], P["b1"], padding=1))
    a2 = F.relu(F.conv2d(a1, P["W2"], P["b2"], padding=1))
    a3 = F.relu(F.conv2d(a2, P["W3"], P["b3"], padding=1))
    g = a3.mean(dim=(2, 3))
    h = F.relu(F.linear(g, P["F1"], P["c1"]))
    o = F.linear(h, P["F2"], P["c2"])
    yt = torch.tensor(y, dtype=torch.float64)
    fit = yt[:, 0]
    bce = F.binary_cross_entropy_with_logits(o[:, 0], fit, reduction="none")
    v = o[:, 1:4]
    cos = (v * yt[:, 1:4]).sum(1) / torch.sqrt((v * v).sum(1) + N.NORM_EPS)
    sl1 = F.smooth_l1_loss(o[:, 4], yt[:, 4], beta=N.SMOOTH_L1_BETA, reduction="none")
    loss = (bce + fit * (1 - cos.abs()) + fit * sl1).mean()
    loss.backward()
    loss = loss.detach()
    grads = np.concatenate([P[k].grad.numpy().reshape(-1) for k, _ in N.SHAPES])
    return float(loss), grads, o.detach().numpy()


def _batch(seed, T=6):
    rng = np.random.default_rng(seed)
    X = rng.normal(0, 0.3, (T, 4, 8, 8))
    X[:, :, 5:, 6:] = 0.0     # an empty corner
    y = np.zeros((T, 5))
    y[:, 0] = rng.integers(0, 2, T)
    n = rng.normal(0, 1, (T, 3))
    y[:, 1:4] = n / np.linalg.norm(n, axis=1, keepdims=True)
    y[:, 4] = rng.normal(0, 0.03, T)
    return X, y


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.normal(0, 3, 2000), rng.normal(0, 1e-3, 500),
                        1.0 + np.arange(8) * 2.0 ** -9, -(1.0 + np.arange(8) * 2.0 ** -9)])
    x32 = x.astype(np.float32)   # the GPU rounds fp32 values
    ref = torch.tensor(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(N.bf16(x32.astype(np.float64)), ref)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert N.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    assert N.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6


def test_forward_loss_and_gradients_match_torch_autograd():
    theta = N.init_params(7)
    X, y = _batch(3)
    loss, grad, o = N.loss_and_grad(theta, X, y, rounding=False)
    tl, tg, to = _torch_net(theta, X, y)
    assert np.allclose(o, to, rtol=1e-10, atol=1e-12)
    assert abs(loss - tl) <= 1e-12 * max(1.0, abs(tl))
    assert np.allclose(grad, tg, rtol=1e-8, atol=1e-14)


def test_gradients_match_finite_differences():
    theta = N.init_params(11)
    # non-zero biases: with zero biases an all-empty 3x3 window sits exactly on the ReLU kink
    P = N.unflatten(theta.copy())
    brng = np.random.default_rng(12)
    for k in ("b1", "b2", "b3", "c1", "c2"):
        P[k][:] = brng.normal(0, 0.05, P[k].shape)
    theta = N.flatten(P)
    X, y = _batch(5, T=3)
    _, grad, _ = N.loss_and_grad(theta, X, y, rounding=False)
    rng = np.random.default_rng(2)
    # a few coordinates of every parameter block
    o, idx = 0, []
    for _, shp in N.SHAPES:
        n = int(np.prod(shp))
        idx += list(o + rng.choice(n, min(4, n), replace=False))
        o += n
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (N.loss_and_grad(tp, X, y, rounding=False)[0] - N.loss_and_grad(tm, X, y, rounding=False)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 + 1e-4 * abs(grad[i]), (i, fd, grad[i])


def test_rounding_points_hold_bf16_values():
    theta = N.init_params(3)
    X, y = _batch(9)
    o, c = N.forward(theta, X, rounding=True)
    for k in ("a0", "a1", "a2", "a3", "g", "h"):
        assert np.array_equal(N.bf16(c[k]), c[k]), k
    # with rounding the result stays close to the fp64 net (BF16 keeps 8 significant bits)
    o64, _ = N.forward(theta, X, rounding=False)
    assert np.abs(o - o64).max() <= 0.05 * max(1.0, np.abs(o64).max())


def test_tile_inputs_of_hand_built_tiles():
    H, W = 8, 16
    rng = np.zeros((H, W), np.float32)
    beams = np.zeros((H, W, 3), np.float32)
    beams[..., 0] = 1.0   # every ray along +x: p = (r, 0, 0)
    rng[0, 3] = 0.0
    rng[1, 2] = 5.0       # tile 0: first valid pixel in raster order is (1, 2)
    rng[4, 7] = 7.5
    X, anchors, nv = N.tile_inputs(rng, beams)
    assert X.shape == (2, 4, 8, 8) and list(nv) == [2, 0]
    assert anchors[0].tolist() == [5.0, 0.0, 0.0]
    assert X[0, 0, 1, 2] == 0.0 and X[0, 0, 4, 7] == 2.5 and X[0, 1, 4, 7] == 2.5
    assert np.count_nonzero(X[0]) == 2 and np.count_nonzero(X[1]) == 0


def test_labels_are_planes_relative_to_the_anchor():
    planes = np.array([[0.0, 0.0, 1.0, 1.7], [1.0, 0.0, 0.0, 12.0]], np.float32)
    anchors = np.array([[3.0, 4.0, -1.7], [12.0, 1.0, 0.5]], np.float32)
    y = N.labels(np.array([1, 0]), planes, anchors)
    assert np.allclose(y[0], [1, 0, 0, 1, 1.7 - (-1.7)])
    assert np.array_equal(y[1], np.zeros(5))


def test_adam_matches_torch():
    rng = np.random.default_rng(4)
    theta = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(3)]
    p = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-3)
    m = np.zeros(50)
    v = np.zeros(50)
    t = theta.copy()
    for k, g in enumerate(grads):
        opt.zero_grad()
        p.grad = torch.tensor(g)
        opt.step()
        t, m, v = N.adam(t, g, m, v, k + 1, 1e-3)
    assert np.allclose(t, p.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_param_count():
    assert N.N_PARAMS == 58853
