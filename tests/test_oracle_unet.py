"""Pins of the warm-start U-Net's CPU reference (oracle/unet_ref.py), no GPU.

The GPU network's forward, backward and weight-gradient kernels are judged
against oracle/unet_ref.py; these tests pin that reference to the
architecture it states, with definitions written out independently of the
PyTorch operators it calls:
  * the 3x3 convolution equals the explicit nine-tap sum with the weight
    layout w[tap][cout][cin], tap = 3 (dy + 1) + (dx + 1), zero padding;
  * 2x2 average pooling and nearest upsampling equal their block
    definitions, and pooling is a quarter of upsampling's adjoint;
  * every layer of forward() equals the architecture (channel counts,
    pooling, upsampling, the order of each skip concatenation) recomputed
    with those explicit operations from the previous layers' outputs; a
    planted swap of the concatenation order fails this check;
  * loss_and_grads() returns the gradient of its own loss: central
    differences in float64 agree with every layer's weight and bias
    gradients.
"""
import numpy as np
import pytest
import torch

from oracle import unet_ref as U

CH = {"e0": (16, 16), "e1": (16, 32), "e2": (32, 64), "b1": (64, 128), "b2": (128, 64),
      "d2": (128, 32), "d1": (64, 16), "d0": (32, 16), "out": (16, 16)}


def params(seed=0, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    out = {}
    for name, (cin, cout) in CH.items():
        w = torch.randn(9, cout, cin, generator=g, dtype=torch.float64) * scale / np.sqrt(9 * cin)
        b = torch.randn(cout, generator=g, dtype=torch.float64) * 0.05
        out[name] = (w, b)
    return out


def conv_taps(x, wb):
    """y[n, co, h, w] = b[co] + sum_{dy, dx, ci} w[3 (dy+1) + (dx+1)][co][ci] x[n, ci, h+dy, w+dx]."""
    w, b = (t.numpy() for t in wb)
    x = x.numpy() if isinstance(x, torch.Tensor) else x
    n, ci, hh, ww = x.shape
    xp = np.zeros((n, ci, hh + 2, ww + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.broadcast_to(b[None, :, None, None], (n, w.shape[1], hh, ww)).copy()
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            tap = 3 * (dy + 1) + (dx + 1)
            shifted = xp[:, :, 1 + dy:1 + dy + hh, 1 + dx:1 + dx + ww]
            y += np.einsum("oc,nchw->nohw", w[tap], shifted)
    return y


def pool_blocks(x):
    n, c, hh, ww = x.shape
    return x.reshape(n, c, hh // 2, 2, ww // 2, 2).mean(axis=(3, 5))


def up_blocks(x):
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def relu(a):
    return np.maximum(a, 0.0)


def layer_errors(p, x):
    """Largest relative deviation of each forward() layer from the
    architecture recomputed with the explicit operations above."""
    acts = {}
    y = U.forward(p, x, acts)
    a = {k: v.numpy() for k, v in acts.items()}
    expect = {
        "e0": relu(conv_taps(x, p["e0"])),
        "e1": relu(conv_taps(pool_blocks(a["e0"]), p["e1"])),
        "e2": relu(conv_taps(pool_blocks(a["e1"]), p["e2"])),
        "b1": relu(conv_taps(pool_blocks(a["e2"]), p["b1"])),
        "b2": relu(conv_taps(a["b1"], p["b2"])),
        "d2": relu(conv_taps(np.concatenate([up_blocks(a["b2"]), a["e2"]], axis=1), p["d2"])),
        "d1": relu(conv_taps(np.concatenate([up_blocks(a["d2"]), a["e1"]], axis=1), p["d1"])),
        "d0": relu(conv_taps(np.concatenate([up_blocks(a["d1"]), a["e0"]], axis=1), p["d0"])),
        "out": conv_taps(a["d0"], p["out"]),
    }
    got = dict(a, out=y.numpy())
    return {k: float(np.abs(got[k] - v).max() / max(np.abs(v).max(), 1e-300)) for k, v in expect.items()}


def test_conv_is_the_nine_tap_sum():
    g = torch.Generator().manual_seed(1)
    x = torch.randn(2, 5, 6, 7, generator=g, dtype=torch.float64)
    wb = (torch.randn(9, 4, 5, generator=g, dtype=torch.float64), torch.randn(4, generator=g, dtype=torch.float64))
    np.testing.assert_allclose(U._conv(x, wb).numpy(), conv_taps(x, wb), rtol=0, atol=1e-13)
    # a single tap: the weight of tap (dy, dx) = (-1, +1) picks x[h - 1, w + 1]
    w = torch.zeros(9, 1, 1, dtype=torch.float64)
    w[3 * 0 + 2, 0, 0] = 1.0
    y = U._conv(x[:, :1], (w, torch.zeros(1, dtype=torch.float64)))[0, 0]
    np.testing.assert_array_equal(y[1:, :-1].numpy(), x[0, 0, :-1, 1:].numpy())


def test_pool_and_upsample_blocks_and_adjoint():
    g = torch.Generator().manual_seed(2)
    x = torch.randn(2, 3, 8, 6, generator=g, dtype=torch.float64)
    y = torch.randn(2, 3, 4, 3, generator=g, dtype=torch.float64)
    np.testing.assert_allclose(U.pool(x).numpy(), pool_blocks(x.numpy()), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(U.up(y).numpy(), up_blocks(y.numpy()))
    # <pool x, y> = <x, up y> / 4, and pooling undoes upsampling
    lhs = float((U.pool(x) * y).sum())
    rhs = float((x * U.up(y)).sum()) / 4.0
    assert lhs == pytest.approx(rhs, rel=1e-13)
    np.testing.assert_allclose(U.pool(U.up(y)).numpy(), y.numpy(), rtol=0, atol=1e-15)
    # the concatenation puts its first argument's channels first
    c = U.cat(x[:, :1], x[:, 1:])
    np.testing.assert_array_equal(c.numpy(), x.numpy())


def test_every_layer_follows_the_architecture():
    g = torch.Generator().manual_seed(3)
    x = torch.randn(2, 16, 8, 8, generator=g, dtype=torch.float64)
    errs = layer_errors(params(3), x)
    assert max(errs.values()) <= 1e-12, errs


def test_planted_concat_swap_is_caught(monkeypatch):
    """The same check on a reference whose skip concatenation puts the skip
    first: the decoder layers must fail."""
    g = torch.Generator().manual_seed(4)
    x = torch.randn(2, 16, 8, 8, generator=g, dtype=torch.float64)
    p = params(4)
    # a swapped order only changes the channel order, so the decoders' input
    # widths must stay equal: d2 takes 64 + 64, d1 32 + 32, d0 16 + 16
    monkeypatch.setattr(U, "cat", lambda a, b: torch.cat([b, a], dim=1))
    errs = layer_errors(p, x)
    assert errs["d2"] > 1e-3 and errs["d1"] > 1e-3 and errs["d0"] > 1e-3, errs
    assert errs["e0"] <= 1e-12 and errs["b2"] <= 1e-12


def test_loss_and_grads_match_central_differences():
    g = torch.Generator().manual_seed(5)
    x = torch.randn(2, 16, 8, 8, generator=g, dtype=torch.float64)
    target = torch.randn(2, 2, 8, 8, generator=g, dtype=torch.float64)
    p = params(5, scale=1.5)
    loss, _, grads = U.loss_and_grads(p, x, target)
    rng = np.random.default_rng(5)
    h = 1e-6
    for name, (w, b) in p.items():
        gw, gb = grads[name]
        assert gw.shape == w.shape and gb.shape == b.shape
        picks = [("w", tuple(int(rng.integers(0, s)) for s in w.shape)) for _ in range(3)]
        picks.append(("b", (int(rng.integers(0, b.shape[0])),)))
        for kind, idx in picks:
            vals = []
            for sgn in (1.0, -1.0):
                q = {k: (ww.clone(), bb.clone()) for k, (ww, bb) in p.items()}
                (q[name][0] if kind == "w" else q[name][1])[idx] += sgn * h
                vals.append(U.loss_and_grads(q, x, target)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            an = float((gw if kind == "w" else gb)[idx])
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-9 * max(abs(loss), 1.0)), (name, kind, idx, an, fd)
