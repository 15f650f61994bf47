"""CPU FP64 reference of the warm-start U-Net (test infrastructure only).

Only the tests may use this module.  It restates the network with plain
PyTorch CPU operators in float64 -- 3x3 convolutions with zero padding, 2x2
average pooling, nearest 2x upsampling, channel concatenation, ReLU -- and
gets gradients from autograd, so the GPU's hand-written forward, backward and
weight-gradient kernels can be checked against it.

Architecture (channels; H x W halves at each pooling):
  e0 = relu(conv(x, 16 -> 16));  e1 = relu(conv(pool(e0), 16 -> 32));
  e2 = relu(conv(pool(e1), 32 -> 64));  b1 = relu(conv(pool(e2), 64 -> 128));
  b2 = relu(conv(b1, 128 -> 64));  d2 = relu(conv([up(b2), e2], 128 -> 32));
  d1 = relu(conv([up(d2), e1], 64 -> 16));  d0 = relu(conv([up(d1), e0], 32 -> 16));
  y  = conv(d0, 16 -> 16)  (channels 0 and 1 are the prediction)
Weights are given as {name: (w[9][cout][cin], b[cout])} with tap = 3 (dy + 1) + (dx + 1).

Pins (tests/test_oracle_unet.py): the convolution against an explicit
nine-tap sum, pooling and upsampling against their block definitions and
each other's adjoint, every layer of forward() against the architecture
above written with those explicit loops (a planted swap of the skip
concatenation fails it), and the gradients of loss_and_grads() against
central differences of its loss.
"""
import torch
import torch.nn.functional as F

NAMES = ("e0", "e1", "e2", "b1", "b2", "d2", "d1", "d0", "out")


def _conv(x, wb):
    w, b = wb
    cout, cin = w.shape[1], w.shape[2]
    k = w.permute(1, 2, 0).reshape(cout, cin, 3, 3)   # [co][ci][ky][kx]
    return F.conv2d(x, k, b, padding=1)


def pool(t):
    """2x2 average pooling (each output the mean of its 2x2 input block)."""
    return F.avg_pool2d(t, 2)


def up(t):
    """Nearest 2x upsampling (each input value copied to its 2x2 output block)."""
    return F.interpolate(t, scale_factor=2, mode="nearest")


def cat(a, b):
    """Channel concatenation, a's channels first."""
    return torch.cat([a, b], dim=1)


def forward(params, x, acts=None):
    """x: float64 [N, 16, H, W] (NCHW); returns y [N, 16, H, W].  If acts is a
    dict, the layer outputs e0 .. d0 are stored in it."""
    r = torch.relu
    e0 = r(_conv(x, params["e0"]))
    e1 = r(_conv(pool(e0), params["e1"]))
    e2 = r(_conv(pool(e1), params["e2"]))
    b1 = r(_conv(pool(e2), params["b1"]))
    b2 = r(_conv(b1, params["b2"]))
    d2 = r(_conv(cat(up(b2), e2), params["d2"]))
    d1 = r(_conv(cat(up(d2), e1), params["d1"]))
    d0 = r(_conv(cat(up(d1), e0), params["d0"]))
    if acts is not None:
        acts.update(e0=e0, e1=e1, e2=e2, b1=b1, b2=b2, d2=d2, d1=d1, d0=d0)
    return _conv(d0, params["out"])


def loss_and_grads(params, x, target):
    """MSE of channels 0..1 against target [N, 2, H, W]; gradients of every weight and bias."""
    p = {k: (w.detach().clone().requires_grad_(True), b.detach().clone().requires_grad_(True))
         for k, (w, b) in params.items()}
    y = forward(p, x)
    loss = ((y[:, :2] - target) ** 2).mean()
    loss.backward()
    return loss.item(), y.detach(), {k: (w.grad, b.grad) for k, (w, b) in p.items()}
