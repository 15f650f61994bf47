"""Learned warm start: a 4-level U-Net on BF16 tensor cores (include/pic_poisson_nn.h).

The network maps the normalised mode residual r_m of a previous-step iterate
(two channels, Re and Im, plus the mode's shift ratio lambda_m mu / D) on the
r-z grid of one mode to an approximate correction d_m ~ A_m^{-1} r_m.  Every
layer runs in the library's kernels: BF16 3x3 convolutions on the tcgen05
tensor cores (TMA-staged implicit GEMM, FP32 accumulators in tensor memory;
mma.sync for widths the tensor-core tiling does not take), their data and weight gradients, pooling,
upsampling, the loss and Adam on FP32 master weights.  This module only
allocates tensors and sequences the calls.

Architecture (channels; one 2x2 pooling per level):
  e0 = relu(conv(x, 16->16));  e1 = relu(conv(pool e0, 16->32));
  e2 = relu(conv(pool e1, 32->64));  b1 = relu(conv(pool e2, 64->128));
  b2 = relu(conv(b1, 128->64));  d2 = relu(conv([up b2, e2], 128->32));
  d1 = relu(conv([up d2, e1], 64->16));  d0 = relu(conv([up d1, e0], 32->16));
  y = conv(d0, 16->16), channels 0, 1 used.   ~225k trained parameters.
H and W must be divisible by 8.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import binding as B

LAYERS = (("e0", 16, 16), ("e1", 16, 32), ("e2", 32, 64), ("b1", 64, 128), ("b2", 128, 64),
          ("d2", 128, 32), ("d1", 64, 16), ("d0", 32, 16), ("out", 16, 16))
IN_CH = 16
OUT_USED = 2

_SIGS = {
    "pic_nn_conv3x3": "vivvvvi iiiiv",
    "pic_nn_conv3x3_mma_sync": "vivvvvi iiiiv",
    "pic_nn_conv_tc_status": "v",
    "pic_nn_flip_weights": "viivv",
    "pic_nn_conv3x3_wgrad": "viviiiivvvsv",
    "pic_nn_relu_bwd": "vvlv",
    "pic_nn_pool2": "vviiiiiv",
    "pic_nn_up2": "vviiiiiiv",
    "pic_nn_copy_channels": "viiviiliv",
    "pic_nn_mse": "vvliivvvv",
    "pic_nn_adam": "vvvvlffffivv",
    "pic_nn_add": "vvlv",
    "pic_nn_to_bf16": "vvlv",
    "pic_nn_pack_modes": "vviiivvvv",
    "pic_nn_unpack_modes": "vivfiiivv",
    "pic_nn_pack_target": "viiivvvv",
    "pic_nn_gather_batch": "vvvvilvvv",
    "pic_nn_restrict2": "viiivv",
    "pic_nn_prolong2": "viiivv",
    "pic_nn_minres_step": "vvvvliidvvvv",
}
_lib = None


def nn_lib():
    """The library with argument types of the pic_nn_* entry points."""
    global _lib
    if _lib is not None:
        return _lib
    lib = B.load()
    code = {"v": ctypes.c_void_p, "i": ctypes.c_int, "l": ctypes.c_long, "f": ctypes.c_float,
            "d": ctypes.c_double, "s": ctypes.c_size_t}
    for name, sig in _SIGS.items():
        sig = sig.replace(" ", "")
        f = getattr(lib, name)
        f.argtypes = [code[c] for c in sig]
        f.restype = ctypes.c_int
    lib.pic_nn_wgrad_scratch_floats.argtypes = [ctypes.c_int] * 5
    lib.pic_nn_wgrad_scratch_floats.restype = ctypes.c_size_t
    _lib = lib
    return lib


def P(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ok(status):
    if status != B.OK:
        raise B.PicPoissonError(status, B.last_error())


def _st():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class UNet:
    """Weights (FP32 master + BF16 copies), Adam state and the forward / backward passes."""

    def __init__(self, seed: int = 0, in_used: int = 3, device: str = "cuda"):
        self.device = device
        g = torch.Generator().manual_seed(seed)
        self.w, self.b, self.wb, self.wt = {}, {}, {}, {}
        self.gw, self.gb, self.m, self.v = {}, {}, {}, {}
        for name, cin, cout in LAYERS:
            fan_in = 9 * (in_used if name == "e0" else cin)
            w = torch.randn(9, cout, cin, generator=g, dtype=torch.float32) * math.sqrt(2.0 / fan_in)
            if name == "e0":
                w[:, :, in_used:] = 0.0
            if name == "out":
                w *= 0.1
                w[:, OUT_USED:, :] = 0.0
            self.w[name] = w.to(device)
            self.b[name] = torch.zeros(cout, dtype=torch.float32, device=device)
            self.wb[name] = torch.empty(9, cout, cin, dtype=torch.bfloat16, device=device)
            self.wt[name] = torch.empty(9, cin, cout, dtype=torch.bfloat16, device=device)
            self.gw[name] = torch.zeros_like(self.w[name])
            self.gb[name] = torch.zeros_like(self.b[name])
            for key in ("w", "b"):
                src = self.w[name] if key == "w" else self.b[name]
                self.m[(name, key)] = torch.zeros_like(src)
                self.v[(name, key)] = torch.zeros_like(src)
        self.steps = 0
        self._bufs = {}
        self.sync_bf16()

    def n_params(self):
        """Trained parameters (the padded input / output channels excluded)."""
        n = 0
        for name, cin, cout in LAYERS:
            ci = 3 if name == "e0" else cin
            co = OUT_USED if name == "out" else cout
            n += 9 * ci * co + co
        return n

    def sync_bf16(self):
        lib = nn_lib()
        for name, cin, cout in LAYERS:
            _ok(lib.pic_nn_to_bf16(P(self.w[name]), P(self.wb[name]), self.w[name].numel(), _st()))
            _ok(lib.pic_nn_flip_weights(P(self.wb[name]), cout, cin, P(self.wt[name]), _st()))

    def state(self):
        return {name: (self.w[name].detach().cpu().clone(), self.b[name].detach().cpu().clone())
                for name, _, _ in LAYERS}

    def load_state(self, st):
        for name, _, _ in LAYERS:
            self.w[name].copy_(st[name][0].to(self.device))
            self.b[name].copy_(st[name][1].to(self.device))
        self.sync_bf16()

    # ------------------------------------------------------------------ buffers
    def _buffers(self, n, h, w):
        key = (n, h, w)
        if key in self._bufs:
            return self._bufs[key]
        if h % 8 or w % 8:
            raise ValueError("U-Net input height and width must be divisible by 8")
        bf = dict(dtype=torch.bfloat16, device=self.device)
        s = {0: (h, w), 1: (h // 2, w // 2), 2: (h // 4, w // 4), 3: (h // 8, w // 8)}
        shapes = {"e0": (0, 16), "p0": (1, 16), "e1": (1, 32), "p1": (2, 32), "e2": (2, 64), "p2": (3, 64),
                  "b1": (3, 128), "b2": (3, 64), "c2": (2, 128), "d2": (2, 32), "c1": (1, 64), "d1": (1, 16),
                  "c0": (0, 32), "d0": (0, 16)}
        buf = {}
        for k, (lv, c) in shapes.items():
            hh, ww = s[lv]
            buf[k] = torch.empty(n, hh, ww, c, **bf)
            buf["g" + k] = torch.empty(n, hh, ww, c, **bf)
        buf["y"] = torch.empty(n, h, w, 16, dtype=torch.float32, device=self.device)
        buf["gy"] = torch.empty(n, h, w, 16, **bf)
        buf["tmp"] = torch.empty(n, h, w, 16, **bf)     # pooling adjoints (largest: level 0, 16 ch)
        lib = nn_lib()
        sizes = {"e0": (16, 16, 0), "e1": (16, 32, 1), "e2": (32, 64, 2), "b1": (64, 128, 3), "b2": (128, 64, 3),
                 "d2": (128, 32, 2), "d1": (64, 16, 1), "d0": (32, 16, 0), "out": (16, 16, 0)}
        need = max(lib.pic_nn_wgrad_scratch_floats(ci, co, n, *s[lv]) for ci, co, lv in sizes.values())
        buf["wg"] = torch.empty(int(need), dtype=torch.float32, device=self.device)
        buf["loss_scratch"] = torch.empty((n * h * w * 16 + 255) // 256, dtype=torch.float32, device=self.device)
        buf["loss"] = torch.zeros(1, dtype=torch.float32, device=self.device)
        buf["levels"] = s
        self._bufs[key] = buf
        return buf

    # ------------------------------------------------------------------ passes
    # pic_nn_conv3x3 (tcgen05 where the shape tiles) or pic_nn_conv3x3_mma_sync (legacy path, for comparison)
    conv_entry = "pic_nn_conv3x3"

    def _conv(self, name, x, cin, y, cout, n, hw, relu, y32=None, transposed=False):
        w = self.wt[name] if transposed else self.wb[name]
        bias = None if transposed else self.b[name]
        _ok(getattr(nn_lib(), self.conv_entry)(P(x), cin, P(w), P(bias), P(y), P(y32), cout, n, hw[0], hw[1],
                                               int(relu), _st()))

    def forward(self, x):
        """x: BF16 [n, h, w, 16]; returns the FP32 output [n, h, w, 16] (a buffer, reused)."""
        lib = nn_lib()
        n, h, w, _ = x.shape
        b = self._buffers(n, h, w)
        s = b["levels"]
        self._x = x
        st = _st()
        self._conv("e0", x, 16, b["e0"], 16, n, s[0], True)
        _ok(lib.pic_nn_pool2(P(b["e0"]), P(b["p0"]), n, *s[0], 16, 0, st))
        self._conv("e1", b["p0"], 16, b["e1"], 32, n, s[1], True)
        _ok(lib.pic_nn_pool2(P(b["e1"]), P(b["p1"]), n, *s[1], 32, 0, st))
        self._conv("e2", b["p1"], 32, b["e2"], 64, n, s[2], True)
        _ok(lib.pic_nn_pool2(P(b["e2"]), P(b["p2"]), n, *s[2], 64, 0, st))
        self._conv("b1", b["p2"], 64, b["b1"], 128, n, s[3], True)
        self._conv("b2", b["b1"], 128, b["b2"], 64, n, s[3], True)
        for lo, hi, cu, cs, src in ((3, 2, 64, 128, ("b2", "e2", "c2")), (2, 1, 32, 64, ("d2", "e1", "c1")),
                                    (1, 0, 16, 32, ("d1", "e0", "c0"))):
            up, skip, cat = src
            _ok(lib.pic_nn_up2(P(b[up]), P(b[cat]), n, *s[lo], cu, cs, 0, st))
            _ok(lib.pic_nn_copy_channels(P(b[skip]), cs - cu, 0, P(b[cat]), cs, cu, n * s[hi][0] * s[hi][1],
                                         cs - cu, st))
            dname = {"c2": "d2", "c1": "d1", "c0": "d0"}[cat]
            cout = {"d2": 32, "d1": 16, "d0": 16}[dname]
            self._conv(dname, b[cat], cs, b[dname], cout, n, s[hi], True)
        self._conv("out", b["d0"], 16, None, 16, n, s[0], False, y32=b["y"])
        return b["y"]

    def loss_backward(self, target):
        """MSE of output channels 0..1 against target FP32 [n, h, w, 2]; fills the gradients."""
        lib = nn_lib()
        x = self._x
        n, h, w, _ = x.shape
        b = self._buffers(n, h, w)
        s = b["levels"]
        st = _st()
        _ok(lib.pic_nn_mse(P(b["y"]), P(target), n * h * w, 16, OUT_USED, P(b["gy"]), P(b["loss_scratch"]),
                           P(b["loss"]), st))
        wg, nwg = b["wg"], b["wg"].numel()

        def wgrad(name, inp, cin, gout, cout, lv):
            _ok(lib.pic_nn_conv3x3_wgrad(P(inp), cin, P(gout), cout, n, *s[lv], P(self.gw[name]),
                                         P(self.gb[name]), P(wg), nwg, st))

        def relu_bwd(act, g):
            _ok(lib.pic_nn_relu_bwd(P(act), P(g), act.numel(), st))

        wgrad("out", b["d0"], 16, b["gy"], 16, 0)
        self._conv("out", b["gy"], 16, b["gd0"], 16, n, s[0], False, transposed=True)
        for dname, cat, cin, cout, lv, up, skip, cu in (("d0", "c0", 32, 16, 0, "d1", "e0", 16),
                                                        ("d1", "c1", 64, 16, 1, "d2", "e1", 32),
                                                        ("d2", "c2", 128, 32, 2, "b2", "e2", 64)):
            relu_bwd(b[dname], b["g" + dname])
            wgrad(dname, b[cat], cin, b["g" + dname], cout, lv)
            self._conv(dname, b["g" + dname], cout, b["g" + cat], cin, n, s[lv], False, transposed=True)
            pix = n * s[lv][0] * s[lv][1]
            _ok(lib.pic_nn_copy_channels(P(b["g" + cat]), cin, cu, P(b["g" + skip]), cin - cu, 0, pix, cin - cu, st))
            _ok(lib.pic_nn_up2(P(b["g" + cat]), P(b["g" + up]), n, *s[lv + 1], cu, cin, 1, st))
        relu_bwd(b["b2"], b["gb2"])
        wgrad("b2", b["b1"], 128, b["gb2"], 64, 3)
        self._conv("b2", b["gb2"], 64, b["gb1"], 128, n, s[3], False, transposed=True)
        relu_bwd(b["b1"], b["gb1"])
        wgrad("b1", b["p2"], 64, b["gb1"], 128, 3)
        self._conv("b1", b["gb1"], 128, b["gp2"], 64, n, s[3], False, transposed=True)
        for ename, pin, pname, cin, cout, lv in (("e2", "p1", "p2", 32, 64, 2), ("e1", "p0", "p1", 16, 32, 1),
                                                 ("e0", None, "p0", 16, 16, 0)):
            tmp = b["tmp"].view(-1)[: b[ename].numel()].view(b[ename].shape)
            _ok(lib.pic_nn_pool2(P(b["g" + pname]), P(tmp), n, *s[lv], cout, 1, st))
            _ok(lib.pic_nn_add(P(b["g" + ename]), P(tmp), tmp.numel(), st))
            relu_bwd(b[ename], b["g" + ename])
            wgrad(ename, x if pin is None else b[pin], cin, b["g" + ename], cout, lv)
            if pin is not None:
                self._conv(ename, b["g" + ename], cout, b["g" + pin], cin, n, s[lv], False, transposed=True)
        return b["loss"]

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        lib = nn_lib()
        self.steps += 1
        st = _st()
        for name, cin, cout in LAYERS:
            _ok(lib.pic_nn_adam(P(self.w[name]), P(self.gw[name]), P(self.m[(name, "w")]), P(self.v[(name, "w")]),
                                self.w[name].numel(), lr, b1, b2, eps, self.steps, P(self.wb[name]), st))
            _ok(lib.pic_nn_adam(P(self.b[name]), P(self.gb[name]), P(self.m[(name, "b")]), P(self.v[(name, "b")]),
                                self.b[name].numel(), lr, b1, b2, eps, self.steps, None, st))
            _ok(lib.pic_nn_flip_weights(P(self.wb[name]), cout, cin, P(self.wt[name]), st))
