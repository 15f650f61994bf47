"""Learned warm start (GPU): network kernels vs the FP64 CPU oracle, training,
and what the trained network gains over the previous-step guess.

The U-Net runs in BF16 with FP32 accumulation, so its outputs and gradients
agree with the FP64 oracle to BF16 accuracy (relative errors of a few 1e-3
per layer); the tolerances below allow for that.
"""
import ctypes
import math

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from oracle import unet_ref
from paper_2609_07172_gb300 import FP64, MIXED, Plan, binding as B, workloads as W
from paper_2609_07172_gb300 import learned as LW
from paper_2609_07172_gb300.unet import LAYERS, P, UNet, _ok, _st, nn_lib

pytestmark = pytest.mark.gpu


def bf(x):
    return x.to(torch.bfloat16)


def rel(a, b):
    return float((a - b).norm() / b.norm())


def conv_ref(x, w, b):
    """x [n,h,w,ci], w [9][co][ci] (float64) -> [n,h,w,co] via the CPU conv2d."""
    k = w.permute(1, 2, 0).reshape(w.shape[1], w.shape[2], 3, 3)
    return F.conv2d(x.permute(0, 3, 1, 2), k, b, padding=1).permute(0, 2, 3, 1)


@pytest.mark.parametrize("cin,cout", [(16, 16), (32, 64), (128, 32), (64, 128), (16, 8)])
def test_conv3x3_matches_cpu(cin, cout):
    g = torch.Generator().manual_seed(cin * 7 + cout)
    n, h, w = 3, 10, 13                       # ragged: 390 pixels is not a multiple of 64
    x = bf(torch.randn(n, h, w, cin, generator=g))
    wt = bf(torch.randn(9, cout, cin, generator=g) / math.sqrt(9 * cin))
    bias = torch.randn(cout, generator=g)
    out = torch.empty(n, h, w, cout, dtype=torch.bfloat16, device="cuda")
    out32 = torch.empty(n, h, w, cout, dtype=torch.float32, device="cuda")
    xc, wc, bc = x.cuda(), wt.cuda(), bias.cuda()
    _ok(nn_lib().pic_nn_conv3x3(P(xc), cin, P(wc), P(bc), P(out), P(out32), cout, n, h, w, 1, _st()))
    ref = torch.relu(conv_ref(x.double(), wt.double(), bias.double()))
    assert rel(out32.cpu().double(), ref) < 1e-5            # FP32 accumulation of exact BF16 products
    assert rel(out.cpu().double(), ref) < 1e-2              # BF16 output rounding


def tc_status():
    st = ctypes.c_int(-1)
    _ok(nn_lib().pic_nn_conv_tc_status(ctypes.byref(st)))
    return st.value


# widths the tcgen05 tiling takes: 128 pixels of a row (w a multiple of 128) or
# 128 / w whole rows (w = 16, 32, 64; ragged last row block when h % (128 / w) != 0)
TC_SHAPES = [(2, 5, 256), (3, 9, 128), (2, 7, 64), (2, 25, 32), (1, 11, 16)]
TC_CHANNELS = [(16, 16), (16, 32), (32, 64), (64, 128), (128, 64), (128, 32), (64, 16), (32, 16), (16, 48)]


@pytest.mark.parametrize("cin,cout", TC_CHANNELS)
@pytest.mark.parametrize("n,h,w", TC_SHAPES)
def test_conv3x3_tcgen05_matches_cpu_and_mma_sync(n, h, w, cin, cout):
    """The tcgen05 implicit GEMM (TMA zero fill as the padding, FP32 in TMEM)
    against the FP64 CPU convolution and against the mma.sync kernel."""
    g = torch.Generator().manual_seed(n * 1000 + h * 100 + w + cin * 7 + cout)
    x = bf(torch.randn(n, h, w, cin, generator=g))
    wt = bf(torch.randn(9, cout, cin, generator=g) / math.sqrt(9 * cin))
    bias = torch.randn(cout, generator=g)
    xc, wc, bc = x.cuda(), wt.cuda(), bias.cuda()
    outs = {}
    for name in ("pic_nn_conv3x3", "pic_nn_conv3x3_mma_sync"):
        out = torch.full((n, h, w, cout), float("nan"), dtype=torch.bfloat16, device="cuda")
        out32 = torch.full((n, h, w, cout), float("nan"), dtype=torch.float32, device="cuda")
        _ok(getattr(nn_lib(), name)(P(xc), cin, P(wc), P(bc), P(out), P(out32), cout, n, h, w, 1, _st()))
        torch.cuda.synchronize()
        outs[name] = (out.cpu(), out32.cpu())
    assert tc_status() == 0
    ref = torch.relu(conv_ref(x.double(), wt.double(), bias.double()))
    out, out32 = outs["pic_nn_conv3x3"]
    assert torch.isfinite(out32).all() and torch.isfinite(out.float()).all()
    assert rel(out32.double(), ref) < 1e-5
    assert rel(out.double(), ref) < 1e-2
    # the same sums in another order: FP32 rounding apart
    assert rel(out32.double(), outs["pic_nn_conv3x3_mma_sync"][1].double()) < 1e-5
    # no ReLU, FP32 output only (the data-gradient convolution's form)
    out32b = torch.full((n, h, w, cout), float("nan"), dtype=torch.float32, device="cuda")
    _ok(nn_lib().pic_nn_conv3x3(P(xc), cin, P(wc), None, None, P(out32b), cout, n, h, w, 0, _st()))
    torch.cuda.synchronize()
    assert tc_status() == 0
    assert rel(out32b.cpu().double(), conv_ref(x.double(), wt.double(), None)) < 1e-5


def test_conv_gradients_match_autograd():
    g = torch.Generator().manual_seed(5)
    n, h, w, cin, cout = 2, 12, 16, 32, 16
    x = bf(torch.randn(n, h, w, cin, generator=g))
    wt = bf(torch.randn(9, cout, cin, generator=g) / math.sqrt(9 * cin))
    dy = bf(torch.randn(n, h, w, cout, generator=g))
    lib = nn_lib()
    xc, wc, dyc = x.cuda(), wt.cuda(), dy.cuda()
    wflip = torch.empty(9, cin, cout, dtype=torch.bfloat16, device="cuda")
    _ok(lib.pic_nn_flip_weights(P(wc), cout, cin, P(wflip), _st()))
    dx32 = torch.empty(n, h, w, cin, dtype=torch.float32, device="cuda")
    _ok(lib.pic_nn_conv3x3(P(dyc), cout, P(wflip), None, None, P(dx32), cin, n, h, w, 0, _st()))
    need = lib.pic_nn_wgrad_scratch_floats(cin, cout, n, h, w)
    scratch = torch.empty(int(need), dtype=torch.float32, device="cuda")
    dw = torch.empty(9, cout, cin, dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    _ok(lib.pic_nn_conv3x3_wgrad(P(xc), cin, P(dyc), cout, n, h, w, P(dw), P(db), P(scratch), need, _st()))
    xr = x.double().requires_grad_(True)
    wr = wt.double().requires_grad_(True)
    br = torch.zeros(cout, dtype=torch.float64, requires_grad=True)
    y = conv_ref(xr, wr, br)
    (y * dy.double()).sum().backward()
    assert rel(dx32.cpu().double(), xr.grad) < 1e-5
    assert rel(dw.cpu().double(), wr.grad) < 1e-5
    assert rel(db.cpu().double(), br.grad) < 1e-5


def test_pool_and_upsample_adjoints():
    g = torch.Generator().manual_seed(9)
    n, h, w, c = 2, 8, 12, 16
    lib = nn_lib()
    a = bf(torch.randn(n, h, w, c, generator=g)).cuda()
    bsmall = bf(torch.randn(n, h // 2, w // 2, c, generator=g)).cuda()
    pa = torch.empty_like(bsmall)
    _ok(lib.pic_nn_pool2(P(a), P(pa), n, h, w, c, 0, _st()))
    pb = torch.empty_like(a)
    _ok(lib.pic_nn_pool2(P(bsmall), P(pb), n, h, w, c, 1, _st()))
    lhs = (pa.double() * bsmall.double()).sum()
    rhs = (a.double() * pb.double()).sum()
    assert float(lhs) == pytest.approx(float(rhs), rel=2e-2)
    ua = torch.empty_like(a)
    _ok(lib.pic_nn_up2(P(bsmall), P(ua), n, h // 2, w // 2, c, c, 0, _st()))
    ub = torch.empty_like(bsmall)
    _ok(lib.pic_nn_up2(P(a), P(ub), n, h // 2, w // 2, c, c, 1, _st()))
    assert float((ua.double() * a.double()).sum()) == pytest.approx(float((bsmall.double() * ub.double()).sum()),
                                                                    rel=2e-2)


def test_unet_forward_and_gradients_match_oracle():
    net = UNet(seed=3)
    g = torch.Generator().manual_seed(11)
    n, h, w = 2, 16, 24
    x = torch.zeros(n, h, w, 16)
    x[..., :3] = torch.randn(n, h, w, 3, generator=g)
    x = bf(x).cuda()
    target = torch.randn(n, h, w, 2, generator=g).cuda()
    y = net.forward(x)
    loss = net.loss_backward(target)
    torch.cuda.synchronize()
    params = {name: (net.wb[name].double().cpu(), net.b[name].double().cpu()) for name, _, _ in LAYERS}
    lref, yref, gref = unet_ref.loss_and_grads(params, x.double().cpu().permute(0, 3, 1, 2),
                                               target.double().cpu().permute(0, 3, 1, 2))
    assert rel(y.double().cpu().permute(0, 3, 1, 2)[:, :2], yref[:, :2]) < 3e-2
    assert float(loss.item()) == pytest.approx(lref, rel=3e-2)
    # BF16 activations and gradients between ~20 layers: per-layer gradients
    # agree to ~10 % in norm with cosine similarity > 0.99; an indexing or
    # wiring error gives O(1) differences and low similarity.
    stats = {}
    for name, _, _ in LAYERS:
        gw, gb = gref[name]
        a = net.gw[name].double().cpu()
        cos = float((a * gw).sum() / (a.norm() * gw.norm()))
        stats[name] = (rel(a, gw), cos)
        if gb.norm() > 0:
            stats[name + ".b"] = (rel(net.gb[name].double().cpu(), gb), 1.0)
    assert max(r for r, _ in stats.values()) < 0.15, stats
    assert min(c for _, c in stats.values()) > 0.99, stats


def test_training_reduces_loss_and_warm_start_beats_previous_guess():
    """Train on a small drifting-wave sequence, then solve a finer sequence:
    the learned step removes more of the initial residual than the
    previous-step guess, and never adds to it (minimal-residual step)."""
    pt = W.annulus(64, 16, 48)                 # training grid (H = 48, W = 64)
    X, Y, gain = LW.training_pairs(pt, steps=12, seed=7)
    net = UNet(seed=0)
    losses = LW.train(net, X, Y, epochs=12, batch=8, lr=2e-3)
    assert losses[-1] < 0.7 * losses[0]
    pe = W.annulus(128, 16, 96)                # evaluation grid: the training grid refined 2x in r and z
    res = LW.evaluate_sequence(net, gain, pe, steps=6, coarse=True, gpu_inputs=False)
    assert res["all_converged"]
    assert res["rel0_learned"] < res["rel0_prev"]
    assert res["cycles_learned"] <= res["cycles_prev"]
    with Plan(pe) as plan:                     # the step never increases the residual
        ws = LW.WarmStart(net, gain, pe, plan)
        rho0 = torch.from_numpy(W.drifting_rho(pe, 0)).cuda()
        rho1 = torch.from_numpy(W.drifting_rho(pe, 1)).cuda()
        plan.solve(rho0, tol=1e-10)
        u0 = plan.get_modes()
        b1 = plan.forward(rho1)
        _, r_prev = plan.mode_residual(u0, b1)
        gu = ws.guess(b1, u0)
        _, r_new = plan.mode_residual(gu, b1)
    assert r_new <= r_prev * (1 + 1e-12)


def test_training_target_and_batch_gather_kernels():
    """pic_nn_pack_target (per-mode unit-RMS FP32 targets) and
    pic_nn_gather_batch (sample gather with sign flips) against plain torch."""
    lib = nn_lib()
    nr, nz, nm = 24, 16, 9
    g = torch.Generator(device="cpu").manual_seed(8)
    x = torch.randn(nz, nr, nm, 2, generator=g, dtype=torch.float64).cuda() * torch.arange(1, nm + 1).view(1, 1, nm, 1).cuda()
    rms = torch.empty(nm, dtype=torch.float32, device="cuda")
    scratch = torch.empty(256 * nm, dtype=torch.float64, device="cuda")
    y = torch.empty(nm, nz, nr, 2, dtype=torch.float32, device="cuda")
    _ok(lib.pic_nn_pack_target(P(x), nr, nz, nm, P(rms), P(scratch), P(y), _st()))
    em = x.permute(2, 0, 1, 3)
    comp_rms = em.pow(2).mean(dim=(1, 2, 3)).sqrt()          # per real component
    assert torch.allclose(rms.double(), comp_rms * 2 ** 0.5, rtol=1e-6)   # of |x|
    assert torch.allclose(y.double(), em / comp_rms.view(nm, 1, 1, 1), rtol=1e-6, atol=1e-6)
    # gather with signs
    n, pix = 7, nz * nr
    X = torch.randn(n, nz, nr, 16, generator=g).to(torch.bfloat16).cuda()
    Y = torch.randn(n, nz, nr, 2, generator=g).cuda()
    idx = torch.tensor([5, 0, 3, 3], dtype=torch.int64).cuda()
    sign = torch.tensor([1.0, -1.0, -1.0, 1.0]).cuda()
    xb = torch.empty(4, nz, nr, 16, dtype=torch.bfloat16, device="cuda")
    yb = torch.empty(4, nz, nr, 2, device="cuda")
    _ok(lib.pic_nn_gather_batch(P(X), P(Y), P(idx), P(sign), 4, pix, P(xb), P(yb), _st()))
    torch.cuda.synchronize()
    want_x = X[idx].clone()
    want_x[..., :2] *= sign.view(-1, 1, 1, 1).to(torch.bfloat16)
    assert torch.equal(xb, want_x)
    assert torch.equal(yb, Y[idx] * sign.view(-1, 1, 1, 1))
