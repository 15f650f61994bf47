"""Learned warm start: training pairs from the solver, training on the GPU, and
the warm-start step used between solves of a sequence.

Reading of the specification: the network sees the new charge density and
the previous-step potential through their mode residual
r_m = b_m - A_m phi_hat_(t-1),m (that residual is what a correction must
undo), plus a per-cell shift ratio that carries the mode index, and predicts
the correction phi_hat_t,m - phi_hat_(t-1),m.  Training pairs come from plain
solves of a drifting-wave sequence.  At a finer grid than the training grid
the residual is restricted 2:1 (finite-volume sum), the network runs on the
coarse grid and its correction is prolongated back -- a learned coarse-grid
correction.  The step length along the predicted direction d is chosen to
minimise the residual, alpha = <r, A d> / <A d, A d>, so the warm start is
never worse than the previous-step guess (alpha = 0 recovers it); the
multigrid then iterates to the same tolerance as without it.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np
import torch

from . import binding as B
from . import workloads as W
from .unet import P, UNet, _ok, _st, nn_lib


def shift_feature(p, dtype=np.float32):
    """Per-cell, per-mode input feature lambda_m mu_i / D_i (interior cell),
    shape (nz, nr, nm): the relative strength of mode m's diagonal shift."""
    nm = p.ntheta // 2 + 1
    dr = (p.r_out - p.r_in) / p.nr
    dz = (p.z1 - p.z0) / p.nz
    da = p.theta_span / p.ntheta
    r = p.r_centres()
    lam = 4.0 / da ** 2 * np.sin(np.pi * np.arange(nm) / p.ntheta) ** 2
    d_int = 2.0 * r * (dz / dr + dr / dz)
    ratio = (dr * dz / r)[:, None] * lam[None, :] / d_int[:, None]
    return np.ascontiguousarray(np.broadcast_to(ratio[None], (p.nz, p.nr, nm)), dtype=dtype)


def mode_rms(x):
    """Per-mode RMS over the cells of a mode-layout tensor (nz, nr, nm, 2)."""
    return x.pow(2).sum(dim=(0, 1, 3)).div(x.shape[0] * x.shape[1]).sqrt()


class Packer:
    """Device buffers that turn mode-layout residuals into network inputs."""

    def __init__(self, p, device="cuda"):
        self.p = p
        self.nm = p.ntheta // 2 + 1
        self.shift = torch.from_numpy(shift_feature(p)).to(device)
        self.rms = torch.empty(self.nm, dtype=torch.float32, device=device)
        self.scratch = torch.empty(256 * self.nm + 2048, dtype=torch.float64, device=device)
        self.x = torch.empty(self.nm, p.nz, p.nr, 16, dtype=torch.bfloat16, device=device)

    def pack(self, r):
        _ok(nn_lib().pic_nn_pack_modes(P(r), P(self.shift), self.p.nr, self.p.nz, self.nm, P(self.rms),
                                       P(self.scratch), P(self.x), _st()))
        return self.x, self.rms


def training_pairs(p, steps, seed=7, limit=None, tol=1e-11):
    """Pairs (network input, normalised correction) from plain FP64 solves of the
    drifting-wave sequence on problem p (`steps` steps, N_theta/2+1 modes each).
    Returns X (BF16 [n, nz, nr, 16]), Y (FP32 [n, nz, nr, 2]) and a gain.
    Each target is the correction scaled to unit RMS: the network learns the
    direction of the correction; its length is set at use by the
    minimal-residual step, so the returned gain is 1."""
    dev = torch.device("cuda")
    pk = Packer(p)
    nm = pk.nm
    xs, es, rr = [], [], []
    rms_t = torch.empty(nm, dtype=torch.float32, device=dev)   # the targets' per-mode RMS
    with B.Plan(p, graph=True) as plan:
        uprev = torch.zeros(plan.mode_shape, dtype=torch.float64, device=dev)
        for t in range(steps):
            rho = torch.from_numpy(W.drifting_rho(p, t, base_seed=seed)).to(dev)
            bhat = plan.forward(rho)
            r, _ = plan.mode_residual(uprev, bhat, want_r=True)
            plan.solve(rho, tol=tol)
            u = plan.get_modes()
            e = u - uprev
            x, rms_r = pk.pack(r)
            xs.append(x.clone())
            rr.append(rms_r.clone())
            y = torch.empty(nm, p.nz, p.nr, 2, dtype=torch.float32, device=dev)
            _ok(nn_lib().pic_nn_pack_target(P(e), p.nr, p.nz, nm, P(rms_t), P(pk.scratch), P(y), _st()))
            es.append(y)
            uprev = u
    X = torch.cat(xs)
    Y = torch.cat(es)
    gain = 1.0
    if limit:
        X, Y = X[:limit], Y[:limit]
    return X.contiguous(), Y.contiguous(), gain


def train(net, X, Y, epochs=20, batch=16, lr=1e-3, seed=0, log=None):
    """Adam on MSE with random sign flips (the correction is odd in the residual);
    returns the mean loss of every epoch."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    pix = X.shape[1] * X.shape[2]
    steps = max(1, n // batch) * epochs
    losses = []
    t0 = time.time()
    k = 0
    xb = torch.empty((batch,) + tuple(X.shape[1:]), dtype=X.dtype, device=X.device)
    yb = torch.empty((batch,) + tuple(Y.shape[1:]), dtype=Y.dtype, device=Y.device)
    for ep in range(epochs):
        ep_losses = []
        perm = torch.randperm(n, generator=g)
        for s in range(n // batch):
            # the batch's sample order and sign flips are drawn on the host;
            # the gather and the flips run in a kernel
            idx = perm[s * batch:(s + 1) * batch].to(torch.int64).to(X.device)
            sign = (torch.randint(0, 2, (batch,), generator=g) * 2 - 1).float().to(X.device)
            _ok(nn_lib().pic_nn_gather_batch(P(X), P(Y), P(idx), P(sign), batch, pix, P(xb), P(yb), _st()))
            net.forward(xb)
            loss = net.loss_backward(yb)
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * k / steps))
            net.adam(cur)
            k += 1
            ep_losses.append(loss.clone())
        losses.append(float(torch.stack(ep_losses).mean().item()))
        if log:
            log(f"epoch {ep}: mean loss {losses[-1]:.4f} ({time.time() - t0:.1f} s)")
    return losses


class WarmStart:
    """The learned initial iterate for a solver plan on problem p (training
    grid or twice it in r and z), driven by a trained UNet."""

    def __init__(self, net, gain, p, plan, coarse=True):
        self.net, self.gain, self.p, self.plan = net, float(gain), p, plan
        self.coarse = coarse
        dev = torch.device("cuda")
        self.nm = p.ntheta // 2 + 1
        pc = W.annulus(p.nr // 2, p.ntheta, p.nz // 2, r_in=p.r_in, r_out=p.r_out, z0=p.z0, z1=p.z1,
                       theta_span=p.theta_span) if coarse else p
        self.pc = pc
        self.packer = Packer(pc)
        f64 = dict(dtype=torch.float64, device=dev)
        self.r = torch.empty(plan.mode_shape, **f64)
        self.rc = torch.empty(pc.nz, pc.nr, self.nm, 2, **f64) if coarse else self.r
        self.dc = torch.empty(pc.nz, pc.nr, self.nm, 2, **f64)
        self.d = torch.empty(plan.mode_shape, **f64) if coarse else self.dc
        self.bd = torch.empty(plan.mode_shape, **f64)
        self.zero = torch.zeros(plan.mode_shape, **f64)
        self.guess_buf = torch.empty(plan.mode_shape, **f64)
        self.scratch = torch.empty(2048, **f64)
        self.alpha = torch.zeros(1, **f64)

    def guess(self, bhat, uprev):
        """phi_hat_(t-1) + alpha d for the new right-hand side bhat (all on the device, no sync)."""
        lib = nn_lib()
        st = _st()
        p, pc, nm = self.p, self.pc, self.nm
        _ok(B.load().pic_poisson_mode_residual(self.plan._plan, P(uprev), P(bhat), P(self.r), None))
        if self.coarse:
            _ok(lib.pic_nn_restrict2(P(self.r), p.nr, p.nz, nm, P(self.rc), st))
        x, rms = self.packer.pack(self.rc)
        y = self.net.forward(x)
        _ok(lib.pic_nn_unpack_modes(P(y), 16, P(rms), self.gain, pc.nr, pc.nz, nm, P(self.dc), st))
        if self.coarse:
            _ok(lib.pic_nn_prolong2(P(self.dc), p.nr, p.nz, nm, P(self.d), st))
        return self._step(uprev)

    def _step(self, uprev):
        """uprev + alpha d, alpha minimising the residual (self.r holds b - A uprev)."""
        _ok(B.load().pic_poisson_mode_residual(self.plan._plan, P(self.d), P(self.zero), P(self.bd), None))
        _ok(nn_lib().pic_nn_minres_step(P(uprev), P(self.d), P(self.r), P(self.bd), self.r.numel() // 2, self.nm,
                                        self.p.ntheta, -1.0, P(self.scratch), P(self.guess_buf), P(self.alpha),
                                        _st()))
        return self.guess_buf

    def coarse_bound(self, bhat, uprev, ucur):
        """The best guess a predictor on the network's 2:1 coarse grid could
        give: the exact correction ucur - uprev of this step (ucur the solved
        modes), averaged onto the coarse grid and prolongated back, then the
        same minimal-residual step -- an upper bound on what the learned
        correction can achieve, since the network outputs coarse-grid fields."""
        lib = nn_lib()
        st = _st()
        p, nm = self.p, self.nm
        _ok(B.load().pic_poisson_mode_residual(self.plan._plan, P(uprev), P(bhat), P(self.r), None))
        torch.sub(ucur, uprev, out=self.d)
        if self.coarse:
            _ok(lib.pic_nn_restrict2(P(self.d), p.nr, p.nz, nm, P(self.dc), st))
            self.dc.mul_(0.25)   # the restriction sums the four fine cells: their average
            _ok(lib.pic_nn_prolong2(P(self.dc), p.nr, p.nz, nm, P(self.d), st))
        return self._step(uprev)


def evaluate_sequence(net, gain, p, steps, tol=1e-10, coarse=True, gpu_inputs=True, seed=3, precision=B.FP64,
                      bound=False):
    """Drifting-wave sequence solved back to back from (a) the previous-step
    guess and (b) the learned warm start; per-step cycles and device ms
    (the learned side includes its forward transform, residual, inference and
    step).  With bound, also (c) the coarse-grid predictor bound of
    WarmStart.coarse_bound (not timed: it uses the step's solution).  Returns a
    dict of summaries and per-step records."""
    dev = torch.device("cuda")
    base = B.Plan(p, graph=True, precision=precision)
    lrn = B.Plan(p, graph=True, precision=precision)
    ws = WarmStart(net, gain, p, lrn, coarse=coarse)
    ub = torch.zeros(base.mode_shape, dtype=torch.float64, device=dev)
    ul = torch.zeros_like(ub)
    ub_prev = torch.zeros_like(ub)
    ucur = torch.zeros_like(ub)
    phi = torch.empty(p.shape, dtype=torch.float64, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rec = []
    for t in range(steps):
        rho = (W.drifting_rho_torch(p, t, base_seed=seed) if gpu_inputs
               else torch.from_numpy(W.drifting_rho(p, t, base_seed=seed)).to(dev))
        torch.cuda.synchronize()
        e0.record()
        _, ib = base.solve_modes(rho, ub, phi, tol=tol)
        e1.record()
        torch.cuda.synchronize()
        ms_b = e0.elapsed_time(e1)
        base.get_modes(ub)
        e0.record()
        bhat = lrn.forward(rho)
        g = ws.guess(bhat, ul)
        _, il = lrn.solve_modes(rho, g, phi, tol=tol)
        e1.record()
        torch.cuda.synchronize()
        ms_l = e0.elapsed_time(e1)
        lrn.get_modes(ul)
        r = {"t": t, "cycles_prev": ib["cycles"], "cycles_learned": il["cycles"],
             "rel0_prev": ib["rel_res0"], "rel0_learned": il["rel_res0"], "ms_prev": ms_b,
             "ms_learned": ms_l, "alpha": float(ws.alpha.item()),
             "ok": ib["status"] == B.OK and il["status"] == B.OK}
        if bound and t > 0:   # the coarse-grid predictor bound, from the previous step's base solution
            gb = ws.coarse_bound(bhat, ub_prev, base.get_modes(ucur))
            _, ibd = lrn.solve_modes(rho, gb, phi, tol=tol)
            r.update(cycles_bound=ibd["cycles"], rel0_bound=ibd["rel_res0"])
        if bound:
            base.get_modes(ub_prev)
        rec.append(r)
    base.close()
    lrn.close()
    body = rec[1:]     # step 0 starts both from zero
    mean = lambda k: sum(r[k] for r in body) / len(body)
    out = {"steps": steps, "cycles_prev": mean("cycles_prev"), "cycles_learned": mean("cycles_learned"),
           "ms_prev": mean("ms_prev"), "ms_learned": mean("ms_learned"),
           "rel0_prev": mean("rel0_prev"), "rel0_learned": mean("rel0_learned"),
           "alpha_mean": mean("alpha"), "all_converged": all(r["ok"] for r in rec), "records": rec}
    if bound:
        out.update(cycles_coarse_bound=mean("cycles_bound"), rel0_coarse_bound=mean("rel0_bound"))
    return out
