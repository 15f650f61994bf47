"""The no-allocation residual entry point agrees with the planned one (GPU).

pic_poisson_mode_residual_noalloc serves callers that cannot call cudaMalloc
(for example a PIC code whose particle arrays own all device memory, or a
step loop that may not synchronise the device): it takes no plan and keeps
its partial sums in a fixed device array.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import ctypes
import dataclasses
import math

import numpy as np
import pytest
import torch

from helpers import to_modes, with_bias_walls
from paper_2609_07172_gb300 import Plan, binding as B, workloads as W

pytestmark = pytest.mark.gpu


def call_noalloc(p, uhat, bhat, rhat, rel):
    d, keep = B.make_desc(p)
    st = torch.cuda.current_stream().cuda_stream
    status = B.load().pic_poisson_mode_residual_noalloc(
        ctypes.byref(d), ctypes.c_void_p(uhat.data_ptr()), ctypes.c_void_p(bhat.data_ptr()),
        ctypes.c_void_p(rhat.data_ptr()) if rhat is not None else None,
        ctypes.c_void_p(rel.data_ptr()), ctypes.c_void_p(st))
    del keep
    return status


@pytest.mark.parametrize("dims,span", [
    ((96, 16, 40), None), ((512, 128, 200), None),
    # one and two axial rows (the 4- and 3-term Dirichlet axial coefficients),
    # ntheta = 2 (m = 1 is the Nyquist mode, Parseval weight 1) and a
    # quarter-annulus period (lambda_m from dalpha = span / ntheta)
    ((8, 2, 1), None), ((8, 4, 2), None), ((16, 8, 6), math.pi / 2)],
    ids=["96x16x40", "512x128x200", "8x2x1", "8x4x2", "16x8x6_quarter"])
def test_noalloc_residual_matches_planned_twice(dims, span):
    kw = {} if span is None else {"theta_span": span}
    p = with_bias_walls(W.annulus(*dims, **kw))
    rng = np.random.default_rng(21)
    rho = torch.from_numpy(W.rho_plasma(p, seed=13)).cuda()
    with Plan(p) as plan:
        bhat = plan.forward(rho)
        for call in range(2):       # the scratch array keeps the previous call's contents
            uhat = torch.from_numpy(to_modes(rng.standard_normal(p.shape) * (10.0 + 90.0 * call))).cuda()
            r_ref, rel_ref = plan.mode_residual(uhat, bhat)
            r_na = torch.full_like(r_ref, float("nan"))
            rel_na = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            assert call_noalloc(p, uhat, bhat, r_na, rel_na) == B.OK, B.last_error()
            torch.cuda.synchronize()
            scale = r_ref.abs().max().item()
            assert torch.allclose(r_na, r_ref, rtol=0, atol=1e-12 * scale)
            assert rel_na.item() == pytest.approx(rel_ref, rel=1e-12)
            # norm only (no residual output)
            rel2 = torch.zeros(1, dtype=torch.float64, device="cuda")
            assert call_noalloc(p, uhat, bhat, None, rel2) == B.OK
            torch.cuda.synchronize()
            assert rel2.item() == rel_na.item()


def test_noalloc_rejects_oversize_problem():
    p = W.annulus(512, 256, 512)     # 512 * 512 * 129 entries > 16,777,216
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    status = call_noalloc(p, dummy, dummy, None, dummy)
    assert status == B.EINVAL
    assert "at most 16777216 mode entries" in B.last_error()


@pytest.mark.parametrize("field,value", [("theta_span", float("nan")), ("theta_span", float("inf")),
                                         ("r_out", float("inf")), ("z1", float("inf"))])
def test_noalloc_rejects_non_finite_geometry(field, value):
    p = dataclasses.replace(W.annulus(16, 8, 6), **{field: value})
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    assert call_noalloc(p, dummy, dummy, None, dummy) == B.EINVAL
    assert "finite" in B.last_error()
