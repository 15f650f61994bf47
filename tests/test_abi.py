"""Host-side checks of the C-ABI library (no GPU needed).

The library loads, exports every function include/pic_poisson.h declares, and
its host-only entry points (descriptor validation, multigrid hierarchy,
level-0 coefficients) behave as documented.  The coefficient builder is
pinned to the paper's worked stencil example and compared with the oracle's
independent coefficient routine.
"""
import ctypes
import dataclasses
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2609_07172_gb300 import binding as B, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "pic_poisson.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(pic_poisson_\w+)\s*\(", text, re.M)))


def test_library_exports_every_declared_function():
    lib = B.load()
    names = header_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.EXPORTS)


def test_query_hierarchy_paper_grid():
    q = B.query(W.c1_problem())
    assert q["levels"] == 5
    assert q["nr"] == [512, 256, 128, 64, 32]
    assert q["nz"] == [400, 200, 100, 50, 25]
    assert q["n_modes"] == 65
    # three complex FP64 vectors (u, b, b / diag) on every level dominate the workspace
    v0 = 512 * 400 * 65 * 16
    assert 3 * v0 < q["workspace_bytes"] < 3 * v0 * 1.5


def test_query_mixed_has_fp32_levels():
    q64 = B.query(W.c1_problem())
    qm = B.query(W.c1_problem(), precision=B.MIXED)
    assert qm["levels"] == q64["levels"]
    assert qm["workspace_bytes"] < q64["workspace_bytes"] * 1.5


@pytest.mark.parametrize("kw, why", [
    (dict(ntheta=12), "power of two"),
    (dict(ntheta=512), "power of two"),
    (dict(nr=0), "nr and nz"),
    (dict(r_in=0.0), "r_in"),
    (dict(r_in=0.06), "r_in"),
    (dict(z1=-1.0), "z0 < z1"),
    (dict(nr=127, nz=129), "direct-solve limit"),
])
def test_query_rejects_invalid(kw, why):
    base = dict(nr=32, ntheta=16, nz=32)
    base.update(kw)
    with pytest.raises(B.PicPoissonError) as ei:
        B.query(W.Problem(**base))
    assert ei.value.status == B.EINVAL
    assert why in str(ei.value)


def test_precision_and_sweeps_validated():
    d, _ = B.make_desc(W.c0_problem(), precision=7)
    assert B.load().pic_poisson_query(ctypes.byref(d), None) == B.EINVAL
    d, _ = B.make_desc(W.c0_problem(), pre_sweeps=0, post_sweeps=0)
    assert B.load().pic_poisson_query(ctypes.byref(d), None) == B.EINVAL
    lay = B.Layout()
    for prec in (B.FP64, B.MIXED):
        d, _ = B.make_desc(W.c0_problem(), precision=prec, inner_first=65)
        assert B.load().pic_poisson_query(ctypes.byref(d), ctypes.byref(lay)) == (B.EINVAL if prec == B.MIXED
                                                                                  else B.OK)
        d, _ = B.make_desc(W.c0_problem(), precision=prec, inner_first=64)
        assert B.load().pic_poisson_query(ctypes.byref(d), ctypes.byref(lay)) == B.OK


def test_cell_coeffs_worked_example(golden):
    """Library coefficient builder on the appendix's worked stencil cell."""
    g0 = golden("worked_stencil.txt")
    p = W.Problem(nr=3, ntheta=8, nz=3, r_in=0.5, r_out=3.5, z0=-0.5, z1=2.5)
    c = B.cell_coeffs(p, 1, 1)
    assert c[0:4] == pytest.approx([g0["G_r_minus"][0], g0["G_r_plus"][0], g0["G_z_minus"][0],
                                    g0["G_z_plus"][0]], rel=1e-15)
    assert c[4:8] == [0, 0, 0, 0]
    assert c[8] == pytest.approx(g0["mu"][0], rel=1e-15)
    assert c[9] * W.EPS0 == pytest.approx(g0["s_times_eps0"][0], rel=1e-15)
    assert c[10] == pytest.approx(g0["D0_interior"][0], rel=1e-15)
    # east Dirichlet face at r = 2.5: two radial cells, the second centred at r = 2
    pd = W.Problem(nr=2, ntheta=8, nz=3, r_in=0.5, r_out=2.5, z0=-0.5, z1=2.5, phi_r_out=7.0, phi_z0=0.0)
    cd = B.cell_coeffs(pd, 1, 1)
    assert cd[5] == 1 and cd[4] == 0
    assert cd[1] == pytest.approx(g0["GD_r_plus"][0], rel=1e-15)
    assert cd[10] == pytest.approx(g0["D0_dirichlet_east"][0], rel=1e-15)
    assert cd[11] == pytest.approx(g0["rhs_dirichlet_factor"][0] * 7.0, rel=1e-15)


@pytest.mark.parametrize("radial", ["uniform", "stretched"])
def test_cell_coeffs_match_oracle_everywhere(radial):
    """Every coefficient of every cell against the oracle's, on a uniform and
    on a geometrically stretched radial mesh (each cell 1.3 times the one
    inside it: the centre-to-centre and centre-to-wall distances differ)."""
    p = W.annulus(9, 8, 7, phi_r_in=3.0, phi_r_out=-2.0, phi_z0=11.0, phi_z1=5.0)
    if radial == "stretched":
        p = p.with_r_faces(W.stretched_radial_faces(p.r_in, p.r_out, p.nr, 1.3))
    g = oracle.grid_from_problem(p)
    b = oracle.rhs3d(g, np.zeros(p.shape))
    for k in range(p.nz):
        for i in range(p.nr):
            lib = np.array(B.cell_coeffs(p, i, k))
            orc = oracle.cell_coeffs(g, i, k)
            np.testing.assert_allclose(lib[0:4], orc["G"], rtol=1e-14)
            np.testing.assert_array_equal(lib[4:8].astype(bool), orc["dirichlet"])
            assert lib[8] == pytest.approx(orc["mu"], rel=1e-14)
            assert lib[9] == pytest.approx(orc["s"], rel=1e-14)
            assert lib[10] == pytest.approx(orc["D0"], rel=1e-14)
            assert lib[11] == pytest.approx(b[k, 0, i], rel=1e-14, abs=1e-12)


def test_cell_coeffs_rejects_outside():
    with pytest.raises(B.PicPoissonError):
        B.cell_coeffs(W.c0_problem(), 32, 0)


def test_batch_plan_rejects_mismatched_settings_before_touching_the_gpu():
    a, ka = B.make_desc(W.c0_problem())
    b, kb = B.make_desc(W.annulus(16, 8, 16), pre_sweeps=1)
    descs = (B.Desc * 2)(a, b)
    out = ctypes.c_void_p()
    assert B.load().pic_poisson_plan_batch(descs, 2, None, ctypes.byref(out)) == B.EINVAL
    assert "must match problem 0" in B.last_error()
    assert B.load().pic_poisson_plan_batch(descs, 0, None, ctypes.byref(out)) == B.EINVAL
    assert B.load().pic_poisson_plan_batch(descs, 65, None, ctypes.byref(out)) == B.EINVAL


def test_unknown_flags_rejected():
    d, _ = B.make_desc(W.c0_problem(), flags=64)
    assert B.load().pic_poisson_query(ctypes.byref(d), None) == B.EINVAL


def test_cell_coeffs_rejects_non_increasing_faces():
    p = W.annulus(8, 4, 8)
    bad = W.stretched_radial_faces(p.r_in, p.r_out, p.nr, 1.1)
    bad[3] = bad[2]
    with pytest.raises(B.PicPoissonError):
        B.cell_coeffs(p.with_r_faces(bad), 0, 0)


@pytest.mark.parametrize("field,value", [("theta_span", float("nan")), ("theta_span", float("inf")),
                                         ("r_in", float("nan")), ("r_out", float("inf")),
                                         ("z0", float("-inf")), ("z1", float("inf"))])
def test_non_finite_geometry_rejected(field, value):
    """Both the planned entry points and the no-allocation residual refuse
    non-finite geometry (a NaN span would otherwise propagate into lambda_m)."""
    p = dataclasses.replace(W.c0_problem(), **{field: value})
    d, _ = B.make_desc(p)
    assert B.load().pic_poisson_query(ctypes.byref(d), None) == B.EINVAL
    assert "finite" in B.last_error()


def test_library_exports_every_network_function():
    """Every entry point include/pic_poisson_nn.h declares (the learned warm
    start's kernels, the tcgen05 convolution and its status query) is exported."""
    text = open(os.path.join(ROOT, "include", "pic_poisson_nn.h")).read()
    names = sorted(set(re.findall(r"^\s*(?:int|size_t)\s*(pic_nn_\w+)\s*\(", text, re.M)))
    assert len(names) >= 18 and "pic_nn_conv3x3_mma_sync" in names and "pic_nn_conv_tc_status" in names
    lib = B.load()
    for n in names:
        assert hasattr(lib, n), n


def test_autotune_cache_key_separates_geometries(tmp_path):
    """The autotuner's cache key carries each problem's sizes and, when it has
    them, a digest of its face arrays and patches: the headline grid, the same
    grid with stretched axial faces and a composite domain of the same size are
    tuned apart, and a cached entry is returned without touching a GPU."""
    p = W.annulus(64, 16, 48)
    w = 1.02 ** np.arange(p.nz)
    q = p.with_z_faces(p.z0 + (p.z1 - p.z0) * np.r_[0.0, np.cumsum(w)] / w.sum())
    c = p.with_patches([(0, 32, 0, 48), (32, 64, 16, 32)], phi_exposed=12.0)
    keys = {B.tune_key([x], B.FP64, True, 1e-10) for x in (p, q, c)}
    assert len(keys) == 3
    assert B.tune_key([p], B.FP64, True, 1e-10) == B.tune_key([W.annulus(64, 16, 48)], B.FP64, True, 1e-10)
    assert B.tune_key([p], B.FP64, True, 1e-10) != B.tune_key([p], B.MIXED, True, 1e-10)
    cache = tmp_path / "tune.json"
    best = {"pre_sweeps": 1, "post_sweeps": 2, "inner_cycles": 2, "smooth_threads": 128, "smooth_strip": 0,
            "omega": 1.2, "smooth_fused": 0, "fmg": 0, "inner_first": 2}
    import json
    cache.write_text(json.dumps({B.tune_key([q], B.FP64, True, 1e-10): {"best": best, "ms": 1.0, "tried": []}}))
    assert B.autotune([q], [None], tol=1e-10, precision=B.FP64, graph=True, cache=str(cache)) == best
