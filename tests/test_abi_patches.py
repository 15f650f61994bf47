"""Composite-domain descriptors through the C ABI (host only, no GPU).

The library's coefficient builder against the oracle's on every cell of
channel-plume domains; protected faces in the hierarchy the plan would build;
and the descriptor checks.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2609_07172_gb300 import MIXED, binding as B, workloads as W


def _cp(radial):
    p = W.channel_plume(16, 8, 12, phi_r_in=3.0, phi_r_out=-2.0, phi_z0=11.0, phi_z1=5.0)
    p = p.with_patches(p.patches + ((12, 16, 2, 4),), 7.5)   # and an island patch
    if radial == "stretched":
        p = p.with_r_faces(W.stretched_radial_faces(p.r_in, p.r_out, p.nr, 1.2))
    return p


@pytest.mark.parametrize("radial", ["uniform", "stretched"])
def test_patch_cell_coeffs_match_oracle_everywhere(radial):
    p = _cp(radial)
    g = oracle.grid_from_problem(p)
    b = oracle.rhs3d(g, np.zeros(p.shape))
    act = p.active_cells()
    for k in range(p.nz):
        for i in range(p.nr):
            lib = np.array(B.cell_coeffs(p, i, k))
            orc = oracle.cell_coeffs(g, i, k)
            if not act[k, i]:
                assert np.all(lib == 0.0)
                continue
            np.testing.assert_allclose(lib[0:4], orc["G"], rtol=1e-14)
            np.testing.assert_array_equal(lib[4:8].astype(bool), orc["dirichlet"])
            assert lib[8] == pytest.approx(orc["mu"], rel=1e-14)
            assert lib[9] == pytest.approx(orc["s"], rel=1e-14)
            assert lib[10] == pytest.approx(orc["D0"], rel=1e-14)
            assert lib[11] == pytest.approx(b[k, 0, i], rel=1e-14, abs=1e-12)


def test_hierarchy_keeps_patch_edges_on_coarse_faces():
    for p in (W.channel_plume(512, 8, 384), W.channel_plume(64, 8, 48), _cp("uniform")):
        lay = B.query(p)
        for l in range(lay["levels"]):
            sr, sz = p.nr // lay["nr"][l], p.nz // lay["nz"][l]
            for (i0, i1, k0, k1) in p.patches:
                assert i0 % sr == 0 and i1 % sr == 0 and k0 % sz == 0 and k1 % sz == 0, (l, sr, sz)
    # a patch edge at an odd cell stops coarsening in that direction at once
    p = W.annulus(32, 8, 24).with_patches([(0, 32, 0, 11), (0, 16, 11, 24)])
    lay = B.query(p)
    assert all(nz == 24 for nz in lay["nz"][:lay["levels"]])


@pytest.mark.parametrize("patches,why", [
    ([(0, 8, 0, 8), (4, 12, 4, 12)], "overlap"),
    ([(0, 17, 0, 8)], "inside"),
    ([(3, 3, 0, 8)], "non-empty"),
    ([(-1, 4, 0, 8)], "inside"),
])
def test_invalid_patches_rejected(patches, why):
    p = W.annulus(16, 8, 16).with_patches(patches)
    d, _ = B.make_desc(p)
    assert B.load().pic_poisson_query(ctypes.byref(d), ctypes.byref(B.Layout())) == B.EINVAL
    assert why in B.last_error()


def test_patch_limits_and_settings_rejected():
    lay = B.Layout()
    # 65 patches
    p = W.annulus(130, 8, 8).with_patches([(2 * a, 2 * a + 2, 0, 8) for a in range(65)])
    d, _ = B.make_desc(p)
    assert B.load().pic_poisson_query(ctypes.byref(d), ctypes.byref(lay)) == B.EINVAL
    # the fused smoother takes composite domains (per-row coefficient classes)
    d, _ = B.make_desc(W.channel_plume(64, 8, 48), precision=MIXED, smooth_fused=1)
    assert B.load().pic_poisson_query(ctypes.byref(d), ctypes.byref(lay)) == B.OK
    # patch edges on odd cells leave a coarsest level beyond the dense limit
    p = W.annulus(256, 8, 64).with_patches([(1, 255, 1, 63)])
    d, _ = B.make_desc(p)
    assert B.load().pic_poisson_query(ctypes.byref(d), ctypes.byref(lay)) == B.EINVAL
    assert "active cells" in B.last_error()
    # no-allocation residual refuses patches
    d, _ = B.make_desc(W.channel_plume(16, 8, 16))
    fake = ctypes.c_void_p(256)   # never dereferenced: the descriptor is refused first
    assert B.load().pic_poisson_mode_residual_noalloc(ctypes.byref(d), fake, fake, fake, fake, 0) == B.EINVAL
    assert "composite" in B.last_error()


def _stretched_z(p, ratio):
    w = ratio ** np.arange(p.nz)
    return p.with_z_faces(p.z0 + (p.z1 - p.z0) * np.r_[0.0, np.cumsum(w)] / w.sum())


@pytest.mark.parametrize("kind", ["annulus", "stretched_r", "channel_plume"])
def test_axial_faces_cell_coeffs_match_oracle_everywhere(kind):
    """Non-uniform axial faces: every coefficient of every cell against the
    oracle's (south and north conductances differ row by row)."""
    p = W.annulus(10, 8, 12, phi_r_in=3.0, phi_r_out=-2.0, phi_z0=11.0, phi_z1=5.0)
    if kind == "stretched_r":
        p = p.with_r_faces(W.stretched_radial_faces(p.r_in, p.r_out, p.nr, 1.2))
    if kind == "channel_plume":
        p = W.channel_plume(16, 8, 12, phi_z0=11.0).with_patches(((4, 8, 0, 6), (0, 16, 6, 12)), 2.5)
    p = _stretched_z(p, 1.17)
    g = oracle.grid_from_problem(p)
    b = oracle.rhs3d(g, np.zeros(p.shape))
    act = p.active_cells()
    for k in range(p.nz):
        for i in range(p.nr):
            lib = np.array(B.cell_coeffs(p, i, k))
            orc = oracle.cell_coeffs(g, i, k)
            if not act[k, i]:
                assert np.all(lib == 0.0)
                continue
            np.testing.assert_allclose(lib[0:4], orc["G"], rtol=1e-14)
            np.testing.assert_array_equal(lib[4:8].astype(bool), orc["dirichlet"])
            assert lib[8] == pytest.approx(orc["mu"], rel=1e-14)
            assert lib[9] == pytest.approx(orc["s"], rel=1e-14)
            assert lib[10] == pytest.approx(orc["D0"], rel=1e-14)
            assert lib[11] == pytest.approx(b[k, 0, i], rel=1e-14, abs=1e-12)


def test_axial_faces_validated():
    lay = B.Layout()
    p = W.annulus(16, 8, 16)
    bad = list(p.z0 + (p.z1 - p.z0) * np.arange(17) / 16)
    bad[5] = bad[4]
    d, _ = B.make_desc(p.with_z_faces(bad))
    assert B.load().pic_poisson_query(ctypes.byref(d), ctypes.byref(lay)) == B.EINVAL
    assert "z_faces" in B.last_error()
    d, _ = B.make_desc(_stretched_z(p, 1.1), precision=MIXED, smooth_fused=1)
    assert B.load().pic_poisson_query(ctypes.byref(d), ctypes.byref(lay)) == B.EINVAL
    # the coarsest level is solved densely: at most PIC_POISSON_MAX_DENSE cells
    d, _ = B.make_desc(_stretched_z(W.annulus(130, 8, 50), 1.01))   # coarsest 65 x 50
    assert B.load().pic_poisson_query(ctypes.byref(d), ctypes.byref(lay)) == B.EINVAL
    lay2 = B.query(_stretched_z(W.annulus(512, 8, 400), 1.002))
    assert lay2["nr"][-1] * lay2["nz"][-1] <= 1024
    # the no-allocation residual refuses axial faces before touching any pointer
    d, _ = B.make_desc(_stretched_z(p, 1.1))
    fake = ctypes.c_void_p(256)
    assert B.load().pic_poisson_mode_residual_noalloc(ctypes.byref(d), fake, fake, fake, fake, 0) == B.EINVAL
    assert "axial" in B.last_error()


def test_per_row_tables_enlarge_the_workspace():
    """Per-row tables (one coefficient class per row on an axial mesh) cost
    workspace in proportion to the rows; a composite domain adds only its few
    classes and the dense coarsest factors."""
    p = W.annulus(64, 16, 48)
    base = B.query(p)["workspace_bytes"]
    axial = B.query(_stretched_z(p, 1.05))["workspace_bytes"]
    comp = B.query(W.channel_plume(64, 16, 48))["workspace_bytes"]
    assert axial > base and comp > base
    assert axial - base > comp - base
