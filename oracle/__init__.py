"""FP64 CPU oracle for the cylindrical field solve (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

The oracle is the plain definition of the solve: the three-dimensional
seven-point finite-volume system A phi = b of Sec. 3.1 and the appendix
("Cell integration and face fluxes", "Dirichlet faces"), applied cell by cell
in C (``pic_oracle.c``) with no Fourier transform, and solved by conjugate
gradient.  It builds its own face coordinates from a problem's parameters.

Parity pins (tests/test_oracle_pins.py): the appendix's worked stencil and
two-cell examples, the discrete-eigenvalue identity of
Eq. discrete_azimuthal_eigenvalue, dense direct solves on tiny grids, a
closed-form linear potential, a discretely manufactured potential and the
second-order convergence of an analytically manufactured one.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, OpenMP) and return the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int), ("ntheta", ctypes.c_int), ("nz", ctypes.c_int),
        ("r_faces", ctypes.c_void_p), ("z_faces", ctypes.c_void_p),
        ("L_alpha", ctypes.c_double), ("eps0", ctypes.c_double),
        ("phi_rin", ctypes.c_void_p), ("phi_rout", ctypes.c_void_p),
        ("phi_z0", ctypes.c_void_p), ("phi_z1", ctypes.c_void_p),
        ("active", ctypes.c_void_p), ("phi_exposed", ctypes.c_double),
    ]


class _CGInfo(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("converged", ctypes.c_int),
        ("relres_recursive", ctypes.c_double), ("relres_true", ctypes.c_double),
        ("bnorm", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, dp, ip = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
            lib.oracle_set_threads.argtypes = [ip]
            lib.oracle_get_threads.restype = ip
            lib.oracle_cell_coeffs.argtypes = [vp, ip, ip, vp]
            lib.oracle_apply.argtypes = [vp, vp, vp]
            lib.oracle_rhs.argtypes = [vp, vp, vp]
            lib.oracle_residual.argtypes = [vp, vp, vp, vp, vp]
            lib.oracle_cg.argtypes = [vp, vp, vp, dp, ip, ip, vp]
            lib.oracle_cg.restype = ip
            lib.oracle_cg_fixed.argtypes = [vp, vp, vp, ip, vp]
            lib.oracle_cg_fixed.restype = ip
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """A cell grid given by explicit face coordinates and wall potentials.

    active: optional (nz, nr) boolean array of the composite domain's active
    cells (Sec. 2.2: a union of rectangular patches); a face between an active
    and an inactive cell is a Dirichlet face at phi_exposed.  Inactive cells
    are not unknowns: their rows are the identity with b = 0.
    """

    def __init__(self, r_faces, z_faces, ntheta, L_alpha, eps0,
                 phi_rin, phi_rout, phi_z0, phi_z1, active=None, phi_exposed=0.0):
        self.r_faces = _f64(r_faces)
        self.z_faces = _f64(z_faces)
        self.nr = self.r_faces.size - 1
        self.nz = self.z_faces.size - 1
        self.ntheta = int(ntheta)
        self.L_alpha = float(L_alpha)
        self.eps0 = float(eps0)
        self.phi_rin = _f64(np.broadcast_to(phi_rin, (self.nz,)))
        self.phi_rout = _f64(np.broadcast_to(phi_rout, (self.nz,)))
        self.phi_z0 = _f64(np.broadcast_to(phi_z0, (self.nr,)))
        self.phi_z1 = _f64(np.broadcast_to(phi_z1, (self.nr,)))
        self.active = None if active is None else np.ascontiguousarray(active, dtype=np.uint8).reshape(
            self.nz, self.nr)
        self.phi_exposed = float(phi_exposed)
        self._c = _Grid(self.nr, self.ntheta, self.nz,
                        self.r_faces.ctypes.data, self.z_faces.ctypes.data,
                        self.L_alpha, self.eps0,
                        self.phi_rin.ctypes.data, self.phi_rout.ctypes.data,
                        self.phi_z0.ctypes.data, self.phi_z1.ctypes.data,
                        None if self.active is None else self.active.ctypes.data, self.phi_exposed)

    @property
    def shape(self):
        return (self.nz, self.ntheta, self.nr)

    @property
    def ptr(self):
        return ctypes.addressof(self._c)

    def homogeneous(self):
        """The same grid with every wall potential set to zero."""
        return Grid(self.r_faces, self.z_faces, self.ntheta, self.L_alpha, self.eps0,
                    0.0, 0.0, 0.0, 0.0, self.active, 0.0)


def grid_from_problem(p) -> Grid:
    """Build the oracle's own uniform face arrays from a workloads.Problem."""
    rf = getattr(p, "r_faces", None)
    r_faces = np.asarray(rf, dtype=np.float64) if rf is not None else p.r_in + (p.r_out - p.r_in) * np.arange(p.nr + 1) / p.nr
    zf = getattr(p, "z_faces", None)
    z_faces = np.asarray(zf, dtype=np.float64) if zf is not None else p.z0 + (p.z1 - p.z0) * np.arange(p.nz + 1) / p.nz
    rin = np.asarray(p.phi_r_in_z) if p.phi_r_in_z is not None else p.phi_r_in
    rout = np.asarray(p.phi_r_out_z) if p.phi_r_out_z is not None else p.phi_r_out
    active = None
    patches = getattr(p, "patches", None)
    if patches:
        # the composite domain: cells (i, k) with i0 <= i < i1, k0 <= k < k1 of some patch
        active = np.zeros((p.nz, p.nr), dtype=bool)
        for (i0, i1, k0, k1) in patches:
            active[k0:k1, i0:i1] = True
    return Grid(r_faces, z_faces, p.ntheta, p.theta_span, p.eps0, rin, rout, p.phi_z0, p.phi_z1,
                active, getattr(p, "phi_exposed", 0.0))


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def cell_coeffs(g: Grid, i: int, k: int) -> dict:
    """Face conductances and cell factors of r-z cell (i, k)."""
    out = np.zeros(11)
    _load().oracle_cell_coeffs(g.ptr, int(i), int(k), out.ctypes.data)
    return {"G": out[0:4].copy(), "dirichlet": out[4:8].astype(bool), "mu": out[8],
            "s": out[9], "D0": out[10]}


def apply3d(g: Grid, phi) -> np.ndarray:
    """A phi with homogeneous walls (wall data enters only the right-hand side)."""
    phi = _f64(phi).reshape(g.shape)
    out = np.empty_like(phi)
    _load().oracle_apply(g.ptr, phi.ctypes.data, out.ctypes.data)
    return out


def rhs3d(g: Grid, rho) -> np.ndarray:
    """b = s rho + Dirichlet-face contributions."""
    rho = _f64(rho).reshape(g.shape)
    out = np.empty_like(rho)
    _load().oracle_rhs(g.ptr, rho.ctypes.data, out.ctypes.data)
    return out


def residual(g: Grid, rho, phi):
    """(||b - A phi||_2, ||b||_2) of the physical-space system."""
    rho = _f64(rho).reshape(g.shape)
    phi = _f64(phi).reshape(g.shape)
    rn = ctypes.c_double()
    bn = ctypes.c_double()
    _load().oracle_residual(g.ptr, rho.ctypes.data, phi.ctypes.data,
                            ctypes.byref(rn), ctypes.byref(bn))
    return rn.value, bn.value


def relres(g: Grid, rho, phi) -> float:
    rn, bn = residual(g, rho, phi)
    return rn / bn if bn > 0 else rn


def solve3d(g: Grid, rho, tol: float = 1e-15, maxit: int = 200000, stall: int = 200, x0=None):
    """Conjugate-gradient solve of A phi = b; returns (phi, info dict)."""
    rho = _f64(rho).reshape(g.shape)
    phi = np.zeros(g.shape) if x0 is None else _f64(x0).reshape(g.shape).copy()
    info = _CGInfo()
    rc = _load().oracle_cg(g.ptr, rho.ctypes.data, phi.ctypes.data, float(tol), int(maxit),
                           int(stall), ctypes.byref(info))
    if rc != 0:
        raise MemoryError("oracle_cg: allocation failed")
    return phi, {"iterations": info.iterations, "converged": bool(info.converged),
                 "relres_recursive": info.relres_recursive, "relres": info.relres_true,
                 "bnorm": info.bnorm}


def cg_fixed_iterations(g: Grid, rho, iters: int) -> float:
    """Run exactly `iters` CG iterations from zero (timing sample); returns recursive rel-res."""
    rho = _f64(rho).reshape(g.shape)
    phi = np.zeros(g.shape)
    rr = ctypes.c_double()
    rc = _load().oracle_cg_fixed(g.ptr, rho.ctypes.data, phi.ctypes.data, int(iters), ctypes.byref(rr))
    if rc != 0:
        raise MemoryError("oracle_cg_fixed: allocation failed")
    return rr.value
