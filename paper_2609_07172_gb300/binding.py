"""ctypes binding of the pic_poisson C ABI (include/pic_poisson.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Device buffers are PyTorch CUDA tensors (their data_ptr() and the
current stream are handed to the library).  If the shared library is missing
this module raises instead of falling back to any other implementation.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ENOTCONVERGED, ENONFINITE = 0, 1, 2, 3, 4, 5
FP64, MIXED = 0, 1
USE_INITIAL_GUESS, PROFILE, GRAPH, HOST_STAGED = 1, 2, 4, 8
MAX_BATCH = 64
PHASES = ("forward", "smooth", "smooth_coarse", "restrict", "coarse", "prolong", "norm", "inverse", "defect")
MAX_LEVELS = 16
NPHASE = len(PHASES)

EXPORTS = (
    "pic_poisson_query", "pic_poisson_cell_coeffs", "pic_poisson_plan", "pic_poisson_plan_batch",
    "pic_poisson_set_stream", "pic_poisson_solve_batch",
    "pic_poisson_solve", "pic_poisson_solve_host", "pic_poisson_forward", "pic_poisson_inverse",
    "pic_poisson_face_field", "pic_poisson_deposit", "pic_poisson_project",
    "pic_poisson_mode_residual", "pic_poisson_destroy", "pic_poisson_last_error",
    "pic_poisson_measure_fma_peaks", "pic_poisson_mode_residual_noalloc", "pic_poisson_autotune",
    "pic_poisson_solve_modes", "pic_poisson_analyze", "pic_poisson_get_modes",
)


class PicPoissonError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pic_poisson status {status}: {msg}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int), ("ntheta", ctypes.c_int), ("nz", ctypes.c_int),
        ("r_in", ctypes.c_double), ("r_out", ctypes.c_double),
        ("z0", ctypes.c_double), ("z1", ctypes.c_double),
        ("theta_span", ctypes.c_double),
        ("phi_r_in", ctypes.c_double), ("phi_r_out", ctypes.c_double),
        ("phi_z0", ctypes.c_double), ("phi_z1", ctypes.c_double),
        ("phi_r_in_z", ctypes.c_void_p), ("phi_r_out_z", ctypes.c_void_p), ("r_faces", ctypes.c_void_p),
        ("z_faces", ctypes.c_void_p),
        ("eps0", ctypes.c_double),
        ("precision", ctypes.c_int), ("max_cycles", ctypes.c_int),
        ("pre_sweeps", ctypes.c_int), ("post_sweeps", ctypes.c_int),
        ("inner_cycles", ctypes.c_int), ("smooth_threads", ctypes.c_int), ("smooth_strip", ctypes.c_int),
        ("omega", ctypes.c_double), ("smooth_fused", ctypes.c_int), ("local_bottom", ctypes.c_int),
        ("fmg", ctypes.c_int), ("inner_first", ctypes.c_int),
        ("n_patches", ctypes.c_int), ("patches", ctypes.c_void_p), ("phi_exposed", ctypes.c_double),
        ("flags", ctypes.c_uint),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("cycles", ctypes.c_int), ("outer_iterations", ctypes.c_int),
        ("launches", ctypes.c_int),
        ("rel_res0", ctypes.c_double), ("rel_res", ctypes.c_double),
        ("ms_phase", ctypes.c_double * NPHASE), ("launches_phase", ctypes.c_int * NPHASE),
        ("bytes_phase", ctypes.c_double * NPHASE), ("flops_phase", ctypes.c_double * NPHASE),
    ]

    def as_dict(self):
        return {
            "status": self.status, "cycles": self.cycles, "outer_iterations": self.outer_iterations,
            "launches": self.launches, "rel_res0": self.rel_res0, "rel_res": self.rel_res,
            "ms_phase": {p: self.ms_phase[i] for i, p in enumerate(PHASES)},
            "launches_phase": {p: self.launches_phase[i] for i, p in enumerate(PHASES)},
            "bytes_phase": {p: self.bytes_phase[i] for i, p in enumerate(PHASES)},
            "flops_phase": {p: self.flops_phase[i] for i, p in enumerate(PHASES)},
        }


MAX_TUNE = 96


class Tuning(ctypes.Structure):
    _fields_ = [
        ("pre_sweeps", ctypes.c_int), ("post_sweeps", ctypes.c_int), ("inner_cycles", ctypes.c_int),
        ("inner_first", ctypes.c_int), ("smooth_threads", ctypes.c_int), ("smooth_strip", ctypes.c_int), ("omega", ctypes.c_double),
        ("smooth_fused", ctypes.c_int), ("fmg", ctypes.c_int), ("ms", ctypes.c_double), ("tried", ctypes.c_int),
        ("ms_tried", ctypes.c_double * MAX_TUNE), ("pre_tried", ctypes.c_int * MAX_TUNE), ("post_tried", ctypes.c_int * MAX_TUNE),
        ("inner_tried", ctypes.c_int * MAX_TUNE), ("threads_tried", ctypes.c_int * MAX_TUNE),
        ("strip_tried", ctypes.c_int * MAX_TUNE), ("omega_tried", ctypes.c_double * MAX_TUNE),
        ("fused_tried", ctypes.c_int * MAX_TUNE), ("fmg_tried", ctypes.c_int * MAX_TUNE),
        ("first_tried", ctypes.c_int * MAX_TUNE),
    ]


class Layout(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int), ("nr", ctypes.c_int * MAX_LEVELS), ("nz", ctypes.c_int * MAX_LEVELS),
        ("n_modes", ctypes.c_int), ("workspace_bytes", ctypes.c_size_t),
    ]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the shared library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        try:
            path = _build.build()
        except RuntimeError:
            if not os.path.exists(path):
                raise
    if not os.path.exists(path):
        raise RuntimeError(f"pic_poisson library not built: {path} is missing")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    sig = {
        "pic_poisson_query": ([vp, vp], ip),
        "pic_poisson_cell_coeffs": ([vp, ip, ip, vp], ip),
        "pic_poisson_plan": ([vp, vp, vp], ip),
        "pic_poisson_plan_batch": ([vp, ip, vp, vp], ip),
        "pic_poisson_solve_batch": ([vp, vp, vp, dp, vp], ip),
        "pic_poisson_set_stream": ([vp, vp], ip),
        "pic_poisson_solve": ([vp, vp, vp, dp, vp], ip),
        "pic_poisson_solve_host": ([vp, vp, vp, dp, vp], ip),
        "pic_poisson_forward": ([vp, vp, vp], ip),
        "pic_poisson_face_field": ([vp, vp, vp, vp, vp], ip),
        "pic_poisson_deposit": ([vp, vp, vp, vp, ctypes.c_longlong, ctypes.c_double, vp], ip),
        "pic_poisson_project": ([vp, vp, ctypes.c_double, ctypes.c_int, vp], ip),
        "pic_poisson_inverse": ([vp, vp, vp], ip),
        "pic_poisson_mode_residual": ([vp, vp, vp, vp, vp], ip),
        "pic_poisson_destroy": ([vp], ip),
        "pic_poisson_last_error": ([], ctypes.c_char_p),
        "pic_poisson_measure_fma_peaks": ([vp, vp, vp], ip),
        "pic_poisson_mode_residual_noalloc": ([vp, vp, vp, vp, vp, vp], ip),
        "pic_poisson_autotune": ([vp, ip, vp, vp, dp, vp, ip, vp], ip),
        "pic_poisson_solve_modes": ([vp, vp, vp, vp, dp, vp], ip),
        "pic_poisson_analyze": ([vp, vp, vp], ip),
        "pic_poisson_get_modes": ([vp, vp], ip),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def last_error() -> str:
    return load().pic_poisson_last_error().decode()


def _check(status, allow=(OK,)):
    if status not in allow:
        raise PicPoissonError(status, last_error())
    return status


def make_desc(problem, precision=FP64, max_cycles=0, pre_sweeps=-1, post_sweeps=-1, flags=0, inner_cycles=0,
              smooth_threads=0, smooth_strip=0, omega=0.0, smooth_fused=0, local_bottom=0, fmg=0, inner_first=0):
    """Descriptor for a workloads.Problem; returns (Desc, keep-alive buffers)."""
    keep = []
    d = Desc()
    d.nr, d.ntheta, d.nz = problem.nr, problem.ntheta, problem.nz
    d.r_in, d.r_out, d.z0, d.z1 = problem.r_in, problem.r_out, problem.z0, problem.z1
    d.theta_span = problem.theta_span
    d.phi_r_in, d.phi_r_out = problem.phi_r_in, problem.phi_r_out
    d.phi_z0, d.phi_z1 = problem.phi_z0, problem.phi_z1
    for name in ("phi_r_in_z", "phi_r_out_z", "r_faces", "z_faces"):
        vals = getattr(problem, name, None)
        if vals is not None:
            arr = (ctypes.c_double * len(vals))(*vals)
            keep.append(arr)
            setattr(d, name, ctypes.addressof(arr))
    patches = getattr(problem, "patches", None)
    if patches:
        flat = [int(v) for q in patches for v in q]
        arr = (ctypes.c_int * len(flat))(*flat)
        keep.append(arr)
        d.n_patches = len(patches)
        d.patches = ctypes.addressof(arr)
        d.phi_exposed = float(getattr(problem, "phi_exposed", 0.0))
    d.eps0 = problem.eps0
    d.precision = precision
    d.max_cycles = max_cycles
    d.pre_sweeps = pre_sweeps
    d.post_sweeps = post_sweeps
    d.inner_cycles = inner_cycles
    d.smooth_threads = smooth_threads
    d.smooth_strip = smooth_strip
    d.omega = omega
    d.smooth_fused = smooth_fused
    d.local_bottom = local_bottom
    d.fmg = fmg
    d.inner_first = inner_first
    d.flags = flags
    return d, keep


def query(problem, **kw) -> dict:
    d, _keep = make_desc(problem, **kw)
    lay = Layout()
    _check(load().pic_poisson_query(ctypes.byref(d), ctypes.byref(lay)))
    return {"levels": lay.levels, "nr": list(lay.nr[:lay.levels]), "nz": list(lay.nz[:lay.levels]),
            "n_modes": lay.n_modes, "workspace_bytes": lay.workspace_bytes}


def cell_coeffs(problem, i, k) -> list:
    d, _keep = make_desc(problem)
    out = (ctypes.c_double * 12)()
    _check(load().pic_poisson_cell_coeffs(ctypes.byref(d), int(i), int(k), out))
    return list(out)


def measure_fma_peaks(stream=None):
    import torch
    st = torch.cuda.current_stream().cuda_stream if stream is None else stream
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().pic_poisson_measure_fma_peaks(ctypes.c_void_p(st), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def _dev_ptr(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """A solver plan for one problem (wraps pic_poisson_plan / solve / destroy)."""

    def __init__(self, problem, precision=FP64, max_cycles=0, pre_sweeps=-1, post_sweeps=-1,
                 profile=False, initial_guess=False, stream=None, inner_cycles=0, graph=False,
                 smooth_threads=0, smooth_strip=0, omega=0.0, smooth_fused=0, local_bottom=0, fmg=0,
                 host_staged=False, inner_first=0):
        import torch
        self.problem = problem
        flags = ((PROFILE if profile else 0) | (USE_INITIAL_GUESS if initial_guess else 0)
                 | (GRAPH if graph else 0) | (HOST_STAGED if host_staged else 0))
        self._desc, self._keep = make_desc(problem, precision, max_cycles, pre_sweeps, post_sweeps, flags,
                                           inner_cycles, smooth_threads, smooth_strip, omega,
                                           smooth_fused, local_bottom, fmg, inner_first)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self._plan = ctypes.c_void_p()
        _check(load().pic_poisson_plan(ctypes.byref(self._desc), ctypes.c_void_p(self.stream.cuda_stream),
                                       ctypes.byref(self._plan)))
        self.shape = (problem.nz, problem.ntheta, problem.nr)
        self.n_modes = problem.ntheta // 2 + 1
        self.mode_shape = (problem.nz, problem.nr, self.n_modes, 2)

    def close(self):
        if self._plan:
            load().pic_poisson_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream):
        self.stream = stream
        _check(load().pic_poisson_set_stream(self._plan, ctypes.c_void_p(stream.cuda_stream)))

    def solve(self, rho, phi=None, tol=1e-10):
        """Solve into phi (allocated if None); returns (phi, info dict).

        Raises PicPoissonError for every status except OK and ENOTCONVERGED
        (reported in info["status"]).
        """
        import torch
        if phi is None:
            phi = torch.empty(self.shape, dtype=torch.float64, device=rho.device)
        info = Info()
        st = load().pic_poisson_solve(self._plan, _dev_ptr(rho, self.shape, "rho"),
                                      _dev_ptr(phi, self.shape, "phi"), float(tol), ctypes.byref(info))
        _check(st, allow=(OK, ENOTCONVERGED))
        return phi, info.as_dict()

    def solve_host(self, rho_host, phi_host, tol=1e-10):
        """Solve from host tensors (CPU, float64, contiguous).  Pinned tensors are
        read and written in place by the transforms unless the plan was made
        with host_staged=True; pageable ones go through device staging copies."""
        for t, name in ((rho_host, "rho_host"), (phi_host, "phi_host")):
            if t.is_cuda or not t.is_contiguous() or tuple(t.shape) != self.shape:
                raise ValueError(f"{name} must be a contiguous CPU tensor of shape {self.shape}")
        info = Info()
        st = load().pic_poisson_solve_host(self._plan, ctypes.c_void_p(rho_host.data_ptr()),
                                           ctypes.c_void_p(phi_host.data_ptr()), float(tol), ctypes.byref(info))
        _check(st, allow=(OK, ENOTCONVERGED))
        return info.as_dict()

    def solve_modes(self, rho, uhat_guess, phi=None, tol=1e-10):
        """Solve starting from a mode-layout initial iterate; returns (phi, info)."""
        import torch
        if phi is None:
            phi = torch.empty(self.shape, dtype=torch.float64, device=rho.device)
        info = Info()
        st = load().pic_poisson_solve_modes(self._plan, _dev_ptr(rho, self.shape, "rho"),
                                            _dev_ptr(uhat_guess, self.mode_shape, "uhat_guess"),
                                            _dev_ptr(phi, self.shape, "phi"), float(tol), ctypes.byref(info))
        _check(st, allow=(OK, ENOTCONVERGED))
        return phi, info.as_dict()

    def analyze(self, phi, uhat=None):
        """Mode coefficients (1/N DFT) of a potential."""
        import torch
        if uhat is None:
            uhat = torch.empty(self.mode_shape, dtype=torch.float64, device=phi.device)
        _check(load().pic_poisson_analyze(self._plan, _dev_ptr(phi, self.shape, "phi"),
                                          _dev_ptr(uhat, self.mode_shape, "uhat")))
        return uhat

    def get_modes(self, uhat=None):
        """The mode-space iterate of the last solve."""
        import torch
        if uhat is None:
            uhat = torch.empty(self.mode_shape, dtype=torch.float64, device="cuda")
        _check(load().pic_poisson_get_modes(self._plan, _dev_ptr(uhat, self.mode_shape, "uhat")))
        return uhat

    def face_field(self, phi, er=None, ea=None, ez=None):
        """E = -grad phi on the cell faces: (E_r (nz, nt, nr+1), E_alpha (nz, nt, nr),
        E_z (nz+1, nt, nr)) as new or given CUDA float64 tensors."""
        import torch
        nz, nt, nr = self.shape
        dev = phi.device
        er = torch.empty((nz, nt, nr + 1), dtype=torch.float64, device=dev) if er is None else er
        ea = torch.empty((nz, nt, nr), dtype=torch.float64, device=dev) if ea is None else ea
        ez = torch.empty((nz + 1, nt, nr), dtype=torch.float64, device=dev) if ez is None else ez
        _check(load().pic_poisson_face_field(self._plan, _dev_ptr(phi, self.shape, "phi"),
                                             _dev_ptr(er, (nz, nt, nr + 1), "er"), _dev_ptr(ea, self.shape, "ea"),
                                             _dev_ptr(ez, (nz + 1, nt, nr), "ez")))
        return er, ea, ez

    def node_shape(self):
        nz, nt, nr = self.shape
        return (nz + 1, nt, nr + 1)

    def deposit(self, r, alpha, z, weight, nodes=None):
        """Add the CIC nodal number density of particles (CUDA float64 1-D
        tensors r, alpha, z) to `nodes` (created zeroed if None); returns it."""
        import torch
        n = r.numel()
        for t, name in ((r, "r"), (alpha, "alpha"), (z, "z")):
            if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != n:
                raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of {n} entries")
        if nodes is None:
            nodes = torch.zeros(self.node_shape(), dtype=torch.float64, device=r.device)
        _check(load().pic_poisson_deposit(self._plan, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(alpha.data_ptr()),
                                          ctypes.c_void_p(z.data_ptr()), int(n), float(weight),
                                          _dev_ptr(nodes, self.node_shape(), "nodes")))
        return nodes

    def project(self, nodes, charge, rho=None, accumulate=False):
        """rho (=, or += if accumulate) charge * volume-consistent projection of `nodes`."""
        import torch
        if rho is None:
            rho = torch.zeros(self.shape, dtype=torch.float64, device=nodes.device)
        _check(load().pic_poisson_project(self._plan, _dev_ptr(nodes, self.node_shape(), "nodes"), float(charge),
                                          1 if accumulate else 0, _dev_ptr(rho, self.shape, "rho")))
        return rho

    def forward(self, rho, bhat=None):
        import torch
        if bhat is None:
            bhat = torch.empty(self.mode_shape, dtype=torch.float64, device=rho.device)
        _check(load().pic_poisson_forward(self._plan, _dev_ptr(rho, self.shape, "rho"),
                                          _dev_ptr(bhat, self.mode_shape, "bhat")))
        return bhat

    def inverse(self, phihat, phi=None):
        import torch
        if phi is None:
            phi = torch.empty(self.shape, dtype=torch.float64, device=phihat.device)
        _check(load().pic_poisson_inverse(self._plan, _dev_ptr(phihat, self.mode_shape, "phihat"),
                                          _dev_ptr(phi, self.shape, "phi")))
        return phi

    def mode_residual(self, uhat, bhat, want_r=True):
        import torch
        r = torch.empty(self.mode_shape, dtype=torch.float64, device=uhat.device) if want_r else None
        rel = ctypes.c_double()
        _check(load().pic_poisson_mode_residual(
            self._plan, _dev_ptr(uhat, self.mode_shape, "uhat"), _dev_ptr(bhat, self.mode_shape, "bhat"),
            _dev_ptr(r, self.mode_shape, "rhat") if want_r else None, ctypes.byref(rel)))
        return r, rel.value


class BatchPlan:
    """One plan for several independent problems (wraps pic_poisson_plan_batch / solve_batch)."""

    def __init__(self, problems, precision=FP64, max_cycles=0, pre_sweeps=-1, post_sweeps=-1,
                 profile=False, initial_guess=False, stream=None, inner_cycles=0, graph=False,
                 smooth_threads=0, smooth_strip=0, omega=0.0, smooth_fused=0, local_bottom=0, fmg=0,
                 inner_first=0):
        import torch
        self.problems = list(problems)
        n = len(self.problems)
        if not 1 <= n <= MAX_BATCH:
            raise ValueError(f"batch of {n} problems; 1..{MAX_BATCH} supported")
        flags = ((PROFILE if profile else 0) | (USE_INITIAL_GUESS if initial_guess else 0)
                 | (GRAPH if graph else 0))
        self._descs = (Desc * n)()
        self._keep = []
        for i, p in enumerate(self.problems):
            d, keep = make_desc(p, precision, max_cycles, pre_sweeps, post_sweeps, flags, inner_cycles,
                                smooth_threads, smooth_strip, omega, smooth_fused, local_bottom, fmg, inner_first)
            self._descs[i] = d
            self._keep.extend(keep)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        self._plan = ctypes.c_void_p()
        _check(load().pic_poisson_plan_batch(self._descs, n, ctypes.c_void_p(self.stream.cuda_stream),
                                             ctypes.byref(self._plan)))
        self.shapes = [(p.nz, p.ntheta, p.nr) for p in self.problems]

    def close(self):
        if self._plan:
            load().pic_poisson_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, rhos, phis=None, tol=1e-10):
        """Solve all problems; returns (phis, [info dicts]).  Raises except for OK / ENOTCONVERGED."""
        import torch
        n = len(self.problems)
        if phis is None:
            phis = [torch.empty(sh, dtype=torch.float64, device=r.device) for sh, r in zip(self.shapes, rhos)]
        rp = (ctypes.c_void_p * n)(*[_dev_ptr(r, sh, "rho").value for r, sh in zip(rhos, self.shapes)])
        fp = (ctypes.c_void_p * n)(*[_dev_ptr(f, sh, "phi").value for f, sh in zip(phis, self.shapes)])
        infos = (Info * n)()
        st = load().pic_poisson_solve_batch(self._plan, rp, fp, float(tol), infos)
        _check(st, allow=(OK, ENOTCONVERGED))
        return phis, [i.as_dict() for i in infos]


def tune_key(problems, precision, graph, tol):
    """Cache key of an autotuning: every problem's sizes, plus a digest of its
    face arrays and patches when it has them (two problems of one size but
    different meshes or domains are tuned apart), the precision, the graph
    flag and the tolerance."""
    import hashlib

    def geometry(p):
        extra = (p.r_faces, p.z_faces, p.patches, p.phi_exposed if p.patches else None)
        tag = "%dx%dx%d" % (p.nr, p.ntheta, p.nz)
        if any(x is not None for x in extra[:3]):
            tag += ":" + hashlib.sha1(repr(extra).encode()).hexdigest()[:12]
        return tag
    return "|".join(geometry(p) for p in problems) + "|%d|%d|%g" % (precision, graph, tol)


def autotune(problems, rhos, tol=1e-10, precision=FP64, graph=False, repeats=3, cache=None):
    """Tuned solver settings for `problems` (pic_poisson_autotune), as Plan keyword arguments.

    cache: optional JSON file; results are stored under a key made of the
    problem sizes, precision, graph flag and tolerance and reused when present.
    """
    import json
    import os
    import torch
    problems = list(problems)
    key = tune_key(problems, precision, graph, tol)
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            return table[key]["best"]
    n = len(problems)
    descs = (Desc * n)()
    keep = []
    for i, p in enumerate(problems):
        d, k = make_desc(p, precision, 0, -1, -1, GRAPH if graph else 0)
        descs[i] = d
        keep.extend(k)
    shapes = [(p.nz, p.ntheta, p.nr) for p in problems]
    phis = [torch.empty(sh, dtype=torch.float64, device=r.device) for sh, r in zip(shapes, rhos)]
    rp = (ctypes.c_void_p * n)(*[_dev_ptr(r, sh, "rho").value for r, sh in zip(rhos, shapes)])
    fp = (ctypes.c_void_p * n)(*[_dev_ptr(f, sh, "phi").value for f, sh in zip(phis, shapes)])
    out = Tuning()
    st = torch.cuda.current_stream().cuda_stream
    _check(load().pic_poisson_autotune(descs, n, rp, fp, float(tol), ctypes.c_void_p(st), int(repeats),
                                       ctypes.byref(out)))
    best = {"pre_sweeps": out.pre_sweeps, "post_sweeps": out.post_sweeps, "inner_cycles": out.inner_cycles,
            "smooth_threads": out.smooth_threads, "smooth_strip": out.smooth_strip, "omega": out.omega,
            "smooth_fused": out.smooth_fused, "fmg": out.fmg, "inner_first": out.inner_first}
    tried = [{"pre": out.pre_tried[i], "post": out.post_tried[i], "inner": out.inner_tried[i],
              "threads": out.threads_tried[i], "strip": out.strip_tried[i], "omega": out.omega_tried[i],
              "fused": out.fused_tried[i], "fmg": out.fmg_tried[i], "first": out.first_tried[i],
              "ms": out.ms_tried[i]}
             for i in range(out.tried)]
    if cache:
        table = {}
        if os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
        table[key] = {"best": best, "ms": out.ms, "tried": tried}
        with open(cache, "w") as f:
            json.dump(table, f, indent=1)
    return dict(best, ms=out.ms, tried=tried)
