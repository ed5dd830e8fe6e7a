"""FP64 CPU oracle for block 3MG deblurring -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  It shares no code with the CUDA library (`paper_2002_02328_gb300`)
and never imports it.  The arithmetic lives in `bd3mg_oracle.c` (plain C,
double precision, plain definitions); this module only builds it with gcc and
marshals numpy arrays through ctypes.

Parity status per function (what pins it is in the tests named):
  apply_H / apply_HT ........ pinned (scipy.ndimage.convolve per depth; adjoint
                              identity; delta PSF)            tests/test_oracle_ops.py
  apply_V / apply_VT ........ pinned (numpy.diff; adjoint)    tests/test_oracle_ops.py
  objective ................. pinned (hand-computed fixture tests/golden/objective_hand.txt;
                              closed forms)                   tests/test_oracle_objective.py
  gradient / gradient_at .... pinned (central finite differences of objective)
  apply_A ................... pinned (majorisation inequality, tangency)
  pinv2_solve ............... pinned (numpy.linalg.pinv)
  step / run (3MG) .......... pinned (dense least-squares solve when lambda=0 and
                              the box is inactive; per-voxel closed form for H=I;
                              monotone descent; stationarity)  tests/test_oracle_3mg.py
  penalty mode 1 (joint X-Y hyperbolic + kappa ||V^Z x||^2, as printed in Section 3.1):
                              pinned (hand-computed fixture case C; closed form
                              along z with numpy.diff; reduction to the per-axis
                              mode along x; finite differences; majorisation,
                              tangency, exact quadratic Z majorant; descent and
                              stationarity)       tests/test_oracle_objective.py, test_oracle_3mg.py
  penalty mode 2 (isotropic hyperbolic term over X, Y and Z):
                              pinned (hand-computed fixture case D; reduction to
                              the per-axis mode along each single axis; invariance
                              under axis permutation; finite differences;
                              majorisation, tangency; descent and stationarity)
                                                  tests/test_oracle_objective.py, test_oracle_3mg.py
  ablation variants (run_variant; Section 3.2, Table 1): A = L I with the
  Lipschitz bound, D = -g, the Fletcher-Reeves conjugate direction with the
  majorant's closed-form step, the Jacobi block schedule with curvature
  inflation: pinned (Hessian eigenvalues below the bound; dense gradient
  descent; scipy CG on least squares; Jacobi = sequential for decoupled slabs;
  monotone descent)                   tests/test_oracle_variants.py
Workload-level values of the paper (SNR on FlyBrain/Aneurysm): parity unpinned
(datasets not available).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bd3mg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("px", ctypes.c_int), ("py", ctypes.c_int), ("pz", ctypes.c_int),
                ("psf", ctypes.c_void_p),
                ("lambda_", ctypes.c_double), ("delta", ctypes.c_double), ("eta", ctypes.c_double),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("penalty", ctypes.c_int), ("kappa", ctypes.c_double)]


class _Variant(ctypes.Structure):
    _fields_ = [("metric", ctypes.c_int), ("lipschitz", ctypes.c_double), ("direction", ctypes.c_int),
                ("schedule", ctypes.c_int), ("inflation", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math", "-ffp-contract=off",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.POINTER(_Problem)
            dp = ctypes.c_void_p
            lib.orc_apply_H.argtypes = [P, dp, dp]
            lib.orc_apply_HT.argtypes = [P, dp, dp]
            lib.orc_apply_V.argtypes = [P, ctypes.c_int, dp, dp]
            lib.orc_apply_VT.argtypes = [P, ctypes.c_int, dp, dp]
            lib.orc_objective.argtypes = [P, dp, dp, dp]
            lib.orc_objective.restype = ctypes.c_double
            lib.orc_gradient.argtypes = [P, dp, dp, dp]
            lib.orc_apply_A.argtypes = [P, dp, dp, dp]
            lib.orc_pinv2_solve.argtypes = [dp, dp, dp, ctypes.c_double]
            lib.orc_pinv2_solve.restype = ctypes.c_int
            lib.orc_3mg_step.argtypes = [P, dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
            lib.orc_3mg.argtypes = [P, dp, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, dp]
            lib.orc_gradient_at.argtypes = [P, dp, dp, ctypes.c_int, dp, dp]
            V = ctypes.POINTER(_Variant)
            lib.orc_lipschitz_bound.argtypes = [P]
            lib.orc_lipschitz_bound.restype = ctypes.c_double
            lib.orc_3mg_step_v.argtypes = [P, V, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp]
            lib.orc_3mg_v.argtypes = [P, V, dp, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, dp, dp]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleProblem:
    """Holds the problem description (PSF as float32 [nz,pz,py,px], parameters)."""

    def __init__(self, shape, psf, lam=1e-2, delta=1e-2, eta=1.0, xmin=0.0, xmax=1.0, penalty=0, kappa=0.0):
        self.shape = tuple(int(s) for s in shape)
        nz, ny, nx = self.shape
        self.psf = _f32(psf)
        assert self.psf.ndim == 4 and self.psf.shape[0] == nz
        pz, py, px = self.psf.shape[1:]
        assert px % 2 == 1 and py % 2 == 1 and pz % 2 == 1
        self.params = (float(lam), float(delta), float(eta), float(xmin), float(xmax))
        self.penalty, self.kappa = int(penalty), float(kappa)
        self._c = _Problem(nx, ny, nz, px, py, pz, self.psf.ctypes.data, *self.params, self.penalty, self.kappa)

    @classmethod
    def from_synth(cls, prob):
        return cls(prob.shape, prob.psf, prob.lam, prob.delta, prob.eta, prob.xmin, prob.xmax,
                   getattr(prob, "penalty", 0), getattr(prob, "kappa", 0.0))

    @property
    def ref(self):
        return ctypes.byref(self._c)

    def _vol(self, a) -> np.ndarray:
        a = _f64(a)
        assert a.shape == self.shape, (a.shape, self.shape)
        return a


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def apply_H(op: OracleProblem, x) -> np.ndarray:
    x = op._vol(x)
    out = np.empty_like(x)
    _load().orc_apply_H(op.ref, _ptr(x), _ptr(out))
    return out


def apply_HT(op: OracleProblem, r) -> np.ndarray:
    r = op._vol(r)
    out = np.empty_like(r)
    _load().orc_apply_HT(op.ref, _ptr(r), _ptr(out))
    return out


def apply_V(op: OracleProblem, axis: int, x) -> np.ndarray:
    """axis 0 = X (fastest), 1 = Y, 2 = Z."""
    x = op._vol(x)
    out = np.empty_like(x)
    _load().orc_apply_V(op.ref, int(axis), _ptr(x), _ptr(out))
    return out


def apply_VT(op: OracleProblem, axis: int, q) -> np.ndarray:
    q = op._vol(q)
    out = np.empty_like(q)
    _load().orc_apply_VT(op.ref, int(axis), _ptr(q), _ptr(out))
    return out


def objective(op: OracleProblem, y, x, parts: bool = False):
    y = _f32(y)
    x = op._vol(x)
    pr = np.zeros(3)
    f = _load().orc_objective(op.ref, _ptr(y), _ptr(x), _ptr(pr))
    return (f, pr) if parts else f


def gradient(op: OracleProblem, y, x) -> np.ndarray:
    y = _f32(y)
    x = op._vol(x)
    g = np.empty_like(x)
    _load().orc_gradient(op.ref, _ptr(y), _ptr(x), _ptr(g))
    return g


def gradient_at(op: OracleProblem, y, x, idx) -> np.ndarray:
    y = _f32(y)
    x = op._vol(x)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.shape[0])
    _load().orc_gradient_at(op.ref, _ptr(y), _ptr(x), int(idx.shape[0]), _ptr(idx), _ptr(out))
    return out


def apply_A(op: OracleProblem, xt, v) -> np.ndarray:
    xt = op._vol(xt)
    v = op._vol(v)
    out = np.empty_like(v)
    _load().orc_apply_A(op.ref, _ptr(xt), _ptr(v), _ptr(out))
    return out


def pinv2_solve(B, c, rtol: float = 1e-12):
    B = _f64(np.asarray(B).reshape(4))
    c = _f64(np.asarray(c).reshape(2))
    u = np.zeros(2)
    rank = _load().orc_pinv2_solve(_ptr(B), _ptr(c), _ptr(u), float(rtol))
    return u, int(rank)


def step(op: OracleProblem, y, x, d, z0: int = 0, z1: Optional[int] = None, rtol: float = 1e-12):
    """One (restricted) 3MG step; returns (x_new, d_new, info dict)."""
    y = _f32(y)
    x = op._vol(x).copy()
    d = op._vol(d).copy()
    z1 = op.shape[0] if z1 is None else z1
    info = np.zeros(8)
    _load().orc_3mg_step(op.ref, _ptr(y), _ptr(x), _ptr(d), int(z0), int(z1), float(rtol), _ptr(info))
    return x, d, dict(B=info[:4].reshape(2, 2), c=info[4:6], u=info[6:8])


def run(op: OracleProblem, y, x0, n_sweeps: int, bounds: Optional[Sequence[int]] = None,
        order: Optional[Sequence[int]] = None, d0=None, rtol: float = 1e-12, trace: bool = True):
    """n_sweeps sweeps of 3MG (block form if bounds has more than one slab).

    Returns (x, d, f_trace) with f_trace[k] = f(x^k), k = 0..n_sweeps.
    """
    y = _f32(y)
    x = op._vol(x0).copy()
    d = np.zeros_like(x) if d0 is None else op._vol(d0).copy()
    if bounds is None:
        bounds = [0, op.shape[0]]
    b = np.ascontiguousarray(bounds, dtype=np.int32)
    ns = len(bounds) - 1
    o = np.ascontiguousarray(order if order is not None else range(ns), dtype=np.int32)
    assert o.shape[0] == ns
    ft = np.zeros(n_sweeps + 1)
    _load().orc_3mg(op.ref, _ptr(y), _ptr(x), _ptr(d), int(n_sweeps), int(ns), _ptr(b), _ptr(o),
                    float(rtol), _ptr(ft) if trace else None)
    return x, d, (ft if trace else None)


# ---------------------------------------------------------------------------
# Ablation variants (Section 3.2, Table 1) and block schedules
# ---------------------------------------------------------------------------
METRIC_MAJORANT, METRIC_LIPSCHITZ = 0, 1
DIR_MEMORY_GRADIENT, DIR_GRADIENT, DIR_CONJUGATE = 0, 1, 2
SCHEDULE_SEQUENTIAL, SCHEDULE_JACOBI = 0, 1


def lipschitz_bound(op: OracleProblem) -> float:
    """Upper bound on the Lipschitz constant of grad f (||H||_1 ||H||_inf + 2 eta
    + the penalty's Hessian bound)."""
    return float(_load().orc_lipschitz_bound(op.ref))


def _variant(metric=0, lipschitz=0.0, direction=0, schedule=0, inflation=1.0):
    return _Variant(int(metric), float(lipschitz), int(direction), int(schedule), float(inflation))


def run_variant(op: OracleProblem, y, x0, n_sweeps: int, bounds: Optional[Sequence[int]] = None,
                order: Optional[Sequence[int]] = None, rtol: float = 1e-12, **variant):
    """n_sweeps sweeps of an ablation variant (keywords: metric, lipschitz,
    direction, schedule, inflation).  Returns (x, d, f_trace)."""
    y = _f32(y)
    x = op._vol(x0).copy()
    d = np.zeros_like(x)
    if bounds is None:
        bounds = [0, op.shape[0]]
    b = np.ascontiguousarray(bounds, dtype=np.int32)
    ns = len(bounds) - 1
    o = np.ascontiguousarray(order if order is not None else range(ns), dtype=np.int32)
    state = np.zeros(2 * ns)
    ft = np.zeros(n_sweeps + 1)
    v = _variant(**variant)
    _load().orc_3mg_v(op.ref, ctypes.byref(v), _ptr(y), _ptr(x), _ptr(d), int(n_sweeps), int(ns), _ptr(b), _ptr(o),
                      float(rtol), _ptr(state), _ptr(ft))
    return x, d, ft
