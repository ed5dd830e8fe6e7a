"""Thin ctypes binding of the C ABI in include/bd3mg.h.

Argument marshalling only: every step of the iteration runs in the CUDA
library `libbd3mg.so` built in-tree by `paper_2002_02328_gb300.build`.  There is
no CPU fallback: if the library is missing, `load()` raises.  PyTorch supplies
device memory (through the allocator hook) and streams.

The functions named like the C entry points (`bd3mg_create`, `bd3mg_iterate`,
...) take and return Python objects; `Solver` wraps one context.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libbd3mg.so")
_lock = threading.Lock()
_lib = None

STATUS = {0: "BD3MG_OK", 1: "BD3MG_EINVAL", 2: "BD3MG_ENOMEM", 3: "BD3MG_ECUDA", 4: "BD3MG_ETIMEOUT",
          5: "BD3MG_ENONFINITE", 6: "BD3MG_ESTATE", 7: "BD3MG_EUNSUPPORTED"}
FP32, BF16_GRADIENT, BF16_DIRECTIONS = 0, 1, 2
PENALTY_PER_AXIS, PENALTY_JOINT_XY, PENALTY_ISOTROPIC = 0, 1, 2
METRIC_MAJORANT, METRIC_LIPSCHITZ = 0, 1
DIR_MEMORY_GRADIENT, DIR_GRADIENT, DIR_CONJUGATE = 0, 1, 2
SCHEDULE_COLOURED, SCHEDULE_JACOBI = 0, 1
PSF_AUTO, PSF_DENSE = 0, 1
UPDATE_AUTO, UPDATE_SEPARATE, UPDATE_FUSED = 0, 1, 2
FAULT_NONE, FAULT_SKIP_COPY, FAULT_SKIP_ARRIVE = 0, 1, 2

# Every symbol include/bd3mg.h declares (checked by the CPU test-suite).
EXPORTED = ["bd3mg_params_default", "bd3mg_create", "bd3mg_iterate", "bd3mg_iterate_async", "bd3mg_objective",
            "bd3mg_gradient", "bd3mg_get_x", "bd3mg_get_d", "bd3mg_set_x", "bd3mg_last_step", "bd3mg_apply_H",
            "bd3mg_apply_HT", "bd3mg_slab_colours", "bd3mg_plan_slab_colours", "bd3mg_factor_psf",
            "bd3mg_launches_per_iteration", "bd3mg_profile_iteration", "bd3mg_objective_noalloc",
            "bd3mg_batch_create", "bd3mg_volume_count", "bd3mg_objectives", "bd3mg_get_volume", "bd3mg_set_stopping",
            "bd3mg_stopped", "bd3mg_set_escalation", "bd3mg_escalated", "bd3mg_save", "bd3mg_load",
            "bd3mg_autotune", "bd3mg_inject_fault", "bd3mg_error_string",
            "bd3mg_status_string", "bd3mg_destroy", "bd3mg_lipschitz"]


class Bd3mgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("px", ctypes.c_int), ("py", ctypes.c_int), ("pz", ctypes.c_int),
                ("psf", ctypes.c_void_p),
                ("lambda_", ctypes.c_double), ("delta", ctypes.c_double), ("eta", ctypes.c_double),
                ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("precision", ctypes.c_int), ("nslabs", ctypes.c_int), ("slab_bounds", ctypes.c_void_p),
                ("pinv_rtol", ctypes.c_double), ("zchunk", ctypes.c_int),
                ("penalty", ctypes.c_int), ("kappa", ctypes.c_double),
                ("refresh_every", ctypes.c_int), ("barrier_timeout_ms", ctypes.c_int),
                ("separate_update", ctypes.c_int),
                ("metric", ctypes.c_int), ("lipschitz", ctypes.c_double), ("direction", ctypes.c_int),
                ("schedule", ctypes.c_int), ("inflation", ctypes.c_double), ("curv_rows", ctypes.c_int),
                ("psf_mode", ctypes.c_int), ("persistent", ctypes.c_int)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


def load(path: str = LIB_PATH):
    """Load libbd3mg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        P = ctypes.POINTER(Params)
        sig = {
            "bd3mg_params_default": (None, [P]),
            "bd3mg_create": (ip, [P, vp, vp, ip, vp, ctypes.POINTER(Allocator), ctypes.POINTER(vp)]),
            "bd3mg_iterate": (ip, [vp, ip, vp]),
            "bd3mg_iterate_async": (ip, [vp, ip]),
            "bd3mg_objective": (ip, [vp, vp, vp]),
            "bd3mg_gradient": (ip, [vp, vp, ip, vp]),
            "bd3mg_get_x": (ip, [vp, vp, ip]),
            "bd3mg_get_d": (ip, [vp, vp, ip]),
            "bd3mg_set_x": (ip, [vp, vp, ip]),
            "bd3mg_last_step": (ip, [vp, vp]),
            "bd3mg_apply_H": (ip, [vp, vp, vp]),
            "bd3mg_apply_HT": (ip, [vp, vp, vp]),
            "bd3mg_slab_colours": (ip, [vp, vp, vp]),
            "bd3mg_plan_slab_colours": (ip, [ip, vp, ip, vp, vp]),
            "bd3mg_factor_psf": (ip, [ip, ip, ip, ip, vp, vp, vp, vp, vp]),
            "bd3mg_launches_per_iteration": (ip, [vp]),
            "bd3mg_profile_iteration": (ip, [vp, vp, vp]),
            "bd3mg_batch_create": (ip, [ip, P, vp, vp, ip, vp, ctypes.POINTER(Allocator), ctypes.POINTER(vp)]),
            "bd3mg_volume_count": (ip, [vp]),
            "bd3mg_objectives": (ip, [vp, vp]),
            "bd3mg_get_volume": (ip, [vp, ip, ip, vp, ip]),
            "bd3mg_set_stopping": (ip, [vp, dp, vp]),
            "bd3mg_stopped": (ip, [vp, vp]),
            "bd3mg_objective_noalloc": (ip, [P, vp, vp, vp, vp, ctypes.c_char_p, ctypes.c_size_t]),
            "bd3mg_set_escalation": (ip, [vp, dp]),
            "bd3mg_escalated": (ip, [vp, ctypes.POINTER(ctypes.c_longlong)]),
            "bd3mg_inject_fault": (ip, [vp, ip]),
            "bd3mg_save": (ip, [vp, ctypes.c_char_p]),
            "bd3mg_load": (ip, [vp, ctypes.c_char_p]),
            "bd3mg_autotune": (ip, [ip, P, vp, ip, vp, ip, ctypes.c_char_p, ctypes.POINTER(ip), ctypes.POINTER(ip),
                                    ctypes.POINTER(dp)]),
            "bd3mg_error_string": (ctypes.c_char_p, [vp]),
            "bd3mg_lipschitz": (ip, [vp, ctypes.c_void_p]),
            "bd3mg_status_string": (ctypes.c_char_p, [ip]),
            "bd3mg_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(ctx, status: int):
    if status != 0:
        lib = load()
        msg = lib.bd3mg_error_string(ctx).decode() if ctx else lib.bd3mg_status_string(status).decode()
        raise Bd3mgError(status, msg)


def _torch():
    import torch
    return torch


def _torch_allocator():
    """Allocator hook backed by PyTorch's caching allocator (device memory from torch)."""
    torch = _torch()

    def _alloc(user, nbytes, stream):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                          stream if stream else 0))
        except Exception:
            return None

    def _free(user, ptr, nbytes, stream):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    fa, ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
    return Allocator(fa, ff, None), (fa, ff)


def make_params(shape, psf: np.ndarray, lam=1e-2, delta=1e-2, eta=1.0, xmin=0.0, xmax=1.0,
                slabs: Optional[Sequence[int]] = None, precision: int = FP32, pinv_rtol: float = 1e-12,
                zchunk: int = 0, penalty: int = 0, kappa: float = 0.0, refresh_every: int = 0,
                barrier_timeout_ms: int = 0, separate_update: int = 0, metric: int = 0, lipschitz: float = 0.0,
                direction: int = 0, schedule: int = 0, inflation: float = 0.0, psf_mode: int = 0,
                curv_rows: int = 0, persistent: int = 0):
    """Build a Params struct; returns (params, keepalive) -- keep both alive until create returns."""
    nz, ny, nx = (int(s) for s in shape)
    psf = np.ascontiguousarray(psf, dtype=np.float32)
    assert psf.ndim == 4 and psf.shape[0] == nz, psf.shape
    pz, py, px = psf.shape[1:]
    p = Params()
    load().bd3mg_params_default(ctypes.byref(p))
    p.nx, p.ny, p.nz, p.px, p.py, p.pz = nx, ny, nz, px, py, pz
    p.psf = psf.ctypes.data
    p.lambda_, p.delta, p.eta, p.xmin, p.xmax = float(lam), float(delta), float(eta), float(xmin), float(xmax)
    p.precision = int(precision)
    p.pinv_rtol = float(pinv_rtol)
    p.zchunk = int(zchunk)
    p.penalty, p.kappa = int(penalty), float(kappa)
    p.refresh_every, p.barrier_timeout_ms = int(refresh_every), int(barrier_timeout_ms)
    p.separate_update = int(separate_update)
    p.metric, p.lipschitz, p.direction = int(metric), float(lipschitz), int(direction)
    p.schedule, p.inflation = int(schedule), float(inflation)
    p.psf_mode = int(psf_mode)
    p.curv_rows = int(curv_rows)
    p.persistent = int(persistent)
    keep = [psf]
    if slabs is not None and len(slabs) > 2:
        b = np.ascontiguousarray(slabs, dtype=np.int32)
        p.nslabs = len(slabs) - 1
        p.slab_bounds = b.ctypes.data
        keep.append(b)
    else:
        p.nslabs = 1
    return p, keep


def bd3mg_plan_slab_colours(bounds: Sequence[int], pz: int):
    """Host-only slab colouring; returns (colour array, number of colours)."""
    b = np.ascontiguousarray(bounds, dtype=np.int32)
    col = np.zeros(len(bounds) - 1, np.int32)
    nc = ctypes.c_int()
    st = load().bd3mg_plan_slab_colours(len(bounds) - 1, b.ctypes.data, int(pz), col.ctypes.data, ctypes.byref(nc))
    _check(None, st)
    return col, nc.value


def bd3mg_factor_psf(psf: np.ndarray):
    """Host-only rank-1 factoring; returns (fx, fy, fz, residual) or raises Bd3mgError."""
    psf = np.ascontiguousarray(psf, dtype=np.float32)
    nz, pz, py, px = psf.shape
    fx, fy, fz = np.zeros((nz, px), np.float32), np.zeros((nz, py), np.float32), np.zeros((nz, pz), np.float32)
    res = ctypes.c_double()
    st = load().bd3mg_factor_psf(nz, px, py, pz, psf.ctypes.data, fx.ctypes.data, fy.ctypes.data, fz.ctypes.data,
                                 ctypes.byref(res))
    if st != 0:
        raise Bd3mgError(st, f"PSF not separable (residual {res.value:.3g})")
    return fx, fy, fz, res.value


def bd3mg_objective_noalloc(params: Params, x, y, f_out, stream=None):
    """f(x) into the 4-double device tensor f_out without any device allocation.

    x, y: contiguous float32 CUDA tensors [nz][ny][nx] (nx a multiple of 4).
    Raises Bd3mgError with the library's message on failure.
    """
    import torch
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    err = ctypes.create_string_buffer(256)
    st = load().bd3mg_objective_noalloc(ctypes.byref(params), ctypes.c_void_p(_ptr(x)), ctypes.c_void_p(_ptr(y)),
                                        ctypes.c_void_p(_ptr(f_out)), ctypes.c_void_p(int(s)), err, 256)
    if st != 0:
        raise Bd3mgError(st, err.value.decode())


def _ptr(t) -> int:
    return int(t.data_ptr())


def bd3mg_create(params: Params, y, x0=None, stream=None, use_torch_allocator: bool = True):
    """Create a context from torch tensors y (and x0), on the GPU or on the host.

    Returns (ctx handle, keepalive).  Host tensors are copied from host memory.
    """
    torch = _torch()
    lib = load()
    on_dev = bool(y.is_cuda)
    y = y.contiguous()
    if x0 is not None:
        x0 = x0.contiguous()
        assert bool(x0.is_cuda) == on_dev
    s = stream if stream is not None else (torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0)
    keep = [y, x0]
    alloc_p = None
    if use_torch_allocator:
        al, cbs = _torch_allocator()
        keep += [al, cbs]
        alloc_p = ctypes.byref(al)
    ctx = ctypes.c_void_p()
    st = lib.bd3mg_create(ctypes.byref(params), ctypes.c_void_p(_ptr(y)),
                          ctypes.c_void_p(_ptr(x0)) if x0 is not None else None, int(on_dev),
                          ctypes.c_void_p(int(s)), alloc_p, ctypes.byref(ctx))
    if st != 0:
        msg = lib.bd3mg_error_string(ctx).decode() if ctx.value else lib.bd3mg_status_string(st).decode()
        if ctx.value:
            lib.bd3mg_destroy(ctx)
        raise Bd3mgError(st, msg)
    return ctx, keep


class Solver:
    """One block-3MG context over a single volume (plain or slab form)."""

    def __init__(self, shape, psf, y, x0=None, lam=1e-2, delta=1e-2, eta=1.0, xmin=0.0, xmax=1.0,
                 slabs=None, precision: int = FP32, pinv_rtol: float = 1e-12, zchunk: int = 0, stream=None,
                 use_torch_allocator: bool = True, penalty: int = 0, kappa: float = 0.0, refresh_every: int = 0,
                 barrier_timeout_ms: int = 0, separate_update: int = 0, metric: int = 0, lipschitz: float = 0.0,
                 direction: int = 0, schedule: int = 0, inflation: float = 0.0, psf_mode: int = 0,
                 curv_rows: int = 0, persistent: int = 0):
        torch = _torch()
        self.shape = tuple(int(s) for s in shape)
        self.n = int(np.prod(self.shape))
        self.nslabs = 1 if slabs is None or len(slabs) <= 2 else len(slabs) - 1
        params, keep = make_params(shape, psf, lam, delta, eta, xmin, xmax, slabs, precision, pinv_rtol, zchunk,
                                   penalty, kappa, refresh_every, barrier_timeout_ms, separate_update, metric,
                                   lipschitz, direction, schedule, inflation, psf_mode, curv_rows, persistent)
        if not isinstance(y, torch.Tensor):
            y = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32))
        if x0 is not None and not isinstance(x0, torch.Tensor):
            x0 = torch.from_numpy(np.ascontiguousarray(x0, dtype=np.float32))
        self.device = y.device
        self._ctx, self._keep = bd3mg_create(params, y, x0, stream, use_torch_allocator)
        self._keep.append(keep)
        self._lib = load()

    # -- lifecycle
    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.bd3mg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, st):
        _check(self._ctx, st)

    # -- iteration
    def iterate(self, n: int, trace: bool = True):
        """Run n sweeps; returns the FP64 objective trace (n+1 values) or None."""
        buf = np.zeros(n + 1) if trace else None
        self._c(self._lib.bd3mg_iterate(self._ctx, int(n), buf.ctypes.data if trace else None))
        return buf

    def iterate_async(self, n: int):
        self._c(self._lib.bd3mg_iterate_async(self._ctx, int(n)))

    def objective(self, parts: bool = False):
        f = ctypes.c_double()
        pr = np.zeros(3)
        self._c(self._lib.bd3mg_objective(self._ctx, ctypes.byref(f), pr.ctypes.data))
        return (f.value, pr) if parts else f.value

    def gradient(self, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        f = ctypes.c_double()
        self._c(self._lib.bd3mg_gradient(self._ctx, ctypes.c_void_p(_ptr(out)), int(out.is_cuda), ctypes.byref(f)))
        return out, f.value

    def get_x(self, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        self._c(self._lib.bd3mg_get_x(self._ctx, ctypes.c_void_p(_ptr(out)), int(out.is_cuda)))
        return out

    def get_d(self, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        self._c(self._lib.bd3mg_get_d(self._ctx, ctypes.c_void_p(_ptr(out)), int(out.is_cuda)))
        return out

    def set_x(self, x):
        torch = _torch()
        if not isinstance(x, torch.Tensor):
            x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
        x = x.contiguous()
        self._c(self._lib.bd3mg_set_x(self._ctx, ctypes.c_void_p(_ptr(x)), int(x.is_cuda)))

    def set_stopping(self, tol: float = 0.0, f_target=None):
        """Stop once ||x^k - x^{k-1}|| <= tol ||x^{k-1}|| or f(x^k) <= f_target (None: no target)."""
        t = None if f_target is None else np.array([float(f_target)], np.float64)
        self._c(self._lib.bd3mg_set_stopping(self._ctx, float(tol), None if t is None else t.ctypes.data))

    def stopped(self) -> int:
        """Sweeps after which the solve stopped, or -1 while it runs."""
        k = np.zeros(1, np.int32)
        self._c(self._lib.bd3mg_stopped(self._ctx, k.ctypes.data))
        return int(k[0])

    def set_escalation(self, tol: float):
        """BF16 gradient: switch to an FP32 gradient once f decreases by <= tol |f| per iteration."""
        self._c(self._lib.bd3mg_set_escalation(self._ctx, float(tol)))

    def escalated(self) -> int:
        """Iteration count at which the context switched to an FP32 gradient, or -1."""
        at = ctypes.c_longlong()
        self._c(self._lib.bd3mg_escalated(self._ctx, ctypes.byref(at)))
        return int(at.value)

    def inject_fault(self, kind: int = FAULT_SKIP_COPY):
        """Test hook: make the next iterations' bounded device waits run out (bd3mg_inject_fault)."""
        self._c(self._lib.bd3mg_inject_fault(self._ctx, int(kind)))

    def save(self, path: str):
        """Checkpoint x, d and the iteration count to `path`."""
        self._c(self._lib.bd3mg_save(self._ctx, os.fsencode(path)))

    def load(self, path: str):
        """Resume from a checkpoint written by save() of an identical context."""
        self._c(self._lib.bd3mg_load(self._ctx, os.fsencode(path)))

    def last_step(self) -> np.ndarray:
        """Per slab: [B00, B01, B11, c0, c1, u0, u1, rank] of its latest update."""
        buf = np.zeros((self.nslabs, 8))
        self._c(self._lib.bd3mg_last_step(self._ctx, buf.ctypes.data))
        return buf

    def apply_H(self, t, adjoint: bool = False):
        torch = _torch()
        t = t.contiguous()
        out = torch.empty_like(t)
        fn = self._lib.bd3mg_apply_HT if adjoint else self._lib.bd3mg_apply_H
        self._c(fn(self._ctx, ctypes.c_void_p(_ptr(t)), ctypes.c_void_p(_ptr(out))))
        return out

    def colours(self):
        col = np.zeros(self.nslabs, np.int32)
        nc = ctypes.c_int()
        self._c(self._lib.bd3mg_slab_colours(self._ctx, col.ctypes.data, ctypes.byref(nc)))
        return col, nc.value

    KERNEL_CLASSES = ("objective", "residual", "gradient", "curvature", "update", "dense")

    def profile_iteration(self):
        """One iteration with CUDA events around every launch: {class: (ms, launches)}."""
        ms = np.zeros(len(Solver.KERNEL_CLASSES))
        cnt = np.zeros(len(Solver.KERNEL_CLASSES), np.int32)
        self._c(self._lib.bd3mg_profile_iteration(self._ctx, ms.ctypes.data, cnt.ctypes.data))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(self.KERNEL_CLASSES)}

    def lipschitz(self) -> float:
        """The metric constant L (the caller's, else the library's Lipschitz bound)."""
        L = np.zeros(1)
        self._c(self._lib.bd3mg_lipschitz(self._ctx, L.ctypes.data))
        return float(L[0])

    def launches_per_iteration(self) -> int:
        return int(self._lib.bd3mg_launches_per_iteration(self._ctx))

    @classmethod
    def from_problem(cls, prob, x0=None, device="cuda", slabs="auto", **kw):
        torch = _torch()
        y = torch.from_numpy(prob.y).to(device)
        if x0 is not None:
            x0 = torch.from_numpy(np.ascontiguousarray(x0, np.float32)).to(device)
        sl = prob.slabs if slabs == "auto" else slabs
        kw.setdefault("penalty", getattr(prob, "penalty", 0))
        kw.setdefault("kappa", getattr(prob, "kappa", 0.0))
        return cls(prob.shape, prob.psf, y, x0, lam=prob.lam, delta=prob.delta, eta=prob.eta, xmin=prob.xmin,
                   xmax=prob.xmax, slabs=sl, **kw)


class BatchSolver:
    """Many independent volumes iterated in lockstep by one context (plain 3MG each)."""

    def __init__(self, problems, x0s=None, device="cuda", zchunk: int = 0, stream=None,
                 use_torch_allocator: bool = True, precision: int = FP32, separate_update: int = 0,
                 curv_rows: int = 0, persistent: int = 0):
        torch = _torch()
        lib = load()
        self.shapes = [tuple(int(s) for s in p.shape) for p in problems]
        self.nvol = len(problems)
        arr = (Params * self.nvol)()
        keep = []
        ys, xs = [], []
        precs = list(precision) if isinstance(precision, (list, tuple)) else [precision] * self.nvol
        for v, p in enumerate(problems):
            prm, k = make_params(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax, p.slabs, precs[v], 1e-12,
                                 zchunk, getattr(p, "penalty", 0), getattr(p, "kappa", 0.0),
                                 separate_update=separate_update, curv_rows=curv_rows, persistent=persistent)
            arr[v] = prm
            keep.append(k)
            yt = torch.from_numpy(np.ascontiguousarray(p.y, np.float32)).to(device)
            ys.append(yt)
            if x0s is not None and x0s[v] is not None:
                xs.append(torch.from_numpy(np.ascontiguousarray(x0s[v], np.float32)).to(device))
            else:
                xs.append(None)
        on_dev = bool(ys[0].is_cuda)
        yptr = (ctypes.c_void_p * self.nvol)(*[_ptr(t) for t in ys])
        xptr = (ctypes.c_void_p * self.nvol)(*[(_ptr(t) if t is not None else None) for t in xs])
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        alloc_p = None
        if use_torch_allocator:
            al, cbs = _torch_allocator()
            keep += [al, cbs]
            alloc_p = ctypes.byref(al)
        ctx = ctypes.c_void_p()
        st = lib.bd3mg_batch_create(self.nvol, arr, yptr, xptr, int(on_dev), ctypes.c_void_p(int(s)), alloc_p,
                                    ctypes.byref(ctx))
        if st != 0:
            msg = lib.bd3mg_error_string(ctx).decode() if ctx.value else lib.bd3mg_status_string(st).decode()
            if ctx.value:
                lib.bd3mg_destroy(ctx)
            raise Bd3mgError(st, msg)
        self._ctx, self._keep, self._lib = ctx, [arr, keep, ys, xs], lib

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.bd3mg_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, st):
        _check(self._ctx, st)

    def iterate(self, n: int, trace: bool = True):
        """n lockstep iterations; returns the (nvol, n+1) objective traces or None."""
        buf = np.zeros((self.nvol, n + 1)) if trace else None
        self._c(self._lib.bd3mg_iterate(self._ctx, int(n), buf.ctypes.data if trace else None))
        return buf

    def iterate_async(self, n: int):
        self._c(self._lib.bd3mg_iterate_async(self._ctx, int(n)))

    def set_stopping(self, tol: float = 0.0, f_target=None):
        """Per volume: stop once ||x^k - x^{k-1}|| <= tol ||x^{k-1}|| or f(x^k) <= f_target[v]."""
        t = None if f_target is None else np.ascontiguousarray(f_target, np.float64)
        if t is not None and t.shape != (self.nvol,):
            raise ValueError("f_target needs one value per volume")
        self._c(self._lib.bd3mg_set_stopping(self._ctx, float(tol), None if t is None else t.ctypes.data))
        self._keep_t = t

    def stopped(self) -> np.ndarray:
        """Per volume: sweeps after which it stopped, or -1 while it runs."""
        k = np.zeros(self.nvol, np.int32)
        self._c(self._lib.bd3mg_stopped(self._ctx, k.ctypes.data))
        return k

    def objectives(self):
        f = np.zeros(self.nvol)
        self._c(self._lib.bd3mg_objectives(self._ctx, f.ctypes.data))
        return f

    def get(self, vol: int, which: int = 0, out=None):
        """Volume vol's x (which=0), d (1) or g (2) as a CUDA tensor."""
        torch = _torch()
        if out is None:
            out = torch.empty(self.shapes[vol], dtype=torch.float32, device="cuda")
        self._c(self._lib.bd3mg_get_volume(self._ctx, int(vol), int(which), ctypes.c_void_p(_ptr(out)),
                                           int(out.is_cuda)))
        return out

    def set_escalation(self, tol: float):
        """BF16 gradient: switch to an FP32 gradient once f decreases by <= tol |f| per iteration."""
        self._c(self._lib.bd3mg_set_escalation(self._ctx, float(tol)))

    def escalated(self) -> int:
        """Iteration count at which the context switched to an FP32 gradient, or -1."""
        at = ctypes.c_longlong()
        self._c(self._lib.bd3mg_escalated(self._ctx, ctypes.byref(at)))
        return int(at.value)

    def save(self, path: str):
        """Checkpoint x, d and the iteration count to `path`."""
        self._c(self._lib.bd3mg_save(self._ctx, os.fsencode(path)))

    def load(self, path: str):
        """Resume from a checkpoint written by save() of an identical context."""
        self._c(self._lib.bd3mg_load(self._ctx, os.fsencode(path)))

    def profile_iteration(self):
        ms = np.zeros(len(Solver.KERNEL_CLASSES))
        cnt = np.zeros(len(Solver.KERNEL_CLASSES), np.int32)
        self._c(self._lib.bd3mg_profile_iteration(self._ctx, ms.ctypes.data, cnt.ctypes.data))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(Solver.KERNEL_CLASSES)}

    def lipschitz(self) -> np.ndarray:
        """The metric constant L of each volume."""
        L = np.zeros(self.nvol)
        self._c(self._lib.bd3mg_lipschitz(self._ctx, L.ctypes.data))
        return L

    def launches_per_iteration(self) -> int:
        return int(self._lib.bd3mg_launches_per_iteration(self._ctx))


def autotune(problems, iters: int = 10, cache_path: Optional[str] = None, precision: int = FP32):
    """Fastest work shape for these volumes (bd3mg_autotune): (zchunk, curvature tile rows, ms per
    iteration or -1 if cached)."""
    torch = _torch()
    lib = load()
    n = len(problems)
    arr = (Params * n)()
    keep, ys = [], []
    for v, p in enumerate(problems):
        prm, k = make_params(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax, p.slabs, precision, 1e-12, 0)
        arr[v] = prm
        keep.append(k)
        ys.append(torch.from_numpy(np.ascontiguousarray(p.y, np.float32)).cuda())
    yptr = (ctypes.c_void_p * n)(*[_ptr(t) for t in ys])
    z = ctypes.c_int()
    rows = ctypes.c_int()
    ms = ctypes.c_double()
    s = torch.cuda.current_stream().cuda_stream
    st = lib.bd3mg_autotune(n, arr, yptr, 1, ctypes.c_void_p(int(s)), int(iters),
                            os.fsencode(cache_path) if cache_path else None, ctypes.byref(z), ctypes.byref(rows),
                            ctypes.byref(ms))
    if st != 0:
        raise Bd3mgError(st, lib.bd3mg_status_string(st).decode())
    return int(z.value), int(rows.value), float(ms.value)
