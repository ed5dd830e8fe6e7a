"""Failure detection on the GPU, without faulting, trapping or hanging it.

* A bounded device wait that runs out: the fault flag makes the first CTA of
  every curvature launch leave one slice copy out, so the shared-memory
  barrier it waits on never completes; the wait gives up after the context's
  limit (50 ms here), the CTA drains its other copies and returns, the call
  reports BD3MG_ETIMEOUT and the context is poisoned (BD3MG_ESTATE after).  The
  CUDA context stays usable: a new context afterwards reproduces, bit for bit,
  a run made before the fault.
* An allocation that fails: an allocator hook that returns NULL after a few
  successful allocations makes creation report BD3MG_ENOMEM (the partial state
  is released), and creation works again afterwards.
* The exact-refresh period and the wait limit are parameters: out-of-range
  values are rejected, and refreshing every iteration changes the iterates
  only by the FP32 drift the refresh bounds.
(Non-finite input reporting BD3MG_ENONFINITE is covered in test_gpu_ops.py.)
"""
import ctypes

import numpy as np
import pytest

from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


def _problem():
    return synth.tiny_problem(shape=(12, 32, 40), psf_shape=(5, 5, 5), seed=91, n_ellipsoids=6,
                              slabs=[0, 3, 7, 12])


def test_device_wait_runs_out_and_reports_timeout(cuda_lib):
    p = _problem()
    with cuda_lib.Solver.from_problem(p) as ref:
        tr_ref = ref.iterate(4)
        x_ref = ref.get_x().cpu().numpy()
    s = cuda_lib.Solver.from_problem(p, barrier_timeout_ms=50)
    try:
        s.iterate(1)
        s.inject_fault(cuda_lib.FAULT_SKIP_COPY)
        with pytest.raises(cuda_lib.Bd3mgError) as e:
            s.iterate(1)
        assert e.value.status == 4, str(e.value)                       # BD3MG_ETIMEOUT
        with pytest.raises(cuda_lib.Bd3mgError) as e2:
            s.iterate(1)
        assert e2.value.status == 6                                     # poisoned: BD3MG_ESTATE
    finally:
        s.close()
    with cuda_lib.Solver.from_problem(p) as again:
        tr = again.iterate(4)
        x = again.get_x().cpu().numpy()
    assert np.array_equal(tr, tr_ref) and np.array_equal(x, x_ref)


def test_fault_flag_off_changes_nothing(cuda_lib):
    p = _problem()
    with cuda_lib.Solver.from_problem(p) as a, cuda_lib.Solver.from_problem(p, barrier_timeout_ms=50) as b:
        b.inject_fault(cuda_lib.FAULT_SKIP_COPY)
        b.inject_fault(cuda_lib.FAULT_NONE)
        assert np.array_equal(a.iterate(5), b.iterate(5))
    with cuda_lib.Solver.from_problem(p) as c:
        with pytest.raises(cuda_lib.Bd3mgError, match="fault kind"):
            c.inject_fault(7)


def test_allocation_failure_reports_enomem(cuda_lib):
    import torch
    p = _problem()
    lib = cuda_lib.load()
    params, keep = cuda_lib.make_params(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax, p.slabs)
    y = torch.from_numpy(p.y).cuda()
    held, calls = {}, [0]

    def alloc(user, nbytes, stream):
        calls[0] += 1
        if calls[0] > 3:
            return None                                                  # the fourth allocation fails
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
        held[t.data_ptr()] = t
        return t.data_ptr()

    def free(user, ptr, nbytes, stream):
        held.pop(ptr, None)

    al = cuda_lib.Allocator(cuda_lib._ALLOC_FN(alloc), cuda_lib._FREE_FN(free), None)
    ctx = ctypes.c_void_p()
    s = torch.cuda.current_stream().cuda_stream
    st = lib.bd3mg_create(ctypes.byref(params), ctypes.c_void_p(y.data_ptr()), None, 1, ctypes.c_void_p(s),
                          ctypes.byref(al), ctypes.byref(ctx))
    assert st == 2, lib.bd3mg_status_string(st)                          # BD3MG_ENOMEM
    if ctx.value:
        lib.bd3mg_destroy(ctx)
    torch.cuda.synchronize()
    assert calls[0] == 4 and not held                                    # every successful block returned
    with cuda_lib.Solver.from_problem(p) as ok:
        tr = ok.iterate(3)
    assert np.all(np.isfinite(tr)) and tr[-1] < tr[0]


def test_refresh_period_and_wait_limit_parameters(cuda_lib):
    p = _problem()
    for kw in (dict(refresh_every=-1), dict(barrier_timeout_ms=-5), dict(barrier_timeout_ms=600001)):
        with pytest.raises(cuda_lib.Bd3mgError) as e:
            cuda_lib.Solver.from_problem(p, **kw)
        assert e.value.status == 1
    with cuda_lib.Solver.from_problem(p) as a, cuda_lib.Solver.from_problem(p, refresh_every=1) as b:
        ta, tb = a.iterate(40), b.iterate(40)
        xa, xb = a.get_x().cpu().numpy(), b.get_x().cpu().numpy()
    assert np.max(np.abs(ta - tb) / np.abs(ta)) <= 1e-6
    assert np.linalg.norm(xa - xb) <= 1e-5 * np.linalg.norm(xa)
