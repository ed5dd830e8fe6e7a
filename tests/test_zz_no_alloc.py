"""GPU check of bd3mg_objective_noalloc, the objective entry point that allocates
no device memory (for callers that may not allocate: plug-ins inside a host
framework that owns all device memory, latency-critical loops that must not
take the allocator's locks or the synchronisation cudaFree implies).

It is compared, through the C ABI, with the context entry point bd3mg_objective
on two calls in a row with different iterates, within the objective tolerance
the other parity tests use (relative 1e-5).  The file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_objective_matches_context_objective(cuda_lib):
    import torch
    p = synth.workload_plain_small()                       # 64x64x24, nx multiple of 4
    params, keep = cuda_lib.make_params(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax)
    y = torch.from_numpy(p.y).cuda()
    starts = [p.y, synth.uniform_start(p.y, seed=2)]
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with cuda_lib.Solver.from_problem(p) as s:
        for x0 in starts:
            x = torch.from_numpy(np.ascontiguousarray(x0)).cuda()
            s.set_x(x)
            f_ref, parts_ref = s.objective(parts=True)
            out.fill_(-1.0)
            cuda_lib.bd3mg_objective_noalloc(params, x, y, out)
            torch.cuda.synchronize()
            f, f1, f2, f3 = out.cpu().numpy()
            assert abs(f - f_ref) <= 1e-5 * abs(f_ref)
            np.testing.assert_allclose([f1, f2, f3], parts_ref, rtol=1e-5, atol=1e-9 * abs(f_ref))


def test_noalloc_rejects_oversized_and_misaligned_volumes(cuda_lib):
    import torch
    fx, fy, fz = synth.gaussian_factors(4096, 3, 3, 3, 0.5, 1.0)
    big_shape = (4096, 4096, 4096)                       # plan far beyond the static scratch
    params, keep = cuda_lib.make_params(big_shape, synth.dense_psf(fx, fy, fz))
    t = torch.zeros(64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(cuda_lib.Bd3mgError) as e:
        cuda_lib.bd3mg_objective_noalloc(params, t, t, out)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    fx, fy, fz = synth.gaussian_factors(4, 3, 3, 3, 0.5, 1.0)
    params, keep = cuda_lib.make_params((4, 8, 6), synth.dense_psf(fx, fy, fz))   # nx = 6: not a multiple of 4
    with pytest.raises(cuda_lib.Bd3mgError) as e:
        cuda_lib.bd3mg_objective_noalloc(params, t, t, out)
    assert e.value.status == 1 and "multiple of 4" in str(e.value)
