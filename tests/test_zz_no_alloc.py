"""GPU check of bd3mg_objective_noalloc, the objective entry point that allocates
no device memory (for callers that may not allocate: plug-ins inside a host
framework that owns all device memory, latency-critical loops that must not
take the allocator's locks or the synchronisation cudaFree implies).

It is compared, through the C ABI, with the context entry point bd3mg_objective
on two calls in a row with different iterates, within the objective tolerance
the other parity tests use (relative 1e-5): on the 64x64x24 workload, and on a
ragged 36x37x21 volume (nx = 36: rows of 144 bytes, not a multiple of 32, so
the call's unpadded rows differ from the context's padded pitch) in every
penalty mode.  Free device memory is unchanged across repeated calls.  The
file is named so that pytest collects it last.
"""
import dataclasses

import numpy as np
import pytest

from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


def _compare(cuda_lib, p):
    import torch
    params, keep = cuda_lib.make_params(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax,
                                        penalty=p.penalty, kappa=p.kappa)
    y = torch.from_numpy(np.ascontiguousarray(p.y)).cuda()
    starts = [p.y, synth.uniform_start(p.y, seed=2)]
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with cuda_lib.Solver.from_problem(p) as s:
        for x0 in starts:
            x = torch.from_numpy(np.ascontiguousarray(x0)).cuda()
            s.set_x(x)
            f_ref, parts_ref = s.objective(parts=True)
            out.fill_(-1.0)
            cuda_lib.bd3mg_objective_noalloc(params, x, y, out)
            f, f1, f2, f3 = out.cpu().numpy()
            assert abs(f - f_ref) <= 1e-5 * abs(f_ref)
            np.testing.assert_allclose([f1, f2, f3], parts_ref, rtol=1e-5, atol=1e-9 * abs(f_ref))


def test_noalloc_objective_matches_context_objective(cuda_lib):
    _compare(cuda_lib, synth.workload_plain_small())       # 64x64x24


@pytest.mark.parametrize("mode,kappa", [(0, 0.0), (1, 0.3), (2, 0.0)])
def test_noalloc_objective_ragged_every_penalty_mode(cuda_lib, mode, kappa):
    p = synth.tiny_problem(shape=(21, 37, 36), psf_shape=(5, 5, 5), seed=7, n_ellipsoids=6)
    _compare(cuda_lib, dataclasses.replace(p, penalty=mode, kappa=kappa))


def test_noalloc_objective_allocates_no_device_memory(cuda_lib):
    import torch
    p = synth.tiny_problem(shape=(21, 37, 36), psf_shape=(5, 5, 5), seed=8, n_ellipsoids=6)
    params, keep = cuda_lib.make_params(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax)
    y = torch.from_numpy(np.ascontiguousarray(p.y)).cuda()
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    cuda_lib.bd3mg_objective_noalloc(params, y, y, out)     # first call: per-device set-up, module load
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    vals = []
    for _ in range(5):
        cuda_lib.bd3mg_objective_noalloc(params, y, y, out)
        vals.append(float(out[0].item()))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert len(set(vals)) == 1 and np.isfinite(vals[0])


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


def test_noalloc_reports_non_finite_input(cuda_lib):
    import torch
    p = synth.tiny_problem(shape=(21, 37, 36), psf_shape=(5, 5, 5), seed=9, n_ellipsoids=6)
    params, keep = cuda_lib.make_params(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax)
    y = torch.from_numpy(np.ascontiguousarray(p.y)).cuda()
    x = y.clone()
    x[3, 5, 7] = float("nan")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(cuda_lib.Bd3mgError) as e:
        cuda_lib.bd3mg_objective_noalloc(params, x, y, out)
    assert e.value.status == 5            # BD3MG_ENONFINITE
    assert not np.isfinite(out[0].item())
    cuda_lib.bd3mg_objective_noalloc(params, y, y, out)     # the next call is unaffected
    assert np.isfinite(out[0].item())
