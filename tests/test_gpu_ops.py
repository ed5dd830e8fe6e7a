"""GPU parity of the operators, objective and gradient against the FP64 oracle.

Every call goes through the C ABI (libbd3mg.so via the ctypes binding).
Tolerances: FP32 arithmetic against FP64 -- relative L2 error 2e-6 for single
operator applications, 1e-5 for the objective and gradient (the parity bound
for one iteration).  Beside each L2 bound an element-wise bound, max|a - b|
over max|b|, catches errors confined to a few voxels (a boundary row, a tile
seam) that the volume norm would dilute: 1e-5 for an operator (a separable
pass of at most 11 + 11 + 11 FP32 taps of a sum-1 PSF rounds each output by at
most ~33 ulp of max|x|, 2e-6 of it, and max|Hx| is not below a fifth of max|x|
here), 2e-5 for the gradient (the residual entering H^T carries the same
rounding).
"""
import numpy as np
import pytest

import oracle
from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [  # (nz, ny, nx), (px, py, pz)
    ((7, 19, 45), (3, 3, 3)),        # ragged tiles in x and y
    ((5, 33, 70), (7, 5, 5)),        # px != py
    ((1, 16, 32), (5, 5, 1)),        # single slice, no z blur
    ((3, 8, 8), (3, 3, 7)),          # nz < pz, one partial tile
    ((12, 40, 33), (9, 9, 7)),       # the largest supported-in-configs PSF
    ((9, 17, 64), (11, 11, 11)),     # largest compiled radii
]


def _problem(shape, psf_shape, seed=0):
    return synth.tiny_problem(shape=shape, psf_shape=psf_shape, sxy=(0.5, 2.0), sz=1.0, seed=seed,
                              n_ellipsoids=4)


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _maxrel(a, b):
    """Largest element-wise error, relative to the largest reference magnitude."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("shape,psf_shape", SHAPES)
def test_H_and_HT_match_oracle(cuda_lib, shape, psf_shape):
    import torch
    p = _problem(shape, psf_shape)
    op = oracle.OracleProblem.from_synth(p)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape).astype(np.float32)
    with cuda_lib.Solver.from_problem(p) as s:
        xt = torch.from_numpy(x).cuda()
        hx = s.apply_H(xt).cpu().numpy()
        htx = s.apply_H(xt, adjoint=True).cpu().numpy()
    hx_ref, htx_ref = oracle.apply_H(op, x), oracle.apply_HT(op, x)
    assert _rel(hx, hx_ref) <= 2e-6
    assert _rel(htx, htx_ref) <= 2e-6
    assert _maxrel(hx, hx_ref) <= 1e-5
    assert _maxrel(htx, htx_ref) <= 1e-5


def test_gpu_adjoint_identity(cuda_lib):
    import torch
    shape, psf_shape = (11, 29, 51), (7, 7, 5)
    p = _problem(shape, psf_shape, seed=2)
    rng = np.random.default_rng(3)
    x = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    r = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    with cuda_lib.Solver.from_problem(p) as s:
        lhs = torch.dot(s.apply_H(x).double().ravel(), r.double().ravel()).item()
        rhs = torch.dot(x.double().ravel(), s.apply_H(r, adjoint=True).double().ravel()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("shape,psf_shape", SHAPES[:5])
def test_objective_and_gradient_match_oracle(cuda_lib, shape, psf_shape):
    p = _problem(shape, psf_shape, seed=4)
    x0 = synth.uniform_start(p.y, seed=4) * 1.3 - 0.1      # some voxels outside the box
    op = oracle.OracleProblem.from_synth(p)
    with cuda_lib.Solver.from_problem(p, x0=x0) as s:
        f, parts = s.objective(parts=True)
        g, fg = s.gradient()
        g = g.cpu().numpy()
    f_ref, parts_ref = oracle.objective(op, p.y, x0, parts=True)
    g_ref = oracle.gradient(op, p.y, x0)
    assert abs(f - f_ref) <= 1e-5 * abs(f_ref)
    assert abs(fg - f_ref) <= 1e-5 * abs(f_ref)
    np.testing.assert_allclose(parts, parts_ref, rtol=1e-5, atol=1e-9 * abs(f_ref))
    assert _rel(g, g_ref) <= 1e-5
    assert _maxrel(g, g_ref) <= 2e-5


def test_non_separable_psf_takes_the_dense_path(cuda_lib):
    import torch
    shape = (4, 16, 16)
    psf = synth.random_psf(4, (3, 3, 3), seed=1)
    y = np.random.default_rng(2).uniform(0, 1, size=shape).astype(np.float32)
    op = oracle.OracleProblem(shape, psf)
    with cuda_lib.Solver(shape, psf, torch.from_numpy(y).cuda()) as s:
        f = s.objective()
    f_ref = oracle.objective(op, y, y)
    assert abs(f - f_ref) <= 1e-5 * abs(f_ref)


def test_invalid_arguments_are_rejected(cuda_lib):
    import torch
    shape = (4, 16, 16)
    fx, fy, fz = synth.gaussian_factors(4, 3, 3, 3, 0.5, 1.0)
    psf = synth.dense_psf(fx, fy, fz)
    y = torch.zeros(shape, device="cuda")
    with pytest.raises(cuda_lib.Bd3mgError) as e:
        cuda_lib.Solver(shape, psf, y, lam=-1.0)
    assert e.value.status == 1
    with pytest.raises(cuda_lib.Bd3mgError) as e:
        cuda_lib.Solver(shape, psf, y, slabs=[0, 3, 2, 4])
    assert e.value.status == 1
    with pytest.raises(cuda_lib.Bd3mgError) as e:
        cuda_lib.Solver(shape, psf, y, xmin=1.0, xmax=0.0)
    assert e.value.status == 1


def test_non_finite_input_poisons_context(cuda_lib):
    import torch
    p = _problem((4, 16, 32), (3, 3, 3))
    y = p.y.copy()
    y[1, 3, 5] = np.nan
    with cuda_lib.Solver(p.shape, p.psf, torch.from_numpy(y).cuda()) as s:
        with pytest.raises(cuda_lib.Bd3mgError) as e:
            s.iterate(2)
        assert e.value.status == 5
        with pytest.raises(cuda_lib.Bd3mgError) as e:
            s.objective()
        assert e.value.status == 6            # sticky


def test_host_buffers_accepted(cuda_lib):
    import torch
    p = _problem((6, 20, 36), (5, 5, 3))
    op = oracle.OracleProblem.from_synth(p)
    with cuda_lib.Solver(p.shape, p.psf, torch.from_numpy(p.y)) as s:   # host y
        f = s.objective()
        x = s.get_x(torch.empty(p.shape, dtype=torch.float32))          # host out
    assert abs(f - oracle.objective(op, p.y, p.y)) <= 1e-5 * abs(f)
    np.testing.assert_array_equal(x.numpy(), p.y)
