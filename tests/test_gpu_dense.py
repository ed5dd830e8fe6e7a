"""GPU parity of the dense (non-separable) PSF path against the FP64 oracle.

The paper's blur is a rotated Gaussian per depth (Section 3.1), which does not
factor; its experiments use 11x11x21 and 5x5x11 kernels (Sections 3.2, 3.3).
The dense path applies the taps as given.  Bounds as for the separable path:
H and H^T within relative L2 2e-6 and element-wise 1e-5 of max|ref| (a dense
sum of up to 2541 FP32 products of a sum-1 PSF rounds each output by a few ulp
of the input's magnitude times the square root of the tap count, far below
these); objective and gradient 1e-5; iterates after a few iterations or sweeps
2e-5 and the trace 1e-5.  A separable PSF forced onto the dense path gives the
separable path's iterates to 1e-5.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2002_02328_gb300 import synth
from tests.test_gpu_3mg import _colour_major

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _maxrel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _dense_problem(shape, psf_shape, seed, slabs=None, **kw):
    psf = synth.rotated_gaussian_psf(shape[0], psf_shape, seed)
    return synth.make_problem_dense(f"dense-{shape}", shape, 6, psf, 0.02, seed, slabs=slabs, **kw)


@pytest.mark.parametrize("shape,psf_shape", [
    ((7, 19, 45), (3, 3, 3)),          # ragged tiles
    ((24, 40, 45), (11, 11, 21)),      # the paper's FlyBrain kernel; nz equal to its depth extent
    ((16, 37, 33), (5, 5, 11)),        # the paper's Aneurysm kernel
    ((3, 8, 8), (7, 9, 5)),            # nz < pz, px != py, one partial tile
])
def test_dense_H_and_HT_match_oracle(cuda_lib, shape, psf_shape):
    import torch
    p = _dense_problem(shape, psf_shape, seed=1)
    op = oracle.OracleProblem.from_synth(p)
    x = np.random.default_rng(2).standard_normal(shape).astype(np.float32)
    with cuda_lib.Solver.from_problem(p) as s:
        xt = torch.from_numpy(x).cuda()
        hx = s.apply_H(xt).cpu().numpy()
        htx = s.apply_H(xt, adjoint=True).cpu().numpy()
    hr, htr = oracle.apply_H(op, x), oracle.apply_HT(op, x)
    assert _rel(hx, hr) <= 2e-6 and _rel(htx, htr) <= 2e-6
    assert _maxrel(hx, hr) <= 1e-5 and _maxrel(htx, htr) <= 1e-5


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_dense_objective_and_gradient_match_oracle(cuda_lib, mode):
    p = _dense_problem((12, 40, 33), (7, 7, 9), seed=3)
    p = dataclasses.replace(p, penalty=mode, kappa=0.3 if mode == 1 else 0.0)
    x0 = synth.uniform_start(p.y, seed=4) * 1.3 - 0.1
    op = oracle.OracleProblem.from_synth(p)
    with cuda_lib.Solver.from_problem(p, x0=x0) as s:
        f, parts = s.objective(parts=True)
        g, fg = s.gradient()
        g = g.cpu().numpy()
    f_ref, parts_ref = oracle.objective(op, p.y, x0, parts=True)
    g_ref = oracle.gradient(op, p.y, x0)
    assert abs(f - f_ref) <= 1e-5 * abs(f_ref) and abs(fg - f_ref) <= 1e-5 * abs(f_ref)
    np.testing.assert_allclose(parts, parts_ref, rtol=1e-5, atol=1e-9 * abs(f_ref))
    assert _rel(g, g_ref) <= 1e-5 and _maxrel(g, g_ref) <= 2e-5


def test_dense_plain_iterations_match_oracle(cuda_lib):
    p = _dense_problem((13, 45, 70), (11, 11, 9), seed=5)
    op = oracle.OracleProblem.from_synth(p)
    oracle.set_threads(oracle.max_threads())
    xr, _, fr = oracle.run(op, p.y, p.y, 12)
    with cuda_lib.Solver.from_problem(p) as s:
        tr = s.iterate(12)
        x = s.get_x().cpu().numpy()
    assert _rel(x, xr) <= 2e-5
    assert np.max(np.abs(tr - fr) / np.abs(fr)) <= 1e-5
    assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:]))


def test_dense_slab_sweeps_match_oracle(cuda_lib):
    bounds = [0, 5, 9, 16, 24]
    p = _dense_problem((24, 36, 40), (5, 5, 11), seed=6, slabs=bounds)
    op = oracle.OracleProblem.from_synth(p)
    _, order = _colour_major(bounds, 11)
    oracle.set_threads(oracle.max_threads())
    xr, _, fr = oracle.run(op, p.y, p.y, 5, bounds=bounds, order=order)
    with cuda_lib.Solver.from_problem(p) as s:
        tr = s.iterate(5)
        x = s.get_x().cpu().numpy()
    assert _rel(x, xr) <= 2e-5
    assert np.max(np.abs(tr - fr) / np.abs(fr)) <= 1e-5


def test_dense_path_on_separable_psf_equals_separable_path(cuda_lib):
    p = synth.tiny_problem(shape=(13, 45, 70), psf_shape=(5, 5, 5), seed=7, n_ellipsoids=6)
    with cuda_lib.Solver.from_problem(p) as a, cuda_lib.Solver.from_problem(p, psf_mode=cuda_lib.PSF_DENSE) as b:
        ta, tb = a.iterate(20), b.iterate(20)
        xa, xb = a.get_x().cpu().numpy(), b.get_x().cpu().numpy()
    assert _rel(xb, xa) <= 1e-5
    np.testing.assert_allclose(tb, ta, rtol=1e-5)


def test_dense_limits_are_rejected(cuda_lib):
    import torch
    shape = (4, 16, 16)
    y = torch.zeros(shape, device="cuda")
    with pytest.raises(cuda_lib.Bd3mgError) as e:          # xy radius 6: beyond the dense kernels
        cuda_lib.Solver(shape, synth.random_psf(4, (13, 13, 3), seed=1), y)
    assert e.value.status == 7
    with pytest.raises(cuda_lib.Bd3mgError) as e:          # BF16 gradient on the dense path
        cuda_lib.Solver(shape, synth.random_psf(4, (3, 3, 3), seed=1), y, precision=cuda_lib.BF16_GRADIENT)
    assert e.value.status == 7
