"""Pins of the oracle's ablation variants (Section 3.2, Table 1) and block schedules.

- The Lipschitz bound dominates the largest eigenvalue of the Hessian of f
  (dense, by central differences of the pinned gradient) at random points in
  every penalty mode, and its blur part dominates ||H||_2^2 of the dense matrix.
- D = -g with A = L I is gradient descent with step 1/L: on the least-squares
  case it equals the textbook iteration with the dense matrix (numpy).  The
  memory-gradient subspace with A = L I gives the same iterates (the gradient
  lies in the subspace, so the isotropic majorant's minimiser ignores d).
- The conjugate direction (Fletcher-Reeves) with the exact majorant of a
  quadratic is an exact line search, so it equals linear conjugate gradients
  (scipy) on the least-squares case; with A = L I its first step is the
  gradient step and it descends monotonically.
- The Jacobi schedule equals the sequential one when the slabs do not couple
  (no z blur, no penalty), and with the curvature inflated by the number of
  slabs it descends monotonically on a coupled problem.
"""
import numpy as np
import pytest
from scipy.sparse.linalg import cg

import oracle
from paper_2002_02328_gb300 import synth


def _matrix(op):
    n = int(np.prod(op.shape))
    M = np.zeros((n, n))
    for m in range(n):
        e = np.zeros(n)
        e[m] = 1.0
        M[:, m] = oracle.apply_H(op, e.reshape(op.shape)).ravel()
    return M


def _hessian(op, y, x, h=1e-6):
    n = x.size
    Hs = np.zeros((n, n))
    for m in range(n):
        e = np.zeros(n)
        e[m] = h
        gp = oracle.gradient(op, y, x + e.reshape(x.shape)).ravel()
        gm = oracle.gradient(op, y, x - e.reshape(x.shape)).ravel()
        Hs[:, m] = (gp - gm) / (2 * h)
    return 0.5 * (Hs + Hs.T)


@pytest.mark.parametrize("mode,kappa", [(0, 0.0), (1, 0.4), (2, 0.0)])
def test_lipschitz_bound_dominates_the_hessian(mode, kappa):
    p = synth.tiny_problem(shape=(3, 4, 5), psf_shape=(3, 3, 3), sxy=(0.5, 1.2), sz=0.7, seed=3)
    op = oracle.OracleProblem(p.shape, p.psf, lam=0.05, delta=0.05, eta=1.0, penalty=mode, kappa=kappa)
    L = oracle.lipschitz_bound(op)
    rng = np.random.default_rng(mode)
    worst = 0.0
    for _ in range(3):
        # small differences (the penalty's curvature is largest near t = 0) and some voxels outside the box
        x = 0.5 + 0.01 * rng.standard_normal(p.shape)
        x[0, 0, :2] = [1.3, -0.2]
        worst = max(worst, float(np.max(np.linalg.eigvalsh(_hessian(op, p.y, x)))))
    assert worst <= L
    M = _matrix(op)
    pen = 8 * 0.05 / 0.05 + 8 * kappa if mode == 1 else 12 * 0.05 / 0.05
    assert np.linalg.norm(M, 2) ** 2 <= L - 2.0 - pen + 1e-12


def _least_squares_case(seed=1):
    p = synth.tiny_problem(shape=(4, 6, 6), psf_shape=(3, 3, 3), sxy=(0.5, 0.9), sz=0.6, seed=seed)
    return p, oracle.OracleProblem(p.shape, p.psf, lam=0.0, delta=0.1, eta=0.0)


@pytest.mark.parametrize("direction", [oracle.DIR_GRADIENT, oracle.DIR_MEMORY_GRADIENT])
def test_lipschitz_metric_is_gradient_descent(direction):
    p, op = _least_squares_case()
    M = _matrix(op)
    L = 1.5 * np.linalg.norm(M, 2) ** 2
    y = p.y.astype(np.float64).ravel()
    x0 = synth.uniform_start(p.y, seed=2).astype(np.float64)
    xr = x0.ravel().copy()
    for _ in range(7):
        xr = xr - (M.T @ (M @ xr - y)) / L
    x, _, ft = oracle.run_variant(op, p.y, x0, 7, metric=oracle.METRIC_LIPSCHITZ, lipschitz=L, direction=direction)
    np.testing.assert_allclose(x.ravel(), xr, rtol=0, atol=1e-12 * np.linalg.norm(xr))


def test_conjugate_direction_with_exact_majorant_is_linear_cg():
    p, op = _least_squares_case()
    M = _matrix(op)
    y = p.y.astype(np.float64).ravel()
    x0 = synth.uniform_start(p.y, seed=1).astype(np.float64)
    its = []
    cg(M.T @ M, M.T @ y, x0=x0.ravel().copy(), rtol=1e-300, atol=0.0, maxiter=6,
       callback=lambda xk: its.append(xk.copy()))
    for k in range(1, 7):
        x, _, _ = oracle.run_variant(op, p.y, x0, k, direction=oracle.DIR_CONJUGATE)
        np.testing.assert_allclose(x.ravel(), its[k - 1], rtol=0, atol=1e-9 * np.linalg.norm(its[k - 1]))


def test_conjugate_direction_with_lipschitz_metric_descends():
    p = synth.tiny_problem(shape=(6, 10, 12), psf_shape=(3, 3, 3), seed=4)
    op = oracle.OracleProblem.from_synth(p)
    L = oracle.lipschitz_bound(op)
    x1g, _, _ = oracle.run_variant(op, p.y, p.y, 1, metric=1, lipschitz=L, direction=oracle.DIR_GRADIENT)
    x1c, _, _ = oracle.run_variant(op, p.y, p.y, 1, metric=1, lipschitz=L, direction=oracle.DIR_CONJUGATE)
    np.testing.assert_array_equal(x1g, x1c)
    g0 = oracle.gradient(op, p.y, p.y.astype(np.float64))
    np.testing.assert_allclose(x1g, p.y - g0 / L, rtol=0, atol=1e-12)
    _, _, ft = oracle.run_variant(op, p.y, p.y, 60, metric=1, lipschitz=L, direction=oracle.DIR_CONJUGATE)
    assert np.all(np.diff(ft) <= 1e-13 * np.abs(ft[1:]))
    # the descent lemma for a step 1/L along -g
    assert ft[1] <= ft[0] - 0.5 * np.sum(g0 * g0) / L * (1 - 1e-9)


def test_jacobi_equals_sequential_when_slabs_decouple():
    # no z blur and no penalty: the objective is a sum over slices
    p = synth.tiny_problem(shape=(8, 10, 12), psf_shape=(3, 3, 1), seed=5)
    op = oracle.OracleProblem(p.shape, p.psf, lam=0.0, delta=0.1, eta=1.0)
    bounds = [0, 3, 5, 8]
    xs, ds, fs = oracle.run_variant(op, p.y, p.y, 6, bounds=bounds, schedule=oracle.SCHEDULE_SEQUENTIAL)
    xj, dj, fj = oracle.run_variant(op, p.y, p.y, 6, bounds=bounds, schedule=oracle.SCHEDULE_JACOBI)
    np.testing.assert_allclose(xj, xs, rtol=0, atol=1e-13)
    np.testing.assert_allclose(fj, fs, rtol=1e-13)


def test_jacobi_with_inflation_descends_on_coupled_slabs():
    p = synth.tiny_problem(shape=(12, 10, 12), psf_shape=(5, 5, 5), seed=6)
    op = oracle.OracleProblem.from_synth(p)
    bounds = [0, 3, 6, 9, 12]
    _, _, fj = oracle.run_variant(op, p.y, synth.uniform_start(p.y, seed=7), 40, bounds=bounds,
                                  schedule=oracle.SCHEDULE_JACOBI, inflation=4.0)
    assert np.all(np.diff(fj) <= 1e-12 * np.abs(fj[1:]))
    _, _, fs = oracle.run_variant(op, p.y, synth.uniform_start(p.y, seed=7), 40, bounds=bounds)
    assert fs[-1] < fs[0] and fj[-1] < fj[0]
