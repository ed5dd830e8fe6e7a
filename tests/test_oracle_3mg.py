"""Pins for the oracle's 3MG iteration (CPU only).

* quadratic case (lambda = 0, eta = 0): the memory-gradient subspace step with
  exact minimisation is linear conjugate gradients on H^T H x = H^T y, so the
  iterates must equal scipy's CG iterates and converge to numpy's dense
  least-squares solution;
* H = I, lambda = 0: per-voxel closed form with the box penalty;
* synchronous descent f(x^{k+1}) <= f(x^k) (Section 2.4), stationarity (Theorem 1),
  uniqueness of the minimiser of this convex instance, mirror symmetry;
* block (slab) form: a block step only moves its own slab and decreases f.
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


def test_quadratic_case_is_conjugate_gradients():
    p = synth.tiny_problem(shape=(4, 6, 6), psf_shape=(3, 3, 3), sxy=(0.5, 0.9), sz=0.6, seed=1)
    op = oracle.OracleProblem(p.shape, p.psf, lam=0.0, delta=0.1, eta=0.0)
    M = _matrix(op)
    y = p.y.astype(np.float64).ravel()
    x0 = synth.uniform_start(p.y, seed=1).astype(np.float64).ravel()
    its = []
    cg(M.T @ M, M.T @ y, x0=x0.copy(), rtol=1e-300, atol=0.0, maxiter=6, callback=lambda xk: its.append(xk.copy()))
    x = x0.reshape(p.shape)
    d = np.zeros(p.shape)
    for k in range(6):
        x, d, _ = oracle.step(op, p.y, x, d)
        np.testing.assert_allclose(x.ravel(), its[k], rtol=0, atol=1e-9 * np.linalg.norm(its[k]))


def test_quadratic_case_reaches_dense_least_squares():
    # sigma 0.5..0.6 gives a blur matrix with condition number ~9, so the dense
    # solve is itself accurate to ~1e-15.
    p = synth.tiny_problem(shape=(4, 6, 6), psf_shape=(3, 3, 3), sxy=(0.5, 0.6), sz=0.5, seed=2)
    op = oracle.OracleProblem(p.shape, p.psf, lam=0.0, delta=0.1, eta=0.0)
    M = _matrix(op)
    xls = np.linalg.lstsq(M, p.y.astype(np.float64).ravel(), rcond=None)[0]
    x, _, ft = oracle.run(op, p.y, synth.uniform_start(p.y, seed=2), 150)
    assert np.linalg.norm(x.ravel() - xls) <= 1e-9 * np.linalg.norm(xls)


def test_identity_blur_box_closed_form():
    shape = (3, 5, 6)
    psf = np.ones((3, 1, 1, 1), np.float32)
    rng = np.random.default_rng(3)
    y = rng.uniform(-0.8, 1.8, shape).astype(np.float32)
    eta = 1.5
    op = oracle.OracleProblem(shape, psf, lam=0.0, delta=0.1, eta=eta, xmin=0.0, xmax=1.0)
    x, _, _ = oracle.run(op, y, np.zeros(shape), 60)
    yd = y.astype(np.float64)
    expect = np.where(yd > 1.0, (yd + 2 * eta * 1.0) / (1 + 2 * eta),
                      np.where(yd < 0.0, (yd + 2 * eta * 0.0) / (1 + 2 * eta), yd))
    np.testing.assert_allclose(x, expect, atol=1e-12)


@pytest.fixture(scope="module")
def small():
    p = synth.tiny_problem(shape=(6, 12, 10), psf_shape=(3, 3, 3), sxy=(0.5, 1.5), sz=1.0, seed=4,
                           n_ellipsoids=6)
    return p, oracle.OracleProblem.from_synth(p)


def test_first_step_is_steepest_descent(small):
    p, op = small
    x0 = p.y.astype(np.float64)
    g = oracle.gradient(op, p.y, x0)
    _, _, info = oracle.step(op, p.y, x0, np.zeros(p.shape))
    gAg = np.vdot(g, oracle.apply_A(op, x0, g))
    assert info["u"][1] == 0.0
    assert abs(info["u"][0] - np.vdot(g, g) / gAg) <= 1e-13 * abs(info["u"][0])


def test_monotone_descent_and_stationarity(small):
    p, op = small
    x, d, ft = oracle.run(op, p.y, synth.uniform_start(p.y, seed=4), 400)
    assert np.all(np.diff(ft) <= 1e-12 * np.abs(ft[1:]))
    g0 = oracle.gradient(op, p.y, synth.uniform_start(p.y, seed=4).astype(np.float64))
    g = oracle.gradient(op, p.y, x)
    assert np.linalg.norm(g) <= 1e-4 * np.linalg.norm(g0)


def test_unique_minimiser_from_two_starts(small):
    p, op = small
    xa, _, fa = oracle.run(op, p.y, p.y, 800)
    xb, _, fb = oracle.run(op, p.y, synth.uniform_start(p.y, seed=9), 800)
    assert abs(fa[-1] - fb[-1]) <= 1e-10 * abs(fa[-1])
    assert np.linalg.norm(xa - xb) <= 5e-5 * np.linalg.norm(xa)


def test_mirror_symmetry():
    p = synth.tiny_problem(shape=(4, 7, 9), psf_shape=(3, 3, 3), seed=5)
    psf = synth.random_psf(4, (3, 3, 3), seed=6)
    op = oracle.OracleProblem(p.shape, psf, lam=p.lam, delta=p.delta, eta=p.eta)
    op_m = oracle.OracleProblem(p.shape, psf[:, :, :, ::-1], lam=p.lam, delta=p.delta, eta=p.eta)
    y_m = p.y[:, :, ::-1]
    # V^X is a forward difference, so mirroring X changes which voxel a difference is
    # attached to but not the set of values: f is mirror-invariant.
    x, _, ft = oracle.run(op, p.y, p.y, 25)
    xm, _, ftm = oracle.run(op_m, y_m, y_m, 25)
    np.testing.assert_allclose(ft, ftm, rtol=1e-12)
    np.testing.assert_allclose(xm[:, :, ::-1], x, atol=1e-10)


def test_block_step_moves_only_its_slab_and_descends(small):
    p, op = small
    x = p.y.astype(np.float64)
    d = np.zeros(p.shape)
    f0 = oracle.objective(op, p.y, x)
    x1, d1, _ = oracle.step(op, p.y, x, d, 2, 4)
    assert np.all(x1[:2] == x[:2]) and np.all(x1[4:] == x[4:])
    assert np.any(x1[2:4] != x[2:4])
    assert np.all(d1[:2] == 0) and np.all(d1[4:] == 0)
    assert oracle.objective(op, p.y, x1) <= f0


def test_block_form_converges_to_the_same_minimiser(small):
    p, op = small
    xa, _, fa = oracle.run(op, p.y, p.y, 800)
    xs, _, fs = oracle.run(op, p.y, p.y, 800, bounds=[0, 2, 3, 6], order=[0, 2, 1])
    assert np.all(np.diff(fs) <= 1e-12 * np.abs(fs[1:]))
    assert abs(fs[-1] - fa[-1]) <= 1e-10 * abs(fa[-1])
    assert np.linalg.norm(xs - xa) <= 1e-4 * np.linalg.norm(xa)


def test_paper_penalty_descent_stationarity_and_slab_steps():
    """Penalty mode 1 (joint X-Y hyperbolic + kappa ||V^Z x||^2, Section 3.1):
    monotone descent to a stationary point in the plain form, and the slab
    form's sweeps descend to the same objective."""
    p = synth.tiny_problem(shape=(8, 10, 12), psf_shape=(3, 3, 3), seed=50, n_ellipsoids=4)
    op = oracle.OracleProblem(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax, penalty=1, kappa=0.05)
    x0 = synth.uniform_start(p.y, seed=5)
    x, _, ft = oracle.run(op, p.y, x0, 400)
    assert np.all(np.diff(ft) <= 1e-12 * np.abs(ft[1:]))
    g0 = oracle.gradient(op, p.y, x0.astype(np.float64))
    assert np.linalg.norm(oracle.gradient(op, p.y, x)) <= 1e-4 * np.linalg.norm(g0)
    xs, _, fs = oracle.run(op, p.y, x0, 400, bounds=[0, 3, 5, 8], order=[0, 2, 1])
    assert np.all(np.diff(fs) <= 1e-12 * np.abs(fs[1:]))
    assert abs(fs[-1] - ft[-1]) <= 1e-8 * abs(ft[-1])


def test_isotropic_penalty_descent_stationarity_and_slab_steps():
    """Penalty mode 2 (isotropic hyperbolic term over X, Y, Z): monotone descent to
    a stationary point in the plain form, and the slab form's sweeps descend to
    the same objective."""
    p = synth.tiny_problem(shape=(8, 10, 12), psf_shape=(3, 3, 3), seed=51, n_ellipsoids=4)
    op = oracle.OracleProblem(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax, penalty=2)
    x0 = synth.uniform_start(p.y, seed=6)
    x, _, ft = oracle.run(op, p.y, x0, 400)
    assert np.all(np.diff(ft) <= 1e-12 * np.abs(ft[1:]))
    g0 = oracle.gradient(op, p.y, x0.astype(np.float64))
    assert np.linalg.norm(oracle.gradient(op, p.y, x)) <= 1e-4 * np.linalg.norm(g0)
    xs, _, fs = oracle.run(op, p.y, x0, 400, bounds=[0, 3, 5, 8], order=[0, 2, 1])
    assert np.all(np.diff(fs) <= 1e-12 * np.abs(fs[1:]))
    assert abs(fs[-1] - ft[-1]) <= 1e-8 * abs(ft[-1])
