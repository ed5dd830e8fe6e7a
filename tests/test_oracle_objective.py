"""Pins for the oracle's objective, gradient, majorant and 2x2 pseudo-inverse (CPU only)."""
import numpy as np
import pytest

import oracle
from paper_2002_02328_gb300 import synth
from tests.golden_io import load_cases


def _tiny(seed=0, **kw):
    p = synth.tiny_problem(seed=seed, **kw)
    return p, oracle.OracleProblem.from_synth(p)


def test_objective_hand_case_A():
    c = load_cases()["A"]
    op = oracle.OracleProblem(c["shape"], c["psf"], **c["params"])
    f, parts = oracle.objective(op, c["y"], c["x"], parts=True)
    np.testing.assert_allclose(parts, [c["f1"], c["f2"], c["f3"]], rtol=1e-15)
    np.testing.assert_allclose(oracle.gradient(op, c["y"], c["x"]), c["grad"], rtol=1e-15)


def test_objective_hand_case_B():
    c = load_cases()["B"]
    op = oracle.OracleProblem(c["shape"], c["psf"], **c["params"])
    f, parts = oracle.objective(op, c["y"], c["x"], parts=True)
    assert abs(parts[0] - c["f1"]) < 1e-15 and parts[1] == 0.0
    np.testing.assert_allclose(oracle.gradient(op, c["y"], c["x"]), c["grad"], atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_central_differences(seed):
    p, op = _tiny(seed=seed, shape=(4, 6, 7), psf_shape=(3, 3, 3))
    rng = np.random.default_rng(10 + seed)
    x = p.y.astype(np.float64) + 0.3 * rng.standard_normal(p.shape)      # some voxels outside the box
    g = oracle.gradient(op, p.y, x)
    h = 1e-6
    idx = rng.choice(x.size, size=40, replace=False)
    for k in idx:
        e = np.zeros(x.size)
        e[k] = h
        e = e.reshape(x.shape)
        fd = (oracle.objective(op, p.y, x + e) - oracle.objective(op, p.y, x - e)) / (2 * h)
        assert abs(fd - g.ravel()[k]) <= 2e-7 * max(1.0, abs(g.ravel()[k])), (k, fd, g.ravel()[k])


def test_gradient_at_matches_full_gradient():
    p, op = _tiny(seed=3, shape=(5, 7, 8), psf_shape=(5, 3, 3))
    x = synth.uniform_start(p.y, seed=3).astype(np.float64)
    g = oracle.gradient(op, p.y, x)
    idx = np.array([0, 1, 7, 8 * 7 - 1, 100, x.size - 1, x.size // 2])
    np.testing.assert_allclose(oracle.gradient_at(op, p.y, x, idx), g.ravel()[idx], rtol=1e-12, atol=1e-14)


def _q(op, y, x, xp):
    g = oracle.gradient(op, y, x)
    dx = xp - x
    return oracle.objective(op, y, x) + np.vdot(g, dx) + 0.5 * np.vdot(dx, oracle.apply_A(op, x, dx))


def test_majorant_exact_for_pure_least_squares():
    # lambda = 0, eta = 0: f is quadratic with Hessian H^T H, so Q equals f everywhere.
    p, _ = _tiny(seed=4)
    op = oracle.OracleProblem(p.shape, p.psf, lam=0.0, delta=0.1, eta=0.0)
    rng = np.random.default_rng(5)
    for _ in range(5):
        x = rng.standard_normal(p.shape)
        xp = rng.standard_normal(p.shape)
        f = oracle.objective(op, p.y, xp)
        assert abs(_q(op, p.y, x, xp) - f) <= 1e-11 * abs(f)


def test_majorant_exact_for_box_on_one_side():
    # Pure box term with x, x' both above xmax: eta*(x-xmax)^2 is exactly quadratic with curvature 2*eta.
    shape = (3, 4, 5)
    psf = np.zeros((3, 1, 1, 1), np.float32)        # H = 0
    op = oracle.OracleProblem(shape, psf, lam=0.0, delta=0.1, eta=1.7, xmin=0.0, xmax=1.0)
    rng = np.random.default_rng(6)
    x = 1.0 + rng.uniform(0.1, 2.0, shape)
    xp = 1.0 + rng.uniform(0.1, 2.0, shape)
    y = np.zeros(shape, np.float32)
    assert abs(_q(op, y, x, xp) - oracle.objective(op, y, xp)) < 1e-12


def test_majorization_inequality_random_points():
    p, op = _tiny(seed=7, shape=(4, 6, 7), psf_shape=(3, 3, 3))
    rng = np.random.default_rng(8)
    for _ in range(200):
        x = rng.uniform(-0.5, 1.5, p.shape)
        xp = x + rng.standard_normal(p.shape) * rng.choice([1e-3, 1e-1, 1.0])
        q = _q(op, p.y, x, xp)
        f = oracle.objective(op, p.y, xp)
        assert f <= q + 1e-12 * abs(q)


def test_majorant_curvature_is_tight_for_penalty():
    # With H = 0 and eta = 0 only the hyperbolic penalty remains.  Near flat
    # regions (t ~ 0) the half-quadratic weight 1/sqrt(delta^2 + t^2) equals
    # psi''(t), so shrinking the curvature by 30% must break the majorisation
    # for small steps: this pins the weights (a larger A would also pass).
    shape = (3, 4, 5)
    op = oracle.OracleProblem(shape, np.zeros((3, 1, 1, 1), np.float32), lam=1.0, delta=0.5, eta=0.0)
    y = np.zeros(shape, np.float32)
    rng = np.random.default_rng(9)
    violated = False
    for _ in range(50):
        x = 0.3 + 1e-4 * rng.standard_normal(shape)
        dx = 1e-3 * rng.standard_normal(shape)
        g = oracle.gradient(op, y, x)
        q_small = oracle.objective(op, y, x) + np.vdot(g, dx) + 0.35 * np.vdot(dx, oracle.apply_A(op, x, dx))
        if oracle.objective(op, y, x + dx) > q_small:
            violated = True
            break
    assert violated


def test_pinv2_against_numpy():
    rng = np.random.default_rng(11)
    mats = []
    for _ in range(20):
        m = rng.standard_normal((2, 2))
        mats.append(m @ m.T)                         # SPD
    v = rng.standard_normal(2)
    mats.append(np.outer(v, v))                      # rank 1
    mats.append(np.zeros((2, 2)))                    # zero
    mats.append(np.diag([3.0, 0.0]))                 # first 3MG iteration (d = 0)
    mats.append(np.diag([2.0, 2.0]))                 # repeated eigenvalue
    for B in mats:
        c = rng.standard_normal(2)
        u, _ = oracle.pinv2_solve(B, c)
        np.testing.assert_allclose(u, -np.linalg.pinv(B, rcond=1e-12, hermitian=True) @ c, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# Penalty mode 1: the objective as printed in Section 3.1, a joint X-Y
# hyperbolic term plus kappa ||V^Z x||^2.
# ---------------------------------------------------------------------------

def test_paper_penalty_hand_case_C():
    c = load_cases()["C"]
    op = oracle.OracleProblem(c["shape"], c["psf"], **c["params"])
    f, parts = oracle.objective(op, c["y"], c["x"], parts=True)
    np.testing.assert_allclose(parts, [c["f1"], c["f2"], c["f3"]], rtol=1e-14)
    np.testing.assert_allclose(oracle.gradient(op, c["y"], c["x"]), c["grad"], rtol=1e-14)


def test_paper_penalty_along_z_is_the_quadratic_closed_form():
    # nx = ny = 1: the joint term is delta at every voxel (no X or Y neighbour),
    # and the Z term is kappa * sum of squared numpy differences along z.
    shape = (7, 1, 1)
    op = oracle.OracleProblem(shape, np.zeros((7, 1, 1, 1), np.float32), lam=0.3, delta=0.2, eta=0.0,
                              penalty=1, kappa=1.7)
    x = np.random.default_rng(30).standard_normal(shape)
    _, parts = oracle.objective(op, np.zeros(shape, np.float32), x, parts=True)
    assert abs(parts[2] - (0.3 * 0.2 * 7 + 1.7 * np.sum(np.diff(x[:, 0, 0]) ** 2))) <= 1e-13


def test_paper_penalty_along_x_reduces_to_the_per_axis_penalty():
    # ny = nz = 1: with no Y or Z neighbour the joint term is the per-axis X term,
    # and the per-axis mode adds delta for each of the two absent axes.
    shape = (1, 1, 9)
    psf = np.full((1, 1, 1, 3), 1.0 / 3.0, np.float32)
    x = np.random.default_rng(31).uniform(-0.5, 1.5, shape)
    y = np.random.default_rng(32).uniform(0, 1, shape).astype(np.float32)
    kw = dict(lam=0.2, delta=0.3, eta=1.5)
    op0 = oracle.OracleProblem(shape, psf, **kw)
    op1 = oracle.OracleProblem(shape, psf, **kw, penalty=1, kappa=4.0)
    f0, p0 = oracle.objective(op0, y, x, parts=True)
    f1, p1 = oracle.objective(op1, y, x, parts=True)
    assert abs(p1[2] - (p0[2] - 0.2 * 0.3 * 2 * 9)) <= 1e-13
    np.testing.assert_allclose(oracle.gradient(op1, y, x), oracle.gradient(op0, y, x), rtol=1e-13, atol=1e-15)
    v = np.random.default_rng(33).standard_normal(shape)
    np.testing.assert_allclose(oracle.apply_A(op1, x, v), oracle.apply_A(op0, x, v), rtol=1e-13, atol=1e-15)


def _paper(seed, **kw):
    p = synth.tiny_problem(seed=seed, **kw)
    return p, oracle.OracleProblem(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax, penalty=1, kappa=0.05)


@pytest.mark.parametrize("seed", [0, 1])
def test_paper_penalty_gradient_central_differences(seed):
    p, op = _paper(seed, shape=(4, 6, 7), psf_shape=(3, 3, 3))
    rng = np.random.default_rng(40 + seed)
    x = p.y.astype(np.float64) + 0.3 * rng.standard_normal(p.shape)
    g = oracle.gradient(op, p.y, x)
    h = 1e-6
    for k in rng.choice(x.size, size=40, replace=False):
        e = np.zeros(x.size)
        e[k] = h
        e = e.reshape(x.shape)
        fd = (oracle.objective(op, p.y, x + e) - oracle.objective(op, p.y, x - e)) / (2 * h)
        assert abs(fd - g.ravel()[k]) <= 2e-7 * max(1.0, abs(g.ravel()[k])), (k, fd, g.ravel()[k])


def test_paper_penalty_gradient_at_matches_full_gradient():
    p, op = _paper(3, shape=(5, 7, 8), psf_shape=(5, 3, 3))
    x = synth.uniform_start(p.y, seed=3).astype(np.float64)
    g = oracle.gradient(op, p.y, x)
    idx = np.array([0, 1, 7, 8, 8 * 7 - 1, 100, 123, x.size - 1, x.size // 2])
    np.testing.assert_allclose(oracle.gradient_at(op, p.y, x, idx), g.ravel()[idx], rtol=1e-12, atol=1e-14)


def test_paper_penalty_majorisation_and_tangency():
    p, op = _paper(7, shape=(4, 6, 7), psf_shape=(3, 3, 3))
    rng = np.random.default_rng(48)
    for _ in range(200):
        x = rng.uniform(-0.5, 1.5, p.shape)
        xp = x + rng.standard_normal(p.shape) * rng.choice([1e-3, 1e-1, 1.0])
        q = _q(op, p.y, x, xp)
        assert oracle.objective(op, p.y, xp) <= q + 1e-12 * abs(q)
    # tangency: Q and f agree to first order at x, so (Q - f) / (f(x + h v) - f(x))
    # shrinks in proportion to h
    x = rng.uniform(0, 1, p.shape)
    v = rng.standard_normal(p.shape)
    rel = []
    for h in (1e-3, 1e-4):
        f0, f1 = oracle.objective(op, p.y, x), oracle.objective(op, p.y, x + h * v)
        rel.append(abs(_q(op, p.y, x, x + h * v) - f1) / abs(f1 - f0))
    assert rel[1] <= 0.2 * rel[0] and rel[1] < 1e-2, rel


def test_paper_penalty_z_term_majorant_is_exact():
    # lambda = 0, eta = 0, H = 0: only kappa ||V^Z x||^2 remains, a quadratic whose
    # Hessian 2 kappa V^ZT V^Z is the majorant's curvature, so Q equals f everywhere.
    shape = (5, 3, 4)
    op = oracle.OracleProblem(shape, np.zeros((5, 1, 1, 1), np.float32), lam=0.0, delta=0.1, eta=0.0,
                              penalty=1, kappa=0.8)
    y = np.zeros(shape, np.float32)
    rng = np.random.default_rng(49)
    for _ in range(5):
        x, xp = rng.standard_normal(shape), rng.standard_normal(shape)
        f = oracle.objective(op, y, xp)
        assert abs(_q(op, y, x, xp) - f) <= 1e-12 * abs(f)


# ---------------------------------------------------------------------------
# Penalty mode 2: the isotropic hyperbolic term over the three axes,
# lambda sum_n sqrt(delta^2 + [V^X x]_n^2 + [V^Y x]_n^2 + [V^Z x]_n^2).
# ---------------------------------------------------------------------------

def test_isotropic_penalty_hand_case_D():
    c = load_cases()["D"]
    op = oracle.OracleProblem(c["shape"], c["psf"], **c["params"])
    f, parts = oracle.objective(op, c["y"], c["x"], parts=True)
    np.testing.assert_allclose(parts, [c["f1"], c["f2"], c["f3"]], rtol=1e-14)
    np.testing.assert_allclose(oracle.gradient(op, c["y"], c["x"]), c["grad"], rtol=1e-14)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_isotropic_penalty_along_one_axis_reduces_to_the_per_axis_penalty(axis):
    # A volume that extends along one axis only: the isotropic term is that axis's
    # per-axis term, and the per-axis mode adds delta for each of the two absent axes.
    shape = [1, 1, 1]
    shape[2 - axis] = 9
    shape = tuple(shape)
    psf = np.zeros((shape[0], 1, 1, 1), np.float32)
    psf[...] = 1.0
    x = np.random.default_rng(60 + axis).uniform(-0.5, 1.5, shape)
    y = np.random.default_rng(63 + axis).uniform(0, 1, shape).astype(np.float32)
    kw = dict(lam=0.2, delta=0.3, eta=1.5)
    op0 = oracle.OracleProblem(shape, psf, **kw)
    op2 = oracle.OracleProblem(shape, psf, **kw, penalty=2)
    _, p0 = oracle.objective(op0, y, x, parts=True)
    _, p2 = oracle.objective(op2, y, x, parts=True)
    assert abs(p2[2] - (p0[2] - 0.2 * 0.3 * 2 * 9)) <= 1e-13
    np.testing.assert_allclose(oracle.gradient(op2, y, x), oracle.gradient(op0, y, x), rtol=1e-13, atol=1e-15)
    v = np.random.default_rng(66 + axis).standard_normal(shape)
    np.testing.assert_allclose(oracle.apply_A(op2, x, v), oracle.apply_A(op0, x, v), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("perm", [(2, 1, 0), (1, 0, 2), (0, 2, 1)])
def test_isotropic_penalty_is_invariant_under_axis_permutation(perm):
    # With H = I and a box term the objective treats the three axes alike in this
    # mode: permuting the axes of x and y permutes the gradient and the majorant's
    # action and leaves f unchanged (a dropped or mis-weighted axis breaks this).
    shape = (4, 5, 6)
    rng = np.random.default_rng(70)
    x = rng.uniform(-0.5, 1.5, shape)
    y = rng.uniform(0, 1, shape).astype(np.float32)
    v = rng.standard_normal(shape)
    kw = dict(lam=0.15, delta=0.2, eta=0.7, penalty=2)
    op = oracle.OracleProblem(shape, np.ones((shape[0], 1, 1, 1), np.float32), **kw)
    xs, ys, vs = (np.ascontiguousarray(np.transpose(a, perm)) for a in (x, y, v))
    ops = oracle.OracleProblem(xs.shape, np.ones((xs.shape[0], 1, 1, 1), np.float32), **kw)
    assert abs(oracle.objective(ops, ys, xs) - oracle.objective(op, y, x)) <= 1e-12 * abs(oracle.objective(op, y, x))
    np.testing.assert_allclose(oracle.gradient(ops, ys, xs), np.transpose(oracle.gradient(op, y, x), perm),
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(oracle.apply_A(ops, xs, vs), np.transpose(oracle.apply_A(op, x, v), perm),
                               rtol=1e-12, atol=1e-14)


def _iso(seed, **kw):
    p = synth.tiny_problem(seed=seed, **kw)
    return p, oracle.OracleProblem(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax, penalty=2)


@pytest.mark.parametrize("seed", [0, 1])
def test_isotropic_penalty_gradient_central_differences(seed):
    p, op = _iso(seed, shape=(4, 6, 7), psf_shape=(3, 3, 3))
    rng = np.random.default_rng(80 + seed)
    x = p.y.astype(np.float64) + 0.3 * rng.standard_normal(p.shape)
    g = oracle.gradient(op, p.y, x)
    h = 1e-6
    for k in rng.choice(x.size, size=40, replace=False):
        e = np.zeros(x.size)
        e[k] = h
        e = e.reshape(x.shape)
        fd = (oracle.objective(op, p.y, x + e) - oracle.objective(op, p.y, x - e)) / (2 * h)
        assert abs(fd - g.ravel()[k]) <= 2e-7 * max(1.0, abs(g.ravel()[k])), (k, fd, g.ravel()[k])


def test_isotropic_penalty_gradient_at_matches_full_gradient():
    p, op = _iso(3, shape=(5, 7, 8), psf_shape=(5, 3, 3))
    x = synth.uniform_start(p.y, seed=3).astype(np.float64)
    g = oracle.gradient(op, p.y, x)
    idx = np.array([0, 1, 7, 8, 8 * 7 - 1, 8 * 7, 100, 123, x.size - 1, x.size // 2])
    np.testing.assert_allclose(oracle.gradient_at(op, p.y, x, idx), g.ravel()[idx], rtol=1e-12, atol=1e-14)


def test_isotropic_penalty_majorisation_and_tangency():
    p, op = _iso(7, shape=(4, 6, 7), psf_shape=(3, 3, 3))
    rng = np.random.default_rng(88)
    for _ in range(200):
        x = rng.uniform(-0.5, 1.5, p.shape)
        xp = x + rng.standard_normal(p.shape) * rng.choice([1e-3, 1e-1, 1.0])
        q = _q(op, p.y, x, xp)
        assert oracle.objective(op, p.y, xp) <= q + 1e-12 * abs(q)
    x = rng.uniform(0, 1, p.shape)
    v = rng.standard_normal(p.shape)
    rel = []
    for h in (1e-3, 1e-4):
        f0, f1 = oracle.objective(op, p.y, x), oracle.objective(op, p.y, x + h * v)
        rel.append(abs(_q(op, p.y, x, x + h * v) - f1) / abs(f1 - f0))
    assert rel[1] <= 0.2 * rel[0] and rel[1] < 1e-2, rel
