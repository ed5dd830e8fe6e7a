"""GPU parity of the batched form: independent volumes of uneven size, each with
its own PSF ramp and lambda, iterated in lockstep by one context.  Each volume
must follow the FP64 oracle run on that volume alone, and agree with a
single-volume context."""
import numpy as np
import pytest

import oracle
from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _tiny_batch():
    return [
        synth.tiny_problem(shape=(10, 24, 40), psf_shape=(5, 5, 5), sxy=(0.5, 1.5), seed=11, n_ellipsoids=5,
                           lam=2e-2),
        synth.tiny_problem(shape=(7, 33, 21), psf_shape=(7, 7, 7), sxy=(0.8, 2.5), seed=12, n_ellipsoids=4,
                           lam=6e-3),
        synth.tiny_problem(shape=(16, 17, 64), psf_shape=(3, 3, 3), sxy=(0.4, 1.0), seed=13, n_ellipsoids=6,
                           lam=1e-2, eta=0.5),
    ]


def test_batch_matches_oracle_per_volume(cuda_lib):
    probs = _tiny_batch()
    oracle.set_threads(oracle.max_threads())
    with cuda_lib.BatchSolver(probs) as b:
        tr = b.iterate(8)
        xs = [b.get(v).cpu().numpy() for v in range(len(probs))]
    for v, p in enumerate(probs):
        op = oracle.OracleProblem.from_synth(p)
        xr, _, fr = oracle.run(op, p.y, p.y, 8)
        assert _rel(xs[v], xr) <= 2e-5, v
        assert np.max(np.abs(tr[v] - fr) / np.abs(fr)) <= 1e-5, v


def test_batch_of_one_equals_single_context(cuda_lib):
    p = synth.tiny_problem(shape=(12, 40, 36), psf_shape=(5, 5, 5), seed=14, n_ellipsoids=6)
    with cuda_lib.BatchSolver([p]) as b, cuda_lib.Solver.from_problem(p) as s:
        tb = b.iterate(10)
        ts = s.iterate(10)
        xb = b.get(0).cpu().numpy()
        xs = s.get_x().cpu().numpy()
    np.testing.assert_array_equal(xb, xs)
    np.testing.assert_array_equal(tb[0], ts)


def test_batch_volumes_follow_their_own_solves(cuda_lib):
    probs = _tiny_batch()
    with cuda_lib.BatchSolver(probs) as b:
        tb = b.iterate(20)
        fb = b.objectives()
    for v, p in enumerate(probs):
        with cuda_lib.Solver.from_problem(p) as s:
            ts = s.iterate(20)
        np.testing.assert_allclose(tb[v], ts, rtol=1e-6)
        assert abs(fb[v] - ts[-1]) <= 1e-6 * abs(ts[-1])


def test_full_size_batch_members_match_oracle(cuda_lib):
    """The 16-volume recipe at full size, 3 lockstep sweeps: its two smallest
    volumes against the oracle run on each alone (iterate and trace as the tiny
    batch above)."""
    probs = synth.workload_batch(count=16, seed=0)
    order = np.argsort([p.n for p in probs])[:2]
    oracle.set_threads(oracle.max_threads())
    with cuda_lib.BatchSolver(probs) as b:
        tr = b.iterate(3)
        xs = {int(v): b.get(int(v)).cpu().numpy() for v in order}
    for v in order:
        p = probs[int(v)]
        op = oracle.OracleProblem.from_synth(p)
        xr, _, fr = oracle.run(op, p.y, p.y, 3)
        assert _rel(xs[int(v)], xr) <= 2e-5, v
        assert np.max(np.abs(tr[v] - fr) / np.abs(fr)) <= 1e-5, v


def test_uneven_batch_recipe_descends(cuda_lib):
    probs = synth.workload_batch(count=16, seed=0, scale=0.5)
    with cuda_lib.BatchSolver(probs) as b:
        tr = b.iterate(15)
    assert tr.shape == (16, 16)
    assert np.all(np.diff(tr, axis=1) <= 1e-6 * np.abs(tr[:, 1:]))
    assert np.all(tr[:, -1] < tr[:, 0])
