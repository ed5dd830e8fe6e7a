"""GPU parity of the ablation variants (Section 3.2, Table 1) against the oracle's.

Async-GD (A = L I, D = -g), Async-CG (A = L I, Fletcher-Reeves conjugate
direction), the conjugate direction with the half-quadratic majorant, the block
form with the gradient direction, and BP3MG (every slab's step from the same
iterate, curvature inflated by the number of slabs), each run through the C
ABI and compared with oracle.run_variant on the same inputs: the iterate
within relative 2e-5 and the objective trace within 1e-5, the bounds of the
slab-form parity tests.  The library's Lipschitz bound equals the oracle's
(both from the definition, on the factored and on the dense PSF).
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


@pytest.mark.parametrize("mode,kappa", [(0, 0.0), (1, 0.3), (2, 0.0)])
def test_lipschitz_bound_matches_oracle(cuda_lib, mode, kappa):
    p = synth.tiny_problem(shape=(9, 33, 37), psf_shape=(7, 5, 5), seed=41, n_ellipsoids=5)
    p = dataclasses.replace(p, penalty=mode, kappa=kappa)
    with cuda_lib.Solver.from_problem(p, metric=cuda_lib.METRIC_LIPSCHITZ) as s:
        L = s.lipschitz()
    L_ref = oracle.lipschitz_bound(oracle.OracleProblem.from_synth(p))
    assert abs(L - L_ref) <= 1e-5 * L_ref


@pytest.mark.parametrize("metric,direction,n", [
    (1, 1, 40),     # Async-GD: gradient descent with step 1/L
    (1, 2, 40),     # Async-CG: Fletcher-Reeves direction, step from A = L I
    (0, 2, 30),     # conjugate direction with the half-quadratic majorant
    (0, 1, 30),     # steepest descent with the majorant's step
])
def test_plain_variants_match_oracle(cuda_lib, metric, direction, n):
    p = synth.tiny_problem(shape=(13, 45, 70), psf_shape=(5, 5, 5), seed=42, n_ellipsoids=6)
    op = oracle.OracleProblem.from_synth(p)
    L = oracle.lipschitz_bound(op)
    xr, _, fr = oracle.run_variant(op, p.y, p.y, n, metric=metric, lipschitz=L, direction=direction)
    for sep in (2, 1):            # fused-update and separate-update iterations
        with cuda_lib.Solver.from_problem(p, metric=metric, lipschitz=L, direction=direction,
                                          separate_update=sep) as s:
            tr = s.iterate(n)
            x = s.get_x().cpu().numpy()
        assert _rel(x, xr) <= 2e-5
        assert np.max(np.abs(tr - fr) / np.abs(fr)) <= 1e-5
        assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:]))


def test_block_gradient_direction_matches_oracle(cuda_lib):
    bounds = [0, 3, 9, 12, 17, 20, 24]
    p = synth.tiny_problem(shape=(24, 40, 48), psf_shape=(5, 5, 5), seed=43, n_ellipsoids=8, slabs=bounds)
    op = oracle.OracleProblem.from_synth(p)
    _, order = _colour_major(bounds, 5)
    xr, _, fr = oracle.run_variant(op, p.y, p.y, 8, bounds=bounds, order=order, direction=oracle.DIR_GRADIENT)
    with cuda_lib.Solver.from_problem(p, direction=cuda_lib.DIR_GRADIENT) as s:
        tr = s.iterate(8)
        x = s.get_x().cpu().numpy()
    assert _rel(x, xr) <= 2e-5
    assert np.max(np.abs(tr - fr) / np.abs(fr)) <= 1e-5


@pytest.mark.parametrize("inflation", [0.0, 2.5])
def test_jacobi_schedule_matches_oracle(cuda_lib, inflation):
    bounds = [0, 4, 11, 13, 20]
    p = synth.tiny_problem(shape=(20, 36, 40), psf_shape=(7, 7, 7), seed=44, n_ellipsoids=8, slabs=bounds)
    op = oracle.OracleProblem.from_synth(p)
    infl = inflation if inflation > 0 else len(bounds) - 1          # the library's default: the slab count
    x0 = synth.uniform_start(p.y, seed=5)
    xr, _, fr = oracle.run_variant(op, p.y, x0, 10, bounds=bounds, schedule=oracle.SCHEDULE_JACOBI,
                                   inflation=infl)
    with cuda_lib.Solver.from_problem(p, x0=x0, schedule=cuda_lib.SCHEDULE_JACOBI, inflation=inflation) as s:
        col, nc = s.colours()
        assert nc == 1 and s.launches_per_iteration() == 6
        tr = s.iterate(10)
        x = s.get_x().cpu().numpy()
    assert _rel(x, xr) <= 2e-5
    assert np.max(np.abs(tr - fr) / np.abs(fr)) <= 1e-5
    if inflation == 0.0:
        assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:]))


def test_invalid_variants_are_rejected(cuda_lib):
    p = synth.tiny_problem(shape=(4, 16, 16), psf_shape=(3, 3, 3), seed=45)
    for kw in ({"metric": 2}, {"direction": 3}, {"schedule": 2}, {"inflation": 0.5}, {"lipschitz": -1.0}):
        with pytest.raises(cuda_lib.Bd3mgError) as e:
            cuda_lib.Solver.from_problem(p, **kw)
        assert e.value.status == 1
