"""GPU checks of the state the update carries from one iteration to the next:
the residual r = H x - y and the images H d_S of the slabs' memory directions
(H d_S(new) = -u0 H g_S + u1 H d_S, r += H d_S(new)), recomputed exactly
before the first iteration after creation or set_x, and every 256
iterations.  Runs longer than a refresh period must keep the oracle parity of
the 200-iteration test, and a context whose iterate was set from outside
must continue exactly like one created at that iterate."""
import numpy as np
import pytest

import oracle
from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _order(bounds, pz):
    """Colour-major slab order (written independently of the library)."""
    gap = max(pz - 1, 1)
    ends, col = [], []
    for s in range(len(bounds) - 1):
        c = next((k for k, e in enumerate(ends) if bounds[s] - e >= gap), len(ends))
        if c == len(ends):
            ends.append(0)
        ends[c] = bounds[s + 1]
        col.append(c)
    return [s for c in range(len(ends)) for s in range(len(col)) if col[s] == c]


@pytest.mark.parametrize("bounds", [None, [0, 3, 7, 12]])
def test_parity_across_an_exact_refresh(cuda_lib, bounds):
    """300 iterations (the carried r and H d_S are refreshed at iteration 256):
    iterate within 1e-4 and every objective within 1e-5 of the FP64 oracle,
    monotone descent throughout."""
    p = synth.tiny_problem(shape=(12, 32, 40), psf_shape=(5, 5, 5), seed=41, n_ellipsoids=6, slabs=bounds)
    op = oracle.OracleProblem.from_synth(p)
    oracle.set_threads(oracle.max_threads())
    order = _order(bounds, 5) if bounds else None
    xr, _, fr = oracle.run(op, p.y, p.y, 300, bounds=bounds, order=order)
    with cuda_lib.Solver.from_problem(p) as s:
        tr = s.iterate(300)
        x = s.get_x().cpu().numpy()
    assert _rel(x, xr) <= 1e-4
    assert np.max(np.abs(tr - fr) / np.abs(fr)) <= 1e-5
    assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:]))


@pytest.mark.parametrize("bounds", [None, [0, 4, 9, 16]])
def test_set_x_continues_like_a_new_context(cuda_lib, bounds):
    """set_x resets d and recomputes r and H d_S: the next sweeps are bit for
    bit those of a context created at that iterate."""
    p = synth.tiny_problem(shape=(16, 24, 36), psf_shape=(5, 5, 5), seed=42, n_ellipsoids=5, slabs=bounds)
    with cuda_lib.Solver.from_problem(p) as a:
        a.iterate(37, trace=False)
        xm = a.get_x().cpu().numpy()
        a.set_x(xm)
        tr_a = a.iterate(9)
        xa = a.get_x().cpu().numpy()
    with cuda_lib.Solver.from_problem(p, x0=xm) as b:
        tr_b = b.iterate(9)
        xb = b.get_x().cpu().numpy()
    assert np.array_equal(tr_a, tr_b)
    assert np.array_equal(xa, xb)


@pytest.mark.parametrize("bounds,precision", [(None, 0), ([0, 3, 7, 12], 0), (None, 1)])
def test_sweep_objective_from_the_carried_residual(cuda_lib, bounds, precision):
    """Every trace entry takes its data term from the carried residual;
    bd3mg_objective applies H to x afresh.  At the same iterate -- after 5
    iterations, and after 252, shortly before the exact refresh at 256, when the
    carried r has drifted most -- both are within 1e-6 of the FP64 oracle's
    objective at that iterate and of each other: the two differ only in the
    residual entering 1/2 r^2, each an FP32 evaluation (the trace's parity bound
    against the oracle is 1e-5).  The end of a call and the start of the next
    report the same value, bit for bit."""
    p = synth.tiny_problem(shape=(12, 32, 40), psf_shape=(5, 5, 5), seed=43, n_ellipsoids=6, slabs=bounds)
    op = oracle.OracleProblem.from_synth(p)
    with cuda_lib.Solver.from_problem(p, precision=precision) as s:
        for n in (5, 246):
            carried = s.iterate(n)[-1]              # f(x^k) at the end of the call
            exact = s.objective()                   # H x afresh
            ref = oracle.objective(op, p.y, s.get_x().cpu().numpy())
            assert abs(carried - ref) <= 1e-6 * abs(ref), (n, carried, ref)
            assert abs(exact - ref) <= 1e-6 * abs(ref), (n, exact, ref)
            assert s.iterate(1)[0] == carried       # the pass that opens the next sweep
