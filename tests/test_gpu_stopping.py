"""GPU checks of per-volume stopping.  The rule of the paper's scaling
experiment (Section 3.3), ||x^k - x^{k-1}|| <= tol ||x^{k-1}||, and an
objective target are tested on the device before every sweep; a stopped volume
keeps its iterate while the other volumes of the batch run on unchanged."""
import numpy as np
import pytest

from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


def _batch():
    return [
        synth.tiny_problem(shape=(10, 24, 40), psf_shape=(5, 5, 5), sxy=(0.5, 1.5), seed=31, n_ellipsoids=5,
                           lam=2e-2),
        synth.tiny_problem(shape=(7, 33, 21), psf_shape=(7, 7, 7), sxy=(0.8, 2.5), seed=32, n_ellipsoids=4),
        synth.tiny_problem(shape=(16, 17, 64), psf_shape=(3, 3, 3), sxy=(0.4, 1.0), seed=33, n_ellipsoids=6,
                           eta=0.5),
    ]


@pytest.mark.parametrize("precision", [0, 1])
def test_target_stops_one_volume_and_freezes_it(cuda_lib, precision):
    probs = _batch()
    n, k_stop = 30, 8
    with cuda_lib.BatchSolver(probs, precision=precision) as b:
        free = b.iterate(n)
        x_free = [b.get(v).cpu().numpy() for v in range(3)]
    assert np.all(np.diff(free[1]) < 0)                  # strictly decreasing: the first hit is k_stop
    with cuda_lib.BatchSolver(probs, precision=precision) as b:
        b.iterate(k_stop)
        x_at_k = b.get(1).cpu().numpy()
    targets = np.array([-np.inf, free[1][k_stop], -np.inf])
    with cuda_lib.BatchSolver(probs, precision=precision) as b:
        b.set_stopping(0.0, targets)
        tr = b.iterate(n)
        np.testing.assert_array_equal(b.stopped(), [-1, k_stop, -1])
        xs = [b.get(v).cpu().numpy() for v in range(3)]
        tr2 = b.iterate(5)                                # stays stopped across calls
        np.testing.assert_array_equal(b.get(1).cpu().numpy(), xs[1])
    # the stopped volume keeps x^k and repeats f(x^k)
    np.testing.assert_array_equal(xs[1], x_at_k)
    np.testing.assert_array_equal(tr[1][:k_stop + 1], free[1][:k_stop + 1])
    assert np.all(tr[1][k_stop:] == free[1][k_stop]) and np.all(tr2[1] == free[1][k_stop])
    # the others are untouched, bit for bit
    for v in (0, 2):
        np.testing.assert_array_equal(tr[v], free[v])
        np.testing.assert_array_equal(xs[v], x_free[v])


def _host_step_ratios(cuda_lib, prob, slabs, n):
    """||x^k - x^{k-1}|| / ||x^{k-1}|| for k = 1..n from the iterates, in FP64."""
    out = []
    with cuda_lib.Solver.from_problem(prob, slabs=slabs) as s:
        prev = s.get_x().cpu().numpy().astype(np.float64)
        for _ in range(n):
            s.iterate(1)
            cur = s.get_x().cpu().numpy().astype(np.float64)
            out.append(np.linalg.norm(cur - prev) / np.linalg.norm(prev))
            prev = cur
    return np.array(out)


@pytest.mark.parametrize("slabs", [None, [0, 5, 11, 16, 24]])
def test_step_rule_matches_the_iterates(cuda_lib, slabs):
    """The device's step test (lengths from the FP64 subspace sums) stops at the
    first k with ||x^k - x^{k-1}|| <= tol ||x^{k-1}||, measured from the iterates."""
    prob = synth.tiny_problem(shape=(24, 36, 44), psf_shape=(5, 5, 3), seed=34, n_ellipsoids=7)
    n = 60
    ratios = _host_step_ratios(cuda_lib, prob, slabs, n)
    # a tolerance half-way (geometrically) between two neighbouring ratios that
    # are at least 2% apart, near the middle of the run
    srt = np.sort(ratios)
    j = next(j for j in range(len(srt) // 2, len(srt) - 1) if srt[j + 1] > 1.02 * srt[j])
    tol = float(np.sqrt(srt[j] * srt[j + 1]))
    k_host = int(np.nonzero(ratios <= tol)[0][0]) + 1
    with cuda_lib.Solver.from_problem(prob, slabs=slabs) as s:
        s.set_stopping(tol)
        s.iterate(n)
        k_dev = s.stopped()
    assert k_dev == k_host, (k_dev, k_host, tol, ratios[:k_host + 1])


def test_stopping_state_resets(cuda_lib):
    prob = synth.tiny_problem(shape=(8, 20, 24), psf_shape=(3, 3, 3), seed=35, n_ellipsoids=3)
    with cuda_lib.Solver.from_problem(prob, slabs=None) as s:
        free = s.iterate(10)
    with cuda_lib.Solver.from_problem(prob, slabs=None) as s:
        s.set_stopping(0.0, free[3])
        s.iterate(10)
        assert s.stopped() == 3
        s.set_stopping(0.0, None)                      # clears the stop and the target
        assert s.stopped() == -1
        tr = s.iterate(4)
        assert tr[-1] < tr[0]
        s.set_stopping(0.0, tr[-1] * 2.0)              # met at once: stops after 0 sweeps
        s.iterate(2)
        assert s.stopped() == 0
        import torch
        s.set_x(torch.from_numpy(prob.y).cuda())       # a new start clears the stop, keeps the target
        assert s.stopped() == -1


def test_stopping_rejects_bad_arguments(cuda_lib):
    prob = synth.tiny_problem(shape=(6, 16, 16), psf_shape=(3, 3, 3), seed=36)
    with pytest.raises(cuda_lib.Bd3mgError, match="tol"):
        with cuda_lib.Solver.from_problem(prob, slabs=None) as s:
            s.set_stopping(-1.0)
    with pytest.raises(cuda_lib.Bd3mgError, match="NaN"):
        with cuda_lib.Solver.from_problem(prob, slabs=None) as s:
            s.set_stopping(0.0, float("nan"))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("zchunk", [8, 0])
def test_dropping_stopped_volumes_from_the_work_lists_changes_nothing(cuda_lib, precision, zchunk):
    """The synchronous iterate re-plans the gradient, curvature and update launches
    without the volumes that stopped; the asynchronous one keeps launching their
    (empty) items.  With a z-chunk the caller fixed, every running volume keeps
    its items, and both leave every volume bit-identical.  With the cost model's
    chunks (zchunk 0) the re-plan chooses new chunks for the volumes still
    running, which regroups their partial sums: the same sweeps stop and the
    iterates agree to 1e-5."""
    probs = _batch()
    probs[2].slabs = synth.slab_bounds([5, 6, 5])       # one volume in the slab form
    n = 24
    with cuda_lib.BatchSolver(probs, precision=precision, zchunk=zchunk) as b:
        free = b.iterate(n)
    # every volume stops, at different sweeps; a margin far below one sweep's
    # decrease keeps the stopping sweep independent of how the sums are grouped
    targets = np.array([free[0][5], free[1][11], free[2][17]])
    targets = targets + 1e-9 * np.abs(targets)
    runs = []
    for sync in (True, False):
        with cuda_lib.BatchSolver(probs, precision=precision, zchunk=zchunk) as b:
            b.set_stopping(0.0, targets)
            if sync:
                b.iterate(n, trace=False)
            else:
                b.iterate_async(n)
            runs.append(([b.get(v).cpu().numpy() for v in range(3)], b.stopped()))
    np.testing.assert_array_equal(runs[0][1], [5, 11, 17])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    for v in range(3):
        if zchunk:
            np.testing.assert_array_equal(runs[0][0][v], runs[1][0][v])
        else:
            a, b_ = runs[0][0][v].astype(np.float64), runs[1][0][v].astype(np.float64)
            assert np.linalg.norm(a - b_) <= 1e-5 * np.linalg.norm(b_)
