"""GPU checks of the persistent iteration (bd3mg_params.persistent = 1).

The fused-update iteration of plain volumes runs many iterations inside one
cooperative launch: every CTA is resident, takes the work items of a pass from
a queue and waits at a bounded grid-wide barrier before the next pass.  The
per-item code, the item lists and the fixed-order sums are those of the graph
form (two launches per iteration), so iterates, memory directions and traces
must be the same bits, across refreshes (one launch per refresh period) and
for the ablation variants.  A batch with stopping stops the same volumes at
the same sweeps without re-planning the work lists (with a fixed z-chunk the
graph form keeps every running volume's items too, so the iterates agree bit
for bit).  Failure detection: a CTA that never arrives at the barrier, or a
slice copy left out, makes the bounded waits run out and the call report
BD3MG_ETIMEOUT; nothing faults or hangs.
"""
import dataclasses

import numpy as np
import pytest

from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu

FUSED = 2          # BD3MG_UPDATE_FUSED: the graph form of the same iteration


def _run(cuda_lib, p, n, async_=False, **kw):
    with cuda_lib.Solver.from_problem(p, **kw) as s:
        if async_:
            s.iterate_async(n)
            tr = None
        else:
            tr = s.iterate(n)
        return tr, s.get_x().cpu().numpy(), s.get_d().cpu().numpy(), s.launches_per_iteration()


@pytest.mark.parametrize("shape,psf_shape,mode", [
    ((13, 45, 70), (5, 5, 5), 0),       # ragged in x and y
    ((12, 40, 33), (9, 9, 7), 1),       # printed penalty (joint X-Y + kappa Z)
    ((6, 34, 66), (3, 3, 3), 2),        # isotropic penalty
    ((40, 64, 96), (7, 7, 7), 0),       # more items than resident CTAs
])
def test_persistent_equals_graph_iteration(cuda_lib, shape, psf_shape, mode):
    p = synth.tiny_problem(shape=shape, psf_shape=psf_shape, seed=61, n_ellipsoids=6)
    p = dataclasses.replace(p, penalty=mode, kappa=0.3 if mode == 1 else 0.0)
    tg, xg, dg, lg = _run(cuda_lib, p, 25, separate_update=FUSED)
    tp, xp, dp, lp = _run(cuda_lib, p, 25, persistent=1)
    assert lg == 2 and lp == 1
    np.testing.assert_array_equal(xp, xg)
    np.testing.assert_array_equal(dp, dg)
    np.testing.assert_array_equal(tp, tg)


def test_persistent_across_refreshes_and_async(cuda_lib):
    p = synth.tiny_problem(shape=(10, 36, 40), psf_shape=(5, 5, 5), seed=62, n_ellipsoids=6)
    tg, xg, _, _ = _run(cuda_lib, p, 30, separate_update=FUSED, refresh_every=7)
    tp, xp, _, _ = _run(cuda_lib, p, 30, persistent=1, refresh_every=7)
    np.testing.assert_array_equal(xp, xg)
    np.testing.assert_array_equal(tp, tg)
    _, xa, _, _ = _run(cuda_lib, p, 30, async_=True, persistent=1, refresh_every=7)
    np.testing.assert_array_equal(xa, xg)


@pytest.mark.parametrize("metric,direction", [(1, 1), (1, 2), (0, 2)])
def test_persistent_variants_equal_graph_iteration(cuda_lib, metric, direction):
    p = synth.tiny_problem(shape=(9, 33, 37), psf_shape=(7, 7, 7), seed=63, n_ellipsoids=5)
    kw = dict(metric=metric, direction=direction)
    tg, xg, _, _ = _run(cuda_lib, p, 20, separate_update=FUSED, **kw)
    tp, xp, _, _ = _run(cuda_lib, p, 20, persistent=1, **kw)
    np.testing.assert_array_equal(xp, xg)
    np.testing.assert_array_equal(tp, tg)


def _batch():
    return [
        synth.tiny_problem(shape=(10, 24, 40), psf_shape=(5, 5, 5), sxy=(0.5, 1.5), seed=64, n_ellipsoids=5,
                           lam=2e-2),
        synth.tiny_problem(shape=(7, 33, 21), psf_shape=(7, 7, 7), sxy=(0.8, 2.5), seed=65, n_ellipsoids=4),
        synth.tiny_problem(shape=(16, 17, 64), psf_shape=(3, 3, 3), sxy=(0.4, 1.0), seed=66, n_ellipsoids=6,
                           eta=0.5),
    ]


def test_persistent_batch_stops_volumes_inside_the_launch(cuda_lib):
    probs = _batch()
    n = 24
    with cuda_lib.BatchSolver(probs, separate_update=FUSED, zchunk=8) as b:
        free = b.iterate(n)
    targets = np.array([free[0][5], free[1][11], free[2][17]])
    targets = targets + 1e-9 * np.abs(targets)
    runs = []
    for kw in (dict(separate_update=FUSED), dict(persistent=1)):
        with cuda_lib.BatchSolver(probs, zchunk=8, **kw) as b:
            b.set_stopping(0.0, targets)
            tr = b.iterate(n)
            runs.append((tr, [b.get(v).cpu().numpy() for v in range(3)], b.stopped()))
    np.testing.assert_array_equal(runs[0][2], [5, 11, 17])
    np.testing.assert_array_equal(runs[1][2], runs[0][2])
    np.testing.assert_array_equal(runs[1][0], runs[0][0])
    for v in range(3):
        np.testing.assert_array_equal(runs[1][1][v], runs[0][1][v])


def _timeout_then_poisoned(cuda_lib, p, kind):
    s = cuda_lib.Solver.from_problem(p, persistent=1, barrier_timeout_ms=50)
    try:
        s.iterate(2)
        s.inject_fault(kind)
        with pytest.raises(cuda_lib.Bd3mgError) as e:
            s.iterate(3)
        assert e.value.status == 4, str(e.value)                       # BD3MG_ETIMEOUT
        with pytest.raises(cuda_lib.Bd3mgError) as e2:
            s.iterate(1)
        assert e2.value.status == 6                                     # poisoned: BD3MG_ESTATE
    finally:
        s.close()


@pytest.mark.parametrize("kind", ["arrive", "copy"])
def test_persistent_bounded_waits_run_out(cuda_lib, kind):
    p = synth.tiny_problem(shape=(12, 32, 40), psf_shape=(5, 5, 5), seed=67, n_ellipsoids=6)
    ref = _run(cuda_lib, p, 4, persistent=1)
    _timeout_then_poisoned(cuda_lib, p, cuda_lib.FAULT_SKIP_ARRIVE if kind == "arrive" else cuda_lib.FAULT_SKIP_COPY)
    again = _run(cuda_lib, p, 4, persistent=1)       # the CUDA context stays usable
    np.testing.assert_array_equal(again[0], ref[0])
    np.testing.assert_array_equal(again[1], ref[1])


def test_persistent_rejects_other_forms(cuda_lib):
    p = synth.tiny_problem(shape=(8, 24, 24), psf_shape=(3, 3, 3), seed=68, n_ellipsoids=3)
    ps = synth.tiny_problem(shape=(8, 24, 24), psf_shape=(3, 3, 3), seed=68, n_ellipsoids=3, slabs=[0, 4, 8])
    for prob, kw, status in ((ps, {}, 7),                                  # slabs
                             (p, {"precision": 1}, 7),                    # BF16 gradient
                             (p, {"separate_update": 1}, 7),              # separate update pass
                             (p, {"curv_rows": 32}, 7),                   # 32-row FP32 curvature tiles
                             (p, {"psf_mode": 1}, 7),                     # dense PSF path
                             (p, {"persistent": 2}, 1)):
        kw = dict(kw)
        kw.setdefault("persistent", 1)
        with pytest.raises(cuda_lib.Bd3mgError) as e:
            cuda_lib.Solver.from_problem(prob, **kw)
        assert e.value.status == status, (kw, str(e.value))
