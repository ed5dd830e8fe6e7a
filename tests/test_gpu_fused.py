"""GPU checks of the fused-update iteration (volumes without slabs).

Such a context runs an iteration as two passes: the gradient pass applies the
previous iteration's update (x, d, r, H d) as it reads the state and writes
the new state into a second buffer set, then the curvature pass builds and
solves the 2x2 system.  The update arithmetic is that of the separate update
pass, so the iterates must be the same bits as a context created with
separate_update = 1 (the fused form is forced with separate_update = 2;
contexts below 2^24 voxels do not take it by default); only the objective's summation order differs (both sum
FP32 per-thread partials of up to a few hundred terms and FP64 across threads:
trace within 1e-6 relative).
"""
import dataclasses

import numpy as np
import pytest

from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


FUSED = 2          # BD3MG_UPDATE_FUSED (the automatic choice fuses only large contexts)


def _pair(cuda_lib, p, n, **kw):
    out = []
    for sep in (FUSED, 1):
        with cuda_lib.Solver.from_problem(p, separate_update=sep, **kw) as s:
            assert s.launches_per_iteration() == (2 if sep == FUSED else 4)
            tr = s.iterate(n)
            out.append((tr, s.get_x().cpu().numpy(), s.get_d().cpu().numpy()))
    return out


@pytest.mark.parametrize("shape,psf_shape,prec,mode", [
    ((13, 45, 70), (5, 5, 5), 0, 0),       # ragged in x and y
    ((9, 33, 37), (7, 7, 7), 1, 0),        # BF16 gradient
    ((12, 40, 33), (9, 9, 7), 0, 1),       # printed penalty (joint X-Y + kappa Z)
    ((6, 34, 66), (3, 3, 3), 0, 2),        # isotropic penalty
])
def test_fused_iterates_equal_separate_update(cuda_lib, shape, psf_shape, prec, mode):
    p = synth.tiny_problem(shape=shape, psf_shape=psf_shape, seed=21, n_ellipsoids=6)
    p = dataclasses.replace(p, penalty=mode, kappa=0.3 if mode == 1 else 0.0)
    (tf, xf, df), (ts, xs, ds) = _pair(cuda_lib, p, 25, precision=prec)
    np.testing.assert_array_equal(xf, xs)
    np.testing.assert_array_equal(df, ds)
    np.testing.assert_allclose(tf, ts, rtol=1e-6)


def test_fused_across_refreshes(cuda_lib):
    p = synth.tiny_problem(shape=(10, 36, 40), psf_shape=(5, 5, 5), seed=22, n_ellipsoids=6)
    (tf, xf, _), (ts, xs, _) = _pair(cuda_lib, p, 30, refresh_every=7)
    np.testing.assert_array_equal(xf, xs)
    np.testing.assert_allclose(tf, ts, rtol=1e-6)


def test_pending_update_is_applied_before_reads(cuda_lib):
    """iterate_async leaves the last update pending; every reader applies it first."""
    import torch
    p = synth.tiny_problem(shape=(11, 30, 44), psf_shape=(5, 5, 5), seed=23, n_ellipsoids=6)
    with cuda_lib.Solver.from_problem(p, separate_update=FUSED) as a, \
            cuda_lib.Solver.from_problem(p, separate_update=FUSED) as b:
        a.iterate(6)
        xa, fa = a.get_x().cpu().numpy(), a.objective()
        b.iterate_async(3)
        b.iterate_async(3)
        fb = b.objective()
        xb = b.get_x().cpu().numpy()
        np.testing.assert_array_equal(xa, xb)
        assert fa == fb
        # an odd number of passes leaves the state in the second buffer set
        b.iterate_async(1)
        g, _ = b.gradient()
        a.iterate(1)
        np.testing.assert_array_equal(a.get_x().cpu().numpy(), b.get_x().cpu().numpy())
        np.testing.assert_array_equal(a.get_d().cpu().numpy(), b.get_d().cpu().numpy())
        # set_x discards nothing it should keep: both restart from the same point
        x0 = torch.from_numpy(synth.uniform_start(p.y, seed=5)).cuda()
        b.iterate_async(2)
        a.set_x(x0)
        b.set_x(x0)
        ta, tb = a.iterate(4), b.iterate(4)
        np.testing.assert_array_equal(ta, tb)


def test_fused_batch_with_stopping_equals_separate(cuda_lib):
    probs = [
        synth.tiny_problem(shape=(10, 24, 40), psf_shape=(5, 5, 5), seed=31, n_ellipsoids=5, lam=2e-2),
        synth.tiny_problem(shape=(7, 33, 21), psf_shape=(7, 7, 7), seed=32, n_ellipsoids=4, lam=6e-3),
        synth.tiny_problem(shape=(16, 17, 64), psf_shape=(3, 3, 3), seed=33, n_ellipsoids=6),
    ]
    with cuda_lib.BatchSolver(probs, separate_update=1, zchunk=8) as b:
        t0 = b.iterate(30)
    # objective targets halfway between two sweeps' values, so that rounding of
    # the objective cannot move the stopping sweep (8, 13, 21 for the three volumes)
    stop_at = [8, 13, 21]
    target = np.array([0.5 * (t0[v, k - 1] + t0[v, k]) for v, k in enumerate(stop_at)])
    res = []
    for sep in (FUSED, 1):
        with cuda_lib.BatchSolver(probs, separate_update=sep, zchunk=8) as b:
            b.set_stopping(0.0, target)
            tr = b.iterate(30)
            res.append((tr, [b.get(v).cpu().numpy() for v in range(3)], b.stopped()))
    (tf, xf, kf), (ts, xs, ks) = res
    assert list(kf) == list(ks) == stop_at
    for v in range(3):
        np.testing.assert_array_equal(xf[v], xs[v])
    np.testing.assert_allclose(tf, ts, rtol=1e-6)


def test_fused_checkpoint_resume(cuda_lib, tmp_path):
    p = synth.tiny_problem(shape=(9, 28, 36), psf_shape=(5, 5, 5), seed=24, n_ellipsoids=6)
    path = str(tmp_path / "ck.bin")
    with cuda_lib.Solver.from_problem(p, separate_update=FUSED) as a:
        ta = a.iterate(12)
        xa = a.get_x().cpu().numpy()
    with cuda_lib.Solver.from_problem(p, separate_update=FUSED) as b:
        b.iterate_async(5)                 # pending update at the save
        b.save(path)
    with cuda_lib.Solver.from_problem(p, separate_update=FUSED) as c:
        c.load(path)
        tc = c.iterate(7)
        xc = c.get_x().cpu().numpy()
    np.testing.assert_array_equal(xa, xc)
    np.testing.assert_array_equal(ta[5:], tc)
