"""GPU tests of the runtime around the iteration: checkpoint / resume, precision
escalation of the BF16-gradient form, and the z-chunk autotuner."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _prob(slabs=False, seed=0):
    from paper_2002_02328_gb300 import synth
    p = synth.tiny_problem(shape=(16, 40, 48), psf_shape=(5, 5, 5), seed=seed, n_ellipsoids=6)
    if slabs:
        p.slabs = synth.slab_bounds([4, 7, 5])
    return p


@pytest.mark.parametrize("slabs,prec", [(False, 0), (True, 0), (False, 1)])
def test_resume_from_checkpoint_is_bit_exact(cuda_lib, tmp_path, slabs, prec):
    p = _prob(slabs)
    path = str(tmp_path / "ck.bin")
    with cuda_lib.Solver.from_problem(p, precision=prec) as a:
        a.iterate(7)
        a.save(path)
        tr_a = a.iterate(5)
        xa = a.get_x().cpu().numpy()
        da = a.get_d().cpu().numpy()
    with cuda_lib.Solver.from_problem(p, precision=prec) as b:
        b.load(path)
        tr_b = b.iterate(5)
        xb = b.get_x().cpu().numpy()
        db = b.get_d().cpu().numpy()
    assert np.array_equal(xa, xb) and np.array_equal(da, db)
    assert np.array_equal(tr_a, tr_b)


def test_checkpoint_of_another_shape_is_rejected(cuda_lib, tmp_path):
    path = str(tmp_path / "ck.bin")
    with cuda_lib.Solver.from_problem(_prob()) as a:
        a.save(path)
    from paper_2002_02328_gb300 import synth
    q = synth.tiny_problem(shape=(8, 40, 48), psf_shape=(5, 5, 5), seed=1)
    with cuda_lib.Solver.from_problem(q) as b:
        with pytest.raises(cuda_lib.Bd3mgError) as e:
            b.load(path)
        assert e.value.status == 1


def test_escalation_switches_to_fp32_gradient_and_keeps_descending(cuda_lib):
    p = _prob(seed=2)
    with cuda_lib.Solver.from_problem(p) as s32:
        f32 = s32.iterate(300)[-1]
    with cuda_lib.Solver.from_problem(p, precision=cuda_lib.BF16_GRADIENT) as s:
        assert s.escalated() == -1
        s.set_escalation(1e-5)
        tr = s.iterate(300)
        at = s.escalated()
        d = s.get_d().cpu().numpy()
    assert 0 < at < 300
    assert np.all(np.diff(tr) <= 1e-12 * np.abs(tr[1:]))          # monotone across the switch
    assert abs(tr[-1] - f32) <= 1e-6 * abs(f32)
    assert np.all(np.isfinite(d))
    # an FP32 context never escalates
    with cuda_lib.Solver.from_problem(p) as t:
        t.set_escalation(1e-3)
        t.iterate(20)
        assert t.escalated() == -1


def test_autotune_returns_a_candidate_and_caches_it(cuda_lib, tmp_path):
    from paper_2002_02328_gb300 import synth
    probs = [_prob(seed=3), synth.tiny_problem(shape=(12, 33, 29), psf_shape=(5, 5, 5), seed=4)]
    cache = str(tmp_path / "tune.jsonl")
    z, rows, ms = cuda_lib.autotune(probs, iters=3, cache_path=cache)
    assert z in (0, 4, 6, 8, 12, 16, 24, 32, 48) and rows in (16, 32) and ms > 0
    lines = [json.loads(l) for l in open(cache)]
    assert len(lines) == 1 and lines[0]["zchunk"] == z and lines[0]["curv_rows"] == rows
    assert len(lines[0]["candidates (chunk/rows)"]) == 18          # 9 chunks x 2 tile shapes
    z2, rows2, ms2 = cuda_lib.autotune(probs, iters=3, cache_path=cache)
    assert (z2, rows2, ms2) == (z, rows, -1.0)
    # the tuned shape gives the same iterates as the default (the work split only
    # regroups the partial sums)
    with cuda_lib.BatchSolver(probs) as a, cuda_lib.BatchSolver(probs, zchunk=z, curv_rows=rows) as b:
        ta, tb = a.iterate(5), b.iterate(5)
    np.testing.assert_allclose(ta, tb, rtol=1e-6)


@pytest.mark.parametrize("slabs", [False, True])
def test_32_row_curvature_tiles_match_16_row(cuda_lib, slabs):
    """The two FP32 curvature tile shapes compute the same sums in another grouping."""
    from paper_2002_02328_gb300 import synth
    bounds = [0, 4, 11, 13, 20] if slabs else None
    p = synth.tiny_problem(shape=(20, 45, 70), psf_shape=(7, 7, 7), seed=6, n_ellipsoids=8, slabs=bounds)
    with cuda_lib.Solver.from_problem(p, curv_rows=16) as a, cuda_lib.Solver.from_problem(p, curv_rows=32) as b:
        ta, tb = a.iterate(10), b.iterate(10)
        xa, xb = a.get_x().cpu().numpy(), b.get_x().cpu().numpy()
    np.testing.assert_allclose(tb, ta, rtol=1e-6)
    assert np.linalg.norm(xb - xa) <= 1e-5 * np.linalg.norm(xa)
