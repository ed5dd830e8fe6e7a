"""GPU checks of the mixed-precision form: the gradient direction g stored in
BF16 (d, x, r in FP32), FP32 arithmetic, FP64 reductions and 2x2 solve.  Its
iterates differ from the FP32 run by the rounding of g, so it is held to what
the method guarantees instead of to bit agreement: monotone descent of f
(Section 3.1: every step minimises a majorant of f on the subspace),
convergence to the same minimiser as the FP64 oracle, and a stored gradient
within BF16 rounding of the FP32 one."""
import numpy as np
import pytest

import oracle
from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_bf16_first_gradient_is_rounded_fp32_gradient(cuda_lib):
    """At x0 the gradient is computed in FP32 and stored rounded: each element is
    within half a BF16 ulp (2^-9 relative) of the FP32 kernel's."""
    p = synth.tiny_problem(shape=(12, 40, 52), psf_shape=(5, 5, 5), seed=21, n_ellipsoids=6)
    with cuda_lib.Solver.from_problem(p, slabs=None) as s32, \
            cuda_lib.Solver.from_problem(p, slabs=None, precision=cuda_lib.BF16_GRADIENT) as sbf:
        g32, f32 = s32.gradient()
        gbf, fbf = sbf.gradient()
    g32 = g32.cpu().numpy().astype(np.float64)
    gbf = gbf.cpu().numpy().astype(np.float64)
    assert fbf == pytest.approx(f32, rel=1e-12)
    assert np.all(np.abs(gbf - g32) <= 2.0 ** -8 * np.abs(g32))
    # BF16 has 8 significand bits: rounding g32 in numpy gives the same values
    # up to ties, which a random FP32 field essentially never hits.
    u = g32.astype(np.float32).view(np.uint32).astype(np.uint64)
    rnd = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16).astype(np.uint32).view(np.float32)
    assert np.mean(rnd.astype(np.float64) == gbf) > 0.999


def test_bf16_descends_monotonically(cuda_lib):
    p = synth.tiny_problem(shape=(16, 48, 40), psf_shape=(7, 7, 5), seed=22, n_ellipsoids=7)
    with cuda_lib.Solver.from_problem(p, slabs=None, precision=cuda_lib.BF16_GRADIENT) as s:
        tr = s.iterate(60)
    assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:])), np.max(np.diff(tr))
    assert tr[-1] < tr[0]


def test_bf16_reaches_oracle_minimiser(cuda_lib):
    """After enough iterations both precisions sit at the same minimiser: the
    objective gap to the FP64 oracle's long run is below 1e-4 relative."""
    p = synth.tiny_problem(shape=(10, 32, 36), psf_shape=(5, 5, 5), seed=23, n_ellipsoids=5, lam=2e-2)
    oracle.set_threads(oracle.max_threads())
    op = oracle.OracleProblem.from_synth(p)
    _, _, fr = oracle.run(op, p.y, p.y, 400)
    fstar = fr[-1]
    with cuda_lib.Solver.from_problem(p, slabs=None, precision=cuda_lib.BF16_GRADIENT) as s:
        tr = s.iterate(400)
    assert (tr[-1] - fstar) / abs(fstar) <= 1e-4


def test_bf16_batch_and_slab_forms_descend(cuda_lib):
    probs = [
        synth.tiny_problem(shape=(9, 24, 40), psf_shape=(5, 5, 5), seed=24, n_ellipsoids=4),
        synth.tiny_problem(shape=(14, 31, 17), psf_shape=(3, 3, 3), seed=25, n_ellipsoids=4),
    ]
    with cuda_lib.BatchSolver(probs, precision=cuda_lib.BF16_GRADIENT) as b:
        tb = b.iterate(25)
        d1 = b.get(1, which=1).cpu().numpy()
    assert np.all(np.diff(tb, axis=1) <= 1e-6 * np.abs(tb[:, 1:]))
    assert np.all(np.isfinite(d1)) and np.any(d1 != 0)
    p = synth.tiny_problem(shape=(24, 40, 40), psf_shape=(5, 5, 5), seed=26, n_ellipsoids=6)
    with cuda_lib.Solver.from_problem(p, slabs=[0, 6, 12, 18, 24], precision=cuda_lib.BF16_GRADIENT) as s:
        ts = s.iterate(20)
    assert np.all(np.diff(ts) <= 1e-6 * np.abs(ts[1:]))


def test_mixed_batch_precisions_rejected(cuda_lib):
    probs = [synth.tiny_problem(shape=(8, 16, 16), psf_shape=(3, 3, 3), seed=27)] * 2
    with pytest.raises(cuda_lib.Bd3mgError, match="precision"):
        cuda_lib.BatchSolver(probs, precision=[cuda_lib.FP32, cuda_lib.BF16_GRADIENT])


def test_crop_errors_against_oracle(cuda_lib):
    """Errors of every precision against the FP64 oracle on the 128x128x32 crop
    of the 512x512x128 recipe (PSF 9x9x7): f and g at x0 = y, and f and x after
    10 sweeps.  The BF16 forms leave f(x0) unchanged (it does not involve g),
    round g to 8 significand bits, and perturb the later steps (BF16 directions
    also through the rounding of d, H g and H d)."""
    p = synth.workload_mixed(seed=0, crop=True)
    oracle.set_threads(oracle.max_threads())
    op = oracle.OracleProblem.from_synth(p)
    f0 = oracle.objective(op, p.y, p.y)
    g0 = oracle.gradient(op, p.y, p.y)
    n = 10
    xr, _, fr = oracle.run(op, p.y, p.y, n)
    errs = {}
    for prec in (cuda_lib.FP32, cuda_lib.BF16_GRADIENT, cuda_lib.BF16_DIRECTIONS):
        with cuda_lib.Solver.from_problem(p, slabs=None, precision=prec) as s:
            g, f = s.gradient()
            tr = s.iterate(n)
            x = s.get_x().cpu().numpy()
        errs[prec] = dict(f0=abs(f - f0) / abs(f0), g0=_rel(g.cpu().numpy(), g0),
                          f10=abs(tr[-1] - fr[-1]) / abs(fr[-1]), x10=_rel(x, xr))
    print("crop errors vs oracle:", errs)
    e32, ebf = errs[cuda_lib.FP32], errs[cuda_lib.BF16_GRADIENT]
    assert e32["f0"] <= 1e-5 and e32["g0"] <= 1e-5 and e32["f10"] <= 1e-5 and e32["x10"] <= 1e-4
    assert ebf["f0"] <= 1e-5
    assert ebf["g0"] <= 2.0 ** -8                     # per-element rounding bound, in norm
    assert ebf["f10"] <= 1e-4 and ebf["x10"] <= 1e-2
    ebd = errs[cuda_lib.BF16_DIRECTIONS]
    assert ebd["f0"] <= 1e-5 and ebd["g0"] <= 2.0 ** -8
    assert ebd["f10"] <= 1e-4 and ebd["x10"] <= 1e-2


# ---------------------------------------------------------------------------
# BF16 directions (BD3MG_BF16_DIRECTIONS): g, d, H g and H d stored in BF16,
# x, y and r in FP32; fused form only.
# ---------------------------------------------------------------------------

def _bf16_round(a):
    """Round FP32 values to BF16 (nearest even), returned as FP32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16).astype(np.uint32).view(np.float32)


def test_bf16_directions_first_step_rounds_the_stored_direction(cuda_lib):
    """The first iteration (d = 0) takes the BF16 gradient's step: x1 is the BF16
    gradient form's x1 bit for bit, and the stored d1 is its FP32 step rounded
    to BF16 (nearest even)."""
    p = synth.tiny_problem(shape=(12, 40, 52), psf_shape=(5, 5, 5), seed=28, n_ellipsoids=6)
    out = {}
    for prec in (cuda_lib.BF16_GRADIENT, cuda_lib.BF16_DIRECTIONS):
        with cuda_lib.Solver.from_problem(p, slabs=None, precision=prec, separate_update=2) as s:
            s.iterate(1)
            out[prec] = (s.get_x().cpu().numpy(), s.get_d().cpu().numpy())
    (xg, dg), (xd, dd) = out[cuda_lib.BF16_GRADIENT], out[cuda_lib.BF16_DIRECTIONS]
    np.testing.assert_array_equal(xd, xg)
    np.testing.assert_array_equal(dd, _bf16_round(dg))
    assert np.any(dd != 0)


def test_bf16_directions_descend_and_reach_oracle_minimiser(cuda_lib):
    """Near-monotone descent (each step minimises a majorant built from the
    stored directions; the carried residual drifts by their rounding between
    exact refreshes) and the FP64 oracle's minimiser to 1e-4 in objective."""
    p = synth.tiny_problem(shape=(10, 32, 36), psf_shape=(5, 5, 5), seed=23, n_ellipsoids=5, lam=2e-2)
    oracle.set_threads(oracle.max_threads())
    op = oracle.OracleProblem.from_synth(p)
    _, _, fr = oracle.run(op, p.y, p.y, 400)
    fstar = fr[-1]
    with cuda_lib.Solver.from_problem(p, slabs=None, precision=cuda_lib.BF16_DIRECTIONS) as s:
        tr = s.iterate(400)
        f_fresh = s.objective()
    print("bf16 directions: worst rise", float(np.max(np.diff(tr) / np.abs(tr[1:]))),
          "gap", (tr[-1] - fstar) / abs(fstar), "carried vs fresh f", (tr[-1] - f_fresh) / abs(f_fresh))
    assert np.all(np.diff(tr) <= 1e-5 * np.abs(tr[1:]))
    assert (tr[-1] - fstar) / abs(fstar) <= 1e-4
    assert abs(tr[-1] - f_fresh) <= 1e-4 * abs(f_fresh)


def test_bf16_directions_batch_escalation_and_checkpoint(cuda_lib, tmp_path):
    probs = [
        synth.tiny_problem(shape=(9, 24, 40), psf_shape=(5, 5, 5), seed=24, n_ellipsoids=4),
        synth.tiny_problem(shape=(14, 31, 17), psf_shape=(3, 3, 3), seed=25, n_ellipsoids=4),
    ]
    with cuda_lib.BatchSolver(probs, precision=cuda_lib.BF16_DIRECTIONS) as b:
        tb = b.iterate(25)
        d1 = b.get(1, which=1).cpu().numpy()
    assert np.all(np.diff(tb, axis=1) <= 1e-5 * np.abs(tb[:, 1:]))
    assert np.all(np.isfinite(d1)) and np.any(d1 != 0)
    np.testing.assert_array_equal(d1, _bf16_round(d1))            # widened BF16 values
    # escalation to FP32 storage keeps descending
    p = synth.tiny_problem(shape=(16, 48, 40), psf_shape=(7, 7, 5), seed=22, n_ellipsoids=7)
    with cuda_lib.Solver.from_problem(p, slabs=None, precision=cuda_lib.BF16_DIRECTIONS) as s:
        s.set_escalation(1e-3)
        tr = s.iterate(60)
        at = s.escalated()
    assert at >= 0 and tr[-1] < tr[0]
    assert np.all(np.diff(tr) <= 1e-5 * np.abs(tr[1:]))
    # checkpoint / resume in the same mode is bit-exact
    with cuda_lib.Solver.from_problem(p, slabs=None, precision=cuda_lib.BF16_DIRECTIONS) as s:
        s.iterate(7)
        s.save(str(tmp_path / "bd.ckpt"))
        t_a = s.iterate(6)
        x_a = s.get_x().cpu().numpy()
    with cuda_lib.Solver.from_problem(p, slabs=None, precision=cuda_lib.BF16_DIRECTIONS) as s:
        s.load(str(tmp_path / "bd.ckpt"))
        t_b = s.iterate(6)
        x_b = s.get_x().cpu().numpy()
    np.testing.assert_array_equal(t_b, t_a)
    np.testing.assert_array_equal(x_b, x_a)


def test_bf16_directions_other_forms_rejected(cuda_lib):
    p = synth.tiny_problem(shape=(8, 24, 24), psf_shape=(3, 3, 3), seed=29, n_ellipsoids=3)
    ps = synth.tiny_problem(shape=(8, 24, 24), psf_shape=(3, 3, 3), seed=29, n_ellipsoids=3, slabs=[0, 4, 8])
    for prob, kw in ((ps, {}), (p, {"separate_update": 1}), (p, {"penalty": 1}), (p, {"psf_mode": 1})):
        with pytest.raises(cuda_lib.Bd3mgError) as e:
            cuda_lib.Solver.from_problem(prob, precision=cuda_lib.BF16_DIRECTIONS, **kw)
        assert e.value.status == 7, (kw, str(e.value))
