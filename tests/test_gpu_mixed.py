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
    """Errors of both precisions against the FP64 oracle on the 128x128x32 crop
    of the 512x512x128 recipe (PSF 9x9x7): f and g at x0 = y, and f and x after
    10 sweeps.  The BF16 gradient leaves f(x0) unchanged (it does not involve g),
    rounds g to 8 significand bits, and perturbs the later steps."""
    p = synth.workload_mixed(seed=0, crop=True)
    oracle.set_threads(oracle.max_threads())
    op = oracle.OracleProblem.from_synth(p)
    f0 = oracle.objective(op, p.y, p.y)
    g0 = oracle.gradient(op, p.y, p.y)
    n = 10
    xr, _, fr = oracle.run(op, p.y, p.y, n)
    errs = {}
    for prec in (cuda_lib.FP32, cuda_lib.BF16_GRADIENT):
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
