"""GPU parity of penalty modes 1 and 2 against the FP64 oracle, through the C ABI.

Mode 1 is the objective as Section 3.1 prints it: a joint X-Y hyperbolic term
lambda sum_n sqrt(delta^2 + [V^X x]_n^2 + [V^Y x]_n^2) plus kappa ||V^Z x||^2,
with the X and Y differences sharing one half-quadratic weight in the majorant
and the Z term entering through its exact Hessian 2 kappa V^ZT V^Z.  Mode 2 is
the isotropic term lambda sum_n sqrt(delta^2 + sum_a [V^a x]_n^2), one weight
shared by the three differences.  The bounds are those of the per-axis mode:
objective and gradient within relative 1e-5 (ragged shapes spanning several
32x32 tiles, both starts), one iteration
(f, g, x, d, B, c, u) within 1e-5, 200 iterations of the 64x64x24 workload
within 1e-4 on the iterate and 1e-5 on the objective trace, slab sweeps
against the oracle visiting the slabs one after the other in colour-major
order (x 2e-5, trace 1e-5).  With a BF16 gradient the run must descend and end
at the oracle's minimiser within 1e-4.  Batches of mixed modes and invalid
modes or kappa are rejected, and the allocation-free objective honours the
mode.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2002_02328_gb300 import synth
from tests.test_gpu_3mg import _colour_major

pytestmark = pytest.mark.gpu

KAPPA = 0.05


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _joint(p, kappa=KAPPA):
    return dataclasses.replace(p, penalty=1, kappa=kappa)


def _mode(p, mode, kappa=KAPPA):
    return dataclasses.replace(p, penalty=mode, kappa=kappa if mode == 1 else 0.0)


@pytest.mark.parametrize("shape,psf_shape,mode,kappa", [
    ((13, 45, 70), (5, 5, 5), 1, KAPPA),   # ragged in x and y: three by two 32-wide tiles
    ((9, 33, 37), (7, 7, 7), 1, 0.7),      # one column and one row past a tile edge
    ((6, 40, 36), (3, 3, 3), 1, 0.0),      # joint X-Y term alone
    ((13, 45, 70), (5, 5, 5), 2, 0.0),
    ((9, 33, 37), (7, 7, 7), 2, 0.0),
    ((5, 34, 66), (9, 9, 7), 2, 0.0),      # largest compiled radii of the workloads
])
def test_objective_and_gradient_match_oracle(cuda_lib, shape, psf_shape, mode, kappa):
    p = _mode(synth.tiny_problem(shape=shape, psf_shape=psf_shape, seed=61, n_ellipsoids=6), mode, kappa)
    op = oracle.OracleProblem.from_synth(p)
    assert op.penalty == mode and op.kappa == kappa
    for x0 in (p.y, synth.uniform_start(p.y, seed=3)):
        f_ref, parts_ref = oracle.objective(op, p.y, x0, parts=True)
        g_ref = oracle.gradient(op, p.y, x0)
        with cuda_lib.Solver.from_problem(p, x0=x0, slabs=None) as s:
            f, parts = s.objective(parts=True)
            g, fg = s.gradient()
        assert abs(f - f_ref) <= 1e-5 * abs(f_ref)
        assert abs(fg - f_ref) <= 1e-5 * abs(f_ref)
        np.testing.assert_allclose(parts, parts_ref, rtol=1e-5, atol=1e-9 * abs(f_ref))
        assert _rel(g.cpu().numpy(), g_ref) <= 1e-5


def test_modes_change_the_objective(cuda_lib):
    """The three modes give different objectives and gradients on the same data
    (a kernel that ignored the mode would pass the parity test of none)."""
    p = synth.tiny_problem(shape=(8, 24, 28), psf_shape=(3, 3, 3), seed=62, n_ellipsoids=4)
    res = []
    for mode in (0, 1, 2):
        with cuda_lib.Solver.from_problem(_mode(p, mode), slabs=None) as s:
            g, f = s.gradient()
            res.append((g.cpu().numpy(), f))
    for a in range(3):
        for b in range(a + 1, 3):
            assert abs(res[a][1] - res[b][1]) > 1e-3 * abs(res[a][1])
            assert _rel(res[a][0], res[b][0]) > 1e-3


@pytest.fixture(scope="module", params=[1, 2])
def mode_small(request):
    p = _mode(synth.workload_plain_small(), request.param)
    op = oracle.OracleProblem.from_synth(p)
    oracle.set_threads(oracle.max_threads())
    x200, _, ft = oracle.run(op, p.y, p.y, 200)
    return p, op, x200, ft


def test_one_iteration_parity(cuda_lib, mode_small):
    p, op, _, _ = mode_small
    x0 = p.y.astype(np.float64)
    x1_ref, d1_ref, info = oracle.step(op, p.y, x0, np.zeros(p.shape))
    with cuda_lib.Solver.from_problem(p) as s:
        tr = s.iterate(1)
        g1, f1 = s.gradient()
        x1 = s.get_x().cpu().numpy()
        d1 = s.get_d().cpu().numpy()
        st = s.last_step()[0]
    f0_ref = oracle.objective(op, p.y, x0)
    f1_ref = oracle.objective(op, p.y, x1_ref)
    assert abs(tr[0] - f0_ref) <= 1e-5 * abs(f0_ref)
    assert abs(tr[1] - f1_ref) <= 1e-5 * abs(f1_ref)
    assert abs(f1 - f1_ref) <= 1e-5 * abs(f1_ref)
    assert _rel(g1.cpu().numpy(), oracle.gradient(op, p.y, x1_ref)) <= 1e-5
    assert _rel(x1, x1_ref) <= 1e-5
    assert _rel(d1, d1_ref) <= 1e-5
    B = info["B"]
    np.testing.assert_allclose([st[0], st[1], st[2]], [B[0, 0], B[0, 1], B[1, 1]], rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(st[3:5], info["c"], rtol=1e-5, atol=1e-12)
    assert abs(st[5] - info["u"][0]) <= 1e-5 * abs(info["u"][0]) and st[6] == 0.0 and st[7] == 1


def test_200_iterations_parity(cuda_lib, mode_small):
    p, op, x200, ft = mode_small
    with cuda_lib.Solver.from_problem(p) as s:
        tr = s.iterate(200)
        x = s.get_x().cpu().numpy()
    assert _rel(x, x200) <= 1e-4
    assert np.max(np.abs(tr - ft) / np.abs(ft)) <= 1e-5
    assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:]))


@pytest.mark.parametrize("mode", [1, 2])
def test_slab_sweeps_match_sequential_oracle(cuda_lib, mode):
    p = _mode(synth.tiny_problem(shape=(22, 40, 44), psf_shape=(5, 5, 5), seed=63, n_ellipsoids=8), mode)
    bounds = [0, 3, 7, 12, 16, 22]
    _, order = _colour_major(bounds, 5)
    op = oracle.OracleProblem.from_synth(p)
    oracle.set_threads(oracle.max_threads())
    x_ref, d_ref, f_ref = oracle.run(op, p.y, p.y, 30, bounds=bounds, order=order)
    with cuda_lib.Solver.from_problem(p, slabs=bounds) as s:
        tr = s.iterate(30)
        x = s.get_x().cpu().numpy()
    assert _rel(x, x_ref) <= 2e-5
    assert np.max(np.abs(tr - f_ref) / np.abs(f_ref)) <= 1e-5


@pytest.mark.parametrize("mode", [1, 2])
def test_bf16_gradient_reaches_oracle_minimiser(cuda_lib, mode):
    p = _mode(synth.tiny_problem(shape=(10, 32, 36), psf_shape=(5, 5, 5), seed=64, n_ellipsoids=5, lam=2e-2), mode)
    op = oracle.OracleProblem.from_synth(p)
    oracle.set_threads(oracle.max_threads())
    _, _, fr = oracle.run(op, p.y, p.y, 400)
    with cuda_lib.Solver.from_problem(p, slabs=None, precision=cuda_lib.BF16_GRADIENT) as s:
        tr = s.iterate(400)
    assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:]))
    assert (tr[-1] - fr[-1]) / abs(fr[-1]) <= 1e-4


@pytest.mark.parametrize("mode", [1, 2])
def test_batch_matches_single_volume_solves(cuda_lib, mode):
    probs = [_mode(synth.tiny_problem(shape=(9, 24, 40), psf_shape=(5, 5, 5), seed=65, n_ellipsoids=4), mode),
             _mode(synth.tiny_problem(shape=(14, 31, 17), psf_shape=(3, 3, 3), seed=66, n_ellipsoids=4), mode, 0.3)]
    with cuda_lib.BatchSolver(probs) as b:
        tb = b.iterate(20)
    for v, p in enumerate(probs):
        op = oracle.OracleProblem.from_synth(p)
        _, _, f_ref = oracle.run(op, p.y, p.y, 20)
        assert np.max(np.abs(tb[v] - f_ref) / np.abs(f_ref)) <= 1e-5


def test_invalid_modes_rejected(cuda_lib):
    p = synth.tiny_problem(shape=(8, 16, 16), psf_shape=(3, 3, 3), seed=67)
    with pytest.raises(cuda_lib.Bd3mgError, match="penalty mode"):
        cuda_lib.BatchSolver([p, _joint(p)])
    with pytest.raises(cuda_lib.Bd3mgError, match="penalty mode"):
        cuda_lib.BatchSolver([_mode(p, 2), _joint(p)])
    with pytest.raises(cuda_lib.Bd3mgError, match="penalty mode"):
        cuda_lib.Solver.from_problem(dataclasses.replace(p, penalty=3), slabs=None)
    with pytest.raises(cuda_lib.Bd3mgError, match="kappa"):
        cuda_lib.Solver.from_problem(_joint(p, -1.0), slabs=None)


@pytest.mark.parametrize("mode", [1, 2])
def test_noalloc_objective_honours_the_mode(cuda_lib, mode):
    import torch
    p = _mode(synth.workload_plain_small(), mode)
    op = oracle.OracleProblem.from_synth(p)
    x0 = synth.uniform_start(p.y, seed=4)
    params, keep = cuda_lib.make_params(p.shape, p.psf, p.lam, p.delta, p.eta, p.xmin, p.xmax,
                                        penalty=mode, kappa=p.kappa)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    cuda_lib.bd3mg_objective_noalloc(params, torch.from_numpy(x0).cuda(), torch.from_numpy(p.y).cuda(), out)
    torch.cuda.synchronize()
    f_ref = oracle.objective(op, p.y, x0)
    assert abs(out[0].item() - f_ref) <= 1e-5 * abs(f_ref)
