"""Edge cases of the method on the GPU against the FP64 oracle: degenerate
volume shapes (one row, one column, one slice, a volume smaller than the PSF),
a start that already is the minimiser (g = 0: the 2x2 system has rank 0 and
the step must be zero), and the 512x512x128 volume at full size on sampled
gradient voxels."""
import numpy as np
import pytest

import oracle
from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("shape,psf_shape", [
    ((1, 6, 9), (3, 3, 3)),        # one slice
    ((4, 1, 10), (3, 3, 3)),       # one row
    ((3, 7, 1), (3, 3, 3)),        # one column
    ((2, 2, 2), (5, 5, 5)),        # smaller than the PSF
    ((5, 9, 3), (7, 7, 7)),        # thinner than the PSF in x and z
])
def test_degenerate_shapes_match_oracle(cuda_lib, shape, psf_shape):
    p = synth.tiny_problem(shape=shape, psf_shape=psf_shape, seed=11, n_ellipsoids=2)
    op = oracle.OracleProblem.from_synth(p)
    x0 = p.y.astype(np.float64)
    f0 = oracle.objective(op, p.y, x0)
    g0 = oracle.gradient(op, p.y, x0)
    x1, _, _ = oracle.step(op, p.y, x0, np.zeros(p.shape))
    with cuda_lib.Solver.from_problem(p, slabs=None) as s:
        g, f = s.gradient()
        tr = s.iterate(1)
        x = s.get_x().cpu().numpy()
    assert abs(f - f0) <= 1e-5 * abs(f0)
    assert _rel(g.cpu().numpy(), g0) <= 1e-5
    assert abs(tr[0] - f0) <= 1e-5 * abs(f0)
    assert _rel(x, x1) <= 1e-5


def test_minimiser_start_gives_rank_zero_step(cuda_lib):
    """H = I (1x1x1 PSF), y constant inside the box: x = y has r = 0, Vx = 0 and
    zero box distance, so grad f = 0 exactly; the subspace matrix is zero, its
    pseudo-inverse drops both eigenvalues and x must not move."""
    shape = (6, 10, 12)
    y = np.full(shape, 0.4, np.float32)
    psf = np.ones((shape[0], 1, 1, 1), np.float32)
    with cuda_lib.Solver(shape, psf, y) as s:
        g, f = s.gradient()
        tr = s.iterate(3)
        x = s.get_x().cpu().numpy()
        info = s.last_step()
    assert np.all(g.cpu().numpy() == 0.0)
    assert np.array_equal(x, y)
    assert np.all(tr == tr[0])
    assert info[0, 7] == 0 and info[0, 5] == 0.0 and info[0, 6] == 0.0      # rank 0, u = 0


def test_full_size_512_gradient_sampled(cuda_lib):
    """The 512x512x128 recipe at full size (PSF 9x9x7), in the launch shape the
    bench times: the gradient at sampled voxels (corners, faces, interior)."""
    p = synth.workload_mixed(seed=0)
    op = oracle.OracleProblem.from_synth(p)
    oracle.set_threads(oracle.max_threads())
    nz, ny, nx = p.shape
    rng = np.random.default_rng(3)
    corners = [0, nx - 1, nx * (ny - 1), p.n - 1, (nz - 1) * nx * ny, (nz // 2) * nx * ny + (ny // 2) * nx + nx // 2]
    idx = np.concatenate([corners, rng.choice(p.n, size=58, replace=False)]).astype(np.int64)
    with cuda_lib.Solver.from_problem(p, slabs=None) as s:
        g, _ = s.gradient()
        g = g.cpu().numpy().ravel()
    g_ref = oracle.gradient_at(op, p.y, p.y.astype(np.float64), idx)
    assert np.max(np.abs(g[idx] - g_ref)) <= 1e-5 * np.max(np.abs(g_ref))
