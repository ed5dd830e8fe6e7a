"""GPU parity of the block 3MG iteration against the FP64 oracle, through the C ABI.

Parity bounds: objective and gradient within relative 1e-5
after one iteration; iterate within relative 1e-4 (L2) after 200 iterations on
the 64x64x24 workload (PSF 5x5x5).  The slab form is compared with the oracle
visiting the slabs one after the other in colour-major order.  At the full
256x256x64 size the gradient is compared at sampled voxels and the objective in
full; the iteration is checked through properties (descent, determinism).
Beside the L2 bounds, element-wise bounds (max|a - b| over max|b|) catch errors
confined to a few voxels: 2e-5 for g, x and d after one iteration, 1e-3 for
the iterate after 200 iterations and for slab sweeps (a local error the L2 norm
would dilute by the square root of the voxel count is far above these).
"""
import numpy as np
import pytest

import oracle
from paper_2002_02328_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _maxrel(a, b):
    """Largest element-wise error, relative to the largest reference magnitude."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _colour_major(bounds, pz):
    """Reference colouring (written independently of the library): greedy in z,
    a slab joins the first colour whose latest slab ends >= max(pz-1,1) slices before it."""
    gap = max(pz - 1, 1)
    ends, col = [], []
    for s in range(len(bounds) - 1):
        c = next((k for k, e in enumerate(ends) if bounds[s] - e >= gap), len(ends))
        if c == len(ends):
            ends.append(0)
        ends[c] = bounds[s + 1]
        col.append(c)
    order = [s for c in range(len(ends)) for s in range(len(col)) if col[s] == c]
    return np.array(col), order


@pytest.fixture(scope="module")
def plain_small():
    p = synth.workload_plain_small()
    op = oracle.OracleProblem.from_synth(p)
    oracle.set_threads(oracle.max_threads())
    x200, d200, ft = oracle.run(op, p.y, p.y, 200)
    return p, op, x200, ft


def test_one_iteration_parity(cuda_lib, plain_small):
    p, op, _, _ = plain_small
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
    g1_ref = oracle.gradient(op, p.y, x1_ref)
    assert _rel(g1.cpu().numpy(), g1_ref) <= 1e-5
    assert _rel(x1, x1_ref) <= 1e-5
    assert _rel(d1, d1_ref) <= 1e-5
    assert _maxrel(g1.cpu().numpy(), g1_ref) <= 2e-5
    assert _maxrel(x1, x1_ref) <= 2e-5
    assert _maxrel(d1, d1_ref) <= 2e-5
    B = info["B"]
    np.testing.assert_allclose([st[0], st[1], st[2]], [B[0, 0], B[0, 1], B[1, 1]], rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(st[3:5], info["c"], rtol=1e-5, atol=1e-12)
    assert abs(st[5] - info["u"][0]) <= 1e-5 * abs(info["u"][0]) and st[6] == 0.0 and st[7] == 1


def test_200_iterations_parity(cuda_lib, plain_small):
    p, op, x200, ft = plain_small
    with cuda_lib.Solver.from_problem(p) as s:
        tr = s.iterate(200)
        x = s.get_x().cpu().numpy()
    assert _rel(x, x200) <= 1e-4
    assert _maxrel(x, x200) <= 1e-3
    assert np.max(np.abs(tr - ft) / np.abs(ft)) <= 1e-5


def test_determinism_and_iterate_split(cuda_lib):
    p = synth.tiny_problem(shape=(9, 40, 50), psf_shape=(5, 5, 5), seed=3, n_ellipsoids=6)
    with cuda_lib.Solver.from_problem(p) as a, cuda_lib.Solver.from_problem(p) as b:
        ta = a.iterate(30)
        tb1 = b.iterate(10)
        tb2 = b.iterate(20)
        xa, xb = a.get_x().cpu().numpy(), b.get_x().cpu().numpy()
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(ta[:11], tb1)
    np.testing.assert_array_equal(ta[10:], tb2)


@pytest.mark.parametrize("shape,psf_shape,bounds", [
    ((24, 40, 48), (5, 5, 5), [0, 3, 9, 12, 17, 20, 24]),      # uneven slabs, 5-tap z blur
    ((16, 24, 40), (3, 3, 3), [0, 1, 2, 6, 7, 16]),             # one-slice slabs
    ((10, 20, 36), (5, 5, 1), [0, 2, 5, 6, 10]),                # no z blur: adjacent slabs differ in colour
])
def test_slab_form_matches_sequential_oracle(cuda_lib, shape, psf_shape, bounds):
    p = synth.tiny_problem(shape=shape, psf_shape=psf_shape, seed=5, n_ellipsoids=8, sxy=(0.5, 2.0), sz=1.0,
                           slabs=bounds)
    op = oracle.OracleProblem.from_synth(p)
    col_ref, order = _colour_major(bounds, psf_shape[2])
    oracle.set_threads(oracle.max_threads())
    xr, dr, fr = oracle.run(op, p.y, p.y, 6, bounds=bounds, order=order)
    with cuda_lib.Solver.from_problem(p) as s:
        col, nc = s.colours()
        tr = s.iterate(6)
        x = s.get_x().cpu().numpy()
        d = s.get_d().cpu().numpy()
    np.testing.assert_array_equal(col, col_ref)
    assert _rel(x, xr) <= 2e-5
    assert _rel(d, dr) <= 1e-4
    assert _maxrel(x, xr) <= 1e-3
    assert np.max(np.abs(tr - fr) / np.abs(fr)) <= 1e-5
    assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:]))


@pytest.fixture(scope="module")
def full_slabs():
    return synth.workload_slabs()


def test_full_size_gradient_sampled_and_objective(cuda_lib, full_slabs):
    p = full_slabs
    op = oracle.OracleProblem.from_synth(p)
    oracle.set_threads(oracle.max_threads())
    rng = np.random.default_rng(0)
    nz, ny, nx = p.shape
    corners = [0, nx - 1, nx * (ny - 1), p.n - 1, (nz // 2) * nx * ny + (ny // 2) * nx + nx // 2]
    idx = np.concatenate([corners, rng.choice(p.n, size=59, replace=False)]).astype(np.int64)
    with cuda_lib.Solver.from_problem(p) as s:
        g, f = s.gradient()
        g = g.cpu().numpy().ravel()
    g_ref = oracle.gradient_at(op, p.y, p.y.astype(np.float64), idx)
    f_ref = oracle.objective(op, p.y, p.y)
    assert abs(f - f_ref) <= 1e-5 * abs(f_ref)
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g[idx] - g_ref)) <= 1e-5 * scale


def test_full_size_slab_sweeps_descend(cuda_lib, full_slabs):
    p = full_slabs
    with cuda_lib.Solver.from_problem(p) as s:
        col, nc = s.colours()
        tr = s.iterate(20)
    col_ref, _ = _colour_major(p.slabs, 7)
    np.testing.assert_array_equal(col, col_ref)
    assert nc == 3
    assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:]))
    assert tr[-1] < 0.9 * tr[0]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("zchunk", [4, 5])
def test_slab_form_with_short_chunks_matches_oracle(cuda_lib, prec, zchunk):
    """Short z-chunks make work items start and end at every slab edge, where
    slices outside the slab are zero-filled in the curvature ring."""
    bounds = [0, 4, 11, 13, 20]
    p = synth.tiny_problem(shape=(20, 36, 40), psf_shape=(7, 7, 7), seed=9, n_ellipsoids=8, sxy=(0.5, 2.0), sz=1.0,
                           slabs=bounds)
    op = oracle.OracleProblem.from_synth(p)
    _, order = _colour_major(bounds, 7)
    oracle.set_threads(oracle.max_threads())
    xr, _, fr = oracle.run(op, p.y, p.y, 8, bounds=bounds, order=order)
    with cuda_lib.Solver.from_problem(p, precision=prec, zchunk=zchunk) as s:
        tr = s.iterate(8)
        x = s.get_x().cpu().numpy()
    assert np.all(np.isfinite(tr)) and np.all(np.isfinite(x))
    if prec == 0:
        assert _rel(x, xr) <= 2e-5
        assert np.max(np.abs(tr - fr) / np.abs(fr)) <= 1e-5
    else:                                  # BF16 gradient: descent and closeness to the FP32 oracle path
        assert np.all(np.diff(tr) <= 1e-6 * np.abs(tr[1:]))
        assert np.max(np.abs(tr - fr) / np.abs(fr)) <= 1e-3
