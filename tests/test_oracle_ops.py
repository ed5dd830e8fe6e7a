"""Pins for the oracle's linear operators (CPU only).

H is checked against scipy.ndimage.convolve applied with each output depth's
PSF (a library routine), against a hand-computed 1D case, and through the
adjoint identity and an explicit matrix transpose for H^T.  V is checked against
numpy.diff.
"""
import numpy as np
import pytest
from scipy.ndimage import convolve

import oracle
from paper_2002_02328_gb300 import synth
from tests.golden_io import load_cases


def _op(shape, psf, **kw):
    return oracle.OracleProblem(shape, psf, **kw)


@pytest.mark.parametrize("shape,psf_shape", [((5, 7, 9), (3, 5, 3)), ((4, 6, 5), (5, 3, 7)),
                                             ((3, 4, 4), (5, 5, 5))])
def test_H_matches_scipy_convolve_per_depth(shape, psf_shape):
    rng = np.random.default_rng(1)
    psf = synth.random_psf(shape[0], psf_shape, seed=3)        # non-symmetric
    x = rng.standard_normal(shape)
    hx = oracle.apply_H(_op(shape, psf), x)
    for z in range(shape[0]):
        full = convolve(x, psf[z].astype(np.float64), mode="constant", cval=0.0)
        np.testing.assert_allclose(hx[z], full[z], rtol=0, atol=1e-12)


def test_H_hand_case():
    case = load_cases()["B"]
    op = _op(case["shape"], case["psf"], **case["params"])
    np.testing.assert_allclose(oracle.apply_H(op, case["x"]), case["Hx"], atol=1e-15)


@pytest.mark.parametrize("shape,psf_shape", [((5, 7, 9), (3, 5, 3)), ((6, 5, 4), (7, 3, 5))])
def test_adjoint_identity(shape, psf_shape):
    rng = np.random.default_rng(2)
    op = _op(shape, synth.random_psf(shape[0], psf_shape, seed=4))
    x = rng.standard_normal(shape)
    r = rng.standard_normal(shape)
    lhs = np.vdot(oracle.apply_H(op, x), r)
    rhs = np.vdot(x, oracle.apply_HT(op, r))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0)


def test_HT_is_matrix_transpose():
    shape, psf_shape = (3, 4, 5), (3, 3, 3)
    op = _op(shape, synth.random_psf(shape[0], psf_shape, seed=5))
    n = int(np.prod(shape))
    MH = np.zeros((n, n))
    MT = np.zeros((n, n))
    for m in range(n):
        e = np.zeros(n)
        e[m] = 1.0
        MH[:, m] = oracle.apply_H(op, e.reshape(shape)).ravel()
        MT[:, m] = oracle.apply_HT(op, e.reshape(shape)).ravel()
    np.testing.assert_allclose(MT, MH.T, atol=1e-15)


def test_delta_psf_is_identity():
    shape = (4, 5, 6)
    psf = np.zeros((4, 3, 5, 3), np.float32)
    psf[:, 1, 2, 1] = 1.0
    x = np.random.default_rng(3).standard_normal(shape)
    op = _op(shape, psf)
    np.testing.assert_array_equal(oracle.apply_H(op, x), x)
    np.testing.assert_array_equal(oracle.apply_HT(op, x), x)


def test_constant_interior_preserved():
    shape = (9, 11, 13)
    fx, fy, fz = synth.gaussian_factors(shape[0], 3, 3, 3, 0.6, 1.2, 0.8)
    op = _op(shape, synth.dense_psf(fx, fy, fz))
    hx = oracle.apply_H(op, np.ones(shape))
    psf_sums = op.psf.astype(np.float64).sum(axis=(1, 2, 3))
    np.testing.assert_allclose(hx[1:-1, 1:-1, 1:-1], psf_sums[1:-1, None, None] * np.ones((9, 11, 13))[1:-1, 1:-1, 1:-1],
                               rtol=1e-14)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_V_matches_numpy_diff_and_adjoint(axis):
    shape = (4, 5, 6)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(shape)
    q = rng.standard_normal(shape)
    op = _op(shape, np.ones((4, 1, 1, 1), np.float32))
    npax = 2 - axis                              # numpy axis of X is 2
    expect = np.zeros(shape)
    sl = [slice(None)] * 3
    sl[npax] = slice(0, shape[npax] - 1)
    expect[tuple(sl)] = np.diff(x, axis=npax)
    vx = oracle.apply_V(op, axis, x)
    np.testing.assert_allclose(vx, expect, atol=1e-15)
    assert abs(np.vdot(vx, q) - np.vdot(x, oracle.apply_VT(op, axis, q))) < 1e-12
