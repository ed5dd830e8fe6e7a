"""Pins of the FP64 U-Net oracle against things other than itself: scipy's
correlation, brute-force loops, central finite differences, and Adam's closed
form under a constant gradient."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import unet as U


def _rng(seed):
    return np.random.default_rng(seed)


def test_conv3_is_scipy_correlation_summed_over_channels():
    r = _rng(0)
    x = r.normal(size=(5, 6, 7, 3))
    w = r.normal(size=(27, 2, 3))
    b = r.normal(size=2)
    out = U.conv3(x, w, b)
    for co in range(2):
        ref = np.full(x.shape[:3], b[co])
        for ci in range(3):
            k = w[:, co, ci].reshape(3, 3, 3)        # [dz, dy, dx], centred
            ref += ndimage.correlate(x[..., ci], k, mode="constant", cval=0.0)
        np.testing.assert_allclose(out[..., co], ref, rtol=1e-12, atol=1e-12)


def _fd_check(f, arg, grad, idxs, h=1e-6, rtol=1e-6):
    for idx in idxs:
        save = arg[idx]
        arg[idx] = save + h
        fp = f()
        arg[idx] = save - h
        fm = f()
        arg[idx] = save
        fd = (fp - fm) / (2 * h)
        assert abs(fd - grad[idx]) <= rtol * max(1.0, abs(fd)), (idx, fd, grad[idx])


def _some(shape, r, n=6):
    return [tuple(int(r.integers(0, s)) for s in shape) for _ in range(n)]


def test_conv3_backward_finite_differences():
    r = _rng(1)
    x = r.normal(size=(4, 5, 6, 3))
    w = r.normal(size=(27, 2, 3))
    b = r.normal(size=2)
    g = r.normal(size=(4, 5, 6, 2))
    dx, dw, db = U.conv3_backward(x, w, g)
    f = lambda: float(np.sum(U.conv3(x, w, b) * g))
    _fd_check(f, x, dx, _some(x.shape, r))
    _fd_check(f, w, dw, _some(w.shape, r))
    _fd_check(f, b, db, [(0,), (1,)])


def test_maxpool_matches_loops_and_first_maximum_wins_ties():
    r = _rng(2)
    x = r.integers(0, 3, size=(4, 6, 4, 2)).astype(np.float64)     # many ties
    out, arg = U.maxpool2(x)
    dout = r.normal(size=out.shape)
    dx = U.maxpool2_backward(dout, arg)
    ref_dx = np.zeros_like(x)
    for z in range(2):
        for y in range(3):
            for xx in range(2):
                for c in range(2):
                    best, bt = -np.inf, None
                    for a, (az, ay, ax) in enumerate(U.TAPS2):
                        v = x[2 * z + az, 2 * y + ay, 2 * xx + ax, c]
                        if v > best:
                            best, bt = v, (az, ay, ax)
                    assert out[z, y, xx, c] == best
                    ref_dx[2 * z + bt[0], 2 * y + bt[1], 2 * xx + bt[2], c] += dout[z, y, xx, c]
    np.testing.assert_array_equal(dx, ref_dx)
    _, arg0 = U.maxpool2(np.zeros((2, 2, 2, 1)))
    assert arg0.item() == 0


def test_up2_matches_scatter_loops_and_backward_fd():
    r = _rng(3)
    x = r.normal(size=(2, 3, 2, 3))
    w = r.normal(size=(8, 2, 3))
    b = r.normal(size=2)
    out = U.up2(x, w, b)
    ref = np.zeros((4, 6, 4, 2)) + b
    for z in range(2):
        for y in range(3):
            for xx in range(2):
                for a, (az, ay, ax) in enumerate(U.TAPS2):
                    ref[2 * z + az, 2 * y + ay, 2 * xx + ax] += w[a] @ x[z, y, xx]
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)
    g = r.normal(size=out.shape)
    dx, dw, db = U.up2_backward(x, w, g)
    f = lambda: float(np.sum(U.up2(x, w, b) * g))
    _fd_check(f, x, dx, _some(x.shape, r))
    _fd_check(f, w, dw, _some(w.shape, r))
    _fd_check(f, b, db, [(0,), (1,)])


def _tiny_params(widths, cin, seed):
    r = _rng(seed)
    p = {}
    for name, ws, bs in U.layer_shapes(widths, cin):
        fan_in = ws[0] * ws[2]
        p[name + ".w"] = r.normal(scale=np.sqrt(2.0 / fan_in), size=ws)
        p[name + ".b"] = r.normal(scale=0.1, size=bs)
    return p


def test_network_backward_finite_differences():
    widths = (2, 3, 2, 4)
    p = _tiny_params(widths, 2, 4)
    r = _rng(5)
    inp = r.normal(size=(8, 8, 8, 2))
    target = r.normal(size=(8, 8, 8))

    def loss():
        out, _ = U.forward(p, inp, widths)
        return U.mse_loss(out, target)[0]

    out, cache = U.forward(p, inp, widths, keep=True)
    _, dout = U.mse_loss(out, target)
    grads = U.backward(p, cache, dout, widths)
    assert set(grads) == set(p)
    for name in ("enc0a.w", "enc1b.w", "enc3a.b", "enc3b.w", "up2.w", "up0.b", "dec1a.w", "dec0b.b", "head.w",
                 "head.b"):
        _fd_check(loss, p[name], grads[name], _some(p[name].shape, r, 3), h=1e-6, rtol=1e-5)


def test_network_shapes_and_skip_order():
    widths = (2, 3, 2, 4)
    p = _tiny_params(widths, 2, 6)
    inp = _rng(7).normal(size=(8, 16, 8, 2))
    out, cache = U.forward(p, inp, widths, keep=True)
    assert out.shape == (8, 16, 8)
    # decoder 0 input = [encoder level-0 output, upsampled decoder level-1 output]
    np.testing.assert_array_equal(cache["dec0a_in"][..., :2], cache["enc0_out"])
    np.testing.assert_array_equal(cache["dec0a_in"][..., 2:],
                                  U.up2(cache["up0_in"], p["up0.w"], p["up0.b"]))


def test_mse_gradient_and_adam_closed_form():
    r = _rng(8)
    pred, target = r.normal(size=(3, 4, 5)), r.normal(size=(3, 4, 5))
    l, g = U.mse_loss(pred, target)
    assert l == pytest.approx(np.mean((pred - target) ** 2), rel=1e-14)
    _fd_check(lambda: U.mse_loss(pred, target)[0], pred, g, _some(pred.shape, r))
    # constant gradient: bias correction makes every step lr * g / (|g| + eps)
    w0 = r.normal(size=7)
    gc = r.normal(size=7)
    w, m, v = w0.copy(), np.zeros(7), np.zeros(7)
    for t in range(1, 6):
        w_prev = w
        w, m, v = U.adam_step(w, gc, m, v, t, lr=1e-2)
        np.testing.assert_allclose(w_prev - w, 1e-2 * gc / (np.abs(gc) + 1e-8), rtol=1e-10)
