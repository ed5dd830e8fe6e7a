"""FP64 oracle of the learned warm start: a 3D U-Net, its backward pass, MSE
loss and Adam, written from the definitions.  Test infrastructure only (the
tests, the smoke check and the bench's CPU baseline use it; the library never
does).

The network predicts x_hat = y + net([y, s]) where s is the per-depth blur
width map; it has 4 levels of widths C = (16, 32, 64, 128) on the GPU (any
widths here), two 3x3x3 convolutions + bias + ReLU per level, 2x2x2 max
pooling on the way down, a 2x2x2 stride-2 transposed convolution (+ bias, no
activation) on the way up, skip concatenation [encoder, upsampled], and a
1x1x1 head.  The paper has no learned component: the architecture follows the
design readings (inputs [y, sigma_xy(z)], residual output, no normalisation).

Layout: one volume is a float64 array [D, H, W, C] (channels last).  A 3x3x3
weight is [27, Cout, Cin] with tap t = (dz * 3 + dy) * 3 + dx reading input
voxel (z + dz - 1, y + dy - 1, x + dx - 1), zero outside the volume; an up
weight is [8, Cout, Cin] with tap a = (az * 2 + ay) * 2 + ax writing output
voxel (2z + az, 2y + ay, 2x + ax).  Max-pool ties go to the first maximum in
(dz, dy, dx) order.
"""
from typing import Dict, List, Sequence, Tuple

import numpy as np

TAPS3 = [(dz, dy, dx) for dz in range(3) for dy in range(3) for dx in range(3)]
TAPS2 = [(az, ay, ax) for az in range(2) for ay in range(2) for ax in range(2)]


def _shifted(x: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """v[z, y, x] = x[z + dz, y + dy, x + dx], zero outside (offsets in -1..1)."""
    D, H, W = x.shape[:3]
    out = np.zeros_like(x)
    zs, ys, xs = slice(max(0, -dz), min(D, D - dz)), slice(max(0, -dy), min(H, H - dy)), \
        slice(max(0, -dx), min(W, W - dx))
    zt, yt, xt = slice(max(0, dz), min(D, D + dz)), slice(max(0, dy), min(H, H + dy)), \
        slice(max(0, dx), min(W, W + dx))
    out[zs, ys, xs] = x[zt, yt, xt]
    return out


def conv3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[v, co] = b[co] + sum_t sum_ci w[t, co, ci] x[v + t - 1, ci]."""
    out = np.broadcast_to(b, x.shape[:3] + (w.shape[1],)).astype(np.float64).copy()
    for t, (dz, dy, dx) in enumerate(TAPS3):
        out += np.einsum("zyxc,oc->zyxo", _shifted(x, dz - 1, dy - 1, dx - 1), w[t])
    return out


def conv3_backward(x: np.ndarray, w: np.ndarray, dout: np.ndarray):
    """Gradients of conv3 with respect to x, w and b, given dL/dout."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (dz, dy, dx_) in enumerate(TAPS3):
        xs = _shifted(x, dz - 1, dy - 1, dx_ - 1)
        dw[t] = np.einsum("zyxo,zyxc->oc", dout, xs)
        # out[v] reads x[v + s]: the gradient flows back to x[u] from out[u - s]
        dx += _shifted(np.einsum("zyxo,oc->zyxc", dout, w[t]), -(dz - 1), -(dy - 1), -(dx_ - 1))
    db = dout.sum(axis=(0, 1, 2))
    return dx, dw, db


def relu(x):
    return np.maximum(x, 0.0)


def maxpool2(x: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """2x2x2 max pooling; returns (out, arg) with arg the tap (0..7) of the first maximum."""
    D, H, W, C = x.shape
    v = x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).transpose(0, 2, 4, 1, 3, 5, 6).reshape(
        D // 2, H // 2, W // 2, 8, C)
    arg = np.argmax(v, axis=3)                       # numpy returns the first maximum
    return np.take_along_axis(v, arg[:, :, :, None, :], axis=3)[:, :, :, 0, :], arg


def maxpool2_backward(dout: np.ndarray, arg: np.ndarray) -> np.ndarray:
    D, H, W, C = dout.shape
    g = np.zeros((D, H, W, 8, C))
    np.put_along_axis(g, arg[:, :, :, None, :], dout[:, :, :, None, :], axis=3)
    return g.reshape(D, H, W, 2, 2, 2, C).transpose(0, 3, 1, 4, 2, 5, 6).reshape(2 * D, 2 * H, 2 * W, C)


def up2(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """out[2z + az, 2y + ay, 2x + ax, co] = b[co] + sum_ci w[a, co, ci] x[z, y, x, ci]."""
    D, H, W, _ = x.shape
    out = np.empty((2 * D, 2 * H, 2 * W, w.shape[1]))
    for a, (az, ay, ax) in enumerate(TAPS2):
        out[az::2, ay::2, ax::2] = np.einsum("zyxc,oc->zyxo", x, w[a]) + b
    return out


def up2_backward(x: np.ndarray, w: np.ndarray, dout: np.ndarray):
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for a, (az, ay, ax) in enumerate(TAPS2):
        g = dout[az::2, ay::2, ax::2]
        dx += np.einsum("zyxo,oc->zyxc", g, w[a])
        dw[a] = np.einsum("zyxo,zyxc->oc", g, x)
    return dx, dw, dout.sum(axis=(0, 1, 2))


# ---------------------------------------------------------------------------
# Network
# ---------------------------------------------------------------------------

def layer_shapes(widths: Sequence[int] = (16, 32, 64, 128), cin: int = 2) -> List[Tuple[str, tuple, tuple]]:
    """(name, weight shape, bias shape) of every parameter tensor, in a fixed order."""
    c = list(widths)
    out = []
    prev = cin
    for l, cl in enumerate(c):
        out.append((f"enc{l}a", (27, cl, prev), (cl,)))
        out.append((f"enc{l}b", (27, cl, cl), (cl,)))
        prev = cl
    for l in range(len(c) - 2, -1, -1):
        out.append((f"up{l}", (8, c[l], c[l + 1]), (c[l],)))
        out.append((f"dec{l}a", (27, c[l], 2 * c[l]), (c[l],)))
        out.append((f"dec{l}b", (27, c[l], c[l]), (c[l],)))
    out.append(("head", (1, 1, c[0]), (1,)))
    return out


def forward(params: Dict[str, np.ndarray], inp: np.ndarray, widths=(16, 32, 64, 128), keep: bool = False):
    """net(inp) for one volume [D, H, W, cin]; returns (out [D, H, W], cache or None)."""
    L = len(widths)
    cache = {"inp": inp}
    h = inp
    skips = []
    for l in range(L):
        if l > 0:
            h, arg = maxpool2(h)
            cache[f"pool{l}"] = arg
        cache[f"enc{l}a_in"] = h
        h = relu(conv3(h, params[f"enc{l}a.w"], params[f"enc{l}a.b"]))
        cache[f"enc{l}b_in"] = h
        h = relu(conv3(h, params[f"enc{l}b.w"], params[f"enc{l}b.b"]))
        cache[f"enc{l}_out"] = h
        skips.append(h)
    for l in range(L - 2, -1, -1):
        cache[f"up{l}_in"] = h
        u = up2(h, params[f"up{l}.w"], params[f"up{l}.b"])
        h = np.concatenate([skips[l], u], axis=3)
        cache[f"dec{l}a_in"] = h
        h = relu(conv3(h, params[f"dec{l}a.w"], params[f"dec{l}a.b"]))
        cache[f"dec{l}b_in"] = h
        h = relu(conv3(h, params[f"dec{l}b.w"], params[f"dec{l}b.b"]))
    cache["head_in"] = h
    out = np.einsum("zyxc,c->zyx", h, params["head.w"][0, 0]) + params["head.b"][0]
    return out, (cache if keep else None)


def _relu_conv_backward(params, cache, name, dact):
    """Backward through act = relu(conv3(cache[name_in])): returns d(input), dW, db."""
    x = cache[f"{name}_in"]
    w, b = params[f"{name}.w"], params[f"{name}.b"]
    z = conv3(x, w, b)
    dz = dact * (z > 0)
    return conv3_backward(x, w, dz)


def backward(params, cache, dout: np.ndarray, widths=(16, 32, 64, 128)) -> Dict[str, np.ndarray]:
    """Gradients of sum(dout * net(inp)) with respect to every parameter."""
    L = len(widths)
    grads = {}
    h = cache["head_in"]
    grads["head.w"] = np.einsum("zyx,zyxc->c", dout, h)[None, None, :]
    grads["head.b"] = np.array([dout.sum()])
    dh = dout[..., None] * params["head.w"][0, 0][None, None, None, :]
    dskip = [None] * L
    # decoder, from level 0 upward (reverse of the forward order)
    for l in range(0, L - 1):
        dh, grads[f"dec{l}b.w"], grads[f"dec{l}b.b"] = _relu_conv_backward(params, cache, f"dec{l}b", dh)
        dh, grads[f"dec{l}a.w"], grads[f"dec{l}a.b"] = _relu_conv_backward(params, cache, f"dec{l}a", dh)
        c = widths[l]
        dskip[l] = dh[..., :c]
        du = dh[..., c:]
        dh, grads[f"up{l}.w"], grads[f"up{l}.b"] = up2_backward(cache[f"up{l}_in"], params[f"up{l}.w"], du)
    # encoder, from the bottom level upward
    for l in range(L - 1, -1, -1):
        if dskip[l] is not None:
            dh = dh + dskip[l]
        dh, grads[f"enc{l}b.w"], grads[f"enc{l}b.b"] = _relu_conv_backward(params, cache, f"enc{l}b", dh)
        dh, grads[f"enc{l}a.w"], grads[f"enc{l}a.b"] = _relu_conv_backward(params, cache, f"enc{l}a", dh)
        if l > 0:
            dh = maxpool2_backward(dh, cache[f"pool{l}"])
    return grads


def mse_loss(pred: np.ndarray, target: np.ndarray) -> Tuple[float, np.ndarray]:
    """mean((pred - target)^2) and its gradient with respect to pred."""
    diff = pred - target
    return float(np.mean(diff * diff)), 2.0 * diff / diff.size


def adam_step(w, g, m, v, t: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments, step t >= 1); returns new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
