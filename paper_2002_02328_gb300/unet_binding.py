"""Thin ctypes binding of the learned warm start's C ABI (include/bd3mg_unet.h).

Argument marshalling only: the network's forward pass, loss, backward pass and
Adam run in `libbd3mg.so` (tcgen05 BF16 kernels).  There is no CPU fallback:
the library must be built.  PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import binding

EXPORTED = ["bd3mg_unet_create", "bd3mg_unet_param_count", "bd3mg_unet_set_params", "bd3mg_unet_get_params",
            "bd3mg_unet_get_grads", "bd3mg_unet_forward", "bd3mg_unet_loss_grad", "bd3mg_unet_train_step",
            "bd3mg_unet_conv3", "bd3mg_unet_conv3_wgrad", "bd3mg_unet_up", "bd3mg_unet_error_string",
            "bd3mg_unet_destroy", "bd3mg_unet_set_tma_conv"]

_bound = False


class UnetParams(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("widths", ctypes.c_int * 8), ("cin", ctypes.c_int),
                ("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


def load():
    """The library with the U-Net signatures bound."""
    global _bound
    lib = binding.load()
    if _bound:
        return lib
    vp, ip, dp, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "bd3mg_unet_create": (ip, [ctypes.POINTER(UnetParams), vp, ctypes.POINTER(vp)]),
        "bd3mg_unet_param_count": (ll, [vp]),
        "bd3mg_unet_set_params": (ip, [vp, vp]),
        "bd3mg_unet_get_params": (ip, [vp, vp]),
        "bd3mg_unet_get_grads": (ip, [vp, vp]),
        "bd3mg_unet_forward": (ip, [vp, ip, ip, ip, ip, vp, vp, vp]),
        "bd3mg_unet_loss_grad": (ip, [vp, ip, ip, ip, ip, vp, vp, vp, vp]),
        "bd3mg_unet_train_step": (ip, [vp, ip, ip, ip, ip, vp, vp, vp, vp]),
        "bd3mg_unet_conv3": (ip, [ip, ip, ip, ip, vp, ip, ip, vp, ip, vp, ip, vp, ip, vp, ip, vp]),
        "bd3mg_unet_conv3_wgrad": (ip, [ip, ip, ip, ip, vp, ip, ip, vp, ip, ip, vp, vp]),
        "bd3mg_unet_up": (ip, [ip, ip, ip, ip, vp, ip, ip, vp, ip, vp, vp, ip, vp]),
        "bd3mg_unet_error_string": (ctypes.c_char_p, [vp]),
        "bd3mg_unet_destroy": (None, [vp]),
        "bd3mg_unet_set_tma_conv": (ip, [ip]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _bound = True
    return lib


def _p(t):
    return ctypes.c_void_p(int(t.data_ptr())) if t is not None else None


def _stream():
    import torch
    return ctypes.c_void_p(int(torch.cuda.current_stream().cuda_stream))


def _ok(st: int, what: str):
    if st != 0:
        raise binding.Bd3mgError(st, what)


def layer_shapes(widths: Sequence[int] = (16, 32, 64, 128), cin: int = 2) -> List[Tuple[str, tuple, tuple]]:
    """(name, weight shape, bias shape) in the flat-parameter order of the C ABI."""
    c = list(widths)
    out, prev = [], cin
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


def flatten(params: Dict[str, np.ndarray], widths, cin) -> np.ndarray:
    parts = []
    for name, ws, bs in layer_shapes(widths, cin):
        parts += [np.asarray(params[f"{name}.w"], np.float64).reshape(-1),
                  np.asarray(params[f"{name}.b"], np.float64).reshape(-1)]
    return np.concatenate(parts).astype(np.float32)


def unflatten(flat: np.ndarray, widths, cin) -> Dict[str, np.ndarray]:
    out, off = {}, 0
    for name, ws, bs in layer_shapes(widths, cin):
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out[f"{name}.w"] = flat[off:off + nw].reshape(ws)
        off += nw
        out[f"{name}.b"] = flat[off:off + nb].reshape(bs)
        off += nb
    return out


def he_init(widths=(16, 32, 64, 128), cin: int = 2, seed: int = 0) -> Dict[str, np.ndarray]:
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, from a seeded numpy generator."""
    rng = np.random.default_rng([seed, 11])
    p = {}
    for name, ws, bs in layer_shapes(widths, cin):
        fan_in = ws[0] * ws[2] if name != "head" else ws[2]
        if name.startswith("up"):
            fan_in = ws[2]
        std = np.sqrt(2.0 / fan_in) if name != "head" else np.sqrt(1.0 / fan_in) * 0.1
        p[f"{name}.w"] = rng.normal(0.0, std, size=ws)
        p[f"{name}.b"] = np.zeros(bs)
    return p


class UNet:
    """One network (bd3mg_unet) on the current CUDA device and stream."""

    def __init__(self, widths=(16, 32, 64, 128), cin: int = 2, lr: float = 1e-3):
        self.lib = load()
        self.widths, self.cin = tuple(widths), cin
        prm = UnetParams()
        prm.levels = len(widths)
        for i, w in enumerate(widths):
            prm.widths[i] = w
        prm.cin = cin
        prm.lr = lr
        h = ctypes.c_void_p()
        st = self.lib.bd3mg_unet_create(ctypes.byref(prm), _stream(), ctypes.byref(h))
        if st != 0:
            msg = self.lib.bd3mg_unet_error_string(h).decode() if h.value else str(st)
            if h.value:
                self.lib.bd3mg_unet_destroy(h)
            raise binding.Bd3mgError(st, msg)
        self.h = h
        self.nparam = int(self.lib.bd3mg_unet_param_count(h))

    def _c(self, st):
        if st != 0:
            raise binding.Bd3mgError(st, self.lib.bd3mg_unet_error_string(self.h).decode())

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.bd3mg_unet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, params: Dict[str, np.ndarray]):
        flat = np.ascontiguousarray(flatten(params, self.widths, self.cin))
        assert flat.size == self.nparam
        self._c(self.lib.bd3mg_unet_set_params(self.h, flat.ctypes.data))

    def get_flat(self, grads: bool = False) -> np.ndarray:
        out = np.zeros(self.nparam, np.float32)
        fn = self.lib.bd3mg_unet_get_grads if grads else self.lib.bd3mg_unet_get_params
        self._c(fn(self.h, out.ctypes.data))
        return out

    def params(self) -> Dict[str, np.ndarray]:
        return unflatten(self.get_flat(), self.widths, self.cin)

    def grads(self) -> Dict[str, np.ndarray]:
        return unflatten(self.get_flat(True), self.widths, self.cin)

    def forward(self, inp, base=None, out=None):
        """inp: float32 CUDA [B, D, H, W, cin]; base: [B, D, H, W] or None; returns pred [B, D, H, W]."""
        import torch
        B, D, H, W, _ = inp.shape
        if out is None:
            out = torch.empty((B, D, H, W), device=inp.device, dtype=torch.float32)
        self._c(self.lib.bd3mg_unet_forward(self.h, B, D, H, W, _p(inp.contiguous()),
                                            _p(base.contiguous()) if base is not None else None, _p(out)))
        return out

    def loss_grad(self, inp, base, target) -> float:
        B, D, H, W, _ = inp.shape
        loss = ctypes.c_double()
        self._c(self.lib.bd3mg_unet_loss_grad(self.h, B, D, H, W, _p(inp.contiguous()),
                                              _p(base.contiguous()) if base is not None else None,
                                              _p(target.contiguous()), ctypes.byref(loss)))
        return loss.value

    def train_step(self, inp, base, target, want_loss: bool = True):
        B, D, H, W, _ = inp.shape
        loss = ctypes.c_double()
        self._c(self.lib.bd3mg_unet_train_step(self.h, B, D, H, W, _p(inp.contiguous()),
                                               _p(base.contiguous()) if base is not None else None,
                                               _p(target.contiguous()), ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None


def set_tma_conv(enable: bool) -> bool:
    """Choose the TMA-staged 3x3x3 convolution (True, the default) or the row-gather
    implicit GEMM for every convolution; returns the previous setting."""
    return bool(load().bd3mg_unet_set_tma_conv(int(bool(enable))))


def conv3(x, w, bias=None, relu=False, mask=None, cout=None, out=None):
    """One tensor-core 3x3x3 convolution: x bf16 CUDA [B, D, H, W, cin], w bf16 [27, cout, cin]."""
    import torch
    lib = load()
    B, D, H, W, cin = x.shape
    cout = w.shape[1]
    if out is None:
        out = torch.empty((B, D, H, W, cout), device=x.device, dtype=torch.bfloat16)
    st = lib.bd3mg_unet_conv3(B, D, H, W, _p(x), x.stride(3), cin, _p(w.contiguous()), cout,
                              _p(bias) if bias is not None else None, int(relu),
                              _p(mask) if mask is not None else None, mask.stride(3) if mask is not None else 0,
                              _p(out), out.stride(3), _stream())
    _ok(st, "bd3mg_unet_conv3")
    return out


def conv3_wgrad(x, dz):
    """dW [27, cout, cin] (float32) of a 3x3x3 convolution from its input x and output gradient dz."""
    import torch
    lib = load()
    B, D, H, W, cin = x.shape
    cout = dz.shape[-1]
    dw = torch.empty((27, cout, cin), device=x.device, dtype=torch.float32)
    st = lib.bd3mg_unet_conv3_wgrad(B, D, H, W, _p(x), x.stride(3), cin, _p(dz), dz.stride(3), cout, _p(dw),
                                    _stream())
    _ok(st, "bd3mg_unet_conv3_wgrad")
    return dw


def up(x, w, bias=None):
    """2x2x2 stride-2 transposed convolution: x bf16 [B, D, H, W, cin], w bf16 [8, cout, cin]."""
    import torch
    lib = load()
    B, D, H, W, cin = x.shape
    cout = w.shape[1]
    out = torch.empty((B, 2 * D, 2 * H, 2 * W, cout), device=x.device, dtype=torch.bfloat16)
    st = lib.bd3mg_unet_up(B, D, H, W, _p(x), x.stride(3), cin, _p(w.contiguous()), cout,
                           _p(bias) if bias is not None else None, _p(out), out.stride(3), _stream())
    _ok(st, "bd3mg_unet_up")
    return out
