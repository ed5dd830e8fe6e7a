"""Learned warm start for block 3MG: training pairs made by the method itself, the
U-Net trained on them with the library's tensor-core kernels, and 3MG started
from the network's prediction (with plain 3MG as fallback).

Pipeline (all numerics in libbd3mg.so; this module only orchestrates):
  1. crops: independent volumes of the mixed-precision recipe (PSF 9x9x7,
     sigma_xy(z) of the 0.5 -> 3.0 ramp over 128 slices evaluated at a random
     depth offset z0, noise 0.01, texture 0.05, the recipe's ellipsoid density);
  2. targets: each crop's observation y solved by plain 3MG (batched contexts,
     a fixed number of iterations) -> pairs (y, x_3mg);
  3. training: inputs [y, sigma_xy(z)], residual output x_hat = y + net(...),
     MSE against x_3mg, Adam, mini-batches of crops;
  4. solve: x_hat from the network, checked against y by the objective (the
     start with the lower f is used: plain 3MG remains the fallback), then 3MG.
"""
from __future__ import annotations

import time
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import binding, synth, unet_binding

C2_DEPTH = 128                       # depth of the ramp's reference volume
C2_SXY = (0.5, 3.0)


def ramp(z0: int, nz: int, depth: int = C2_DEPTH) -> Tuple[float, float]:
    """sigma_xy at the first and last slice of a crop starting at depth z0 of the ramp
    0.5 -> 3.0 over `depth` slices (the 512x512x128 recipe's ramp for depth 128)."""
    lo, hi = C2_SXY
    s = lambda z: lo + (hi - lo) * z / (depth - 1)
    return s(z0), s(z0 + nz - 1)


def crop_params(k: int, shape=(48, 128, 128), seed: int = 0, source_shape=None, n_sources: int = 0):
    """Where crop k of the training set comes from: (source volume, z0, y0, x0, sigma ramp).

    With source volumes (source_shape given) the crop is a window of one of n_sources
    phantoms of that shape; otherwise it is an independent volume of the crop's own shape
    (source -1, offsets 0).  z0 is the crop's depth offset on the ramp."""
    nz, ny, nx = shape
    rng = np.random.default_rng([seed, 31, k])
    depth = source_shape[0] if source_shape is not None else C2_DEPTH
    z0 = int(rng.integers(0, depth - nz + 1)) if nz < depth else 0
    if source_shape is None:
        return -1, z0, 0, 0, ramp(z0, nz, depth)
    src = int(rng.integers(0, n_sources))
    y0 = int(rng.integers(0, source_shape[1] - ny + 1))
    x0 = int(rng.integers(0, source_shape[2] - nx + 1))
    return src, z0, y0, x0, ramp(z0, nz, depth)


def make_crops(count: int, shape=(48, 128, 128), seed: int = 0, source_shape=(128, 512, 512),
               source_ellipsoids: int = 800, n_sources: int = 4, noise: float = 0.01, texture: float = 0.05):
    """Observations of `count` crops as a CUDA float32 tensor [count, D, H, W] and their sigma
    ramps [count, 2].

    Phantoms: n_sources volumes of source_shape with source_ellipsoids ellipsoids each
    (synth.phantom on the host, seeds distinct from the evaluation volume's), crops taken at
    random windows; with source_shape None every crop is an independent phantom of its own
    shape at the same ellipsoid density.  Each crop is then blurred by the library's own
    depth-variant H for its ramp (one context per distinct ramp) and gets seeded Gaussian
    noise from a CUDA generator."""
    import torch
    nz, ny, nx = shape
    ys = torch.empty((count,) + tuple(shape), dtype=torch.float32, device="cuda")
    ramps = np.empty((count, 2))
    sources = []
    if source_shape is not None:
        for s in range(n_sources):
            ph = synth.phantom(tuple(source_shape), source_ellipsoids, 1000 + 7 * seed + s, texture)
            sources.append(torch.from_numpy(ph.astype(np.float32)).cuda())
    n_ell = max(2, int(round(800 * nz * ny * nx / (128 * 512 * 512))))
    ctxs = {}
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed * 7919 + 13)
    zeros = torch.zeros(tuple(shape), dtype=torch.float32, device="cuda")
    try:
        for k in range(count):
            src, z0, y0, x0, sxy = crop_params(k, shape, seed, source_shape, n_sources)
            ramps[k] = sxy
            if z0 not in ctxs:
                ctxs[z0] = binding.Solver(shape, psf_of(shape, sxy), zeros)
            if src >= 0:
                xt = sources[src][z0:z0 + nz, y0:y0 + ny, x0:x0 + nx].contiguous()
            else:
                xt = torch.from_numpy(synth.phantom(shape, n_ell, seed * 100003 + 17 * k + 5, texture)
                                      .astype(np.float32)).cuda()
            ys[k] = ctxs[z0].apply_H(xt) + noise * torch.randn(tuple(shape), generator=gen, device="cuda")
    finally:
        for c in ctxs.values():
            c.close()
    torch.cuda.synchronize()
    return ys, ramps


def crop_problem(y_dev, sxy, lam=1e-2, delta=1e-2, eta=1.0) -> synth.Problem:
    """The restoration problem of one crop (y copied to the host)."""
    y = y_dev.detach().cpu().numpy().astype(np.float32)
    return synth.Problem(name="crop", shape=tuple(y.shape), psf=psf_of(y.shape, sxy), y=y, x_true=None, lam=lam,
                         delta=delta, eta=eta, xmin=0.0, xmax=1.0, slabs=None, meta={"sxy": tuple(sxy)})


def psf_of(shape, sxy) -> np.ndarray:
    nz = shape[0]
    fx, fy, fz = synth.gaussian_factors(nz, 9, 9, 7, sxy[0], sxy[1], 1.0)
    return synth.dense_psf(fx, fy, fz)


def solve_targets(ys_dev, ramps, iters: int = 100, chunk: int = 32, lam=1e-2, delta=1e-2, eta=1.0):
    """x_3mg of every crop: plain 3MG from y, `iters` lockstep iterations per batch of `chunk`
    volumes.  ys_dev: CUDA [count, D, H, W]; returns a CUDA float32 tensor of the same shape."""
    import torch
    count = ys_dev.shape[0]
    out = torch.empty_like(ys_dev)
    for c0 in range(0, count, chunk):
        probs = [crop_problem(ys_dev[k], ramps[k], lam, delta, eta) for k in range(c0, min(count, c0 + chunk))]
        with binding.BatchSolver(probs) as bs:
            bs.iterate(iters, trace=False)
            for j in range(len(probs)):
                bs.get(j, 0, out[c0 + j])
    torch.cuda.synchronize()
    return out


def net_input(y, sxy: Sequence[float]):
    """[D, H, W, 2] float32 CUDA input: y and the per-depth blur width sigma_xy(z)."""
    import torch
    D = y.shape[0]
    s = torch.linspace(float(sxy[0]), float(sxy[1]), D, device=y.device, dtype=torch.float32)
    return torch.stack([y, s.view(D, 1, 1).expand_as(y)], dim=-1).contiguous()


def train(net: unet_binding.UNet, ys_dev, ramps, targets, train_idx: Sequence[int], epochs: int = 1,
          batch: int = 4, seed: int = 0, time_budget_s: Optional[float] = None, log=None):
    """Adam over mini-batches of crops; returns the per-step loss list."""
    import torch
    rng = np.random.default_rng([seed, 41])
    losses = []
    t0 = time.perf_counter()
    idx = np.asarray(train_idx)
    for ep in range(epochs):
        order = rng.permutation(idx)
        for b0 in range(0, len(order) - batch + 1, batch):
            sel = order[b0:b0 + batch]
            inp = torch.stack([net_input(ys_dev[k], ramps[k]) for k in sel])
            base = ys_dev[sel]
            tgt = targets[sel]
            losses.append(net.train_step(inp, base, tgt, want_loss=True))
            if time_budget_s is not None and time.perf_counter() - t0 > time_budget_s:
                return losses
        if log:
            log(f"epoch {ep}: loss {np.mean(losses[-max(1, len(order) // batch):]):.4g}")
    return losses


def predict(net: unet_binding.UNet, y_dev, sxy):
    """x_hat = y + net([y, sigma_xy]) for one volume (CUDA [D, H, W])."""
    inp = net_input(y_dev, sxy)[None]
    return net.forward(inp, y_dev[None])[0]


def choose_start(prob: synth.Problem, x_hat) -> Tuple[object, float, float]:
    """The start with the lower objective: (start, f(x_hat), f(y)).  Plain 3MG's start y is the
    fallback whenever the network does not improve on it."""
    import torch
    y = torch.from_numpy(prob.y).cuda()
    with binding.Solver.from_problem(prob, slabs=None) as s:
        fy = s.objective()
        s.set_x(x_hat)
        fx = s.objective()
    return (x_hat if fx < fy else y), fx, fy
