"""Seeded synthetic inputs for the depth-variant deblurring problem (Section 3.1).

This module makes INPUTS only: ellipsoid phantoms, per-depth Gaussian PSFs, the
degraded observation y = H x_bar + b (Eq. "model"), start points and slab
partitions.  It holds none of the 3MG arithmetic (no objective, gradient,
majorant or subspace solve).  Both the FP64 oracle and the CUDA library consume
exactly the arrays returned here (y and the PSF are rounded to float32 once, so
both sides read identical values).

The paper's own volumes (FlyBrain, Aneurysm) are not available; the phantoms
below stand in for them with the shapes and value ranges of the workloads the
library is measured on.  The forward model used to synthesise y calls
scipy.ndimage.convolve1d (a library routine) with the separable Gaussian
factors; it is data synthesis, not part of either implementation.

Array layout everywhere: C order [nz][ny][nx] (x fastest), PSF [nz][pz][py][px]
with tap offset a in [-r, r] stored at index a + r, applied as a convolution
(Hx)(i,j,z) = sum_{a,b,c} h_z(a,b,c) x(i-a, j-b, z-c), zero outside the volume,
using the PSF of the OUTPUT depth z.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclass
class Problem:
    """One restoration problem: observation, PSF and penalty parameters."""
    name: str
    shape: Tuple[int, int, int]          # (nz, ny, nx)
    psf: np.ndarray                      # float32 [nz, pz, py, px]
    y: np.ndarray                        # float32 [nz, ny, nx]
    x_true: np.ndarray                   # float32 [nz, ny, nx]
    lam: float = 1e-2
    delta: float = 1e-2
    eta: float = 1.0
    xmin: float = 0.0
    xmax: float = 1.0
    slabs: Optional[List[int]] = None    # slab boundaries z_0=0 < ... < z_S=nz
    meta: dict = field(default_factory=dict)
    penalty: int = 0                     # 0 per-axis; 1 joint X-Y + kappa ||V^Z x||^2; 2 isotropic X, Y, Z
    kappa: float = 0.0

    @property
    def n(self) -> int:
        nz, ny, nx = self.shape
        return nz * ny * nx


def phantom(shape, n_ellipsoids: int, seed: int, texture_sigma: float = 0.0) -> np.ndarray:
    """Sum of axis-aligned ellipsoids with intensities U[0,1] (float64).

    Centres are uniform over the volume, semi-axes U[0.05, 0.25] x (extent of
    the axis), intensities U[0,1]; overlapping ellipsoids add.  An optional
    i.i.d. N(0, texture_sigma^2) texture is added everywhere.
    """
    nz, ny, nx = shape
    dims = np.array([nz, ny, nx], dtype=np.float64)
    rng = np.random.default_rng([seed, 0])
    centres = rng.uniform(0.0, 1.0, size=(n_ellipsoids, 3)) * dims
    semi = rng.uniform(0.05, 0.25, size=(n_ellipsoids, 3)) * dims
    semi = np.maximum(semi, 0.5)
    inten = rng.uniform(0.0, 1.0, size=n_ellipsoids)
    vol = np.zeros(shape, dtype=np.float64)
    for e in range(n_ellipsoids):
        sl = []
        d2 = []
        for ax in range(3):
            lo = max(0, int(np.floor(centres[e, ax] - semi[e, ax])))
            hi = min(int(dims[ax]), int(np.ceil(centres[e, ax] + semi[e, ax])) + 1)
            if hi <= lo:
                break
            coords = np.arange(lo, hi, dtype=np.float64)
            sl.append(slice(lo, hi))
            d2.append(((coords - centres[e, ax]) / semi[e, ax]) ** 2)
        if len(sl) < 3:
            continue
        inside = (d2[0][:, None, None] + d2[1][None, :, None] + d2[2][None, None, :]) <= 1.0
        vol[sl[0], sl[1], sl[2]] += inten[e] * inside
    if texture_sigma > 0.0:
        trng = np.random.default_rng([seed, 2])
        vol += trng.normal(0.0, texture_sigma, size=shape)
    return vol


def gaussian_factors(nz: int, px: int, py: int, pz: int, sxy_lo: float, sxy_hi: float,
                     sz: float = 1.0):
    """Per-depth 1D Gaussian factors, each normalised to sum 1 (float64).

    sigma_xy(z) rises linearly from sxy_lo at z=0 to sxy_hi at z=nz-1; sigma_z
    is constant.  Returns (fx [nz,px], fy [nz,py], fz [nz,pz]).
    """
    def g1(p, s):
        r = (p - 1) // 2
        a = np.arange(-r, r + 1, dtype=np.float64)
        if s <= 0:
            v = (a == 0).astype(np.float64)
        else:
            v = np.exp(-0.5 * (a / s) ** 2)
        return v / v.sum()

    fx = np.zeros((nz, px))
    fy = np.zeros((nz, py))
    fz = np.zeros((nz, pz))
    for z in range(nz):
        s = sxy_lo if nz == 1 else sxy_lo + (sxy_hi - sxy_lo) * z / (nz - 1)
        fx[z] = g1(px, s)
        fy[z] = g1(py, s)
        fz[z] = g1(pz, sz)
    return fx, fy, fz


def dense_psf(fx: np.ndarray, fy: np.ndarray, fz: np.ndarray) -> np.ndarray:
    """Outer product per depth -> float32 [nz, pz, py, px]."""
    h = fz[:, :, None, None] * fy[:, None, :, None] * fx[:, None, None, :]
    return h.astype(np.float32)


def blur_separable(x: np.ndarray, fx: np.ndarray, fy: np.ndarray, fz: np.ndarray) -> np.ndarray:
    """Depth-variant blur with separable per-output-depth factors (float64).

    Used only to synthesise observations; calls scipy.ndimage.convolve1d.
    """
    from scipy.ndimage import convolve1d

    nz = x.shape[0]
    pz = fz.shape[1]
    rz = (pz - 1) // 2
    out = np.empty_like(x, dtype=np.float64)
    for z in range(nz):
        w = np.zeros(x.shape[1:], dtype=np.float64)
        for ci in range(pz):
            c = ci - rz
            zs = z - c
            if 0 <= zs < nz:
                w += fz[z, ci] * x[zs]
        w = convolve1d(w, fy[z], axis=0, mode="constant", cval=0.0)
        w = convolve1d(w, fx[z], axis=1, mode="constant", cval=0.0)
        out[z] = w
    return out


def observe(x_true: np.ndarray, fx, fy, fz, noise_sigma: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng([seed, 1])
    y = blur_separable(x_true, fx, fy, fz)
    if noise_sigma > 0:
        y = y + rng.normal(0.0, noise_sigma, size=y.shape)
    return y.astype(np.float32)


def uniform_start(y: np.ndarray, seed: int) -> np.ndarray:
    """x0 with entries U[0, max(y)] (the paper's initialisation, Section 3.1)."""
    rng = np.random.default_rng([seed, 3])
    return rng.uniform(0.0, float(np.max(y)), size=y.shape).astype(np.float32)


def slab_bounds(thicknesses: Sequence[int]) -> List[int]:
    b = [0]
    for t in thicknesses:
        b.append(b[-1] + int(t))
    return b


def make_problem(name: str, shape, n_ellipsoids: int, psf_shape, sxy, sz: float,
                 noise: float, seed: int, lam=1e-2, delta=1e-2, eta=1.0,
                 xmin=0.0, xmax=1.0, texture: float = 0.0, slabs=None) -> Problem:
    nz, ny, nx = shape
    px, py, pz = psf_shape
    xt = phantom(shape, n_ellipsoids, seed, texture)
    fx, fy, fz = gaussian_factors(nz, px, py, pz, sxy[0], sxy[1], sz)
    y = observe(xt, fx, fy, fz, noise, seed)
    return Problem(name=name, shape=tuple(shape), psf=dense_psf(fx, fy, fz), y=y,
                   x_true=xt.astype(np.float32), lam=lam, delta=delta, eta=eta,
                   xmin=xmin, xmax=xmax, slabs=slabs,
                   meta=dict(n_ellipsoids=n_ellipsoids, psf_shape=tuple(psf_shape), sxy=tuple(sxy),
                             sz=sz, noise=noise, seed=seed, texture=texture))


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
C1_SLABS = [4, 14, 6, 10, 5, 12, 7, 6]


def workload_plain_small(seed: int = 0) -> Problem:
    """64x64x24 volume, 40 ellipsoids, PSF 5x5x5, sigma_xy 0.5->2.0, noise 0.02."""
    return make_problem("plain-64x64x24", (24, 64, 64), 40, (5, 5, 5), (0.5, 2.0), 1.0, 0.02, seed)


def workload_slabs(seed: int = 0, slabs: bool = True) -> Problem:
    """256x256x64 volume, 200 ellipsoids, PSF 7x7x7, sigma_xy 0.5->3.0, 8 slabs."""
    return make_problem("slabs-256x256x64", (64, 256, 256), 200, (7, 7, 7), (0.5, 3.0), 1.0, 0.02,
                        seed, slabs=slab_bounds(C1_SLABS) if slabs else None)


def workload_mixed(seed: int = 0, crop: bool = False) -> Problem:
    """512x512x128 (or the 128x128x32 crop recipe), 800 ellipsoids + texture, PSF 9x9x7."""
    if crop:
        return make_problem("mixed-crop-128x128x32", (32, 128, 128), 800 * 128 * 128 * 32 // (512 * 512 * 128),
                            (9, 9, 7), (0.5, 3.0), 1.0, 0.01, seed, texture=0.05)
    return make_problem("mixed-512x512x128", (128, 512, 512), 800, (9, 9, 7), (0.5, 3.0), 1.0, 0.01,
                        seed, texture=0.05)


def batch_shapes(count: int = 16, seed: int = 0):
    """Uneven volume shapes and per-volume parameters for the batched form."""
    rng = np.random.default_rng([seed, 7])
    out = []
    for _ in range(count):
        nx = int(rng.integers(96, 385))
        ny = int(rng.integers(96, 385))
        nz = int(rng.integers(32, 97))
        lo = float(rng.uniform(0.4, 1.0))
        hi = float(rng.uniform(1.5, 3.0))
        lam = float(np.exp(rng.uniform(np.log(5e-3), np.log(5e-2))))
        out.append(dict(shape=(nz, ny, nx), sxy=(lo, hi), lam=lam))
    return out


def workload_batch(count: int = 16, seed: int = 0, scale: float = 1.0) -> List[Problem]:
    """count volumes of uneven size (96..384)^2 x (32..96), PSF 7x7x7 each with its own ramp.

    scale < 1 shrinks every extent (used for small test batches).
    """
    probs = []
    for k, s in enumerate(batch_shapes(count, seed)):
        nz, ny, nx = s["shape"]
        if scale != 1.0:
            nz, ny, nx = (max(4, int(round(nz * scale))), max(8, int(round(ny * scale))),
                          max(8, int(round(nx * scale))))
        n_ell = max(4, int(round(200 * (nz * ny * nx) / (256 * 256 * 64))))
        probs.append(make_problem(f"batch{k}-{nx}x{ny}x{nz}", (nz, ny, nx), n_ell, (7, 7, 7), s["sxy"],
                                  1.0, 0.02, seed * 1000 + k + 1, lam=s["lam"]))
    return probs


def tiny_problem(shape=(6, 10, 12), psf_shape=(3, 3, 3), sxy=(0.6, 1.2), sz=0.8, noise=0.02,
                 seed=0, n_ellipsoids=4, **kw) -> Problem:
    """Small problem for brute-force checks."""
    return make_problem(f"tiny-{shape}", shape, n_ellipsoids, psf_shape, sxy, sz, noise, seed, **kw)


def rotated_gaussian_psf(nz: int, psf_shape, seed: int, sxy=(0.5, 2.5), sz=(1.0, 3.0)) -> np.ndarray:
    """Depth-variant rotated Gaussian PSF (float32 [nz][pz][py][px]), one per
    output depth: standard deviations sigma_x, sigma_y ~ U[sxy], sigma_z ~ U[sz]
    and an xy rotation theta ~ U[0, pi) drawn per depth, taps sampled at integer
    offsets and normalised to sum 1 in FP64.  Not separable in x and y."""
    px, py, pz = psf_shape
    rng = np.random.default_rng([seed, 7])
    rx, ry, rz = (px - 1) // 2, (py - 1) // 2, (pz - 1) // 2
    c, b, a = np.meshgrid(np.arange(-rz, rz + 1), np.arange(-ry, ry + 1), np.arange(-rx, rx + 1), indexing="ij")
    out = np.zeros((nz, pz, py, px))
    for z in range(nz):
        sx, sy = rng.uniform(*sxy, size=2)
        szz = rng.uniform(*sz)
        th = rng.uniform(0.0, np.pi)
        u = np.cos(th) * a + np.sin(th) * b
        v = -np.sin(th) * a + np.cos(th) * b
        h = np.exp(-0.5 * (u * u / (sx * sx) + v * v / (sy * sy) + c * c / (szz * szz)))
        out[z] = h / h.sum()
    return out.astype(np.float32)


def blur_dense(x: np.ndarray, psf: np.ndarray) -> np.ndarray:
    """H x in FP64 for a dense PSF of the output depth (data synthesis only):
    out[z] = sum_c conv2d(x[z - c], h_z[c]), zero outside the volume."""
    from scipy.ndimage import convolve
    nz = x.shape[0]
    pz = psf.shape[1]
    rz = (pz - 1) // 2
    xd = x.astype(np.float64)
    out = np.zeros_like(xd)
    for z in range(nz):
        for ci in range(pz):
            zs = z - (ci - rz)
            if 0 <= zs < nz:
                out[z] += convolve(xd[zs], psf[z, ci].astype(np.float64), mode="constant", cval=0.0)
    return out


def make_problem_dense(name: str, shape, n_ellipsoids: int, psf: np.ndarray, noise: float, seed: int,
                       lam=1e-2, delta=1e-2, eta=1.0, xmin=0.0, xmax=1.0, slabs=None) -> Problem:
    """A problem whose observation is blurred by a given dense PSF."""
    xt = phantom(shape, n_ellipsoids, seed)
    rng = np.random.default_rng([seed, 1])
    y = blur_dense(xt, psf)
    if noise > 0:
        y = y + rng.normal(0.0, noise, size=y.shape)
    return Problem(name=name, shape=tuple(shape), psf=np.ascontiguousarray(psf, np.float32),
                   y=y.astype(np.float32), x_true=xt.astype(np.float32), lam=lam, delta=delta, eta=eta,
                   xmin=xmin, xmax=xmax, slabs=slabs,
                   meta=dict(n_ellipsoids=n_ellipsoids, psf_shape=tuple(psf.shape[1:][::-1]), noise=noise,
                             seed=seed, psf="rotated Gaussian per depth"))


def workload_rotated_256x256x24(seed: int = 0, slabs=None) -> Problem:
    """The shape of the paper's comparison experiment (Section 3.2): 256x256x24
    volume, depth-variant rotated Gaussian PSF of 11x11x21 taps, noise 0.04; a
    phantom of 200 ellipsoids per 256x256x64 (75 here) stands in for FlyBrain."""
    psf = rotated_gaussian_psf(24, (11, 11, 21), seed, sxy=(0.5, 2.5), sz=(1.0, 4.0))
    return make_problem_dense("rotated-256x256x24", (24, 256, 256), 75, psf, 0.04, seed, slabs=slabs)


def workload_rotated_155x154x79(seed: int = 0, slabs=None) -> Problem:
    """The shape of the paper's scaling experiment (Section 3.3): 155x154x79
    volume (x, y, z), depth-variant rotated Gaussian PSF of 5x5x11 taps, noise
    0.04; a phantom of 90 ellipsoids stands in for Aneurysm."""
    psf = rotated_gaussian_psf(79, (5, 5, 11), seed, sxy=(0.4, 1.2), sz=(1.0, 2.5))
    return make_problem_dense("rotated-155x154x79", (79, 154, 155), 90, psf, 0.04, seed, slabs=slabs)


def random_psf(nz: int, psf_shape, seed: int) -> np.ndarray:
    """A non-separable, non-symmetric positive PSF per depth (float32), each summing to 1."""
    px, py, pz = psf_shape
    rng = np.random.default_rng([seed, 5])
    h = rng.uniform(0.0, 1.0, size=(nz, pz, py, px))
    h /= h.sum(axis=(1, 2, 3), keepdims=True)
    return h.astype(np.float32)
