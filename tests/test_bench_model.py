"""The bench's byte model and bookkeeping, on the CPU.

The roofline the bench reports divides algorithmic bytes by measured time, so
the byte model is pinned here by hand counts: a plain FP32 iteration moves
80 B per voxel (objective 8, gradient 12, curvature 20, update 40), and the
8-slab 256x256x64 workload's zones (each slab widened by the PSF's z radius 3)
cover 106 of the 64 slices' worth of planes, which puts one curvature launch
at 35.30 MB on average over the three colours.  The launch count of the exact
refreshes and the SNR formula are pinned as well.
"""
import os
import sys
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _prob(shape):
    nz, ny, nx = shape
    return SimpleNamespace(shape=shape, n=nz * ny * nx)


def test_plain_iteration_moves_80_bytes_per_voxel():
    p = _prob((128, 512, 512))
    b = bench.algorithmic_bytes(p, None, 3)
    per_voxel = {k: v / p.n for k, v in b.items()}
    assert per_voxel == {"objective": 8.0, "residual": 0.0, "gradient": 12.0, "curvature": 20.0, "update": 40.0,
                         "dense": 0.0}
    assert sum(per_voxel.values()) == 80.0
    bf = bench.algorithmic_bytes(p, None, 3, g_bytes=2)
    assert bf["gradient"] / p.n == 10.0 and bf["curvature"] / p.n == 18.0 and bf["update"] / p.n == 38.0


def test_fused_iteration_moves_64_bytes_per_voxel():
    """Two passes: gradient reads x, g, d, r, H g, H d and writes x, d, r, H d, g;
    curvature reads g, d, x, H d and writes H g."""
    p = _prob((128, 512, 512))
    b = bench.algorithmic_bytes(p, None, 4, fused=True)
    per_voxel = {k: v / p.n for k, v in b.items()}
    assert per_voxel == {"objective": 0.0, "residual": 0.0, "gradient": 44.0, "curvature": 20.0, "update": 0.0,
                         "dense": 0.0}
    bf = bench.algorithmic_bytes(p, None, 4, g_bytes=2, fused=True)
    assert bf["gradient"] / p.n == 40.0 and bf["curvature"] / p.n == 18.0


def test_block_workload_zones_and_curvature_bytes():
    p = _prob((64, 256, 256))
    bounds = [0, 4, 18, 24, 34, 39, 51, 58, 64]
    # zone of each slab: [z0 - 3, z1 + 3) clipped to [0, 64)
    zone_slices = [7, 20, 12, 16, 11, 18, 13, 9]
    assert sum(zone_slices) == 106
    b = bench.algorithmic_bytes(p, bounds, 3)
    plane = 256 * 256
    assert b["curvature"] == 12.0 * p.n + 8.0 * 106 * plane
    assert b["update"] == 20.0 * p.n + 20.0 * 106 * plane
    # the three colour launches of a sweep share the curvature bytes
    assert abs(b["curvature"] / 3 - 35302058.67) < 1.0


def test_refresh_launches():
    assert bench.refresh_launches(0, 1) == 2          # before iteration 0
    assert bench.refresh_launches(0, 256) == 2
    assert bench.refresh_launches(0, 257) == 4        # and before iteration 256
    assert bench.refresh_launches(5, 30) == 0
    assert bench.refresh_launches(250, 10) == 2


def test_snr_db():
    ref = np.random.default_rng(0).uniform(0.5, 1.5, size=(4, 5, 6))
    assert abs(bench.snr_db(0.9 * ref, ref) - 20.0) < 1e-12      # ||ref||^2 / ||0.1 ref||^2 = 100
    assert abs(bench.snr_db(np.zeros_like(ref), ref)) < 1e-12


def test_dense_tap_count():
    """Valid taps of one dense-PSF iteration, by brute force on a tiny shape."""
    shape, psf = (5, 4, 6), (3, 3, 5)
    nz, ny, nx = shape
    px, py, pz = psf

    def valid(n, p, lo, hi, outs):
        r = (p - 1) // 2
        return sum(1 for o in outs for a in range(-r, r + 1) if lo <= o - a < hi)
    xy = valid(nx, px, 0, nx, range(nx)) * valid(ny, py, 0, ny, range(ny))
    want = xy * valid(nz, pz, 0, nz, range(nz))
    bounds = [0, 2, 5]
    for z0, z1 in zip(bounds[:-1], bounds[1:]):
        want += xy * valid(nz, pz, z0, z1, range(max(0, z0 - 2), min(nz, z1 + 2)))
    assert bench.dense_taps(shape, psf, bounds) == want
    assert bench.fp32_fma_peak(2070.0) == 152 * 128 * 2 * 2070e6 / 1e12
