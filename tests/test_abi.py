"""CPU checks of the C ABI: the library loads, exports every symbol the header
declares, and its host-only planning helpers behave (no GPU calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2002_02328_gb300 import binding, build, synth, unet_binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bd3mg_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(binding.EXPORTED) | set(unet_binding.EXPORTED)


def test_status_strings(lib):
    assert lib.bd3mg_status_string(0) == b"ok"
    assert b"unsupported" in lib.bd3mg_status_string(7)


def test_params_default(lib):
    p = binding.Params()
    p.penalty, p.kappa, p.barrier_timeout_ms = 7, 3.5, 9   # the defaults must reach the struct's last fields
    p.psf_mode, p.persistent = 3, 5
    lib.bd3mg_params_default(ctypes.byref(p))
    assert p.psf_mode == binding.PSF_AUTO and p.persistent == 0
    assert p.lambda_ == 1e-2 and p.delta == 1e-2 and p.eta == 1.0 and p.xmax == 1.0 and p.nslabs == 1
    assert p.penalty == binding.PENALTY_PER_AXIS and p.kappa == 0.0
    assert p.refresh_every == 0 and p.barrier_timeout_ms == 0      # library defaults: 256 iterations, 2 s


def test_slab_colouring_of_the_8_slab_workload(lib):
    bounds = synth.slab_bounds(synth.C1_SLABS)          # [0,4,18,24,34,39,51,58,64]
    col, nc = binding.bd3mg_plan_slab_colours(bounds, 7)
    # gap needed: 6 slices.  Slabs 0,2,4,6 / 1,3,7 / 5 (slab 5 is only 5 slices after slab 3).
    np.testing.assert_array_equal(col, [0, 1, 0, 1, 0, 2, 0, 1])
    assert nc == 3


def test_slab_colouring_rules(lib):
    col, nc = binding.bd3mg_plan_slab_colours([0, 2, 5, 6, 10], 1)     # no z blur: gap 1
    np.testing.assert_array_equal(col, [0, 1, 0, 1])
    col, nc = binding.bd3mg_plan_slab_colours([0, 10], 9)
    assert nc == 1 and col[0] == 0
    # any two slabs of one colour are >= max(pz-1,1) apart
    rng = np.random.default_rng(0)
    for _ in range(50):
        t = rng.integers(1, 8, size=rng.integers(2, 12))
        b = list(np.concatenate([[0], np.cumsum(t)]))
        pz = int(rng.choice([1, 3, 5, 7, 9]))
        col, nc = binding.bd3mg_plan_slab_colours(b, pz)
        for s in range(len(t)):
            for s2 in range(s + 1, len(t)):
                if col[s] == col[s2]:
                    assert b[s2] - b[s + 1] >= max(pz - 1, 1)
    with pytest.raises(binding.Bd3mgError):
        binding.bd3mg_plan_slab_colours([0, 3, 3, 5], 3)


def test_same_colour_zones_are_disjoint(lib):
    """The update adds H D u to r over each slab's zone [z0 - max(rz, 1), z1 + rz)
    for all slabs of a colour in one launch: the colouring must make those zones
    disjoint (one writer per voxel of r), for every slab layout and PSF depth."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        t = rng.integers(1, 10, size=rng.integers(2, 14))
        b = list(np.concatenate([[0], np.cumsum(t)]))
        nz = b[-1]
        pz = int(rng.choice([1, 3, 5, 7, 9, 11]))
        rz = (pz - 1) // 2
        col, nc = binding.bd3mg_plan_slab_colours(b, pz)
        for c in range(nc):
            cover = np.zeros(nz, np.int64)
            for s in np.nonzero(col == c)[0]:
                cover[max(0, b[s] - max(rz, 1)):min(nz, b[s + 1] + rz)] += 1
            assert cover.max() <= 1, (b, pz, col)


def test_psf_factoring(lib):
    fx, fy, fz = synth.gaussian_factors(6, 7, 5, 3, 0.5, 3.0, 1.0)
    psf = synth.dense_psf(fx, fy, fz)
    gx, gy, gz, res = binding.bd3mg_factor_psf(psf)
    assert res <= 1e-6
    rebuilt = gz[:, :, None, None].astype(np.float64) * gy[:, None, :, None] * gx[:, None, None, :]
    np.testing.assert_allclose(rebuilt, psf, rtol=0, atol=1e-6 * psf.max())
    with pytest.raises(binding.Bd3mgError):
        binding.bd3mg_factor_psf(synth.random_psf(3, (3, 3, 3), seed=0))
