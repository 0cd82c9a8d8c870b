"""The synthetic inputs, on the CPU: each seeded generator against the recipe it states (media
ranges and normalisation, layer structure, unit-mass sources, uneven cuts), and the named
workloads against their stated geometry (grid, partition, overlap, PML, points per wavelength,
right-hand-side counts)."""
import math

import numpy as np
import pytest

from paper_1807_04180_gb300 import workloads as W


@pytest.mark.parametrize("n,parts,jitter,seed", [(2048, 32, 8, 3), (2048, 32, 8, 4), (512, 8, 8, 3), (100, 7, 3, 1)])
def test_uneven_cuts(n, parts, jitter, seed):
    cuts = W.uneven_cuts(n, parts, seed, jitter)
    w = np.diff(cuts)
    base = n // parts
    assert cuts[0] == 0 and cuts[-1] == n and len(cuts) == parts + 1
    assert w.min() >= max(1, base - jitter) and w.max() <= base + jitter + 1
    assert np.array_equal(cuts, W.uneven_cuts(n, parts, seed, jitter))        # seeded


def test_gaussian_sum_medium_range_and_band():
    n, h, e = 64, 1.0 / 64, 5
    c = W.gaussian_sum_medium((n, n), h, e, seed=2)
    assert c.shape == (n + 2 * e, n + 2 * e)
    inner = c[e:-e, e:-e]
    assert inner.min() == pytest.approx(1.5) and inner.max() == pytest.approx(4.5)   # normalised to [cmin, cmax]
    assert np.array_equal(c[:e, e:-e], np.repeat(inner[:1], e, axis=0))             # band: nearest interior value
    assert np.array_equal(c[e:-e, -e:], np.repeat(inner[:, -1:], e, axis=1))
    assert np.array_equal(c, W.gaussian_sum_medium((n, n), h, e, seed=2))
    assert not np.array_equal(c, W.gaussian_sum_medium((n, n), h, e, seed=3))


def test_layered_medium_layers():
    n, h, e = 128, 1.0 / 128, 4
    c = W.layered_medium((n, n), h, e, seed=3)
    inner = c[e:-e, e:-e]
    vals = np.unique(inner)
    assert len(vals) <= 6 and vals.min() >= 1.5 and vals.max() <= 4.5
    # interfaces are separated by L/6 - 2 x 0.05 L > 0, so along depth (first axis) every
    # column passes the layers in order: the speed changes at most 5 times down a column
    for j in range(0, n, 7):
        col = inner[:, j]
        assert np.count_nonzero(np.diff(col)) <= 5


def test_point_sources_unit_mass_in_the_interior():
    n, h, e = 40, 1.0 / 40, 6
    f = W.random_point_sources((n, n), h, e, count=9, seed=5)
    assert f.shape == (9, n + 2 * e, n + 2 * e)
    for r in range(9):
        assert np.count_nonzero(f[r]) == 1
        assert f[r].sum() * h ** 2 == pytest.approx(1.0)
        (i, j), = np.argwhere(f[r] != 0)
        # positions ~ U[0.05, 0.95] L, so the node is inside the interior (not the band)
        assert e <= i < e + n and e <= j < e + n


def test_gaussian_source_unit_mass():
    n, h, e = 128, 1.0 / 128, 3
    f = W.gaussian_source((n, n), h, e, (0.5, 0.45), 4 * h)
    assert f.real.sum() * h ** 2 == pytest.approx(1.0, rel=1e-6)
    assert np.all(f[:e] == 0) and np.all(f[:, -e:] == 0)


def test_named_workloads_geometry():
    wl = W.heterogeneous_2d()
    assert wl.n == (1024, 1024) and wl.parts == (16, 16) and wl.ov == 2 and wl.npml == 10
    assert wl.c.shape == (1048, 1048) and wl.nrhs == 1
    assert np.all(np.diff(wl.cuts[0]) == 64)
    c_min = wl.c.min()
    assert c_min == pytest.approx(1.5)
    assert 2 * math.pi * c_min / wl.omega == pytest.approx(10 * wl.h)        # 10 points per wavelength at c_min
    wb = W.layered_2d_batched()
    assert wb.n == (2048, 2048) and wb.parts == (32, 32) and wb.nrhs == 64 and wb.c.shape == (2072, 2072)
    for cuts in wb.cuts:
        w = np.diff(cuts)
        assert w.sum() == 2048 and w.min() >= 56 and w.max() <= 73
    assert 2 * math.pi * 1.5 / wb.omega == pytest.approx(10 * wb.h)
    w3 = W.constant_3d(n=48, parts=2)
    assert w3.dim == 3 and w3.ov == 1 and w3.npml == 6 and w3.c.shape == (62, 62, 62)
    assert w3.f.real.sum() * w3.h ** 3 == pytest.approx(1.0, rel=1e-3)       # unit-mass Gaussian
