"""Pins of the oracle's voxelization against facts fixed outside it.

* one atom: each voxel holds the integral of the normal density over the
  voxel, taken here by numerical quadrature of exp(-t^2/2) (no erf);
* mass: the grid sums to the product of normal-CDF differences over the
  support cube (scipy's ndtr, a different routine from erf);
* an integer-voxel translation shifts the grid exactly;
* linearity in atoms and features, clipping at the grid edge;
* the float32 centroid rule on dyadic coordinates equals the exact mean.
"""

import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import fusion_oracle as O


def _q(lo, hi, sigma):
    f = lambda t: math.exp(-0.5 * (t / sigma) ** 2) / (sigma * math.sqrt(2.0 * math.pi))
    return integrate.quad(f, lo, hi, epsabs=1e-15, epsrel=1e-13)[0]


def test_single_atom_at_voxel_centre_matches_quadrature():
    rng = np.random.default_rng(1)
    f = rng.normal(size=19).astype(np.float32)
    origin = np.zeros(3, dtype=np.float32)
    xyz = np.array([[8.5, 8.5, 8.5]], dtype=np.float32)
    G = O.voxelize(xyz, f[None], origin, 16, 1.0, 1.0, 3)
    q = {m: _q(m - 0.5, m + 0.5, 1.0) for m in range(-3, 4)}
    for mz in range(-4, 5):
        for my in range(-4, 5):
            for mx in range(-4, 5):
                v = G[8 + mz, 8 + my, 8 + mx]
                if max(abs(mz), abs(my), abs(mx)) > 3:
                    assert np.all(v == 0.0)
                else:
                    exp = f.astype(np.float64) * q[mz] * q[my] * q[mx]
                    np.testing.assert_allclose(v, exp, rtol=1e-11, atol=1e-15)
    # nothing outside the 7^3 cube
    assert np.count_nonzero(G[..., 0]) == 343


@pytest.mark.parametrize("h,sigma,k", [(0.5, 1.5, 5), (1.0, 0.7, 2), (0.75, 1.0, 4)])
def test_off_centre_atom_general_spacing(h, sigma, k):
    origin = np.array([-3.25, 1.5, 0.125], dtype=np.float32)
    x = np.array([[1.3, 5.71, 4.02]], dtype=np.float32)
    f = np.ones((1, 1), dtype=np.float32)
    n = 20
    G = O.voxelize(x, f, origin, n, h, sigma, k)
    ci = [int(math.floor(float(np.float32(np.float32(x[0, d] - origin[d]) / np.float32(h))))) for d in range(3)]
    d = [float(x[0, i]) - float(origin[i]) for i in range(3)]
    for iz in range(ci[2] - k, ci[2] + k + 1, 2):
        for iy in range(ci[1] - k, ci[1] + k + 1, 3):
            for ix in range(ci[0] - k, ci[0] + k + 1):
                exp = (_q(ix * h - d[0], (ix + 1) * h - d[0], sigma) *
                       _q(iy * h - d[1], (iy + 1) * h - d[1], sigma) *
                       _q(iz * h - d[2], (iz + 1) * h - d[2], sigma))
                np.testing.assert_allclose(G[iz, iy, ix, 0], exp, rtol=1e-10, atol=1e-16)


def test_mass_equals_cdf_product_for_in_grid_supports():
    rng = np.random.default_rng(7)
    n, h, sigma, k = 24, 1.0, 1.0, 3
    origin = np.array([10.0, -5.0, 2.0], dtype=np.float32)
    xyz = (origin + rng.uniform(4.0, 20.0, size=(40, 3))).astype(np.float32)
    feat = rng.normal(size=(40, 19)).astype(np.float32)
    G = O.voxelize(xyz, feat, origin, n, h, sigma, k)
    exp = np.zeros(19)
    for a in range(40):
        p = 1.0
        for d in range(3):
            ci = math.floor(float(np.float32(xyz[a, d] - origin[d])))
            lo = float(origin[d]) + (ci - k) * h
            hi = float(origin[d]) + (ci + k + 1) * h
            p *= stats.norm.cdf((hi - float(xyz[a, d])) / sigma) - stats.norm.cdf((lo - float(xyz[a, d])) / sigma)
        exp += feat[a].astype(np.float64) * p
    np.testing.assert_allclose(G.sum(axis=(0, 1, 2)), exp, rtol=1e-11, atol=1e-11)


def test_integer_voxel_translation_shifts_grid_exactly():
    rng = np.random.default_rng(3)
    n = 20
    origin = np.array([1.0, 2.0, -3.0], dtype=np.float32)
    xyz = (origin + np.round(rng.uniform(5, 11, size=(12, 3)) * 64) / 64).astype(np.float32)
    feat = rng.normal(size=(12, 19)).astype(np.float32)
    G = O.voxelize(xyz, feat, origin, n, 1.0, 1.0, 3)
    s = np.array([2, 3, -1])           # (x, y, z) shift in voxels
    G2 = O.voxelize((xyz + s).astype(np.float32), feat, origin, n, 1.0, 1.0, 3)
    # G2[z + sz, y + sy, x + sx] == G[z, y, x] wherever both are in the grid
    a = G[1:n - 2, 0:n - 3, 0:n - 2]
    b = G2[0:n - 3, 3:n, 2:n]
    assert np.array_equal(a, b)


def test_linearity_in_atoms_and_features():
    rng = np.random.default_rng(5)
    origin = np.zeros(3, dtype=np.float32)
    xa = rng.uniform(2, 14, size=(5, 3)).astype(np.float32)
    xb = rng.uniform(2, 14, size=(4, 3)).astype(np.float32)
    fa = rng.normal(size=(5, 19)).astype(np.float32)
    fb = rng.normal(size=(4, 19)).astype(np.float32)
    Ga = O.voxelize(xa, fa, origin, 16, 1.0, 1.0, 3)
    Gb = O.voxelize(xb, fb, origin, 16, 1.0, 1.0, 3)
    Gab = O.voxelize(np.concatenate([xa, xb]), np.concatenate([fa, fb]), origin, 16, 1.0, 1.0, 3)
    np.testing.assert_allclose(Gab, Ga + Gb, rtol=0, atol=1e-14)
    G2 = O.voxelize(xa, 2.0 * fa, origin, 16, 1.0, 1.0, 3)
    np.testing.assert_allclose(G2, 2.0 * Ga, rtol=0, atol=1e-14)


def test_clipping_at_grid_edge_is_a_window_of_a_larger_grid():
    rng = np.random.default_rng(9)
    n = 12
    origin = np.zeros(3, dtype=np.float32)
    xyz = rng.uniform(-2.5, 14.5, size=(10, 3)).astype(np.float32)
    feat = rng.normal(size=(10, 19)).astype(np.float32)
    G = O.voxelize(xyz, feat, origin, n, 1.0, 1.0, 3)
    big_origin = np.full(3, -8.0, dtype=np.float32)
    Gb = O.voxelize(xyz, feat, big_origin, n + 16, 1.0, 1.0, 3)
    np.testing.assert_allclose(G, Gb[8:8 + n, 8:8 + n, 8:8 + n], rtol=0, atol=1e-14)


def test_atom_outside_grid_contributes_nothing():
    origin = np.zeros(3, dtype=np.float32)
    xyz = np.array([[-4.01, 5, 5], [5, 5, 20.5]], dtype=np.float32)
    G = O.voxelize(xyz, np.ones((2, 19), dtype=np.float32), origin, 16, 1.0, 1.0, 3)
    assert not G.any()


def test_containing_voxel_on_boundary_and_centroid_rule():
    assert int(O.containing_voxel(np.float32(3.0), np.float32(0.0), 1.0)) == 3
    assert int(O.containing_voxel(np.float32(-0.5), np.float32(0.0), 1.0)) == -1
    # dyadic ligand coordinates: the float32 sum is exact, so the centroid is the mean
    rng = np.random.default_rng(2)
    lig = (np.round(rng.uniform(-20, 20, size=(16, 3)) * 256) / 256).astype(np.float32)
    o = O.grid_origin(lig, 48, 1.0)
    np.testing.assert_array_equal(o.astype(np.float64), lig.astype(np.float64).mean(axis=0) - 24.0)
