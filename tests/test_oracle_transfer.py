"""Pins of the oracle's grid transfers and coefficient coarsening (Eq. 7, Eq. 17).

Restriction is full weighting 1/4[1 2 1] per axis; prolongation is I = 2^3 R^T.
Checked against: a library trilinear interpolator (scipy), exact reproduction
of linear and quadratic functions by full weighting, and the duality
<R a, b> = 2^-3 <a, I b>.
"""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle
from paper_2608_00760_b300 import inputs

SHAPES = [(9, 9, 9), (17, 9, 5), (5, 9, 17), (33, 17, 9)]


@pytest.mark.parametrize("fine", SHAPES)
def test_prolongation_is_trilinear_interpolation(fine):
    coarse = oracle.coarse_shape(fine)
    rng = np.random.default_rng(1)
    e = rng.standard_normal(coarse) * inputs.interior_mask(coarse)
    uf = oracle.prolong_add(e, np.zeros(fine))
    # scipy's trilinear interpolation of the coarse field (zero boundary) at fine vertices
    axes = [np.arange(n) * 2.0 for n in coarse]
    it = RegularGridInterpolator(axes, e, method="linear")
    pts = np.stack(np.meshgrid(*[np.arange(n, dtype=float) for n in fine], indexing="ij"), -1)
    ref = it(pts.reshape(-1, 3)).reshape(fine) * inputs.interior_mask(fine)
    assert np.abs(uf - ref).max() <= 1e-15 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("fine", SHAPES)
def test_restriction_prolongation_duality(fine):
    coarse = oracle.coarse_shape(fine)
    rng = np.random.default_rng(2)
    a = rng.standard_normal(fine) * inputs.interior_mask(fine)
    b = rng.standard_normal(coarse) * inputs.interior_mask(coarse)
    lhs = np.sum(oracle.restrict(a) * b)
    rhs = np.sum(a * oracle.prolong_add(b, np.zeros(fine))) / 8.0
    assert abs(lhs - rhs) <= 1e-13 * np.sqrt(np.sum(a * a) * np.sum(b * b))


@pytest.mark.parametrize("fine", SHAPES)
def test_full_weighting_reproduces_polynomials(fine):
    nz, ny, nx = fine
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    coarse = oracle.coarse_shape(fine)
    Z, Y, X = np.meshgrid(*[2.0 * np.arange(n) for n in coarse], indexing="ij")
    m = inputs.interior_mask(coarse)
    lin = 0.3 + 1.1 * x - 0.7 * y + 2.0 * z
    assert np.allclose(oracle.restrict(lin)[m], (0.3 + 1.1 * X - 0.7 * Y + 2.0 * Z)[m], atol=1e-12)
    # per axis 1/4 (x-1)^2 + 1/2 x^2 + 1/4 (x+1)^2 = x^2 + 1/2
    quad = x * x + y * y + z * z
    assert np.allclose(oracle.restrict(quad)[m], (X * X + Y * Y + Z * Z + 1.5)[m], rtol=1e-14)
    # coefficient coarsening = the same weighting inside, injection on the boundary
    cc = oracle.coarsen(lin)
    ref = 0.3 + 1.1 * X - 0.7 * Y + 2.0 * Z
    assert np.allclose(cc, ref, atol=1e-12)
    ci = oracle.coarsen(quad, inject=True)
    assert np.allclose(ci, X * X + Y * Y + Z * Z)
    cq = oracle.coarsen(quad)
    assert np.allclose(cq[~m], (X * X + Y * Y + Z * Z)[~m])
    assert np.allclose(cq[m], (X * X + Y * Y + Z * Z + 1.5)[m])


def test_level_count_and_shapes():
    assert oracle.count_levels((257, 257, 257)) == 8
    assert oracle.count_levels((129, 257, 257)) == 7
    assert oracle.count_levels((3, 3, 3)) == 1
    assert oracle.count_levels((33, 17, 9)) == 3
    # coarsening stops as soon as any one axis cannot be halved (shapes are (nz, ny, nx))
    assert oracle.count_levels((17, 10, 17)) == 1
    assert oracle.count_levels((17, 17, 10)) == 1
    assert oracle.count_levels((10, 17, 17)) == 1
    assert oracle.count_levels((17, 3, 17)) == 1
    assert oracle.count_levels((33, 5, 17)) == 2
    w = inputs.constant((129, 257, 257), 1.0)
    H = oracle.Hierarchy(w["D"][:3, :5, :5].copy(), w["mu"][:3, :5, :5].copy(), 1.0)
    assert H.nlev == 1
