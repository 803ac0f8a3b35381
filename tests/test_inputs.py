"""The seeded input recipe (paper_2608_00760_b300/inputs.py) against the
distributions it states: squared-exponential GRFs, the tissue coefficient
relations of Eq. 19, the source blob's placement, the cotangent's density, the
tangent scalings, and reproducibility per seed. The torch variants are drawn on
the CPU device here; they follow the same recipe with other random streams."""
import numpy as np
import pytest

from paper_2608_00760_b300 import inputs


def test_axis_factor_reproduces_the_se_covariance():
    for n, h, corr in ((33, 0.5, 5.0), (65, 1.0 / 64, 0.2), (17, 0.5, 1.0)):
        L = inputs._axis_factor(n, h, corr)
        x = np.arange(n) * h
        C = np.exp(-((x[:, None] - x[None, :]) ** 2) / (2 * corr * corr))
        assert np.abs(L @ L.T - C).max() <= 1e-9


def test_grf_sample_covariance_matches_the_kernel():
    # 4000 draws on a 9 x 9 grid; the sample covariance of vertex pairs against
    # std^2 exp(-r^2 / (2 corr^2)) within a few standard errors
    rng = np.random.default_rng(5)
    n, h, corr, std = 9, 1.0, 2.0, 0.7
    draws = np.stack([inputs.grf((n, n), h, corr, std, rng) for _ in range(4000)])
    assert abs(draws.mean()) <= 0.03
    pairs = [((4, 4), (4, 4)), ((4, 4), (4, 5)), ((4, 4), (5, 6)), ((0, 0), (3, 0)), ((2, 3), (6, 7))]
    for (a, b), (c, d) in pairs:
        r2 = ((a - c) ** 2 + (b - d) ** 2) * h * h
        want = std * std * np.exp(-r2 / (2 * corr * corr))
        got = np.mean(draws[:, a, b] * draws[:, c, d])
        assert abs(got - want) <= 0.05 * std * std, ((a, b), (c, d), got, want)


def test_3d_grf_is_the_kronecker_product_of_axis_factors():
    rng_a, rng_b = np.random.default_rng(9), np.random.default_rng(9)
    shape, h, corr, std = (5, 7, 9), 0.5, 1.5, 0.3
    g = inputs.grf(shape, h, corr, std, rng_a)
    Lz, Ly, Lx = (inputs._axis_factor(n, h, corr) for n in shape)
    xi = rng_b.standard_normal((Lz.shape[1], Ly.shape[1], Lx.shape[1]))
    ref = std * np.einsum("za,yb,xc,abc->zyx", Lz, Ly, Lx, xi)
    assert np.abs(g - ref).max() <= 1e-12


def test_tissue_recipe():
    w = inputs.tissue(33, seed=4)
    D, mu, q, h = w["D"], w["mu"], w["q"], w["h"]
    assert h == 0.5 and D.shape == (33, 33, 33)
    # mu_a = 0.01 exp(g2) and D = 1 / (3 (mu_a + mu_s')) with mu_s' = exp(g1): both lognormal around their medians
    mus = 1.0 / (3.0 * D) - mu
    assert np.all(mu > 0) and np.all(mus > 0)
    assert 0.5 < np.median(mus) < 2.0 and 0.005 < np.median(mu) < 0.02
    assert np.std(np.log(mus)) < 0.6 and np.std(np.log(mu / 0.01)) < 0.6
    # Gaussian blob of sigma 3 mm and peak 1, centred at least min(3 sigma,
    # half the extent) from every face (on this 16 mm grid: the middle)
    k, j, i = np.unravel_index(np.argmax(q), q.shape)
    ext = (33 - 1) * h
    lo = min(3 * 3.0, ext / 2)
    for idx in (k, j, i):
        assert lo - h <= idx * h <= ext - lo + h
    assert 0.9 < q.max() <= 1.0
    zz = np.arange(33) * h
    line = q[k, j, :] / q[k, j, i]
    ref = np.exp(-((zz - zz[i]) ** 2) / (2 * 9.0))
    assert np.abs(line - ref).max() <= 0.1
    # cotangent on about 10% of interior vertices, zero elsewhere
    inner = inputs.interior_mask(w["shape"])
    frac = np.count_nonzero(w["w"][inner]) / inner.sum()
    assert 0.08 < frac < 0.12 and not np.any(w["w"][~inner])
    # tangents: dD = 0.1 D xi, dmu = 0.1 mu xi with xi ~ N(0, 1)
    assert abs(np.std(w["dD"] / D) - 0.1) < 0.005 and abs(np.std(w["dmu"] / mu) - 0.1) < 0.005
    assert abs(np.std(w["dq"]) - 1.0) < 0.02


def test_seeds_reproduce_and_roles_are_independent():
    # 41^3 at 0.5 mm: 20 mm per axis, so the blob centre (at least 9 mm from
    # every face) still moves with the seed
    a, b, c = inputs.tissue(41, seed=3), inputs.tissue(41, seed=3), inputs.tissue(41, seed=4)
    for k in ("D", "mu", "q", "w", "dq", "dD", "dmu"):
        assert np.array_equal(a[k], b[k])
        assert not np.array_equal(a[k], c[k]), k
    k, j, i = np.unravel_index(np.argmax(a["q"]), a["q"].shape)
    assert all(9.0 - 0.5 <= idx * 0.5 <= 20.0 - 9.0 + 0.5 for idx in (k, j, i))
    # a VI batch's sample b is the tissue draw of seed (seed, b)
    vb = inputs.vi_batch(17, 3, seed=6)
    for s in range(3):
        assert np.array_equal(vb["D"][s], inputs.tissue(17, seed=(6, s))["D"])
    assert not np.array_equal(vb["D"][0], vb["D"][1])


def test_unit_cube_recipe():
    w = inputs.unit_cube(17, seed=2)
    assert w["h"] == 1.0 / 16 and np.all(w["mu"] == 0.1)
    assert abs(np.std(np.log(w["D"])) - 0.5) < 0.2
    assert w["q"].min() >= 0.0 and w["q"].max() <= 1.0 and abs(w["q"].mean() - 0.5) < 0.02


def test_tissue_torch_follows_the_same_recipe_on_the_cpu_device():
    torch = pytest.importorskip("torch")
    w = inputs.tissue_torch((33, 33, 33), 11, device="cpu")
    D, mu, q, cot = (w[k].numpy() for k in ("D", "mu", "q", "w"))
    assert all(w[k].dtype == torch.float64 for k in w)
    mus = 1.0 / (3.0 * D) - mu
    assert np.all(mu > 0) and np.all(mus > 0)
    assert 0.5 < np.median(mus) < 2.0 and 0.005 < np.median(mu) < 0.02
    k, j, i = np.unravel_index(np.argmax(q), q.shape)
    for idx in (k, j, i):
        assert 8.0 - 0.5 <= idx * 0.5 <= 8.0 + 0.5     # 16 mm per axis: the centre is the middle
    inner = inputs.interior_mask((33, 33, 33))
    assert 0.08 < np.count_nonzero(cot[inner]) / inner.sum() < 0.12 and not np.any(cot[~inner])
    again = inputs.tissue_torch((33, 33, 33), 11, device="cpu")
    assert all(torch.equal(w[k], again[k]) for k in w)
