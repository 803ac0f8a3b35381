"""Seeded synthetic inputs for the diffusion-absorption solver.

This module generates data only; it holds none of the solver's arithmetic and
is the one module that both the CUDA path's tests/benchmarks and the CPU oracle
consume. The paper's own inputs (Monte Carlo tissue volumes, Sec. 2.5.1) are not
available, so the fields below stand in for them with the shapes and value
distributions of the workloads that are benchmarked:

* ``grf``: a Gaussian random field on the vertex grid with squared-exponential
  covariance ``std^2 exp(-r^2 / (2 corr^2))``. The kernel is separable, so the
  field is drawn exactly as ``std * (Lz x Ly x Lx) xi`` where ``L_d = V sqrt(Lam)``
  comes from the 1-D covariance matrix of axis d (negative eigenvalues clipped
  to zero; eigenvalues below 1e-12 of the largest dropped, which changes the
  field by far less than FP64 rounding of the solver).
* ``unit_cube``: the small unit-cube case, 33^3 at h = 1/32: D = exp(g), g a GRF
  with corr 0.2, std 0.5, mean 0; mu constant 0.1; q i.i.d. U[0,1]; the JVP
  tangent on q is N(0,1); the VJP cotangent is N(0,1).
* ``tissue``: tissue-like coefficients in mm (Eq. 19): mus' = 1.0 exp(g1),
  mua = 0.01 exp(g2), g1, g2 GRFs (corr 5 mm, std 0.3), D = 1/(3 (mua + mus')),
  h = 0.5 mm; q a Gaussian blob (sigma 3 mm, peak 1) centred uniformly at
  least 3 sigma from the boundary; the cotangent is N(0,1) on a random 10% of
  interior vertices and 0 elsewhere; the tangent is dq ~ N(0,1),
  dD = 0.1 D xi1, dmu = 0.1 mu xi2 with xi ~ N(0,1).

* ``vi_batch``: the Monte Carlo samples of one variational-inference step
  (Sec. 2.5: every sample evaluates the forward model and its gradient): B
  ``tissue`` problems on one grid, sample b drawn from the seed (seed, b), so
  each sample has its own GRFs for log mus' and log mua, its own source and
  cotangent.

* ``tissue_torch``: the ``tissue`` recipe drawn on a CUDA device with torch's
  seeded generator, for request streams that need fresh inputs at 257^3
  faster than numpy draws them (same distributions, different random streams).

Random streams come from ``numpy.random.SeedSequence(seed).spawn`` with one
child per role, each driving a PCG64 generator, so every role is reproducible
on its own. A seed may be an int or a tuple of ints.
"""
from __future__ import annotations

import numpy as np

ROLES = ("g1", "g2", "q", "w_mask", "w", "dq", "dD", "dmu")


def _rngs(seed: int) -> dict:
    ss = np.random.SeedSequence(seed)
    return {name: np.random.Generator(np.random.PCG64(s)) for name, s in zip(ROLES, ss.spawn(len(ROLES)))}


def _axis_factor(n: int, h: float, corr: float) -> np.ndarray:
    x = np.arange(n) * h
    C = np.exp(-((x[:, None] - x[None, :]) ** 2) / (2.0 * corr * corr))
    lam, V = np.linalg.eigh(C)
    lam = np.clip(lam, 0.0, None)
    keep = lam > 1e-12 * lam.max()
    return V[:, keep] * np.sqrt(lam[keep])


def grf(shape, h: float, corr: float, std: float, rng: np.random.Generator) -> np.ndarray:
    """Zero-mean SE-covariance Gaussian random field on a (nz, ny, nx) or (ny, nx) vertex grid."""
    if len(shape) == 2:
        Ly, Lx = (_axis_factor(n, h, corr) for n in shape)
        xi = rng.standard_normal((Ly.shape[1], Lx.shape[1]))
        return np.ascontiguousarray(std * (Ly @ xi @ Lx.T))
    nz, ny, nx = shape
    Lz, Ly, Lx = (_axis_factor(n, h, corr) for n in (nz, ny, nx))
    xi = rng.standard_normal((Lz.shape[1], Ly.shape[1], Lx.shape[1]))
    t = np.tensordot(xi, Lx, axes=([2], [1]))          # (rz, ry, nx)
    t = np.tensordot(t, Ly, axes=([1], [1]))           # (rz, nx, ny)
    t = np.tensordot(t, Lz, axes=([0], [1]))           # (nx, ny, nz)
    return np.ascontiguousarray(std * t.transpose(2, 1, 0))


def interior_mask(shape) -> np.ndarray:
    m = np.zeros(shape, dtype=bool)
    m[1:-1, 1:-1, 1:-1] = True
    return m


def unit_cube(n: int = 33, seed: int = 0, shape=None) -> dict:
    """Unit-cube workload: D = exp(GRF(0.2, 0.5)), mu = 0.1, q ~ U[0,1], h = 1/(n-1)."""
    shape = tuple(shape) if shape is not None else (n, n, n)
    h = 1.0 / (max(shape) - 1)
    r = _rngs(seed)
    D = np.exp(grf(shape, h, 0.2, 0.5, r["g1"]))
    mu = np.full(shape, 0.1)
    q = r["q"].uniform(0.0, 1.0, size=shape)
    w = r["w"].standard_normal(shape)
    dq = r["dq"].standard_normal(shape)
    dD = 0.1 * D * r["dD"].standard_normal(shape)
    dmu = 0.1 * mu * r["dmu"].standard_normal(shape)
    return dict(name="unit_cube", shape=shape, h=h, D=D, mu=mu, q=q, w=w, dq=dq, dD=dD, dmu=dmu)


def tissue(n: int = 129, seed: int = 0, shape=None, h: float = 0.5) -> dict:
    """Tissue-like workload in mm (Eq. 19 coefficients), Gaussian-blob source."""
    shape = tuple(shape) if shape is not None else (n, n, n)
    r = _rngs(seed)
    mus = 1.0 * np.exp(grf(shape, h, 5.0, 0.3, r["g1"]))
    mua = 0.01 * np.exp(grf(shape, h, 5.0, 0.3, r["g2"]))
    D = 1.0 / (3.0 * (mua + mus))
    mu = mua
    sig = 3.0
    ext = [(s - 1) * h for s in shape]
    lo = [min(3 * sig, e / 2) for e in ext]
    c = [r["q"].uniform(l, e - l) for l, e in zip(lo, ext)]   # (z, y, x) centre
    z, y, x = (np.arange(s) * h for s in shape)
    q = (np.exp(-((z - c[0]) ** 2) / (2 * sig * sig))[:, None, None]
         * np.exp(-((y - c[1]) ** 2) / (2 * sig * sig))[None, :, None]
         * np.exp(-((x - c[2]) ** 2) / (2 * sig * sig))[None, None, :])
    inner = interior_mask(shape)
    sel = (r["w_mask"].random(shape) < 0.10) & inner
    w = np.where(sel, r["w"].standard_normal(shape), 0.0)
    dq = r["dq"].standard_normal(shape)
    dD = 0.1 * D * r["dD"].standard_normal(shape)
    dmu = 0.1 * mu * r["dmu"].standard_normal(shape)
    return dict(name="tissue", shape=shape, h=h, D=np.ascontiguousarray(D), mu=np.ascontiguousarray(mu),
                q=np.ascontiguousarray(q), w=w, dq=dq, dD=dD, dmu=dmu)


_FACTORS = {}


def _axis_factor_torch(n, h, corr, device):
    import torch
    key = (n, h, corr, str(device))
    if key not in _FACTORS:
        _FACTORS[key] = torch.from_numpy(np.ascontiguousarray(_axis_factor(n, h, corr))).to(device).float()
    return _FACTORS[key]


def tissue_torch(shape, seed: int, h: float = 0.5, device="cuda", keys=("D", "mu", "q", "w", "dq", "dD", "dmu")):
    """``tissue`` coefficients, source, cotangent and tangents as float64 tensors on a CUDA device."""
    import torch
    shape = tuple(shape)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = dict(dtype=torch.float64, device=device)

    def field(corr, std):
        # the Kronecker products in FP32 (the field is an input, not solver
        # arithmetic), then FP64
        Lz, Ly, Lx = (_axis_factor_torch(n, h, corr, device) for n in shape)
        xi = torch.randn((Lz.shape[1], Ly.shape[1], Lx.shape[1]), generator=g, dtype=torch.float32,
                         device=device)
        t = torch.einsum("abc,xc->abx", xi, Lx)
        t = torch.einsum("abx,yb->ayx", t, Ly)
        return std * torch.einsum("ayx,za->zyx", t, Lz).double()

    mus = torch.exp(field(5.0, 0.3))
    mua = 0.01 * torch.exp(field(5.0, 0.3))
    out = {"D": (1.0 / (3.0 * (mua + mus))).contiguous(), "mu": mua.contiguous()}
    sig = 3.0
    ext = [(n - 1) * h for n in shape]
    lo = [min(3 * sig, e / 2) for e in ext]
    u = torch.rand(3, generator=g, **f64).tolist()
    c = [l + (e - 2 * l) * r for l, e, r in zip(lo, ext, u)]
    z, y, x = (torch.arange(n, **f64) * h for n in shape)
    out["q"] = (torch.exp(-((z - c[0]) ** 2) / (2 * sig * sig))[:, None, None]
                * torch.exp(-((y - c[1]) ** 2) / (2 * sig * sig))[None, :, None]
                * torch.exp(-((x - c[2]) ** 2) / (2 * sig * sig))[None, None, :]).contiguous()
    if "w" in keys:
        inner = torch.zeros(shape, dtype=torch.bool, device=device)
        inner[1:-1, 1:-1, 1:-1] = True
        sel = (torch.rand(shape, generator=g, **f64) < 0.10) & inner
        out["w"] = torch.where(sel, torch.randn(shape, generator=g, **f64), torch.zeros((), **f64))
    if "dq" in keys:
        out["dq"] = torch.randn(shape, generator=g, **f64)
    if "dD" in keys:
        out["dD"] = 0.1 * out["D"] * torch.randn(shape, generator=g, **f64)
    if "dmu" in keys:
        out["dmu"] = 0.1 * out["mu"] * torch.randn(shape, generator=g, **f64)
    return {k: out[k] for k in keys}


def tissue2d(n: int = 257, seed: int = 0, shape=None, h: float = 0.5) -> dict:
    """The tissue recipe on a (ny, nx) grid for the 2D solver: the same GRF
    coefficients (Eq. 19), a 2D Gaussian-blob source, cotangent and tangents."""
    shape = tuple(shape) if shape is not None else (n, n)
    r = _rngs(seed)
    mus = 1.0 * np.exp(grf(shape, h, 5.0, 0.3, r["g1"]))
    mua = 0.01 * np.exp(grf(shape, h, 5.0, 0.3, r["g2"]))
    D = 1.0 / (3.0 * (mua + mus))
    sig = 3.0
    ext = [(s - 1) * h for s in shape]
    lo = [min(3 * sig, e / 2) for e in ext]
    c = [r["q"].uniform(l, e - l) for l, e in zip(lo, ext)]   # (y, x) centre
    y, x = (np.arange(s) * h for s in shape)
    q = np.exp(-((y - c[0]) ** 2) / (2 * sig * sig))[:, None] * np.exp(-((x - c[1]) ** 2) / (2 * sig * sig))[None, :]
    inner = np.zeros(shape, dtype=bool)
    inner[1:-1, 1:-1] = True
    sel = (r["w_mask"].random(shape) < 0.10) & inner
    w = np.where(sel, r["w"].standard_normal(shape), 0.0)
    return dict(name="tissue2d", shape=shape, h=h, D=np.ascontiguousarray(D), mu=np.ascontiguousarray(mua),
                q=np.ascontiguousarray(q), w=w, dq=r["dq"].standard_normal(shape),
                dD=0.1 * D * r["dD"].standard_normal(shape), dmu=0.1 * mua * r["dmu"].standard_normal(shape))


def _gauss_filter_torch(x, h, corr, axis):
    """x convolved along one axis with the Gaussian of std corr / sqrt(2) (zero padding)."""
    import torch
    s = corr / np.sqrt(2.0) / h
    r = int(np.ceil(4 * s))
    t = torch.arange(-r, r + 1, dtype=x.dtype, device=x.device)
    k = torch.exp(-0.5 * (t / s) ** 2)
    y = x.movedim(axis, -1)
    shp = y.shape
    y = torch.nn.functional.conv1d(y.reshape(-1, 1, shp[-1]), k.view(1, 1, -1), padding=r)
    return y.reshape(shp).movedim(-1, axis), float(torch.sqrt((k * k).sum()))


def grf_filter_torch(shape, h, corr, std, gen, device):
    """Zero-mean Gaussian random field with (approximately) SE covariance
    std^2 exp(-r^2 / (2 corr^2)): white noise filtered by a Gaussian of std
    corr / sqrt(2) along each axis and normalised to unit variance. Linear cost,
    for grids whose 1-D covariance factors would be too costly to decompose."""
    import torch
    x = torch.randn(shape, generator=gen, dtype=torch.float32, device=device)
    norm = 1.0
    for ax in range(len(shape)):
        x, nk = _gauss_filter_torch(x, h, corr, ax)
        norm *= nk
    return (std / norm) * x.double()


def tissue2d_torch(shape, seed: int, h: float = 0.5, device="cuda"):
    """The 2D tissue recipe on a CUDA device (filtered-noise GRFs): D, mu, q, w, dq, dD, dmu."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f64 = dict(dtype=torch.float64, device=device)
    mus = torch.exp(grf_filter_torch(shape, h, 5.0, 0.3, g, device))
    mua = 0.01 * torch.exp(grf_filter_torch(shape, h, 5.0, 0.3, g, device))
    D = 1.0 / (3.0 * (mua + mus))
    sig = 3.0
    ext = [(n - 1) * h for n in shape]
    lo = [min(3 * sig, e / 2) for e in ext]
    u = torch.rand(2, generator=g, **f64).tolist()
    c = [l + (e - 2 * l) * r for l, e, r in zip(lo, ext, u)]
    y, x = (torch.arange(n, **f64) * h for n in shape)
    q = (torch.exp(-((y - c[0]) ** 2) / (2 * sig * sig))[:, None] * torch.exp(-((x - c[1]) ** 2) / (2 * sig * sig))[None, :])
    inner = torch.zeros(shape, dtype=torch.bool, device=device)
    inner[1:-1, 1:-1] = True
    sel = (torch.rand(shape, generator=g, **f64) < 0.10) & inner
    w = torch.where(sel, torch.randn(shape, generator=g, **f64), torch.zeros((), **f64))
    return dict(D=D.contiguous(), mu=mua.contiguous(), q=q.contiguous(), w=w, h=h, shape=tuple(shape))


def vi_batch(n: int = 129, batch: int = 64, seed: int = 0, shape=None, h: float = 0.5,
             keys=("D", "mu", "q", "w")) -> dict:
    """B tissue samples stacked along a leading axis: arrays of shape (B, nz, ny, nx)."""
    out = {k: [] for k in keys}
    w = None
    for b in range(batch):
        w = tissue(n, seed=(seed, b), shape=shape, h=h)
        for k in keys:
            out[k].append(w[k])
    res = {k: np.stack(v) for k, v in out.items()}
    res.update(name="vi_batch", shape=(batch,) + tuple(w["shape"]), h=h)
    return res


def constant(shape, h: float, D: float = 1.0, mu: float = 0.1) -> dict:
    """Constant coefficients (used for closed-form checks)."""
    return dict(shape=tuple(shape), h=h, D=np.full(shape, float(D)), mu=np.full(shape, float(mu)))


def sine_mode(shape, p) -> np.ndarray:
    """prod_d sin(p_d pi x_d) with x_d = i_d / (n_d - 1); zero on the boundary."""
    nz, ny, nx = shape
    pz, py, px = p
    z = np.sin(pz * np.pi * np.arange(nz) / (nz - 1))
    y = np.sin(py * np.pi * np.arange(ny) / (ny - 1))
    x = np.sin(px * np.pi * np.arange(nx) / (nx - 1))
    s = z[:, None, None] * y[None, :, None] * x[None, None, :]
    s[0], s[-1], s[:, 0], s[:, -1], s[:, :, 0], s[:, :, -1] = 0, 0, 0, 0, 0, 0
    return s
