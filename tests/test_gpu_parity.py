"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (written here, derived in the design notes):
  * converged results (both sides at relative residual 1e-10): relative L2
    error <= 1e-8, the bound the solver's accuracy target states;
  * identical schedules (same fixed cycle count m): the two sides run the same
    arithmetic in a different rounding order (FMA contraction, precomputed
    faces and reciprocals), so they agree to <= 1e-11 relative;
  * dot-product (adjoint) identities: <= 1e-10 relative.
"""
import numpy as np
import pytest

import oracle
from paper_2608_00760_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_CONV = 1e-8
TOL_SAME = 1e-11
TOL_DOT = 1e-10


@pytest.fixture(scope="module")
def dmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_00760_b300 import build, dmg
    build.build()
    dmg.lib()
    return dmg


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def N(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a = N(a) if torch.is_tensor(a) else a
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def close(a, b, tol):
    """Relative L2 error <= tol and, entry by entry, |a - b| <= tol max|b|: a
    localised error (one boundary plane of Dbar, one colour, one corner) that
    a whole-field norm would average away still fails the second bound."""
    a = N(a) if torch.is_tensor(a) else np.asarray(a)
    b = N(b) if torch.is_tensor(b) else np.asarray(b)
    e2 = rel(a, b)
    mb = float(np.max(np.abs(b))) if b.size else 0.0
    einf = float(np.max(np.abs(a - b))) / (mb if mb > 0 else 1.0) if b.size else 0.0
    assert e2 <= tol and einf <= tol, "relative L2 %.3e, max-entry %.3e, tolerance %.1e" % (e2, einf, tol)
    return True


WORKLOADS = [
    ("unit_cube", dict(n=17)),
    ("unit_cube", dict(n=33)),
    ("tissue", dict(n=33)),
    ("tissue", dict(shape=(17, 33, 65))),
    ("unit_cube", dict(shape=(33, 9, 17))),
]


def make(name, kw, seed=0):
    return getattr(inputs, name)(seed=seed, **kw)


@pytest.mark.parametrize("name,kw", WORKLOADS)
def test_forward_and_vjp_converged(dmg, name, kw):
    w = make(name, kw)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    u = S.solve(T(w["q"]))
    info_f = S.last_info
    assert info_f.rel_residual <= 1e-10
    qb, Db, mb = S.vjp(u, T(w["w"]))
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ur, _, _ = H.solve(w["q"], rtol=1e-10)
    qbr, Dbr, mbr, _ = H.vjp(ur, w["w"], rtol=1e-10)
    assert close(u, ur, TOL_CONV)
    assert close(qb, qbr, TOL_CONV)
    assert close(Db, Dbr, TOL_CONV)
    assert close(mb, mbr, TOL_CONV)
    # Dirichlet boundary: outputs are zero there, Dbar is not
    m = inputs.interior_mask(w["shape"])
    assert not N(u)[~m].any() and not N(qb)[~m].any() and not N(mb)[~m].any()
    # the GPU's residual, recomputed by the oracle operator
    r = oracle.residual(w["D"], w["mu"], w["h"], w["q"] * m, N(u))
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(w["q"][m])


@pytest.mark.parametrize("m", [1, 2, 5])
@pytest.mark.parametrize("name,kw", WORKLOADS[:4])
def test_fixed_cycles_match_oracle_schedule(dmg, name, kw, m):
    w = make(name, kw, seed=1)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], fixed_cycles=m)
    u = S.solve(T(w["q"]))
    assert S.last_info.cycles == m
    qb, Db, mb = S.vjp(u, T(w["w"]), cycles=m)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ur, _, _ = H.solve(w["q"], fixed=m)
    lam = H.adjoint(w["w"], fixed=m)[0]
    Dbr, mbr = oracle.grad(w["D"], w["h"], ur, lam)
    assert close(u, ur, TOL_SAME)
    assert close(qb, lam, TOL_SAME)
    assert close(Db, Dbr, TOL_SAME)
    assert close(mb, mbr, TOL_SAME)


def test_fixed_cycles_match_oracle_schedule_129(dmg):
    # 129^3: the FP64 cycle runs five grid levels (129, 65, 33, 17, 9) and the
    # shared-memory tail below them; two cycles forward and two transposed
    # cycles must be the oracle's schedule to rounding, entry by entry
    w = make("tissue", dict(n=129), seed=12)
    m = 2
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], fixed_cycles=m)
    assert len(S.levels()) == 7
    u = S.solve(T(w["q"]))
    qb, Db, mb = S.vjp(u, T(w["w"]), cycles=m)
    S.close()
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ur, _, _ = H.solve(w["q"], fixed=m)
    lam = H.adjoint(w["w"], fixed=m)[0]
    Dbr, mbr = oracle.grad(w["D"], w["h"], ur, lam)
    assert close(u, ur, TOL_SAME)
    assert close(qb, lam, TOL_SAME)
    assert close(Db, Dbr, TOL_SAME)
    assert close(mb, mbr, TOL_SAME)


@pytest.mark.parametrize("opts", [dict(face_mean=1), dict(coarsen=1), dict(symmetric=1),
                                  dict(nu1=1, nu2=1), dict(nu1=3, nu2=1), dict(nu1=0, nu2=2)])
def test_schedule_options_match_oracle(dmg, opts):
    w = make("tissue", dict(n=17), seed=2)
    m = 3
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], fixed_cycles=m, **opts)
    u = S.solve(T(w["q"]))
    qb, Db, mb = S.vjp(u, T(w["w"]), cycles=m)
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"], nu1=opts.get("nu1", 2), nu2=opts.get("nu2", 2),
                         harmonic=bool(opts.get("face_mean", 0)), inject=bool(opts.get("coarsen", 0)),
                         symmetric=bool(opts.get("symmetric", 0)))
    ur, _, _ = H.solve(w["q"], fixed=m)
    lam = H.adjoint(w["w"], fixed=m)[0]
    Dbr, mbr = oracle.grad(w["D"], w["h"], ur, lam, harmonic=bool(opts.get("face_mean", 0)))
    assert close(u, ur, TOL_SAME)
    assert close(qb, lam, TOL_SAME)
    assert close(Db, Dbr, TOL_SAME)
    assert close(mb, mbr, TOL_SAME)


def test_count_matched_adjoint_dot_product(dmg):
    w = make("tissue", dict(n=33), seed=3)
    m = 4
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], fixed_cycles=m)
    msk = inputs.interior_mask(w["shape"])
    v = T(w["dq"] * msk)
    Sv = S.solve(v)
    StW, _, _ = S.vjp(None, T(w["w"]), cycles=m, need=(True, False, False))
    lhs = float(torch.sum(T(w["w"] * msk) * Sv))
    rhs = float(torch.sum(StW * v))
    assert abs(lhs - rhs) <= TOL_DOT * np.linalg.norm(w["w"]) * float(torch.linalg.norm(Sv))


def test_jvp_matches_oracle_and_duality(dmg):
    w = make("tissue", dict(n=33), seed=4)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    u = S.solve(T(w["q"]))
    du_q = S.jvp(None, dq=T(w["dq"]))
    du = S.jvp(u, dq=T(w["dq"]), dD=T(w["dD"]), dmu=T(w["dmu"]))
    du_D = S.jvp(u, dD=T(w["dD"]))
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ur, _, _ = H.solve(w["q"], rtol=1e-10)
    ref_q, _ = H.jvp(ur, w["dq"], rtol=1e-10)
    ref, _ = H.jvp(ur, w["dq"], w["dD"], w["dmu"], rtol=1e-10)
    ref_D, _ = H.jvp(ur, np.zeros(w["shape"]), w["dD"], None, rtol=1e-10)
    assert close(du_q, ref_q, TOL_CONV)
    assert close(du, ref, TOL_CONV)
    assert close(du_D, ref_D, TOL_CONV)
    # <w, J t> = <J^T w, t> with both sides converged
    qb, Db, mb = S.vjp(u, T(w["w"]))
    msk = inputs.interior_mask(w["shape"])
    lhs = float(torch.sum(T(w["w"] * msk) * du))
    rhs = float(torch.sum(qb * T(w["dq"] * msk)) + torch.sum(Db * T(w["dD"])) + torch.sum(mb * T(w["dmu"])))
    assert abs(lhs - rhs) <= 1e-8 * abs(lhs)


def test_mixed_precision_matches_fp64_oracle(dmg):
    w = make("tissue", dict(n=65), seed=5)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=dmg.DMG_MIXED)
    u = S.solve(T(w["q"]))
    assert S.last_info.rel_residual <= 1e-10
    qb, Db, mb = S.vjp(u, T(w["w"]))
    assert S.last_info.rel_residual <= 1e-10
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ur, _, _ = H.solve(w["q"], rtol=1e-10)
    qbr, Dbr, mbr, _ = H.vjp(ur, w["w"], rtol=1e-10)
    assert close(u, ur, TOL_CONV)
    assert close(qb, qbr, TOL_CONV)
    assert close(Db, Dbr, TOL_CONV)
    assert close(mb, mbr, TOL_CONV)


@pytest.mark.parametrize("n", [257, 513])
def test_mixed_matches_fp64_gpu_at_full_size(dmg, n):
    # the full-size configurations: mixed precision against the FP64 GPU path
    # (the oracle at these sizes is too slow); both at rtol 1e-10
    w = inputs.tissue_torch((n, n, n), 9, device="cuda", keys=("D", "mu", "q", "w"))
    out = {}
    for prec in (dmg.DMG_FP64, dmg.DMG_MIXED):
        S = dmg.Solver(w["D"], w["mu"], 0.5, precision=prec)
        u = S.solve(w["q"])
        assert S.last_info.rel_residual <= 1e-10
        qb, Db, mb = S.vjp(u, w["w"])
        assert S.last_info.rel_residual <= 1e-10
        out[prec] = (u, qb, Db, mb)
        S.close()
    for a, b in zip(out[dmg.DMG_MIXED], out[dmg.DMG_FP64]):
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) <= 1e-8
        assert float((a - b).abs().max() / b.abs().max()) <= 1e-8


def test_full_size_mixed_certified_by_the_oracle(dmg):
    # The 257^3 workload in the precision the bench times (mixed, rtol 1e-10).
    # Properties that hold at any size, checked with the oracle's own arithmetic:
    # the oracle's operator gives the forward, adjoint and tangent solutions a
    # relative residual within rtol (plus FP64 rounding of the residual itself),
    # and the oracle's gradient formula, applied vertex by vertex to the GPU's
    # u and lambda = qbar, gives the GPU's Dbar and mubar.
    n, h, rtol = 257, 0.5, 1e-10
    w = inputs.tissue_torch((n, n, n), 10, h=h, device="cuda")
    S = dmg.Solver(w["D"], w["mu"], h, precision=dmg.DMG_MIXED, rtol=rtol)
    u = S.solve(w["q"])
    qb, Db, mb = S.vjp(u, w["w"])
    du = S.jvp(u, w["dq"], w["dD"], w["dmu"])
    S.close()
    D, mu, q, wv, dq, dD, dmu = (N(w[k]) for k in ("D", "mu", "q", "w", "dq", "dD", "dmu"))
    u, lam, Db, mb, du = (N(x) for x in (u, qb, Db, mb, du))
    inner = inputs.interior_mask((n, n, n))

    def rel_residual(rhs, x):
        r = (rhs - oracle.apply(D, mu, h, x)) * inner
        return float(np.linalg.norm(r) / np.linalg.norm(rhs * inner))

    bound = rtol * (1 + 1e-2) + 1e-12
    assert rel_residual(q, u) <= bound
    assert rel_residual(wv, lam) <= bound
    assert rel_residual(dq - oracle.dA_apply(D, h, dD, dmu, u), du) <= bound
    Dbr, mbr = oracle.grad(D, h, u, lam)
    # plain numpy norms: numpy arrays also carry a .device attribute
    assert np.linalg.norm(Db - Dbr) <= 1e-12 * np.linalg.norm(Dbr)
    assert np.linalg.norm(mb - mbr) <= 1e-14 * np.linalg.norm(mbr)


def test_host_pointers_give_device_results(dmg):
    w = make("unit_cube", dict(n=17), seed=6)
    S = dmg.Solver(w["D"], w["mu"], w["h"])            # numpy (host) coefficients
    u_dev = S.solve(T(w["q"]))
    u_host = np.zeros(w["shape"])
    assert dmg.dmg_solve(S.ctx, w["q"], u_host, n=S.n) == dmg.DMG_OK
    assert np.array_equal(N(u_dev), u_host)
    qb, Db, mb = np.zeros(w["shape"]), np.zeros(w["shape"]), np.zeros(w["shape"])
    assert dmg.dmg_vjp(S.ctx, u_host, w["w"], 0, qb, Db, mb, n=S.n) == dmg.DMG_OK
    qd, Dd, md = S.vjp(u_dev, T(w["w"]))
    assert np.array_equal(N(qd), qb) and np.array_equal(N(Dd), Db) and np.array_equal(N(md), mb)


def test_edge_cases(dmg):
    # single interior unknown: exact in one cycle
    rng = np.random.default_rng(0)
    D = np.exp(rng.standard_normal((3, 3, 3)))
    mu = np.full((3, 3, 3), 0.3)
    q = rng.uniform(size=(3, 3, 3))
    S = dmg.Solver(T(D), T(mu), 0.5, rtol=1e-14)
    u = S.solve(T(q))
    assert S.last_info.cycles == 1
    assert close(u, oracle.direct_solve(D, mu, 0.5, q), 1e-14)
    # single-level anisotropic grid (3 x 5 x 9 vertices, 21 unknowns)
    D = np.exp(rng.standard_normal((3, 5, 9)))
    mu = np.full((3, 5, 9), 0.1)
    q = rng.uniform(size=(3, 5, 9))
    S = dmg.Solver(T(D), T(mu), 0.2, rtol=1e-13)
    assert S.levels() == [(3, 5, 9)]
    assert close(S.solve(T(q)), oracle.direct_solve(D, mu, 0.2, q), 1e-13)
    # zero source: zero solution, zero cycles
    w = make("unit_cube", dict(n=9))
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    u = S.solve(torch.zeros(w["shape"], dtype=torch.float64, device="cuda"))
    assert S.last_info.cycles == 0 and not bool(u.any())
    # non-convergence within max_cycles: status ENOCONV, last iterate still written
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], max_cycles=1, strict=False)
    u = S.solve(T(w["q"]))
    assert S.last_info.cycles == 1 and S.last_info.rel_residual > 1e-10 and bool(u.any())
    Ss = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], max_cycles=1)
    with pytest.raises(dmg.DMGError) as e:
        Ss.solve(T(w["q"]))
    assert e.value.status == dmg.DMG_ENOCONV
    # NaN input: status ENAN
    qn = w["q"].copy()
    qn[4, 4, 4] = np.nan
    with pytest.raises(dmg.DMGError) as e:
        S.solve(T(qn))
    assert e.value.status == dmg.DMG_ENAN
    # a non-positive-definite operator is rejected at setup
    with pytest.raises(dmg.DMGError) as e:
        dmg.Solver(T(-w["D"]), T(w["mu"]), w["h"])
    assert e.value.status == dmg.DMG_EINVAL


def test_boundary_values_of_inputs_are_ignored(dmg):
    w = make("tissue", dict(n=17), seed=7)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    u1 = S.solve(T(w["q"]))
    q2 = w["q"].copy()
    q2[0] = 5.0
    q2[:, -1] = -2.0
    u2 = S.solve(T(q2))
    assert torch.equal(u1, u2)
    w2 = w["w"].copy()
    w2[:, :, 0] = 3.0
    u_b = N(u1).copy()
    u_b[-1] = 9.0            # a forward solution with garbage on the boundary
    a = S.vjp(u1, T(w["w"]))
    b = S.vjp(T(u_b), T(w2))
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.slow
def test_tissue_129_converged(dmg):
    w = make("tissue", dict(n=129), seed=0)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    u = S.solve(T(w["q"]))
    qb, Db, mb = S.vjp(u, T(w["w"]))
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ur, _, _ = H.solve(w["q"], rtol=1e-10)
    qbr, Dbr, mbr, _ = H.vjp(ur, w["w"], rtol=1e-10)
    for a, b in ((u, ur), (qb, qbr), (Db, Dbr), (mb, mbr)):
        assert close(a, b, TOL_CONV)


FUSED_SHAPES = [(65, 65, 65), (33, 49, 97), (129, 33, 65), (17, 33, 161), (9, 9, 257)]


@pytest.mark.parametrize("shape", FUSED_SHAPES)
@pytest.mark.parametrize("face_mean,nu", [(0, (2, 2)), (1, (2, 2)), (0, (3, 1))])
def test_fp32_vcycle_matches_fp64_vcycle(dmg, shape, face_mean, nu):
    # one mixed refinement step is s * V32(q / s); one FP64 cycle is V64(q). The FP32
    # V-cycle (colour half-sweeps, the prolongation fused into the first
    # post-smoothing half-sweep, ragged rows and planes included) must be the
    # same linear map up to FP32 rounding.
    w = inputs.tissue(shape=shape, seed=8)
    kw = dict(max_cycles=1, strict=False, face_mean=face_mean, nu1=nu[0], nu2=nu[1])
    Sm = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=dmg.DMG_MIXED, inner_cycles=1, **kw)
    S6 = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=dmg.DMG_FP64, **kw)
    for transposed in (False, True):
        if transposed:
            um, _, _ = Sm.vjp(None, T(w["w"]), need=(True, False, False))
            u6, _, _ = S6.vjp(None, T(w["w"]), need=(True, False, False))
        else:
            um, u6 = Sm.solve(T(w["q"])), S6.solve(T(w["q"]))
        assert close(um, N(u6), 2e-6)


@pytest.mark.parametrize("shape", FUSED_SHAPES[:2])
def test_mixed_iterates_track_fp64_iterates(dmg, shape):
    # FP32 rounding in a correction is damped by the later cycles, so converged
    # mixed and FP64 solutions agree far below the solve tolerance, in the same
    # number of cycles.
    w = inputs.tissue(shape=shape, seed=9)
    Sm = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=dmg.DMG_MIXED, inner_cycles=1)
    S6 = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    um, u6 = Sm.solve(T(w["q"])), S6.solve(T(w["q"]))
    assert abs(Sm.last_info.outer - S6.last_info.cycles) <= 1
    assert close(um, N(u6), 1e-12)
    # three FP32 cycles per FP64 step (the default): same total cycle count, a third of the steps
    S3 = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=dmg.DMG_MIXED, inner_cycles=3)
    u3 = S3.solve(T(w["q"]))
    assert S3.last_info.cycles <= S6.last_info.cycles + 3
    assert S3.last_info.outer <= (S6.last_info.cycles + 2) // 3 + 1
    assert S3.last_info.rel_residual <= 1e-10
    assert close(u3, N(u6), 1e-9)


@pytest.mark.parametrize("precision", [0, 1])
def test_long_thin_single_level_grid(dmg, precision):
    # 3 x 3 x 514: one level with 512 unknowns; its FP64 shared-memory tail would
    # not fit, so the FP64 path uses the grid coarse solve, the FP32 path the tail
    rng = np.random.default_rng(4)
    shape = (514, 3, 3)
    D = np.exp(0.3 * rng.standard_normal(shape))
    mu = np.full(shape, 0.05)
    q = rng.uniform(size=shape)
    S = dmg.Solver(T(D), T(mu), 0.1, precision=precision, rtol=1e-12)
    assert S.levels() == [shape]
    u = S.solve(T(q))
    assert close(u, oracle.direct_solve(D, mu, 0.1, q), 1e-10)


# grids small enough that the single-CTA tail starts at the finest level
# (<= 512 interior vertices in FP64, <= 4096 in FP32): each V-cycle must continue
# from the current iterate, so the FP64 solve converges at the V-cycle's rate
@pytest.mark.parametrize("shape", [(5, 5, 5), (9, 9, 9), (5, 9, 17), (17, 17, 17), (9, 17, 33)])
@pytest.mark.parametrize("precision", [0, 1])
def test_tail_at_the_finest_level(dmg, shape, precision):
    w = inputs.tissue(seed=7, shape=shape)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision)
    u = S.solve(T(w["q"]))
    cycles = S.last_info.cycles
    qb, Db, mb = S.vjp(u, T(w["w"]))
    S.close()
    assert cycles <= 16
    H = oracle.Hierarchy(w["D"], w["mu"], w["h"])
    ur, _, _ = H.solve(w["q"], rtol=1e-10)
    qr, Dr, mr, _ = H.vjp(ur, w["w"], rtol=1e-10)
    for got, ref in ((u, ur), (qb, qr), (Db, Dr), (mb, mr)):
        assert close(got, ref, TOL_CONV)
    # the fixed-cycle FP64 iterate equals the oracle's m-cycle iterate (the same V-cycle)
    if precision == 0:
        S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], fixed_cycles=3)
        u3 = S.solve(T(w["q"]))
        S.close()
        ref3, _, _ = H.solve(w["q"], fixed=3)
        assert close(u3, ref3, 1e-11)
