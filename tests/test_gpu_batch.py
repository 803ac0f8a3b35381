"""Batched problems: B independent samples (each with its own D, mu, q and
cotangent) in one context, solved by one launch per kernel and level.

Checked through the C ABI: every sample's solution, adjoint, gradients and
tangent are bit for bit those of the same sample solved alone (so the
single-problem parity tests against the FP64 oracle carry over), each sample
stops at its own cycle count, the per-sample results match the oracle
directly, and the gradients of <w_b, u_b> pass central finite differences with
step 1e-6 on 20 random directions per sample, on small grids and on the
variational-inference workload (64 tissue samples on 129^3 vertices).
"""
import numpy as np
import pytest

import oracle
from paper_2608_00760_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_00760_b300 import build, dmg as m
    build.build()
    return m


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def mixed_batch(shape, seed):
    """Four samples that need different cycle counts: a tissue sample, one with
    strong absorption (few cycles), one with a zero right-hand side (none) and a
    high-contrast diffusion field (more cycles)."""
    ws = [inputs.tissue(seed=(seed, b), shape=shape) for b in range(4)]
    ws[1]["mu"] = ws[1]["mu"] * 1e5
    ws[2]["q"] = np.zeros(shape)
    rng = np.random.default_rng(seed)
    ws[3]["D"] = np.exp(inputs.grf(shape, 0.5, 3.0, 1.5, rng))
    out = {k: np.stack([w[k] for w in ws]) for k in ("D", "mu", "q", "w", "dq", "dD", "dmu")}
    out.update(h=0.5, shape=(4,) + tuple(shape))
    return out


SHAPES = [(33, 33, 33), (17, 33, 65), (9, 17, 33)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", [0, 1])
def test_batch_is_bitwise_the_single_solves(dmg, shape, precision):
    w = mixed_batch(shape, seed=31)
    B = w["shape"][0]
    Sb = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision)
    ub = Sb.solve(T(w["q"]))
    cyc_b, rel_b = Sb.batch_info()
    worst = Sb.last_info
    qb, Db, mb = Sb.vjp(ub, T(w["w"]))
    cyc_vb, _ = Sb.batch_info()
    dub = Sb.jvp(ub, T(w["dq"]), T(w["dD"]), T(w["dmu"]))
    single_cycles = []
    for b in range(B):
        S = dmg.Solver(T(w["D"][b]), T(w["mu"][b]), w["h"], precision=precision)
        u = S.solve(T(w["q"][b]))
        single_cycles.append(S.last_info.cycles)
        assert torch.equal(ub[b], u), b
        assert cyc_b[b] == S.last_info.cycles and rel_b[b] == S.last_info.rel_residual
        q1, D1, m1 = S.vjp(u, T(w["w"][b]))
        assert cyc_vb[b] == S.last_info.cycles
        assert torch.equal(qb[b], q1) and torch.equal(Db[b], D1) and torch.equal(mb[b], m1), b
        du = S.jvp(u, T(w["dq"][b]), T(w["dD"][b]), T(w["dmu"][b]))
        assert torch.equal(dub[b], du), b
        S.close()
    # the samples really stopped at different counts, and the report is the worst
    assert single_cycles[2] == 0 and len(set(single_cycles)) >= 3
    assert worst.cycles == max(single_cycles) and worst.rel_residual == max(rel_b)
    assert not ub[2].any()
    Sb.close()


def test_batch_count_matched_adjoint_is_bitwise(dmg):
    w = mixed_batch((17, 17, 33), seed=32)
    Sb = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    ub = Sb.solve(T(w["q"]))
    qb, Db, mb = Sb.vjp(ub, T(w["w"]), cycles=5)
    for b in range(4):
        S = dmg.Solver(T(w["D"][b]), T(w["mu"][b]), w["h"])
        q1, D1, m1 = S.vjp(ub[b].contiguous(), T(w["w"][b]), cycles=5)
        assert torch.equal(qb[b], q1) and torch.equal(Db[b], D1) and torch.equal(mb[b], m1), b
        S.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_oracle_per_sample(dmg, precision):
    w = inputs.vi_batch(33, 3, seed=33, keys=("D", "mu", "q", "w"))
    Sb = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision)
    ub = Sb.solve(T(w["q"]))
    qb, Db, mb = Sb.vjp(ub, T(w["w"]))
    for b in range(3):
        H = oracle.Hierarchy(w["D"][b], w["mu"][b], w["h"])
        ur, _, _ = H.solve(w["q"][b], rtol=1e-10)
        assert np.linalg.norm(ub[b].cpu().numpy() - ur) <= 1e-8 * np.linalg.norm(ur)
        refs = H.vjp(ur, w["w"][b], rtol=1e-10)[:3]
        for got, ref in zip((qb, Db, mb), refs):
            assert np.linalg.norm(got[b].cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    # dmg_residual reports one pair per sample
    r = Sb.residual(T(w["q"]), ub)
    assert len(r) == 3 and all(rn <= 1e-10 * qn for rn, qn in r)
    Sb.close()


def fd_check(dmg, D, mu, q, wv, h, ndir, seed, grads=None, tol=1e-6):
    """Central differences (step 1e-6) of L_b = <w_b, u_b> along ndir random
    directions per sample against the gradients (qbar, Dbar, mubar) of the
    converged solve: `grads` if given (e.g. from the mixed-precision autograd
    path), else dmg_vjp of an FP64 solve at rtol 1e-13. The perturbed solves run
    a fixed number of FP64 cycles, a few more than an FP64 solve to rtol 1e-13
    needs, so that both sides of a difference run the same iteration (a map
    linear in q and smooth in D, mu). Each directional derivative must agree to
    `tol` relative (to its size, or to 1e-6 of the sum of absolute products
    where it cancels). Returns the worst relative mismatch over samples and
    directions."""
    S = dmg.Solver(D, mu, h, rtol=1e-13)
    u = S.solve(q)
    fixed = max(S.batch_info()[0]) + 3
    qb, Db, mb = S.vjp(u, wv) if grads is None else grads
    S.close()
    del u
    gen = torch.Generator(device="cuda").manual_seed(seed)
    eps, worst = 1e-6, 0.0

    def losses(Dp, mp, qp):
        Sp = dmg.Solver(Dp, mp, h, fixed_cycles=fixed)
        up = Sp.solve(qp)
        Sp.close()
        return (up * wv).flatten(1).sum(1)

    def dot(a, b):
        return (a * b).flatten(1).sum(1)

    for _ in range(ndir):
        dq = torch.randn(D.shape, generator=gen, device="cuda", dtype=torch.float64)
        dD = 0.1 * D * torch.randn(D.shape, generator=gen, device="cuda", dtype=torch.float64)
        dm = 0.1 * mu * torch.randn(D.shape, generator=gen, device="cuda", dtype=torch.float64)
        fd = (losses(D + eps * dD, mu + eps * dm, q + eps * dq) -
              losses(D - eps * dD, mu - eps * dm, q - eps * dq)) / (2 * eps)
        an = dot(qb, dq) + dot(Db, dD) + dot(mb, dm)
        scale = dot(qb.abs(), dq.abs()) + dot(Db.abs(), dD.abs()) + dot(mb.abs(), dm.abs())
        err = ((an - fd).abs() / torch.maximum(an.abs(), 1e-6 * scale)).max().item()
        worst = max(worst, err)
        assert err <= tol, (err, an.tolist(), fd.tolist())
    return worst


# Tolerance of the finite-difference check of gradients from solves converged
# to relative residual 1e-10 (the benchmark's setting). The residual bound
# leaves an error in u and lambda of up to cond(A) * 1e-10 relative; for the
# tissue operator at 129^3 (h = 0.5 mm, D ~ 0.33 mm, mu_a ~ 0.01 / mm) the
# condition number is about 12 D/h^2 / (mu_a + 3 pi^2 D / L^2) ~ 1.3e3, so a
# directional derivative may be off by ~1e-7 relative, and more where its
# terms cancel. 1e-5 bounds that with a margin of ten.
TOL_FD_RTOL10 = 1e-5


def mixed_autograd_grads(dmg, D, mu, q, wv, h, rtol=1e-10):
    """The VI step as the benchmark times it: a mixed-precision solver (FP32
    inner V-cycles, FP64 refinement, rtol 1e-10 unless given),
    u = DMGSolve.apply(q, D, mu), loss = sum_b <w_b, u_b>, loss.backward().
    Returns (q.grad, D.grad, mu.grad)."""
    from paper_2608_00760_b300 import autograd
    S = dmg.Solver(D, mu, h, precision=dmg.DMG_MIXED, rtol=rtol, inner_cycles=3)
    Dg, mg, qg = (x.detach().clone().requires_grad_(True) for x in (D, mu, q))
    u = autograd.DMGSolve.apply(qg, Dg, mg, S, False)
    (u * wv).sum().backward()
    cyc, rel = S.batch_info()
    assert all(r <= rtol for r in rel)
    S.close()
    return qg.grad, Dg.grad, mg.grad


def test_batch_gradients_pass_finite_differences(dmg):
    w = inputs.vi_batch(17, 4, seed=34)
    fd_check(dmg, T(w["D"]), T(w["mu"]), T(w["q"]), T(w["w"]), w["h"], ndir=20, seed=34)


@pytest.mark.parametrize("rtol,tol", [(1e-13, 1e-6), (1e-10, TOL_FD_RTOL10)])
def test_vi_workload_gradients_pass_finite_differences(dmg, rtol, tol):
    # the variational-inference step at full size, 64 samples x 129^3, on the
    # path the benchmark times: mixed precision through the autograd Function,
    # at the benchmark's tolerance and at a tight one
    w = inputs.vi_batch(129, 64, seed=35)
    D, mu, q, wv = T(w["D"]), T(w["mu"]), T(w["q"]), T(w["w"])
    del w
    g = mixed_autograd_grads(dmg, D, mu, q, wv, 0.5, rtol=rtol)
    fd_check(dmg, D, mu, q, wv, 0.5, ndir=20, seed=35, grads=g, tol=tol)


@pytest.mark.parametrize("rtol,tol", [(1e-13, 1e-6), (1e-10, TOL_FD_RTOL10)])
def test_mixed_autograd_batch_gradients_pass_finite_differences(dmg, rtol, tol):
    w = inputs.vi_batch(17, 4, seed=37)
    D, mu, q, wv = T(w["D"]), T(w["mu"]), T(w["q"]), T(w["w"])
    g = mixed_autograd_grads(dmg, D, mu, q, wv, w["h"], rtol=rtol)
    fd_check(dmg, D, mu, q, wv, w["h"], ndir=20, seed=37, grads=g, tol=tol)


def test_mixed_autograd_batch_gradients_match_oracle(dmg):
    # 4 samples x 33^3, mixed precision through the autograd Function: every
    # sample's q, D and mu gradients against the FP64 oracle's pull-back of the
    # same sample (relative L2 and entry by entry <= 1e-8)
    w = inputs.vi_batch(33, 4, seed=38, keys=("D", "mu", "q", "w"))
    qg, Dg, mg = mixed_autograd_grads(dmg, T(w["D"]), T(w["mu"]), T(w["q"]), T(w["w"]), w["h"])
    for b in range(4):
        H = oracle.Hierarchy(w["D"][b], w["mu"][b], w["h"])
        ur, _, _ = H.solve(w["q"][b], rtol=1e-10)
        refs = H.vjp(ur, w["w"][b], rtol=1e-10)[:3]
        for got, ref in zip((qg, Dg, mg), refs):
            g = got[b].cpu().numpy()
            assert np.linalg.norm(g - ref) <= 1e-8 * np.linalg.norm(ref), b
            assert np.max(np.abs(g - ref)) <= 1e-8 * np.max(np.abs(ref)), b


def test_batch_shape_limits(dmg):
    # batch * nz must fit the grid's z dimension; batch >= 1
    p = dmg.dmg_default_params(nx=17, ny=17, nz=17, h=1.0, batch=0)
    D = torch.ones(17 ** 3, dtype=torch.float64, device="cuda")
    st, ctx = dmg.dmg_setup(p, D, D)
    assert st == dmg.DMG_EINVAL and ctx is None
    p = dmg.dmg_default_params(nx=17, ny=17, nz=17, h=1.0, batch=4000)
    st, ctx = dmg.dmg_setup(p, None, None)
    assert st == dmg.DMG_EINVAL and "65535" in dmg.dmg_last_error(None)


def test_batch_backward_through_autograd_function(dmg):
    # the VI step as a sampler runs it: forward of every sample, then
    # loss.backward() through the torch.autograd.Function; each sample's
    # gradients are bitwise those of the same sample through autograd alone
    from paper_2608_00760_b300 import autograd
    w = inputs.vi_batch(17, 3, seed=36)
    Tg = lambda a: T(a).requires_grad_(True)
    D, mu, q = Tg(w["D"]), Tg(w["mu"]), Tg(w["q"])
    u = autograd.solve(q, D, mu, w["h"], precision=1)
    (u * T(w["w"])).sum().backward()
    for b in range(3):
        Db, mub, qb = Tg(w["D"][b]), Tg(w["mu"][b]), Tg(w["q"][b])
        ub = autograd.solve(qb, Db, mub, w["h"], precision=1)
        (ub * T(w["w"][b])).sum().backward()
        assert torch.equal(u[b].detach(), ub.detach())
        for got, ref in ((q.grad[b], qb.grad), (D.grad[b], Db.grad), (mu.grad[b], mub.grad)):
            assert torch.equal(got, ref), b
    autograd.clear_cache()
