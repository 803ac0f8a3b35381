"""Serving: forward, JVP and VJP requests of two grid shapes arrive while others
run, are admitted into slots of per-shape pools as slots free up, and advance
together step by step. Every served result must match the FP64 CPU oracle on
the request's own coefficients and inputs (relative L2 and entry by entry
<= 1e-8, both sides at relative residual 1e-10) and be bit for bit the result
of the same request run alone on a context of batch 1; a request with invalid
coefficients or non-finite input fails alone without disturbing the others.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(17, 17, 17), (9, 17, 33)]


@pytest.fixture(scope="module")
def serve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_00760_b300 import build, serve as m
    build.build()
    return m


TOL_CONV = 1e-8


def oracle_outputs(req, h=0.5):
    """The request's outputs from the FP64 oracle, on the same inputs (drawn
    again from the request's seed) and the same stopping rule."""
    x = {k: v.detach().cpu().numpy() for k, v in req.make_inputs("cuda").items()}
    H = oracle.Hierarchy(x["D"], x["mu"], h)
    u, _, _ = H.solve(x["q"], rtol=1e-10)
    if req.kind == "fwd":
        return {"u": u}
    if req.kind == "jvp":
        du, _ = H.jvp(u, x["dq"], x["dD"], x["dmu"], rtol=1e-10)
        return {"u": u, "du": du}
    qb, Db, mb, _ = H.vjp(u, x["w"], rtol=1e-10)
    return {"u": u, "qbar": qb, "Dbar": Db, "mubar": mb}


def assert_close(got, ref, tol, what):
    got = got.detach().cpu().numpy()
    nb, mb = np.linalg.norm(ref), np.max(np.abs(ref))
    e2 = np.linalg.norm(got - ref) / (nb if nb > 0 else 1.0)
    einf = np.max(np.abs(got - ref)) / (mb if mb > 0 else 1.0)
    assert e2 <= tol and einf <= tol, (what, e2, einf)


def overlapped(served, shape):
    """Some request of this pool was admitted while another one of the same
    pool was between its admission and completion."""
    iv = sorted(r.pool_steps for r in served if r.shape == shape)
    return any(a2 > a1 and a2 < b1 for (a1, b1), (a2, _) in zip(iv, iv[1:]))


@pytest.mark.parametrize("precision", [0, 1])
def test_served_results_equal_alone(serve, precision):
    from paper_2608_00760_b300 import dmg
    reqs = serve.poisson_stream(24, rate=2000.0, shapes=SHAPES, seed=11)
    server = serve.Server(SHAPES, slots={s: 3 for s in SHAPES}, params=dict(precision=precision),
                          budget_bytes=16e9)
    try:
        served, stats = server.run(reqs)
    finally:
        server.close()
    assert stats["requests"] == 24 and stats["ok"] == 24
    assert {r.kind for r in served} == {"fwd", "jvp", "vjp"}
    for s in SHAPES:
        assert overlapped(served, s), s
    for r in served:
        ref = oracle_outputs(r)
        assert set(ref) == set(r.outputs)
        for k in ref:
            assert_close(r.outputs[k], ref[k], TOL_CONV, (r.rid, r.kind, r.shape, k))
        alone = serve.run_alone(r, params=dict(precision=precision))
        assert set(alone) == set(r.outputs)
        for k in alone:
            assert torch.equal(r.outputs[k], alone[k]), (r.rid, r.kind, k)
        assert r.status == dmg.DMG_OK and all(x <= 1e-10 for x in r.rel)


def test_failed_requests_are_isolated(serve):
    from paper_2608_00760_b300 import dmg, inputs
    good = serve.poisson_stream(6, rate=1000.0, shapes=SHAPES[:1], seed=12)

    def bad_coeffs(device):
        x = inputs.tissue_torch(SHAPES[0], 5, device=device, keys=("D", "mu", "q"))
        x["D"] = -x["D"]
        return x

    def nan_source(device):
        x = inputs.tissue_torch(SHAPES[0], 6, device=device, keys=("D", "mu", "q"))
        x["q"][8, 8, 8] = float("nan")
        return x

    bad = [serve.Request(rid=100, kind="fwd", shape=SHAPES[0], make_inputs=bad_coeffs, arrival=0.0),
           serve.Request(rid=101, kind="fwd", shape=SHAPES[0], make_inputs=nan_source, arrival=0.0)]
    server = serve.Server(SHAPES[:1], slots={SHAPES[0]: 4}, budget_bytes=8e9)
    try:
        served, stats = server.run(bad + good)
    finally:
        server.close()
    by = {r.rid: r for r in served}
    assert by[100].status == dmg.DMG_EINVAL and by[101].status == dmg.DMG_ENAN
    for r in good:
        s = by[r.rid]
        assert s.status == dmg.DMG_OK
        alone = serve.run_alone(s)
        assert all(torch.equal(s.outputs[k], alone[k]) for k in alone)


def test_budget_limits_admission(serve):
    # room for the pool and one request's tensors: requests run one after another
    reqs = serve.poisson_stream(4, rate=1e4, shapes=SHAPES[:1], mix=(("fwd", 1),), seed=13)
    probe = serve.Server(SHAPES[:1], slots={SHAPES[0]: 4}, budget_bytes=8e9)
    pool_bytes = probe.pool_bytes
    probe.close()
    server = serve.Server(SHAPES[:1], slots={SHAPES[0]: 4}, budget_bytes=pool_bytes + 1.5 * reqs[0].io_bytes())
    try:
        served, stats = server.run(reqs)
    finally:
        server.close()
    assert stats["ok"] == 4
    iv = sorted(r.pool_steps for r in served)
    assert all(a2 >= b1 for (_, b1), (a2, _) in zip(iv, iv[1:]))


PYRAMID = [(65, 65, 65), (33, 33, 33)]


@pytest.mark.parametrize("precision", [0, 1])
def test_pyramid_pool_batches_levels_across_shapes(serve, precision):
    # 65^3 and 33^3 requests share one pyramid pool: the 65^3 requests' second
    # level and the 33^3 requests' finest level run in the same launches. Every
    # result matches the oracle and is bit for bit the request alone.
    from paper_2608_00760_b300 import dmg
    reqs = serve.poisson_stream(12, rate=2000.0, shapes=PYRAMID, seed=21)
    server = serve.Server(PYRAMID, slots={s: 3 for s in PYRAMID}, params=dict(precision=precision),
                          budget_bytes=16e9, pyramid=True)
    try:
        pools = server.unique_pools()
        assert len(pools) == 1 and pools[0].chain == PYRAMID and pools[0].slots == 6
        served, stats = server.run(reqs)
    finally:
        server.close()
    assert stats["ok"] == 12 and {r.shape for r in served} == set(PYRAMID)
    for r in served:
        ref = oracle_outputs(r)
        for k in ref:
            assert_close(r.outputs[k], ref[k], TOL_CONV, (r.rid, r.kind, r.shape, k))
        alone = serve.run_alone(r, params=dict(precision=precision))
        for k in alone:
            assert torch.equal(r.outputs[k], alone[k]), (r.rid, r.kind, r.shape, k)
        assert r.status == dmg.DMG_OK


def test_pyramid_refusals(serve):
    from paper_2608_00760_b300 import dmg
    # a 17^3 level lies inside the FP32 small-level tail: refused, the server
    # falls back to one pool per shape
    p = dmg.dmg_default_params(nx=33, ny=33, nz=33, h=0.5, precision=dmg.DMG_MIXED)
    st, ctx = dmg.dmg_setup_pyramid(p, [2, 2])
    assert st == dmg.DMG_EINVAL and ctx is None and "tail" in dmg.dmg_last_error(None)
    shapes = [(33, 33, 33), (17, 17, 17)]
    server = serve.Server(shapes, slots={s: 1 for s in shapes}, params=dict(precision=1), budget_bytes=8e9,
                          pyramid=True)
    assert len(server.unique_pools()) == 2
    server.close()
    # whole-context calls are refused on a pyramid
    p = dmg.dmg_default_params(nx=65, ny=65, nz=65, h=0.5)
    st, ctx = dmg.dmg_setup_pyramid(p, [1, 1])
    assert st == dmg.DMG_OK
    q = torch.zeros((65, 65, 65), dtype=torch.float64, device="cuda")
    assert dmg.dmg_solve(ctx, q, torch.empty_like(q), n=q.numel()) == dmg.DMG_EINVAL
    assert "pyramid" in dmg.dmg_last_error(ctx)
    dmg.dmg_destroy(ctx)
