"""dmg_solve_vjp (forward solve and converged pull-back in one call, host
transfers overlapped on a second stream, the adjoint solve beside the forward
one in the twin context) gives bit for bit the results of dmg_solve followed by
dmg_vjp, with host or device arrays, FP64 or mixed, single problems, batches
and 2D grids; so does dmg_solve_vjp_many over a stream of pairs."""
import numpy as np
import pytest

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


CASES = [
    ("tissue33", lambda: inputs.tissue(33, seed=111), 3),
    ("batch", lambda: inputs.vi_batch(17, 3, seed=112), 3),
    ("2d", lambda: inputs.tissue2d(seed=113, shape=(65, 129)), 2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("host", [False, True])
def test_solve_vjp_is_bitwise_solve_then_vjp(dmg, case, precision, host):
    _, make, dim = case
    w = make()
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision, dim=dim)
    q, wv = T(w["q"]), T(w["w"])
    u = S.solve(q)
    ref = (u,) + S.vjp(u, wv)
    if host:
        qh, wh = (np.ascontiguousarray(w[k]) for k in ("q", "w"))
        outs = [np.zeros(q.shape) for _ in range(4)]
        st = dmg.dmg_solve_vjp(S.ctx, qh, wh, *outs, n=S.n)
        got = [torch.from_numpy(o).cuda() for o in outs]
    else:
        got = [torch.empty_like(q) for _ in range(4)]
        fi, ai = dmg.dmg_info(), dmg.dmg_info()
        st = dmg.dmg_solve_vjp(S.ctx, q, wv, *got, fi, ai, n=S.n)
        assert fi.rel_residual <= 1e-10 and ai.rel_residual <= 1e-10
    assert st == dmg.DMG_OK
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    S.close()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("where", ["host", "device", "mixed"])
@pytest.mark.parametrize("twin", [0, 1])
def test_many_pairs_are_bitwise_single_pairs(dmg, case, precision, where, twin):
    # dmg_solve_vjp_many over four pairs (different sources and cotangents, as a
    # sampler streams them): each pair's outputs equal dmg_solve_vjp on that
    # pair, with host arrays (transfers overlapped), device arrays, or both
    # kinds; the adjoint solves in the twin context or after the forward ones
    _, make, dim = case
    w = make()
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision, dim=dim, twin_adjoint=twin)
    rng = np.random.default_rng(7)
    pairs = [(w["q"] * (1.0 + 0.5 * p), w["w"] * rng.standard_normal(w["q"].shape)) for p in range(4)]
    ref = []
    for qa, wa in pairs:
        outs = [torch.empty(w["q"].shape, dtype=torch.float64, device="cuda") for _ in range(4)]
        assert dmg.dmg_solve_vjp(S.ctx, T(qa), T(wa), *outs, n=S.n) == dmg.DMG_OK
        ref.append(outs)

    def arr(a, i):
        dev = where == "device" or (where == "mixed" and i % 2 == 1)
        return T(a) if dev else np.ascontiguousarray(a)

    qs = [arr(qa, i) for i, (qa, _) in enumerate(pairs)]
    ws = [arr(wa, i) for i, (_, wa) in enumerate(pairs)]
    outs = [[arr(np.zeros(w["q"].shape), i) for i in range(4)] for _ in range(4)]
    fi, ai = (dmg.dmg_info * 4)(), (dmg.dmg_info * 4)()
    st = dmg.dmg_solve_vjp_many(S.ctx, qs, ws, *outs, info_fwd=fi, info_adj=ai, n=S.n)
    assert st == dmg.DMG_OK, dmg.dmg_last_error(S.ctx)
    for i in range(4):
        assert fi[i].rel_residual <= 1e-10 and ai[i].rel_residual <= 1e-10
        for k in range(4):
            got = outs[k][i]
            got = got if torch.is_tensor(got) else torch.from_numpy(got).cuda()
            assert torch.equal(got, ref[i][k]), (i, k)
    # outputs may be skipped
    assert dmg.dmg_solve_vjp_many(S.ctx, qs[:2], ws[:2], None, None, outs[2][:2], None, n=S.n) == dmg.DMG_OK
    for i in range(2):
        got = outs[2][i]
        got = got if torch.is_tensor(got) else torch.from_numpy(got).cuda()
        assert torch.equal(got, ref[i][2])
    S.close()


def test_many_pairs_argument_errors(dmg):
    w = inputs.tissue(17, seed=114)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    assert dmg.dmg_solve_vjp_many(S.ctx, [T(w["q"])], [None], n=S.n) == dmg.DMG_EINVAL
    assert dmg.lib().dmg_solve_vjp_many(S.ctx, 0, None, None, None, None, None, None, None, None, None) == \
        dmg.DMG_EINVAL
    S.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_twin_lane_is_bitwise_one_lane(dmg, precision):
    # the adjoint solve in the twin context (twin_adjoint = 1, the default) and in
    # the context itself after the forward one (twin_adjoint = 0)
    w = inputs.tissue(33, seed=114)
    D, mu, q, wv = (T(w[k]) for k in ("D", "mu", "q", "w"))
    A = dmg.Solver(D, mu, w["h"], precision=precision)
    B = dmg.Solver(D, mu, w["h"], precision=precision, twin_adjoint=0)
    bytes_before = dmg.dmg_device_bytes(A.ctx)
    outs = {}
    for name, S in (("twin", A), ("one", B)):
        got = [torch.empty_like(q) for _ in range(4)]
        fi, ai = dmg.dmg_info(), dmg.dmg_info()
        for _ in range(2):   # the first call creates the twin, the second reuses it
            assert dmg.dmg_solve_vjp(S.ctx, q, wv, *got, fi, ai, n=S.n) == dmg.DMG_OK
        outs[name] = (got, fi.cycles, ai.cycles)
    for a, b in zip(outs["twin"][0], outs["one"][0]):
        assert torch.equal(a, b)
    assert outs["twin"][1:] == outs["one"][1:]
    # the twin holds a second copy of the context's device arrays
    assert dmg.dmg_device_bytes(A.ctx) >= 2 * bytes_before - 4096
    assert dmg.dmg_device_bytes(B.ctx) == bytes_before
    # new coefficients reach the twin as well
    w2 = inputs.tissue(33, seed=115)
    D2, mu2 = T(w2["D"]), T(w2["mu"])
    A.set_coefficients(D2, mu2)
    got = [torch.empty_like(q) for _ in range(4)]
    assert dmg.dmg_solve_vjp(A.ctx, q, wv, *got, n=A.n) == dmg.DMG_OK
    F = dmg.Solver(D2, mu2, w["h"], precision=precision, twin_adjoint=0)
    ref = [torch.empty_like(q) for _ in range(4)]
    assert dmg.dmg_solve_vjp(F.ctx, q, wv, *ref, n=F.n) == dmg.DMG_OK
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    for S in (A, B, F):
        S.close()


def test_twin_falls_back_to_one_lane_without_memory(dmg):
    # the twin's first allocation fails (injected): the pair runs in one lane,
    # with the same results; a later call builds the twin
    w = inputs.tissue(33, seed=116)
    D, mu, q, wv = (T(w[k]) for k in ("D", "mu", "q", "w"))
    ref = dmg.Solver(D, mu, w["h"], precision=1, twin_adjoint=0)
    want = [torch.empty_like(q) for _ in range(4)]
    assert dmg.dmg_solve_vjp(ref.ctx, q, wv, *want, n=ref.n) == dmg.DMG_OK
    S = dmg.Solver(D, mu, w["h"], precision=1)
    alone = dmg.dmg_device_bytes(S.ctx)
    got = [torch.empty_like(q) for _ in range(4)]
    dmg.dmg_debug_fail_alloc(1)
    try:
        st = dmg.dmg_solve_vjp(S.ctx, q, wv, *got, n=S.n)
    finally:
        dmg.dmg_debug_fail_alloc(0)
    assert st == dmg.DMG_OK, dmg.dmg_last_error(S.ctx)
    assert dmg.dmg_device_bytes(S.ctx) == alone   # no twin
    for a, b in zip(got, want):
        assert torch.equal(a, b)
    assert dmg.dmg_solve_vjp(S.ctx, q, wv, *got, n=S.n) == dmg.DMG_OK
    assert dmg.dmg_device_bytes(S.ctx) > alone    # the twin now exists
    for a, b in zip(got, want):
        assert torch.equal(a, b)
    S.close()
    ref.close()
