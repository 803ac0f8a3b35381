"""The tiled gradient kernels (arithmetic face mean: each face's differences
formed once per tile and shared, outputs on the device written straight in
the caller's layout) give bit for bit the D-bar and mu-bar of the per-vertex
kernels, which form every face's differences on both of its sides; through
dmg_solve_vjp with device and host outputs and through the stream of pairs,
on 3D grids (odd extents, partial tiles), batches and 2D grids."""
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
    ("tissue33", lambda: inputs.tissue(33, seed=121), 3),
    ("odd", lambda: inputs.tissue(seed=122, shape=(45, 37, 29)), 3),
    ("batch", lambda: inputs.vi_batch(17, 3, seed=123), 3),
    ("2d", lambda: inputs.tissue2d(seed=124, shape=(65, 97)), 2),
]


def pair_outputs(dmg, S, w, host):
    if host:
        outs = [np.zeros(w["q"].shape) for _ in range(4)]
        st = dmg.dmg_solve_vjp(S.ctx, np.ascontiguousarray(w["q"]), np.ascontiguousarray(w["w"]), *outs, n=S.n)
        outs = [torch.from_numpy(o).cuda() for o in outs]
    else:
        outs = [torch.empty(w["q"].shape, dtype=torch.float64, device="cuda") for _ in range(4)]
        st = dmg.dmg_solve_vjp(S.ctx, T(w["q"]), T(w["w"]), *outs, n=S.n)
    assert st == dmg.DMG_OK, dmg.dmg_last_error(S.ctx)
    return outs


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("precision", [0, 1])
def test_tiled_gradient_is_bitwise_per_vertex(dmg, case, precision):
    _, make, dim = case
    w = make()
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision, dim=dim)
    tiled = {h: pair_outputs(dmg, S, w, h) for h in (False, True)}
    dmg.dmg_debug_grad_per_vertex(1)
    try:
        per_vertex = {h: pair_outputs(dmg, S, w, h) for h in (False, True)}
    finally:
        dmg.dmg_debug_grad_per_vertex(0)
    for h in (False, True):
        for k in range(4):
            assert torch.equal(tiled[h][k], per_vertex[h][k]), (h, k)
    assert bool(torch.isfinite(tiled[False][2]).all()) and float(tiled[False][2].abs().max()) > 0
    S.close()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_stream_of_pairs_gradients_are_bitwise_per_vertex(dmg, case):
    # host outputs of even pairs (the tiled kernel writes their staging slots),
    # device outputs of odd ones
    _, make, dim = case
    w = make()
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1, dim=dim)
    rng = np.random.default_rng(5)
    pairs = [(w["q"] * (1.0 + 0.25 * p), w["w"] * rng.standard_normal(w["q"].shape)) for p in range(3)]

    def run():
        arr = lambda a, i: T(a) if i % 2 else np.ascontiguousarray(a)
        outs = [[arr(np.zeros(w["q"].shape), i) for i in range(3)] for _ in range(4)]
        st = dmg.dmg_solve_vjp_many(S.ctx, [arr(p[0], i) for i, p in enumerate(pairs)],
                                    [arr(p[1], i) for i, p in enumerate(pairs)], *outs, n=S.n)
        assert st == dmg.DMG_OK, dmg.dmg_last_error(S.ctx)
        return [[o if torch.is_tensor(o) else torch.from_numpy(o).cuda() for o in col] for col in outs]

    tiled = run()
    dmg.dmg_debug_grad_per_vertex(1)
    try:
        per_vertex = run()
    finally:
        dmg.dmg_debug_grad_per_vertex(0)
    for k in range(4):
        for i in range(3):
            assert torch.equal(tiled[k][i], per_vertex[k][i]), (k, i)
    S.close()
