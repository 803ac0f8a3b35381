"""Prolongation fused into the first post-smoothing half-sweep (FP32 3D levels),
or, on large FP32 levels and in 2D, applied to the one colour that half-sweep
reads.

A red-black half-sweep never reads the old values of the colour it updates,
and the next half-sweep overwrites the other colour without reading it, so the
correction u += P e (Eq. 17) is needed only where the first post half-sweep
reads it. The fused kernel forms it there and never stores it; with the same
rounding steps as the separate prolongation, every result is bit for bit that
of split_prolong = 1 (k_prolong_add, then both half-sweeps)."""
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


def run_pair(dmg, w, split, **kw):
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1, split_prolong=split, **kw)
    n0 = dmg.dmg_launch_count(S.ctx)
    u = S.solve(T(w["q"]))
    cyc = S.last_info.cycles
    S.solve_launches = dmg.dmg_launch_count(S.ctx) - n0
    qb, Db, mb = S.vjp(u, T(w["w"]))
    du = S.jvp(u, T(w["q"][::-1].copy()), T(0.1 * w["D"]), T(0.1 * w["mu"]))
    launches = (S.solve_launches, dmg.dmg_launch_count(S.ctx) - n0)
    S.close()
    return (u, qb, Db, mb, du), cyc, launches


CASES = [
    ((33, 65, 129), {}),
    ((65, 65, 65), {"face_mean": 1}),
    ((33, 33, 33), {"symmetric": 1}),
    ((65, 33, 33), {"nu1": 1, "nu2": 1}),
    ((33, 33, 65), {"nu1": 3, "nu2": 3}),
    ((17, 129, 33), {"coarsen": 1}),
    ((129, 129, 129), {}),
    ((9, 9, 9), {}),
    ((5, 17, 65), {}),
]


@pytest.mark.parametrize("shape,kw", CASES)
def test_fused_is_bitwise_the_split_prolongation(dmg, shape, kw):
    w = inputs.tissue(seed=81, shape=shape)
    fused, cf, lf = run_pair(dmg, w, 0, **kw)
    split, cs, ls = run_pair(dmg, w, 1, **kw)
    assert cf == cs
    for a, b in zip(fused, split):
        assert torch.equal(a, b)
    assert lf[1] <= ls[1]


def test_fused_saves_launches(dmg):
    w = inputs.tissue(seed=82, shape=(129, 129, 129))
    _, cf, lf = run_pair(dmg, w, 0)
    _, cs, ls = run_pair(dmg, w, 1)
    assert cf == cs and lf[0] < ls[0] and lf[1] < ls[1]


def test_without_post_smoothing_nothing_is_fused(dmg):
    # nu2 = 0: the forward cycle has no post-smoothing to fuse into (the
    # transposed cycle of the adjoint post-smooths nu1 times and still fuses)
    w = inputs.tissue(seed=83, shape=(33, 33, 33))
    fused, _, lf = run_pair(dmg, w, 0, nu1=2, nu2=0)
    split, _, ls = run_pair(dmg, w, 1, nu1=2, nu2=0)
    for a, b in zip(fused, split):
        assert torch.equal(a, b)
    assert lf[0] == ls[0] and lf[1] < ls[1]


def test_fused_batch_with_masks(dmg):
    # samples converge at different steps, so later steps run masked
    w = inputs.vi_batch(33, 4, seed=84)
    w["q"][2] *= 1e-3
    w["D"][1] *= 4.0
    out = {}
    for split in (0, 1):
        S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1, split_prolong=split)
        u = S.solve(T(w["q"]))
        out[split] = (u,) + S.vjp(u, T(w["w"])) + (tuple(S.batch_info()[0]),)
        S.close()
    assert out[0][-1] == out[1][-1]
    for a, b in zip(out[0][:-1], out[1][:-1]):
        assert torch.equal(a, b)


def test_split_prolong_is_validated(dmg):
    w = inputs.tissue(seed=85, shape=(17, 17, 17))
    with pytest.raises(dmg.DMGError):
        dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1, split_prolong=2)


def test_one_colour_correction_on_large_levels(dmg):
    # 2 x 129^3 (2 x 129 x 129 x 160 padded vertices >= 2^22): the finest level
    # takes k_prolong_colour32 and a plain half-sweep; the results are those of
    # the full prolongation
    w = inputs.vi_batch(129, 2, seed=86)
    out = {}
    for split in (0, 1):
        S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1, split_prolong=split)
        u = S.solve(T(w["q"]))
        out[split] = (u,) + S.vjp(u, T(w["w"])) + (tuple(S.batch_info()[0]),)
        S.close()
    assert out[0][-1] == out[1][-1]
    for a, b in zip(out[0][:-1], out[1][:-1]):
        assert torch.equal(a, b)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("batch", [1, 3])
def test_2d_one_colour_correction_is_bitwise_the_full_one(dmg, precision, batch):
    # 2D post-smoothing starts from a correction of the colour its first
    # half-sweep reads (k_prolong_colour2); split_prolong = 1 applies the full
    # bilinear correction first
    ws = [inputs.tissue2d(seed=87 + b, shape=(65, 129)) for b in range(batch)]
    st = lambda k: T(np.stack([x[k] for x in ws])) if batch > 1 else T(ws[0][k])
    out = {}
    for split in (0, 1):
        S = dmg.Solver(st("D"), st("mu"), ws[0]["h"], dim=2, precision=precision, split_prolong=split)
        u = S.solve(st("q"))
        out[split] = (u,) + S.vjp(u, st("w"))
        S.close()
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)
