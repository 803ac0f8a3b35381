"""The in-project tile autotuner: dmg_setup with autotune = 1 times the block
shapes of the colour kernels per level and keeps the fastest. The shape only
changes how vertices map to threads, so results are bit for bit those of the
default shape; chosen shapes are valid, and new results are appended to the
file that DMG_TUNE_CACHE names."""
import numpy as np
import pytest

from paper_2608_00760_b300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VALID = {(32, 8), (32, 4), (32, 2), (64, 4), (64, 2), (128, 2), (128, 1), (16, 16), (16, 8), (8, 16), (8, 32)}


@pytest.fixture(scope="module")
def dmg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2608_00760_b300 import build, dmg as m
    build.build()
    return m


def T(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision", [0, 1])
def test_autotuned_results_are_bitwise_the_default(dmg, precision, tmp_path, monkeypatch):
    monkeypatch.setenv("DMG_TUNE_CACHE", str(tmp_path / "tiles.txt"))
    w = inputs.tissue(seed=71, shape=(33, 65, 129 if precision else 65))
    out = {}
    for tune in (0, 1):
        S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=precision, autotune=tune)
        u = S.solve(T(w["q"]))
        out[tune] = (u,) + S.vjp(u, T(w["w"]))
        tiles = S.tiles(fp32=bool(precision))
        assert all(t in VALID for t in tiles)
        if not tune:   # the defaults: 32 x 8 (FP64); FP32 pair kernels by the level's width
            if precision:
                widths = [(s[2] - 2) // 4 + 1 for s in S.levels()]
                assert tiles == [(32, 4) if p > 16 else ((16, 8) if p > 8 else (8, 16)) for p in widths]
            else:
                assert all(t == (32, 8) for t in tiles)
        S.close()
    for a, b in zip(out[0], out[1]):
        assert torch.equal(a, b)


def test_tuned_batch_and_cache_file(dmg, tmp_path, monkeypatch):
    path = tmp_path / "tiles.txt"
    monkeypatch.setenv("DMG_TUNE_CACHE", str(path))
    w = inputs.vi_batch(33, 3, seed=72)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1, autotune=1)
    ub = S.solve(T(w["q"]))
    S.close()
    S0 = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1)
    assert torch.equal(ub, S0.solve(T(w["q"])))
    S0.close()
    lines = path.read_text().split("\n") if path.exists() else []
    # the entries of this batch shape were tuned here (first time in the process) and appended
    assert any(":33x33x33:b3:" in l for l in lines)
