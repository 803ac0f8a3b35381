"""Host logic of the Python binding's Solver (paper_2608_00760_b300/dmg.py) with
dmg_setup stubbed: how array shapes map to grid dimensions and batch size, for
3D and 2D grids, and the errors for shapes that fit neither."""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2608_00760_b300 import dmg  # noqa: E402


@pytest.fixture
def captured(monkeypatch):
    seen = {}

    def setup(params, D, mu, stream=None):
        seen.update(nx=params.nx, ny=params.ny, nz=params.nz, batch=params.batch, h=params.h,
                    precision=params.precision, split_prolong=params.split_prolong)
        return dmg.DMG_OK, None

    monkeypatch.setattr(dmg, "dmg_setup", setup)
    return seen


@pytest.mark.parametrize("shape,dim,want", [
    ((9, 17, 33), 3, dict(nz=9, ny=17, nx=33, batch=1)),
    ((4, 9, 17, 33), 3, dict(nz=9, ny=17, nx=33, batch=4)),
    ((17, 33), 2, dict(nz=1, ny=17, nx=33, batch=1)),
    ((5, 17, 33), 2, dict(nz=1, ny=17, nx=33, batch=5)),
])
def test_shapes_map_to_grid_and_batch(captured, shape, dim, want):
    D = np.ones(shape)
    S = dmg.Solver(D, D, 0.5, dim=dim, precision=dmg.DMG_MIXED, split_prolong=1)
    assert {k: captured[k] for k in want} == want
    assert captured["h"] == 0.5 and captured["precision"] == dmg.DMG_MIXED and captured["split_prolong"] == 1
    assert S.batch == want["batch"] and S.n == int(np.prod(shape)) and S.shape == shape


@pytest.mark.parametrize("shape,dim", [((33,), 3), ((2, 3, 4, 5, 6), 3), ((17, 33), 3), ((2, 3, 17, 33), 2)])
def test_other_shapes_are_refused(captured, shape, dim):
    with pytest.raises(ValueError, match="expected a shape"):
        dmg.Solver(np.ones(shape), np.ones(shape), 0.5, dim=dim)


def test_a_failed_setup_raises_with_the_library_message(monkeypatch):
    monkeypatch.setattr(dmg, "dmg_setup", lambda *a, **k: (dmg.DMG_EINVAL, None))
    monkeypatch.setattr(dmg, "dmg_last_error", lambda ctx=None: "grid 9x9x9: something")
    with pytest.raises(dmg.DMGError, match="something") as e:
        dmg.Solver(np.ones((9, 9, 9)), np.ones((9, 9, 9)), 1.0)
    assert e.value.status == dmg.DMG_EINVAL
