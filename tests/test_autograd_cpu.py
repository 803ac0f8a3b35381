"""Host logic of the torch.autograd integration (paper_2608_00760_b300/autograd.py)
on CPU tensors, with a fake of dmg.Solver that does plain arithmetic: the
context cache (hits, invalidation by in-place changes, eviction that never
destroys a context a live graph still needs), gradient routing and the
recompute option."""
import gc
import weakref

import pytest

torch = pytest.importorskip("torch")

from paper_2608_00760_b300 import autograd  # noqa: E402


class FakeSolver:
    made = []

    def __init__(self, D, mu, h, **params):
        self.D, self.mu, self.h, self.params = D.clone(), mu.clone(), h, params
        self.closed = False
        self.solves = 0
        self.last_need = None
        FakeSolver.made.append(weakref.ref(self))

    def _live(self):
        assert not self.closed, "a closed solver was used"

    def solve(self, q):
        self._live()
        self.solves += 1
        return q / (self.D + self.mu)          # a diagonal "operator" A = D + mu

    def vjp(self, u, w, need=(True, True, True)):
        self._live()
        self.last_need = need
        lam = w / (self.D + self.mu)
        g = -lam * u
        return (lam if need[0] else None, g if need[1] else None, g if need[2] else None)

    def jvp(self, u, dq=None, dD=None, dmu=None):
        self._live()
        rhs = torch.zeros_like(self.D) if dq is None else dq.clone()
        if dD is not None:
            rhs = rhs - dD * u
        if dmu is not None:
            rhs = rhs - dmu * u
        return rhs / (self.D + self.mu)

    def close(self):
        self.closed = True

    def __del__(self):
        self.closed = True


@pytest.fixture(autouse=True)
def fake(monkeypatch):
    monkeypatch.setattr(autograd.dmg, "Solver", FakeSolver)
    monkeypatch.setattr(autograd, "_cache", autograd._Cache(size=3))
    FakeSolver.made.clear()
    yield
    autograd.clear_cache()


def fields(seed, n=5, grad=True):
    g = torch.Generator().manual_seed(seed)
    D = (1.0 + torch.rand((n, n, n), generator=g, dtype=torch.float64)).requires_grad_(grad)
    mu = (0.1 * torch.rand((n, n, n), generator=g, dtype=torch.float64)).requires_grad_(grad)
    q = torch.rand((n, n, n), generator=g, dtype=torch.float64).requires_grad_(grad)
    return q, D, mu


def test_gradients_match_the_fake_operator_and_are_routed():
    q, D, mu = fields(1)
    u = autograd.solve(q, D, mu, 0.5)
    w = torch.rand_like(u)
    (u * w).sum().backward()
    lam = w / (D + mu)
    assert torch.allclose(q.grad, lam) and torch.allclose(D.grad, -lam * u) and torch.allclose(mu.grad, -lam * u)
    # gradients only where asked
    q2, D2, mu2 = fields(2)
    D2.requires_grad_(False)
    u2 = autograd.solve(q2, D2, mu2, 0.5)
    u2.sum().backward()
    s = autograd._cache.items[-1][5]
    assert s.last_need == (True, False, True) and D2.grad is None and mu2.grad is not None


def test_cache_hits_and_invalidation_by_in_place_change():
    q, D, mu = fields(3, grad=False)
    a = autograd._cache.get(D, mu, 0.5, {})
    assert autograd._cache.get(D, mu, 0.5, {}) is a
    assert autograd._cache.get(D, mu, 0.5, {"rtol": 1e-8}) is not a          # other parameters
    D.add_(1.0)                                                                # new version
    b = autograd._cache.get(D, mu, 0.5, {})
    assert b is not a and torch.equal(b.D, D)
    assert autograd._cache.get(D.clone(), mu, 0.5, {}) is not b              # other tensor object


def test_eviction_keeps_contexts_that_live_graphs_still_need():
    outs = []
    for k in range(6):                        # twice the cache size
        q, D, mu = fields(10 + k)
        outs.append((autograd.solve(q, D, mu, 0.5), q, D, mu))
    assert len(autograd._cache.items) == 3
    # the first graph's solver was evicted from the cache but not destroyed
    u0, q0, D0, mu0 = outs[0]
    u0.sum().backward()
    assert q0.grad is not None and torch.allclose(q0.grad, 1.0 / (D0 + mu0))


def test_dropped_solvers_are_destroyed_once_nothing_uses_them():
    refs = []
    for k in range(5):
        q, D, mu = fields(20 + k, grad=False)
        autograd.solve(q, D, mu, 0.5)
        refs.append(FakeSolver.made[-1])
    autograd.clear_cache()
    del q, D, mu
    gc.collect()
    assert all(r() is None for r in refs)


def test_recompute_solves_again_in_backward():
    q, D, mu = fields(4)
    u = autograd.solve(q, D, mu, 0.5, recompute=True)
    s = autograd._cache.items[-1][5]
    assert s.solves == 1
    u.sum().backward()
    assert s.solves == 2 and torch.allclose(q.grad, 1.0 / (D + mu))


def test_forward_mode_uses_the_tangent_rule():
    import torch.autograd.forward_ad as fwAD
    q, D, mu = fields(5, grad=False)
    dq, dD, dmu = (torch.rand_like(q) for _ in range(3))
    with fwAD.dual_level():
        out = autograd.solve(fwAD.make_dual(q, dq), fwAD.make_dual(D, dD), fwAD.make_dual(mu, dmu), 0.5)
        u, du = fwAD.unpack_dual(out)
    ref = (dq - (dD + dmu) * u) / (D + mu)
    assert torch.allclose(du, ref)
