"""The bounds-checked build (libdmg_check.so, compiled with -DDMG_BOUNDS_CHECK,
the library's own stand-in for an external memory checker): every
per-vertex body and colour kernel counts positions outside their arrays and
sample indices outside the batch. A child process loads that build, runs the
solver's paths on odd, thin, batched and 2D grids, and must see zero such
accesses and every call succeed."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
import torch
from paper_2608_00760_b300 import build, dmg
build.build(check=True)
dmg.use_check_library()
from paper_2608_00760_b300 import inputs, serve
T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
runs = []

def run(name, fn):
    try:
        fn()
        runs.append([name, "ok"])
    except Exception as e:
        runs.append([name, repr(e)[:300]])

def full(shape, **kw):
    w = inputs.tissue(seed=1, shape=shape)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], **kw)
    u = S.solve(T(w["q"]))
    S.jvp(u, T(w["dq"]), T(w["dD"]), T(w["dmu"]))
    S.vjp(u, T(w["w"]))
    S.vjp(u, T(w["w"]), cycles=3)
    S.close()

for shape in [(33, 33, 33), (17, 33, 65), (33, 49, 97), (9, 9, 257), (3, 3, 514), (5, 5, 5)]:
    for prec in (0, 1):
        run("3d %s p%d" % (shape, prec), lambda: full(shape, precision=prec))
run("3d harmonic injection", lambda: full((17, 17, 33), precision=1, face_mean=1, coarsen=1))
run("3d autotune", lambda: full((33, 33, 65), precision=1, autotune=1))

def batch():
    w = inputs.vi_batch(17, 3, seed=2)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1)
    u = S.solve(T(w["q"]))
    S.vjp(u, T(w["w"]))
    S.close()
run("batch", batch)

def two_d(prec):
    w = inputs.tissue2d(seed=3, shape=(65, 129))
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], dim=2, precision=prec)
    u = S.solve(T(w["q"]))
    S.jvp(u, T(w["dq"]), T(w["dD"]), T(w["dmu"]))
    S.vjp(u, T(w["w"]))
    S.close()
run("2d p0", lambda: two_d(0))
run("2d p1", lambda: two_d(1))

def extras():
    w = inputs.tissue(seed=4, shape=(17, 17, 17))
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"])
    Le, u = S.response(T(w["q"]), 1.0)
    S.response_vjp(u, T(w["w"]), 1.0)
    S.response_jvp(u, 1.0, dq=T(w["dq"]), dD=T(w["dD"]), dmu=T(w["dmu"]))
    S.vjp_unrolled(T(w["q"]), T(w["w"]), 3)
    outs = [torch.empty_like(u) for _ in range(4)]
    assert dmg.dmg_solve_vjp(S.ctx, T(w["q"]), T(w["w"]), *outs, n=S.n) == dmg.DMG_OK
    S.close()
run("response, unrolled, solve_vjp", extras)

def serving():
    shapes = [(17, 17, 17), (9, 17, 33)]
    server = serve.Server(shapes, slots={s: 3 for s in shapes}, params=dict(precision=1), budget_bytes=8e9)
    try:
        served, st = server.run(serve.poisson_stream(10, 2000.0, shapes, seed=5))
        assert st["ok"] == 10
    finally:
        server.close()
run("serving", serving)

def pyramid(prec):
    shapes = [(65, 65, 65), (33, 33, 33)]
    server = serve.Server(shapes, slots={s: 2 for s in shapes}, params=dict(precision=prec), budget_bytes=8e9,
                          pyramid=True)
    try:
        assert len(server.unique_pools()) == 1
        served, st = server.run(serve.poisson_stream(6, 2000.0, shapes, seed=6))
        assert st["ok"] == 6
    finally:
        server.close()
run("pyramid p0", lambda: pyramid(0))
run("pyramid p1", lambda: pyramid(1))

def many(twin):
    w = inputs.vi_batch(17, 2, seed=7)
    S = dmg.Solver(T(w["D"]), T(w["mu"]), w["h"], precision=1, twin_adjoint=twin)
    hq, hw = np.ascontiguousarray(w["q"]), np.ascontiguousarray(w["w"])
    outs = [[np.zeros(w["q"].shape) for _ in range(2)] for _ in range(4)]
    assert dmg.dmg_solve_vjp_many(S.ctx, [hq, hq], [hw, hw], *outs, n=S.n) == dmg.DMG_OK
    assert dmg.dmg_solve_vjp(S.ctx, hq, hw, *(o[0] for o in outs), n=S.n) == dmg.DMG_OK
    S.set_coefficients(T(w["D"]), T(w["mu"]))
    S.close()
run("solve_vjp_many, solve_vjp, set_coefficients (one lane)", lambda: many(0))
run("solve_vjp_many, solve_vjp, set_coefficients (twin lane)", lambda: many(1))
torch.cuda.synchronize()
print(json.dumps(dict(runs=runs, oob=dmg.dmg_debug_oob_count())))
'''


def test_bounds_checked_build_sees_no_out_of_range_access():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    bad = [x for x in out["runs"] if x[1] != "ok"]
    assert not bad, bad
    assert out["oob"] == 0
