"""Mutation check of the oracle's pins.

The oracle is trusted because CPU tests pin it to things other than itself
(closed forms, a library direct solve, brute-force transposes, finite
differences, an independent numpy V-cycle). This file checks that those pins
are strong enough. Each entry of MUTANTS plants one plausible mistake in a copy
of oracle/dmg_oracle.c: a dropped term, a wrong sign, constant or index, a
transposed operand, or a swapped colour order. The test compiles the copy and
runs the oracle's pin tests against it through DMG_ORACLE_LIB. PY_MUTANTS do
the same to the numpy parts (the 2D solver, the complex-step V-cycle, the
response operator) in a copy of the whole package placed first on the import
path. Every mutant must make at least one pin fail; the unmutated copies must
pass them all.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dmg_oracle.c")
PINS = ["tests/test_oracle_operator.py", "tests/test_oracle_transfer.py", "tests/test_oracle_solver.py",
        "tests/test_oracle_adjoint.py", "tests/test_oracle_grad.py", "tests/test_oracle_response.py",
        "tests/test_oracle_unrolled.py"]

# (what the mistake is, text in dmg_oracle.c, replacement); each text occurs once
MUTANTS = [
    ("arithmetic face mean with a wrong constant",
     "return 0.5 * (a + b);", "return 0.25 * (a + b);"),
    ("harmonic face mean without its factor 2",
     "if (harmonic) return 2.0 * a * b / (a + b);", "if (harmonic) return a * b / (a + b);"),
    ("absorption term dropped from the operator",
     "out[p] = s * ih2 + mu[p] * up;", "out[p] = s * ih2;"),
    ("wrong sign of the neighbour coupling",
     "s += fc * (up - val0(nx, ny, nz, u, a, b, c));", "s += fc * (up + val0(nx, ny, nz, u, a, b, c));"),
    ("z+ neighbour replaced by z-",
     "{0, 1, 0},  {0, 0, -1}, {0, 0, 1}};", "{0, 1, 0},  {0, 0, -1}, {0, 0, -1}};"),
    ("absorption missing from the smoother's diagonal",
     "return s / (h * h) + mu[p];", "return s / (h * h);"),
    ("colour order of every sweep reversed",
     "L->f, L->u, first);\n    orc_gs_half(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, L->f, L->u, 1 - first);",
     "L->f, L->u, 1 - first);\n    orc_gs_half(L->nx, L->ny, L->nz, L->h, H->harmonic, L->D, L->mu, L->f, L->u, first);"),
    ("restriction weights with the y weight in place of the z weight",
     "s += fw(a) * fw(b) * fw(c) *\n                                     r[at(",
     "s += fw(a) * fw(b) * fw(b) *\n                                     r[at("),
    ("prolongation scaled by 2^2 instead of 2^3",
     "8.0 * fw(a) * fw(b) * fw(c) * v", "4.0 * fw(a) * fw(b) * fw(c) * v"),
    ("prolongation offsets z by the y offset",
     "int i = 2 * I + a, j = 2 * J + b, k = 2 * K + c;", "int i = 2 * I + a, j = 2 * J + b, k = 2 * K + b;"),
    ("coefficient coarsening with the x weight in place of the y weight",
     "s += fw(a) * fw(b) * fw(c) *\n                                     Xf[at(",
     "s += fw(a) * fw(a) * fw(c) *\n                                     Xf[at("),
    ("coarse correction not reset to zero",
     "memset(C->u, 0, npts(C) * sizeof(double));\n    vcycle(H, l + 1, transposed);",
     "vcycle(H, l + 1, transposed);"),
    ("symmetric post-smoothing order ignored",
     "int post_first = H->symmetric ? 1 : 0;\n    int npre = transposed",
     "int post_first = 0;\n    int npre = transposed"),
    ("transposed cycle keeps the forward pre-smoothing colour order",
     "int pre_first = transposed ? 1 - post_first : 0;", "int pre_first = transposed ? post_first : 0;"),
    ("transposed cycle does not swap nu1 and nu2",
     "int npre = transposed ? H->nu2 : H->nu1, npost = transposed ? H->nu1 : H->nu2;",
     "int npre = H->nu1, npost = H->nu2;"),
    ("defect with the wrong sign",
     "? f[p] - r[p] : 0.0;", "? r[p] - f[p] : 0.0;"),
    ("forward substitution without the pivot",
     "x[i] = t / l[(size_t)i * n + i];\n    }\n    for (int i = n - 1",
     "x[i] = t;\n    }\n    for (int i = n - 1"),
    ("Cholesky column not divided by the pivot",
     "a[(size_t)i * n + j] = t / d;", "a[(size_t)i * n + j] = t;"),
    ("literal adjoint restricts with 2^2 instead of 2^3",
     "C->ub[p] += 8.0 * t[p];", "C->ub[p] += 4.0 * t[p];"),
    ("transposed Gauss-Seidel step subtracts its right-hand-side cotangent",
     "fbar[p] += t;", "fbar[p] -= t;"),
    ("stopping rule four decades loose",
     "if (fixed == 0 && rel <= rtol) break;", "if (fixed == 0 && rel <= 1e4 * rtol) break;"),
    ("level count checks x twice and y never",
     "(nx - 1) % 2 == 0 && (ny - 1) % 2 == 0 &&", "(nx - 1) % 2 == 0 && (nx - 1) % 2 == 0 &&"),
    ("absorption gradient with the wrong sign",
     "mubar[p] = -lv * uv;", "mubar[p] = lv * uv;"),
    ("diffusion gradient with u_v + u_j",
     "* (lv - lj) * (uv - uj);", "* (lv - lj) * (uv + uj);"),
    ("harmonic face derivative with a for b",
     "if (harmonic) return 2.0 * b * b / ((a + b) * (a + b));",
     "if (harmonic) return 2.0 * a * b / ((a + b) * (a + b));"),
    ("tangent operator takes the neighbour's dD from the centre",
     "orc_face_da(D[q], D[p], harmonic) * dD[q]", "orc_face_da(D[q], D[p], harmonic) * dD[p]"),
    ("tangent operator drops the absorption direction",
     "out[p] = s * ih2 + (dmu ? dmu[p] : 0.0) * u[p];", "out[p] = s * ih2;"),
]


# (file in oracle/, what the mistake is, text, replacement, pin files); each text occurs once
_P2 = ["tests/test_oracle_2d.py"]
_PU = ["tests/test_oracle_unrolled.py"]
_PR = ["tests/test_oracle_response.py"]
PY_MUTANTS = [
    ("dmg2d.py", "absorption term dropped from the 2D operator",
     "out[1:-1, 1:-1] = s / (h * h) + _sh(mu, 0, 0) * uc", "out[1:-1, 1:-1] = s / (h * h)", _P2),
    ("dmg2d.py", "absorption missing from the 2D smoother's diagonal",
     "new = (_sh(f, 0, 0) + off) / (dg + _sh(mu, 0, 0))", "new = (_sh(f, 0, 0) + off) / dg", _P2),
    ("dmg2d.py", "2D y+ neighbour replaced by y-",
     "DIRS = ((-1, 0), (1, 0), (0, -1), (0, 1))", "DIRS = ((-1, 0), (1, 0), (0, -1), (0, -1))", _P2),
    ("dmg2d.py", "2D colours swapped (black first)",
     "return (i + j) & 1", "return (i + j + 1) & 1", _P2),
    ("dmg2d.py", "2D prolongation scaled by 2 instead of 2^2",
     "4.0 * _FW[a] * _FW[b] * ec", "2.0 * _FW[a] * _FW[b] * ec", _P2),
    ("dmg2d.py", "2D transposed cycle does not swap nu1 and nu2",
     "npre, npost = (self.nu2, self.nu1) if transposed else (self.nu1, self.nu2)",
     "npre, npost = (self.nu1, self.nu2)", _P2),
    ("dmg2d.py", "2D absorption gradient with the wrong sign",
     "mb = _zero_boundary(-lam * u)", "mb = _zero_boundary(lam * u)", _P2),
    ("dmg2d.py", "2D harmonic face derivative with a for b",
     "return 2.0 * b * b / ((a + b) * (a + b)) if harmonic", "return 2.0 * a * b / ((a + b) * (a + b)) if harmonic",
     _P2),
    ("dmg2d.py", "2D tangent operator takes the neighbour's dD from the centre",
     "_face_da(Dn, c, harmonic) * dn", "_face_da(Dn, c, harmonic) * dc", _P2),
    ("unrolled.py", "complex-step V-cycle drops the absorption term",
     "out[1:-1, 1:-1, 1:-1] = s / (h * h) + _shift(mu, 0, 0, 0) * uc", "out[1:-1, 1:-1, 1:-1] = s / (h * h)", _PU),
    ("unrolled.py", "complex-step V-cycle prolongs with 2^2",
     "8.0 * _FW[a] * _FW[b] * _FW[c] * ec", "4.0 * _FW[a] * _FW[b] * _FW[c] * ec", _PU),
    ("unrolled.py", "complex-step V-cycle post-smooths black first",
     "gs_half(D, mu, h, f, u, post_first, self.harmonic)", "gs_half(D, mu, h, f, u, 1, self.harmonic)", _PU),
    ("unrolled.py", "complex-step coefficient coarsening injects everywhere",
     "    if not inject:\n        out[1:-1, 1:-1, 1:-1]", "    if False:\n        out[1:-1, 1:-1, 1:-1]", _PU),
    ("unrolled.py", "directional derivative from the real part",
     "return float(np.sum(w * u).imag / eps)", "return float(np.sum(w * u).real / eps)", _PU),
    ("__init__.py", "tangent right-hand side adds dA u instead of subtracting it",
     "rhs = rhs - dA_apply(self.D, self.h, dD, dmu, u, self.harmonic)",
     "rhs = rhs + dA_apply(self.D, self.h, dD, dmu, u, self.harmonic)", PINS),
    ("__init__.py", "pull-back gradients ignore the harmonic face mean",
     "Db, mb = grad(self.D, self.h, u, lam, self.harmonic)", "Db, mb = grad(self.D, self.h, u, lam, False)", PINS),
    ("__init__.py", "tangent operator wrapper swaps the D and mu directions",
     "_ptr(D), _ptr(dD), _ptr(dmu), _ptr(u),", "_ptr(D), _ptr(dmu), _ptr(dD), _ptr(u),", PINS),
    ("__init__.py", "assembled matrix with the wrong sign",
     "vals.append(col[nz_])", "vals.append(-col[nz_])", PINS),
    ("__init__.py", "interior index includes the last plane of every axis",
     "np.meshgrid(np.arange(1, nz - 1), np.arange(1, ny - 1), np.arange(1, nx - 1),",
     "np.meshgrid(np.arange(1, nz), np.arange(1, ny), np.arange(1, nx),", PINS),
    ("__init__.py", "edge mask measures the distance to the lower face only",
     "dist = np.minimum(x, (n - 1) * h - x)", "dist = x", _PR),
    ("__init__.py", "edge mask drops voxels exactly at the edge depth",
     "ok = dist >= edge * (1.0 - 1e-12)", "ok = dist > edge * (1.0 + 1e-12)", _PR),
    ("__init__.py", "response without the absorption factor",
     "return np.where(edge_mask(H.shape, H.h, edge), H.mu * u, 0.0), u",
     "return np.where(edge_mask(H.shape, H.h, edge), u, 0.0), u", _PR),
    ("__init__.py", "response tangent subtracts the absorption direction",
     "t = t + _arr(dmu) * u", "t = t - _arr(dmu) * u", _PR),
    ("__init__.py", "response pull-back misses the explicit absorption term",
     "mb = mb + np.where(m, u * _arr(rbar), 0.0)", "mb = mb + 0.0 * np.where(m, u * _arr(rbar), 0.0)", _PR),
    ("__init__.py", "response pull-back cotangent without the absorption factor",
     "w = np.where(m, H.mu * _arr(rbar), 0.0)", "w = np.where(m, _arr(rbar), 0.0)", _PR),
]


def _compile(text, path):
    c_path = path + ".c"
    with open(c_path, "w") as fh:
        fh.write(text)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", path, c_path, "-lm"])


def _run_pins(lib):
    env = dict(os.environ, DMG_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
                       + PINS, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-1500:] + r.stderr[-500:]


def _package_copy(dest, fname=None, old=None, new=None):
    """A copy of oracle/ under dest (one file mutated), to be imported first."""
    src_dir = os.path.join(ROOT, "oracle")
    shutil.copytree(src_dir, os.path.join(dest, "oracle"), ignore=shutil.ignore_patterns("_build", "__pycache__"))
    if fname is not None:
        path = os.path.join(dest, "oracle", fname)
        with open(path) as fh:
            text = fh.read()
        assert text.count(old) == 1, "mutant of %s: its text occurs %d times" % (fname, text.count(old))
        with open(path, "w") as fh:
            fh.write(text.replace(old, new))


def _run_pins_in_copy(dest, pins, lib):
    # the copy is the working directory (first on sys.path); the repository follows
    # it on PYTHONPATH so the tests' conftest does not put it in front again
    env = dict(os.environ, DMG_ORACLE_LIB=lib, PYTHONPATH=os.pathsep.join([dest, ROOT]))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "--rootdir", ROOT] + [os.path.join(ROOT, p) for p in pins],
                       cwd=dest, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-1500:] + r.stderr[-500:]


@pytest.fixture(scope="module")
def built_lib():
    import oracle
    return oracle.build()


def test_package_copy_is_the_one_imported_and_passes(tmp_path, built_lib):
    dest = str(tmp_path / "copy")
    _package_copy(dest)
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([dest, ROOT]))
    where = subprocess.run([sys.executable, "-c", "import oracle, oracle.dmg2d; print(oracle.__file__)"],
                           cwd=dest, env=env, capture_output=True, text=True, check=True).stdout.strip()
    assert where.startswith(dest)
    pins = sorted({p for m in PY_MUTANTS for p in m[4]})
    rc, out = _run_pins_in_copy(dest, pins, built_lib)
    assert rc == 0, out


def test_every_planted_mistake_in_the_numpy_oracles_fails_a_pin(tmp_path, built_lib):
    jobs = []
    for n, (fname, what, old, new, pins) in enumerate(PY_MUTANTS):
        dest = str(tmp_path / ("m%02d" % n))
        _package_copy(dest, fname, old, new)
        jobs.append((what, dest, pins))
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda j: (j[0],) + _run_pins_in_copy(j[1], j[2], built_lib), jobs))
    survivors = [what for what, rc, _ in results if rc == 0]
    broken = [(what, rc, out) for what, rc, out in results if rc not in (0, 1)]
    assert not broken, "pin runs that did not complete: %r" % broken
    assert not survivors, "planted mistakes no pin catches: %r" % survivors


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


def test_unmutated_copy_passes_every_pin(source, tmp_path):
    lib = str(tmp_path / "liboracle_copy.so")
    _compile(source, lib)
    rc, out = _run_pins(lib)
    assert rc == 0, out


def test_every_planted_mistake_fails_a_pin(source, tmp_path):
    libs = []
    for n, (what, old, new) in enumerate(MUTANTS):
        assert source.count(old) == 1, "mutant %r: its text occurs %d times" % (what, source.count(old))
        lib = str(tmp_path / ("liboracle_mutant%02d.so" % n))
        _compile(source.replace(old, new), lib)
        libs.append((what, lib))
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda wl: (wl[0],) + _run_pins(wl[1]), libs))
    survivors = [what for what, rc, _ in results if rc == 0]
    broken = [(what, rc, out) for what, rc, out in results if rc not in (0, 1)]
    assert not broken, "pin runs that did not complete: %r" % broken
    assert not survivors, "planted mistakes no pin catches: %r" % survivors
