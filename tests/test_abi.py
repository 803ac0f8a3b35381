"""Host-side checks of the C ABI library (no GPU): it builds for sm_103a, loads,
exports every function include/dmg.h declares, and rejects invalid parameters
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dmg():
    from paper_2608_00760_b300 import build, dmg
    build.build()
    dmg.lib()
    return dmg


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dmg_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(dmg):
    names = declared_functions()
    assert len(names) >= 10
    L = ctypes.CDLL(dmg._LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(dmg.EXPORTS)


def test_library_is_built_for_sm_103a(dmg):
    import subprocess
    out = subprocess.run(["cuobjdump", "--list-elf", dmg._LIB_PATH], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_default_params_and_strerror(dmg):
    p = dmg.dmg_default_params()
    assert (p.nu1, p.nu2, p.max_cycles, p.rtol, p.precision, p.inner_cycles) == (2, 2, 100, 1e-10, 0, 3)
    assert (p.batch, p.autotune, p.split_prolong) == (1, 0, 0)
    assert dmg.dmg_strerror(dmg.DMG_OK) == "ok"
    assert dmg.dmg_strerror(dmg.DMG_ENOCONV) == "did not converge"


@pytest.mark.parametrize("bad", [
    dict(nx=2, ny=9, nz=9, h=1.0),                   # too few vertices
    dict(nx=20, ny=20, nz=20, h=1.0),                # even: no coarsening, 18^3 coarsest unknowns > 512
    dict(nx=9, ny=9, nz=9, h=0.0),                   # h <= 0
    dict(nx=9, ny=9, nz=9, h=1.0, nu1=0, nu2=0),     # no smoothing
    dict(nx=9, ny=9, nz=9, h=1.0, precision=7),
    dict(nx=9, ny=9, nz=9, h=1.0, face_mean=3),
    dict(nx=9, ny=9, nz=9, h=1.0, rtol=0.0),
    dict(nx=9, ny=9, nz=9, h=1.0, max_cycles=0),
    dict(nx=9, ny=9, nz=9, h=1.0, inner_cycles=0),
    dict(nx=9, ny=9, nz=9, h=1.0, split_prolong=2),
    dict(nx=9, ny=9, nz=9, h=1.0, twin_adjoint=2),
    dict(nx=65, ny=257, nz=257, h=1.0),              # coarsens to 3x9x9: fine; 7x7x513 is not
    dict(nx=7, ny=7, nz=513, h=1.0),                 # 7 -> 4 stops coarsening at 4x4x257: 1020 unknowns
])
def test_setup_rejects_invalid_params_without_gpu(dmg, bad):
    p = dmg.dmg_default_params(**bad)
    valid = (bad.get("nx"), bad.get("ny"), bad.get("nz")) == (65, 257, 257)
    if valid:
        pytest.skip("valid shape: needs a GPU")
    st, ctx = dmg.dmg_setup(p, 0, 0)
    assert st == dmg.DMG_EINVAL and ctx is None
    assert dmg.dmg_last_error(None) != "" or bad.get("nx") == 2


def test_null_context_calls(dmg):
    assert dmg.dmg_solve(None, 0, 0) == dmg.DMG_EINVAL
    assert dmg.dmg_destroy(None) == dmg.DMG_OK
    assert dmg.dmg_levels(None) == 0


def test_2d_parameter_validation():
    from paper_2608_00760_b300 import dmg
    # nz = 2 is neither 2D nor a valid 3D grid; a 2D grid whose coarsest level is too large is refused
    for (nx, ny, nz), msg in (((17, 17, 2), "3 vertices"), ((33, 34, 1), "unknowns")):
        p = dmg.dmg_default_params(nx=nx, ny=ny, nz=nz, h=1.0)
        st, ctx = dmg.dmg_setup(p, None, None)
        assert st == dmg.DMG_EINVAL and ctx is None and msg in dmg.dmg_last_error(None)


def test_injected_allocation_failure_is_reported_without_a_device():
    # the first allocation of dmg_setup fails (injected on the host before any
    # CUDA call): ENOMEM, no context, and the message names the injection
    from paper_2608_00760_b300 import dmg
    p = dmg.dmg_default_params(nx=17, ny=17, nz=17, h=1.0)
    D = np.ones(17 ** 3)
    dmg.dmg_debug_fail_alloc(1)
    try:
        st, ctx = dmg.dmg_setup(p, D, D)
    finally:
        dmg.dmg_debug_fail_alloc(0)
    assert st == dmg.DMG_ENOMEM and ctx is None
    assert "injected" in dmg.dmg_last_error(None)


def test_ctypes_structs_match_the_header_layout(tmp_path):
    # the binding's mirrors of dmg_params and dmg_info must have the C layout:
    # compile the header with gcc and compare the size and every field offset
    import subprocess
    from paper_2608_00760_b300 import dmg
    lines = ['#include <stdio.h>', '#include "dmg.h"', "int main(void) {"]
    for st in (dmg.dmg_params, dmg.dmg_info):
        name = st.__name__
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in st._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for st in (dmg.dmg_params, dmg.dmg_info):
        name = st.__name__
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert got[(name, f)] == getattr(st, f).offset, (name, f)
    # and the same field names in the same order as the header declares
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "dmg.h")).read(), flags=re.S)
    for st in (dmg.dmg_params, dmg.dmg_info):
        body = re.search(r"typedef struct \{([^}]*)\}\s*%s;" % st.__name__, hdr).group(1)
        names = []
        for decl in body.split(";"):
            decl = re.sub(r"\[[^]]*\]", "", decl).strip()
            if decl:
                names += [v.strip() for v in decl.split(None, 1)[1].split(",")]
        assert names == [f for f, _ in st._fields_], st.__name__


@pytest.mark.parametrize("bad,msg", [
    (dict(nx=9, ny=9, nz=9, h=float("inf")), "h must be > 0"),
    (dict(nx=9, ny=9, nz=9, h=float("nan")), "h must be > 0"),
    (dict(nx=9, ny=9, nz=9, h=1.0, nu1=-1), "nu1, nu2"),
    (dict(nx=9, ny=9, nz=9, h=1.0, nu2=65), "nu1, nu2"),
    (dict(nx=9, ny=9, nz=9, h=1.0, fixed_cycles=-1), "fixed_cycles"),
    (dict(nx=9, ny=9, nz=9, h=1.0, coarsen=2), "bad coarsen"),
    (dict(nx=9, ny=9, nz=9, h=1.0, inner_cycles=17), "inner_cycles"),
    (dict(nx=9, ny=9, nz=9, h=1.0, symmetric=2), "symmetric"),
    (dict(nx=9, ny=9, nz=9, h=1.0, batch=0), "batch must be"),
    (dict(nx=9, ny=9, nz=9, h=1.0, autotune=-1), "autotune"),
    (dict(nx=9, ny=9, nz=9, h=1.0, batch=7282), "batch * nz"),         # 7282 * 9 > 65535
    (dict(nx=2049, ny=1025, nz=1025, h=1.0), "too large"),             # > 2^31 - 1 vertices
    (dict(nx=1025, ny=1025, nz=1993, h=1.0), "padded sample"),         # < 2^31 vertices, padded rows beyond
    (dict(nx=9, ny=9, nz=2, h=1.0), "3 vertices"),
])
def test_each_validation_rule_names_itself(dmg, bad, msg):
    st, ctx = dmg.dmg_setup(dmg.dmg_default_params(**bad), 0, 0)
    assert st == dmg.DMG_EINVAL and ctx is None
    assert msg in dmg.dmg_last_error(None)


def test_fixed_cycles_need_no_rtol(dmg):
    # rtol is only checked when iterating to a tolerance: a fixed-count setup
    # with rtol = 0 passes validation and fails later, at the missing device
    # arrays (NULL coefficient pointers), not at rtol
    st, ctx = dmg.dmg_setup(dmg.dmg_default_params(nx=9, ny=9, nz=9, h=1.0, fixed_cycles=15, rtol=0.0), 0, 0)
    assert ctx is None and "rtol" not in dmg.dmg_last_error(None)


def test_context_free_error_message_is_per_thread(dmg):
    # dmg_last_error(NULL) reports the last failed context-free call of the
    # calling thread: thread A fails, thread B fails with another message, and
    # A still reads its own
    import threading
    bar = threading.Barrier(2)
    seen = {}

    def a():
        dmg.dmg_setup(dmg.dmg_default_params(nx=9, ny=9, nz=9, h=1.0, symmetric=2), 0, 0)
        bar.wait()
        bar.wait()
        seen["a"] = dmg.dmg_last_error(None)

    def b():
        bar.wait()
        dmg.dmg_setup(dmg.dmg_default_params(nx=9, ny=9, nz=9, h=1.0, batch=0), 0, 0)
        seen["b"] = dmg.dmg_last_error(None)
        bar.wait()

    ts = [threading.Thread(target=a), threading.Thread(target=b)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=60)
    assert "symmetric" in seen["a"] and "batch" in seen["b"]


def test_array_arguments_are_checked_before_any_call():
    # the binding passes raw addresses, so it refuses what the C side would
    # misread: other dtypes, strided views and wrong element counts
    torch = pytest.importorskip("torch")
    from paper_2608_00760_b300 import dmg
    a = np.zeros((4, 5, 6))
    assert dmg._ptr(a, 120) == a.ctypes.data and dmg._ptr(None) is None and dmg._ptr(1234) == 1234
    for bad, n in ((a.astype(np.float32), 120), (a[:, :, ::2], 60), (a.T, 120), (a, 121)):
        with pytest.raises(ValueError):
            dmg._ptr(bad, n)
    t = torch.zeros((4, 5, 6), dtype=torch.float64)
    assert dmg._ptr(t, 120) == t.data_ptr()
    for bad, n in ((t.float(), 120), (t.transpose(0, 2), 120), (t[:, :, ::2], 60), (t.to(torch.complex64), 120),
                   (t, 7)):
        with pytest.raises(ValueError):
            dmg._ptr(bad, n)
    with pytest.raises(TypeError):
        dmg._ptr([0.0] * 120, 120)
