"""Host-side checks of kernel logic that is plain C++ (no GPU): programs under
tests/host/ include the kernel header, are compiled by nvcc for the host and
run here."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not found")


def test_fused_prolongation_box_covers_exactly_the_interpolation_supports(tmp_path):
    exe = str(tmp_path / "fuse_box")
    subprocess.check_call([_nvcc(), "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "host", "fuse_box.cu")])
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout


def test_split_row_layout_positions_and_neighbour_offsets(tmp_path):
    exe = str(tmp_path / "geom_layout")
    subprocess.check_call([_nvcc(), "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "host", "geom_layout.cu")])
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout


def _extract_device_function(src, name):
    """Source text of a function defined at column 0 in a CUDA source (from the
    line of its signature to its closing brace at column 0)."""
    start = src.rindex("\n", 0, src.index(" %s(" % name)) + 1
    end = src.index("\n}\n", start) + 3
    return src[start:end]


def test_mixed_precision_conversions_round_like_c(tmp_path):
    # the conversions' own source, pasted into a host program (bit-cast stand-ins
    # for the CUDA intrinsics) and compared with C's conversions
    src = open(os.path.join(ROOT, "paper_2608_00760_b300", "csrc", "kernels.cuh")).read()
    funcs = "\n".join(_extract_device_function(src, n) for n in ("exponent_of", "f64_to_f32_shift",
                                                                 "f32_to_f64_shift"))
    assert funcs.count("__device__ __forceinline__") == 3
    tmpl = open(os.path.join(ROOT, "tests", "host", "bitconv_check.cpp")).read()
    assert tmpl.count("// @EXTRACTED@") == 1
    cpp = tmp_path / "bitconv.cpp"
    cpp.write_text(tmpl.replace("// @EXTRACTED@", funcs))
    exe = str(tmp_path / "bitconv")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-o", exe, str(cpp)])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout


def test_tail_index_decoding_is_exact_division(tmp_path):
    # the host's magic divisor and the kernel's multiply-high division and
    # decode, their own source pasted into a host program
    dev = open(os.path.join(ROOT, "paper_2608_00760_b300", "csrc", "kernels.cuh")).read()
    host = open(os.path.join(ROOT, "paper_2608_00760_b300", "csrc", "dmg.cu")).read()
    funcs = "\n".join([_extract_device_function(host, "magic_div")] +
                      [_extract_device_function(dev, n) for n in ("mdiv", "tail_decode")])
    assert funcs.count("magic_div(int d)") == 1 and funcs.count("__device__ __forceinline__") == 2
    tmpl = open(os.path.join(ROOT, "tests", "host", "tail_decode_check.cpp")).read()
    cpp = tmp_path / "tail_decode.cpp"
    cpp.write_text(tmpl.replace("// @EXTRACTED@", funcs))
    exe = str(tmp_path / "tail_decode")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-o", exe, str(cpp)])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout


def _extract_struct(src, name):
    start = src.index("struct %s {" % name)
    return src[start:src.index("\n};\n", start) + 4]


def test_batch_plane_split_is_exact_division(tmp_path):
    # the runtime's make_geom and the kernels' zsplit, their own source pasted
    # into a host program
    dev = open(os.path.join(ROOT, "paper_2608_00760_b300", "csrc", "kernels.cuh")).read()
    host = open(os.path.join(ROOT, "paper_2608_00760_b300", "csrc", "dmg.cu")).read()
    code = "\n".join([_extract_struct(dev, "Geom"), "enum { kInterior = 0, kCells = 1, kAll = 2 };",
                      _extract_device_function(host, "half_row_pitch"), _extract_device_function(host, "make_geom"),
                      _extract_device_function(dev, "zsplit")])
    assert "Geom make_geom(int nx, int ny, int nz, int nb)" in code
    tmpl = open(os.path.join(ROOT, "tests", "host", "zsplit_check.cpp")).read()
    cpp = tmp_path / "zsplit.cpp"
    cpp.write_text(tmpl.replace("// @EXTRACTED@", code))
    exe = str(tmp_path / "zsplit")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-o", exe, str(cpp)])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout


def test_fused_interpolation_is_bitwise_the_separate_prolongation(tmp_path):
    # fuse_interp (with the box helpers) and prolong_cell, their own source
    dev = open(os.path.join(ROOT, "paper_2608_00760_b300", "csrc", "kernels.cuh")).read()
    a = dev.index("__host__ __device__ constexpr int fuse_lo")
    b = dev.index("\n}\n", dev.index(" fuse_interp(")) + 3
    pc = dev.index(" prolong_cell(")
    start = dev.rindex("template <class T>", 0, pc)
    code = "\n".join([_extract_struct(dev, "Geom"), dev[start:dev.index("\n}\n", pc) + 3], dev[a:b]])
    assert code.count("fuse_interp(") == 1 and code.count("prolong_cell(") == 1
    tmpl = open(os.path.join(ROOT, "tests", "host", "fuse_interp_check.cpp")).read()
    cpp = tmp_path / "fuse_interp.cpp"
    cpp.write_text(tmpl.replace("// @EXTRACTED@", code))
    exe = str(tmp_path / "fuse_interp")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-o", exe, str(cpp)])
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout
