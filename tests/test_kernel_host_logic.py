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
