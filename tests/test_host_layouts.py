"""Host-built device layouts checked on the host: the warp-cube staging
tables (csrc/cube.cpp), the list kernel's super-tile and the complex128
digit images (csrc/oz_image.h).  The warp-cube part: the C++
check in tests/native/ is compiled against the library's own host source and
verifies the mapping, the bounds and the bank-conflict bounds for 30000 random
gates (see the check's header)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_19894_gb300", "csrc")


def test_cube_tables(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "cube_check")
    cmd = [gxx, "-O2", "-std=c++17", "-I", CSRC, "-I", "/usr/local/cuda/include",
           os.path.join(ROOT, "tests", "native", "cube_tables_check.cpp"), os.path.join(CSRC, "cube.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    fields = dict(kv.rsplit("=", 1) for kv in out.stdout.split())
    assert fields["bad"] == "0"
    assert fields["worst_row(q0!=0)"] == "1"
    assert int(fields["worst_row(q0==0)"]) <= 2
    assert fields["worst_chunk"] == "1"
    assert fields["worst_pair"] == "1"


def test_sparse_super_tile_layout(tmp_path):
    """The list kernel's super-tile mapping (make_tile_layout plus the
    kernel's per-thread and per-element offsets): 4096 distinct amplitudes,
    each the one Eq. 3 gathers for its slot, and 4096 distinct slots, for
    3000 random gates (tests/native/sparse_layout_check.cpp)."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "sparse_layout_check")
    cmd = [gxx, "-O2", "-std=c++17", "-I", CSRC, "-I", "/usr/local/cuda/include",
           os.path.join(ROOT, "tests", "native", "sparse_layout_check.cpp"), os.path.join(CSRC, "cube.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    fields = dict(kv.split("=", 1) for kv in out.stdout.split())
    assert fields["bad"] == "0" and int(fields["checked"]) == 9000


def test_digit_images(tmp_path):
    """The complex128 digit images (csrc/oz_image.h) for k = 3..7 in both
    layouts: every digit at its own offset, the rest zero, the digits giving
    back each entry of the real form to 2^(E_n - 49) with its sign
    (tests/native/oz_image_check.cpp)."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "oz_image_check")
    cmd = [gxx, "-O2", "-std=c++17", "-I", CSRC, "-I", "/usr/local/cuda/include",
           os.path.join(ROOT, "tests", "native", "oz_image_check.cpp"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    fields = dict(kv.split("=", 1) for kv in out.stdout.split())
    assert fields["bad"] == "0" and int(fields["images"]) == 96
