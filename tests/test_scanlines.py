"""Host logic of the SGM scanlines (the tables in lfsgm_internal.cuh that the fine and coarse SGM
kernels and the split listing kernel use): built with the host compiler and checked against a
brute-force count.  For every direction of Sec. IV-C (8 and 16 paths) and image shapes down to
1 x 1: each pixel lies on exactly one scanline, a scanline starts where the predecessor p - r
leaves the image and ends where p + r does, scan_index inverts scan_start, the number of
scanlines equals the number of pixels whose predecessor is outside the image, and the bit-field
form of the direction table agrees with it."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
DIRS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1),
        (2, 1), (-2, -1), (2, -1), (-2, 1), (1, 2), (-1, -2), (1, -2), (-1, 2)]
SHAPES = [(1, 1), (1, 7), (7, 1), (2, 2), (2, 3), (3, 2), (5, 17), (17, 5), (32, 32), (31, 64), (40, 56)]


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    cxx, inc = shutil.which("g++"), _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("scan") / "scanline_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", inc, "-I", os.path.join(ROOT, "paper_1907_13449_gb300", "csrc"),
                    os.path.join(HERE, "scanline_check.cpp"), "-o", exe], check=True)
    args = [str(v) for hw in SHAPES for v in hw]
    out = subprocess.run([exe, *args], check=True, capture_output=True, text=True).stdout
    lines = out.split("\n")
    rows = {"bad_dirs": int(lines[0])}
    for line in lines[1:]:
        if line.strip():
            H, W, r, ns, covered, twice, missing, bad_index, bad_ends = map(int, line.split())
            rows[(H, W, r)] = (ns, covered, twice, missing, bad_index, bad_ends)
    return rows


def test_direction_bit_fields_match_the_table(table):
    assert table["bad_dirs"] == 0


@pytest.mark.parametrize("shape", SHAPES)
def test_every_pixel_on_one_scanline(table, shape):
    H, W = shape
    for r, (dx, dy) in enumerate(DIRS):
        ns, covered, twice, missing, bad_index, bad_ends = table[(H, W, r)]
        # brute force: a scanline starts at each pixel whose predecessor p - r is outside the image
        starts = sum(1 for y in range(H) for x in range(W) if not (0 <= x - dx < W and 0 <= y - dy < H))
        assert ns == starts, (shape, r)
        assert covered == H * W and twice == 0 and missing == 0, (shape, r)
        assert bad_index == 0 and bad_ends == 0, (shape, r)
