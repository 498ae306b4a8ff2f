"""Host logic of the batched launch shapes (no GPU needed): `fit_shape` narrows the scenario
width of a shape for a batch smaller than it, and `bgrid` covers every (scenario, cell) item.
A small host program includes the kernels' own header, compiled by nvcc and run on the CPU."""
import itertools
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2608_03778_gb300", "csrc")

SHAPES = [(32, 4), (32, 8), (64, 2), (64, 4), (128, 1), (128, 2), (256, 1), (512, 1), (96, 2)]
SIZES = [1, 2, 3, 5, 8, 16, 17, 31, 32, 33, 63, 64, 65, 100, 128, 300, 512, 4096]
ROWS = [1, 7, 2500, 25000, 10 ** 7]


@pytest.fixture(scope="module")
def table(tmp_path_factory):
    if not shutil.which("nvcc"):
        pytest.skip("nvcc missing")
    d = tmp_path_factory.mktemp("shapes")
    lines = ['#include <cstdio>', '#include "kern_batch.cuh"', "int main() {"]
    for (bx, by), S, R in itertools.product(SHAPES, SIZES, ROWS):
        lines.append(f"{{ dp::BatchShape f = dp::fit_shape(dp::BatchShape{{{bx}, {by}}}, {S}); "
                     f"dim3 g = dp::bgrid({S}, f, {R}); "
                     f'std::printf("{bx} {by} {S} {R} %d %d %u %u\\n", f.bx, f.by, g.x, g.y); }}')
    lines += ["return 0;", "}"]
    src = d / "shapes.cu"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "shapes"
    subprocess.run(["nvcc", "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    return [tuple(int(v) for v in line.split()) for line in out if line]


def test_fit_shape(table):
    for bx, by, S, R, fx, fy, gx, gy in table:
        if S >= bx:
            assert (fx, fy) == (bx, by)
        assert min(S, bx) <= fx <= bx and fy >= 1                         # covers S, never wider
        assert bx * by - fx < fx * fy <= bx * by                          # threads per block kept
        if S < bx and bx & (bx - 1) == 0:
            assert fx & (fx - 1) == 0 and fx < 2 * S                      # power of two, no idle half
        assert 1 <= fx * fy <= 1024


def test_bgrid_covers_every_item(table):
    for bx, by, S, R, fx, fy, gx, gy in table:
        assert gx * fx >= S and (gx - 1) * fx < S                         # scenarios covered, no idle block
        assert 1 <= gy <= 65535
        assert gy * fy >= R or gy == 65535                                # cells covered (grid-stride past 65535)
