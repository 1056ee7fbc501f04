"""Lower-tile enumeration of the digit-pair launches (csrc/oz_tiles.h,
compiled on the CPU with g++): the tiles counted are exactly those that reach
the diagonal, the index -> tile map walks them row by row without gaps or
repeats, and every element on or below the diagonal of a symmetric product
lies in one of them (the recombination kernels read nothing else)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_06377_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "oz_tiles.h"
using namespace ibmi;
int main() {
  int gm, gn, bn;
  while (std::scanf("%d %d %d", &gm, &gn, &bn) == 3) {
    const int n = oz_lower_tiles(gm, gn, bn);
    std::printf("%d", n);
    for (int t = 0; t < n; ++t) {
      int mt, ntl;
      oz_lower_tile(t, gn, bn, mt, ntl);
      std::printf(" %d,%d", mt, ntl);
    }
    std::printf("\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def tiles(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("oz_tiles")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def call(cases):
        out = subprocess.run([str(exe)], input="\n".join(f"{a} {b} {c}" for a, b, c in cases) + "\n",
                             capture_output=True, text=True, check=True).stdout.splitlines()
        res = []
        for line in out:
            f = line.split()
            res.append((int(f[0]), [tuple(int(x) for x in t.split(",")) for t in f[1:]]))
        return res
    return call


@pytest.mark.parametrize("bn", [64, 128, 224])
def test_lower_tiles_are_exactly_those_reaching_the_diagonal(tiles, bn):
    cases = []
    for p in (1, 100, 128, 129, 576, 1024, 2100, 4096, 5120, 8192):
        cases.append(((p + 127) // 128, (p + bn - 1) // bn, bn))
    for (gm, gn, b), (n, got) in zip(cases, tiles(cases)):
        want = [(mt, nt) for mt in range(gm) for nt in range(gn) if nt * b < (mt + 1) * 128]
        assert n == len(want) and got == want, (gm, gn, b)   # row by row, each tile once


@pytest.mark.parametrize("bn", [64, 128, 224])
def test_every_element_on_or_below_the_diagonal_is_covered(tiles, bn):
    for p in (100, 300, 1000, 2100):
        gm, gn = (p + 127) // 128, (p + bn - 1) // bn
        (_, got), = tiles([(gm, gn, bn)])
        cover = set(got)
        for i in range(0, p, 7):
            for j in range(0, i + 1, 5):
                assert (i // 128, j // bn) in cover, (p, bn, i, j)
