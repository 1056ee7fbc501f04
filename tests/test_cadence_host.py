"""Stop-test cadence of the sweeps (csrc/cadence.h, compiled with g++): the
next test comes after about half of the sweeps the observed contraction
predicts, within [gmin, 8]; with nothing observed yet, after gmin."""
import math
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_06377_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include "cadence.h"
int main() {
  int gmin;
  while (std::scanf("%d", &gmin) == 1) {   // gmin, then (r, rho) pairs until r = 0, then target
    ibmi::CheckCadence c;
    c.gmin = c.next = gmin;
    int r; double rho, target;
    std::scanf("%lf", &target);
    while (std::scanf("%d %lf", &r, &rho) == 2 && r > 0) {
      c.after(r, rho, target);
      std::printf("%d %.17g %.17g\n", c.next, c.f, c.sweeps_to(rho, target));
    }
    std::printf("--\n");
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def cadence(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("cadence")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(gmin, target, checks):
        text = f"{gmin} {target!r} " + " ".join(f"{r} {rho!r}" for r, rho in checks) + " 0 0\n"
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
        rows = []
        for line in out:
            if line == "--":
                break
            nxt, f, st = line.split()
            rows.append((int(nxt), float(f), float(st)))
        return rows
    return run


def test_first_test_and_unknown_contraction(cadence):
    rows = cadence(1, 1e-3, [(1, 0.5)])
    assert rows == [(2, 0.0, math.inf)]           # one point: no contraction known
    rows = cadence(3, 1e-3, [(3, 0.5), (6, 0.6)])  # growing residual: unknown again
    assert rows[1][0] == 9 and rows[1][1] == 0.0


def test_gap_is_half_the_predicted_sweeps_within_bounds(cadence):
    target = 1e-6
    # contraction 0.5 per sweep from rho = 1e-2: need log(1e-4)/log(0.5) = 13.3 sweeps, gap floor(6.6) = 6
    rows = cadence(1, target, [(1, 2e-2), (2, 1e-2)])
    nxt, f, st = rows[1]
    assert f == pytest.approx(0.5, rel=1e-12)
    assert st == pytest.approx(math.log(target / 1e-2) / math.log(0.5), rel=1e-12)
    assert nxt == 2 + 6
    # slow contraction: the gap is capped at 8
    rows = cadence(1, target, [(1, 1e-2), (2, 0.99e-2)])
    assert rows[1][0] == 2 + 8
    # fast contraction: at least gmin
    rows = cadence(2, target, [(2, 1e-2), (4, 1e-5)])
    assert rows[1][0] == 4 + 2
    # contraction over several sweeps is taken per sweep
    rows = cadence(1, target, [(1, 1e-1), (4, 1e-1 * 0.5 ** 3)])
    assert rows[1][1] == pytest.approx(0.5, rel=1e-12)


def test_at_target_the_next_test_is_the_next_sweep(cadence):
    rows = cadence(1, 1e-6, [(1, 1e-5), (2, 1e-7)])
    assert rows[1][0] == 3 and rows[1][2] == 0.0
