"""Host choices of the batched executor and the server
(csrc/batch_plan.h, compiled with g++): size buckets, the partitions a bucket
may run with, and the Newton-Schulz hand-over.  Every partition the executor
can pick must pass the library's own plan validation (on a machine without a
GPU a valid plan fails later, at allocation, with IBMI_ERR_OOM)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2502_06377_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstring>
#include "batch_plan.h"
using namespace ibmi;
int main() {
  char c[8];
  long long p;
  while (std::scanf("%7s %lld", c, &p) == 2) {
    if (!std::strcmp(c, "B")) std::printf("%lld\n", (long long)bucket_of(p));
    else if (!std::strcmp(c, "D")) { Shape s = default_shape(p); std::printf("%d %lld\n", s.K, (long long)s.h); }
    else if (!std::strcmp(c, "R")) { Shape s = robust_shape(p); std::printf("%d %lld\n", s.K, (long long)s.h); }
    else if (!std::strcmp(c, "C")) {
      auto v = tune_candidates(p);
      std::printf("%d", (int)v.size());
      for (auto& s : v) std::printf(" %d %lld", s.K, (long long)s.h);
      std::printf("\n");
    } else if (!std::strcmp(c, "T")) {
      int mixed; double req;
      std::scanf("%d %lf", &mixed, &req);
      std::printf("%.17g\n", handover_theta(p, mixed != 0, req));
    }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def bp(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("batch_plan")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def call(*lines):
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True,
                             check=True).stdout.strip().split("\n")
        return [[float(x) if "." in x or "e" in x else int(x) for x in line.split()] for line in out]
    return call


ORDERS = [2, 63, 64, 65, 100, 127, 128, 257, 500, 777, 1000, 1023, 1024, 1025, 1500, 2047, 2048, 3000, 4095,
          4096, 4097, 5000, 8191, 8192, 9000]


def test_buckets_are_the_smallest_multiple_of_their_granularity(bp):
    got = [r[0] for r in bp(*[f"B {p}" for p in ORDERS])]
    for p, pb in zip(ORDERS, got):
        g = 64 if p <= 1024 else (128 if p <= 4096 else 256)
        assert pb >= p and pb % g == 0 and pb - p < g


def _sets(p, K, h):
    return [(max(0, k * p // K - h), min(p, (k + 1) * p // K + h)) for k in range(K)]


def _valid(p, sets):
    lo, hi = zip(*sets)
    if lo[0] != 0 or hi[-1] != p:
        return False
    for k, (a, b) in enumerate(sets):
        if not (0 <= a < b <= p) or (len(sets) > 1 and b - a >= p):
            return False
        if k and not (a > lo[k - 1] and b > hi[k - 1] and a <= hi[k - 1]):
            return False
    return True


def test_every_shape_the_executor_may_pick_is_a_valid_partition(bp):
    import paper_2502_06377_gb300 as ibmi
    buckets = sorted({r[0] for r in bp(*[f"B {p}" for p in ORDERS]) if r[0] >= 128})
    shapes = []
    for pb in buckets:
        (Kd, hd), = bp(f"D {pb}")
        (Kr, hr), = bp(f"R {pb}")
        cand, = bp(f"C {pb}")
        n = cand[0]
        assert n >= 1
        shapes += [(pb, Kd, hd), (pb, Kr, hr)] + [(pb, cand[1 + 2 * i], cand[2 + 2 * i]) for i in range(n)]
        assert 2 <= Kd <= 4 and 2 <= Kr <= 8 and all(2 <= cand[1 + 2 * i] <= 4 for i in range(n))
    for pb, K, h in shapes:
        assert _valid(pb, _sets(pb, K, h)), (pb, K, h)
        if pb > 2048:
            continue   # the library check below allocates on a GPU machine; the small ones suffice
        try:
            plan = ibmi.ibmi_plan(pb, K=K, h=h, precision=ibmi.IBMI_MIXED)
            plan.close()
        except ibmi.IbmiError as e:
            assert e.status != ibmi.IBMI_ERR_INVALID_ARG, (pb, K, h)


def test_robust_partition_has_cores_near_256_rows_and_30_percent_overlap(bp):
    for pb in (512, 1024, 2048, 4096, 8192):
        (K, h), = bp(f"R {pb}")
        m = pb // K
        assert K == min(8, max(2, pb // 256))
        assert 2 * h == pytest.approx(0.3 * m, abs=2)


def test_handover_threshold(bp):
    got = [r[0] for r in bp("T 512 1 0", "T 1024 1 0", "T 1088 1 0", "T 4096 1 0", "T 512 1 0.5", "T 4096 0 0.9")]
    assert got == [3.0, 3.0, 0.9, 0.9, 0.5, 0.0]
