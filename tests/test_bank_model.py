"""The shared-memory bank model that picks the row passes' row strides
(paper_2310_19840_gb300/csrc/bank_model.h), on the CPU.

A small C++ program includes the header and prints, per launch shape, the
chosen strides and their wavefront counts next to those of the fixed strides
used before (FFT scratch n + n/16 + 1, staging W | 1).  Checked: every
stride lies in [length, length + E), it is never worse than the fixed one,
and at the default dealiasing width the cooperative copies into the staging
rows need only the minimum number of wavefronts (two per 32 FP32 complex).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r'''
#include <cstdio>
#include "bank_model.h"
using namespace sbi::bank;
// the fewest wavefronts the cooperative I/O could take: per warp instruction
// ceil(active lanes / E)
long long coop_min(const Geometry& g) {
  const int threads = g.rpc * g.TPR, kstep = threads / g.rpc;
  long long tot = 0;
  for (int w = 0; w * 32 < threads; ++w)
    for (int it = 0; it * kstep < g.W; ++it) {
      int cnt = 0;
      for (int t = 32 * w; t < threads && t < 32 * w + 32; ++t)
        if (t / g.rpc + it * kstep < g.W) ++cnt;
      tot += (cnt + g.E - 1) / g.E;
    }
  return tot;
}
int main() {
  for (int eb : {8, 16}) {
    const int E = 128 / eb;
    for (int NX : {32, 64, 128, 256, 512, 1024, 2048, 4096}) {
      const int n = NX / 2, R = 8, TPR = n / R;
      for (int W : {NX / 4, NX / 8 + 1}) {
        for (int rpc = 1; rpc <= 32; rpc *= 2) {
          if ((rpc * TPR) % 32) continue;
          const Geometry g{n, R, TPR, rpc, W, E};
          const RowStrides s = choose(n, R, TPR, rpc, W, eb, false, false);
          const int fb = n + n / 16 + 1, sw = W | 1;
          auto io = [&](int S) {
            return coop_cost(g, [&](int rl, int k) { return rl * S + pad16(k); }) +
                   coop_cost(g, [&](int rl, int k) { return rl * S + pad16((n - k) & (n - 1)); });
          };
          auto stg = [&](int S) { return coop_cost(g, [&](int rl, int k) { return rl * S + k; }); };
          const long long minio = coop_min(g);
          printf("%d %d %d %d %d %d %lld %lld %d %lld %lld %lld %d\n", eb, NX, W, rpc, s.fbs, fb,
                 fft_cost(g, s.fbs) + io(s.fbs), fft_cost(g, fb) + io(fb), s.sws,
                 stg(s.sws) + c2r_cost(g, s.sws), stg(sw) + c2r_cost(g, sw), stg(s.sws) - minio,
                 E);
        }
      }
    }
  }
}
'''


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ is not available")
    d = tmp_path_factory.mktemp("bank")
    src, exe = d / "bank.cpp", d / "bank"
    src.write_text(PROGRAM)
    inc = os.path.join(ROOT, "paper_2310_19840_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return [list(map(int, ln.split())) for ln in out.splitlines()]


def test_strides_lie_in_range_and_never_lose(rows):
    assert len(rows) > 60
    for eb, nx, w, rpc, fbs, fb, cost, cost_fixed, sws, scost, scost_fixed, _, e in rows:
        assert fb <= fbs < fb + e and w <= sws < w + e, (eb, nx, w, rpc)
        assert cost <= cost_fixed and scost <= scost_fixed, (eb, nx, w, rpc)


def test_cooperative_staging_reaches_the_minimum(rows):
    # at the default dealiasing (W = nx/4); for other widths the model may
    # trade a wavefront of the copies for fewer in the packed inverse's reads
    for eb, nx, w, rpc, *_, excess, e in rows:
        if w == nx // 4:
            assert excess == 0, (eb, nx, w, rpc)


def test_known_gains_of_the_benchmark_shapes(rows):
    # FP32, 8 rows per block: the fixed strides left four rows on a bank group
    by = {(r[0], r[1], r[2], r[3]): r for r in rows}
    r256 = by[(8, 256, 64, 8)]
    r512 = by[(8, 512, 128, 8)]
    assert (r256[6], r256[7]) == (484, 512)
    assert (r512[6], r512[7]) == (904, 1024)
    assert (r512[9], r512[10]) == (192, 256)
