"""Host-side launch shapes of the SIMT coarse stencil (csrc/launch_shape.h).

The coarse stencil of Sec. 2.3 runs one thread per row pair and chunk of
right-hand sides; a CTA may hold at most 256 threads (the kernels'
__launch_bounds__).  The header is plain C++, so it is compiled here with the
host compiler and its shape checked for every dof count n = 2 nv and batch
size R the solver can meet.  No GPU needed.
"""

import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1610_02370_gb300", "csrc", "launch_shape.h")

DRIVER = r"""
#include <cstdio>
#include "launch_shape.h"
int main() {
  for (int n = 2; n <= 128; n += 2)
    for (int R = 1; R <= 256; R++) {
      ddtm::CoarseShape s = ddtm::coarse_shape(n, R);
      std::printf("%d %d %d %d %d %d %d %d\n", n, R, s.rc, s.nch, s.groups, s.per, s.spb, s.threads);
    }
  return 0;
}
"""


@pytest.fixture(scope="module")
def shapes():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "drv.cpp")
        exe = os.path.join(d, "drv")
        with open(src, "w") as f:
            f.write(DRIVER)
        subprocess.run([cxx, "-std=c++17", "-O1", "-I", os.path.dirname(HDR), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = [tuple(int(t) for t in line.split()) for line in out.splitlines()]
    return rows


def test_threads_never_exceed_launch_bounds(shapes):
    for n, R, rc, nch, groups, per, spb, threads in shapes:
        assert 1 <= threads <= 256, (n, R, threads)
        assert threads == spb * per and per == n // 2 * groups, (n, R)


def test_chunks_cover_every_rhs_once(shapes):
    for n, R, rc, nch, groups, per, spb, threads in shapes:
        assert rc in (1, 2, 4) and R % rc == 0 and nch * rc == R, (n, R, rc)
        # the largest of 4, 2, 1 dividing R (16-byte vector loads where possible)
        assert rc == (4 if R % 4 == 0 else 2 if R % 2 == 0 else 1)
        assert 1 <= groups <= nch, (n, R, groups)
        # thread slot g takes chunks g, g + G, ...: every chunk exactly once
        seen = sorted(ch for g in range(groups) for ch in range(g, nch, groups))
        assert seen == list(range(nch))


def test_former_failures_now_fit(shapes):
    by = {(n, R): (threads, spb) for n, R, _, _, _, _, spb, threads in shapes}
    # n = 48 (N_v = 24) with 11, 13, 44 and 48 right-hand sides used to ask for 264..288 threads
    for R in (11, 13, 44, 48, 64, 96):
        threads, spb = by[(48, R)]
        assert threads <= 256 and spb >= 1
