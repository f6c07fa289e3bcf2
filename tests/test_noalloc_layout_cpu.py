"""The scratch layout of the no-allocation entry point, checked on the CPU.

The layout arithmetic lives in plain host C++ (``csrc/noalloc_layout.h``), so
this test compiles it with g++ and checks, for every size the entry point
accepts (1 .. 65536 systems), that each section is aligned for its element
type, that the sections do not overlap and that the whole layout fits the
fixed array sized for the maximum.  No GPU is involved.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1810_03931_gb300", "csrc")

CHECK = r"""
#include <stdio.h>
#include "noalloc_layout.h"
using namespace odegpu;
int main() {
  const size_t max_n = 65536, E = 2;
  const NoAllocLayout big = noalloc_layout(max_n, E);
  if (big.total != 1835264) { printf("total %zu\n", big.total); return 1; }
  for (size_t n = 1; n <= max_n; n++) {
    const NoAllocLayout L = noalloc_layout(n, E);
    // alignment of every section for its element type (and to 256 bytes)
    if (L.nacc % 8 || L.nrej % 8 || L.status % 4 || L.ecnt % 4) { printf("align %zu\n", n); return 2; }
    if (L.nacc % 256 || L.nrej % 256 || L.status % 256 || L.ecnt % 256) { printf("a256 %zu\n", n); return 3; }
    // order and no overlap: head | nacc | nrej | status | ecnt
    if (L.head != 0 || L.nacc < 256) { printf("head %zu\n", n); return 4; }
    if (L.nacc + 8 * n > L.nrej || L.nrej + 8 * n > L.status || L.status + 4 * n > L.ecnt ||
        L.ecnt + 4 * E * n > L.total) { printf("overlap %zu\n", n); return 5; }
    // fits the fixed array, and the array is never larger than needed
    if (L.total > big.total) { printf("fit %zu\n", n); return 6; }
    if (L.total - (L.ecnt + 4 * E * n) >= 256) { printf("slack %zu\n", n); return 7; }
  }
  printf("ok\n");
  return 0;
}
"""


def test_noalloc_layout_aligned_and_fits_for_every_size(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "check_layout.cc"
    src.write_text(CHECK)
    exe = tmp_path / "check_layout"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I" + CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout


def test_noalloc_entry_point_uses_the_layout():
    """The CUDA side takes its section offsets and array size from the same
    header (no second copy of the arithmetic)."""
    src = open(os.path.join(CSRC, "noalloc.cu")).read()
    assert '#include "noalloc_layout.h"' in src
    assert "noalloc_layout(kNoAllocMaxSystems, kMaxE).total" in src
    assert "noalloc_layout(N, kMaxE)" in src
