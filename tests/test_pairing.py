"""The CTA-pair kernel's pairing of tile pairs (csrc/fused_pairing.h), checked on the host.

The kernel's two CTAs share a column tile, and a channel's lower-triangle tile pairs (Eq. 1's
V split into 128 x 128 blocks) are grouped into entries by a closed form.  A wrong entry would
drop or double-count visibilities; the GPU parity tests catch that for the tile counts they run
(1, 2, 4, 5, 7, 8), and this test compiles the same header with g++ and checks every tile count
up to 300: each tile pair exactly once, a single row tile only when the count of tile pairs is
odd, the advertised number of entries, and transposed tile pairs only where a column took one.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1401_8288_gb300", "csrc")
OUT = os.path.join(ROOT, "paper_1401_8288_gb300", "_lib")

CHECKER = r'''
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "fused_pairing.h"
using namespace xc::fused;
int main(int argc, char** argv) {
  if (argc > 1) {  // print one tile count's entries
    const int nb = std::atoi(argv[1]);
    for (int e = 0; e < pair_entries(nb); ++e) {
      int S, r0, r1;
      pair_entry(nb, e, S, r0, r1);
      std::printf("%d %d %d\n", S, r0, r1);
    }
    return 0;
  }
  for (int nb = 1; nb <= 300; ++nb) {
    const int pairs = nb * (nb + 1) / 2, n = pair_entries(nb);
    if (n != (pairs + 1) / 2) { std::printf("nb %d: %d entries\n", nb, n); return 1; }
    std::vector<int> seen(nb * nb, 0);
    int singles = 0, covered = 0;
    for (int e = 0; e < n; ++e) {
      int S, r[2];
      pair_entry(nb, e, S, r[0], r[1]);
      if (S < 0 || S >= nb || r[0] < 0) { std::printf("nb %d entry %d: S %d r0 %d\n", nb, e, S, r[0]); return 1; }
      for (int k = 0; k < 2; ++k) {
        if (r[k] < 0) { ++singles; continue; }
        if (r[k] >= nb || (r[k] < S && !(r[k] == S - 2 && pair_col_kind(nb, S) == kColTakes))) {
          std::printf("nb %d entry %d: row tile %d against column %d\n", nb, e, r[k], S);
          return 1;
        }
        const int I = r[k] > S ? r[k] : S, J = r[k] > S ? S : r[k];
        if (seen[I * nb + J]++) { std::printf("nb %d: tile pair (%d, %d) twice\n", nb, I, J); return 1; }
        ++covered;
      }
    }
    if (covered != pairs || singles != pairs % 2) {
      std::printf("nb %d: %d of %d tile pairs, %d singles\n", nb, covered, pairs, singles);
      return 1;
    }
  }
  std::printf("ok\n");
  return 0;
}
'''


@pytest.fixture(scope="module")
def checker():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    os.makedirs(OUT, exist_ok=True)
    src = os.path.join(OUT, "pairing_check.cpp")
    exe = os.path.join(OUT, "pairing_check")
    with open(src, "w") as f:
        f.write(CHECKER)
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, src, "-o", exe], check=True)
    return exe


def test_every_tile_pair_once_up_to_300_tiles(checker):
    r = subprocess.run([checker], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout


def test_four_tiles_pair_by_column_with_one_transposed(checker):
    # 512 inputs: column 0 pairs rows (0, 1) and (2, 3); columns 1 and 3 have odd counts, so
    # column 3 takes the tile pair (3, 1) as row tile 1 (transposed) and column 1 keeps (1, 2)
    r = subprocess.run([checker, "4"], capture_output=True, text=True, check=True)
    entries = [tuple(int(v) for v in line.split()) for line in r.stdout.split("\n") if line]
    assert entries == [(0, 0, 1), (0, 2, 3), (1, 1, 2), (2, 2, 3), (3, 1, 3)]


def test_odd_counts_keep_one_single(checker):
    # 2 tiles: 3 tile pairs, so one entry holds a single row tile (the odd CTA idles)
    r = subprocess.run([checker, "2"], capture_output=True, text=True, check=True)
    entries = [tuple(int(v) for v in line.split()) for line in r.stdout.split("\n") if line]
    assert entries == [(0, 0, 1), (1, 1, -1)]
