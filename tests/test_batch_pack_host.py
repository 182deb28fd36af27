"""Host check of the batched / served input word: each observation's camera
and point packed into one 32-bit word (pack_obs_index in the multi-problem
engine's header).  Valid indices must come back unchanged, and an index out
of range (negative or past the problem's count) must decode to a value the
device's validation still reports as out of range.  The header is compiled
by nvcc into a host-only program (no CUDA call is made, so no GPU is needed).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_15271_b300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

PROGRAM = r"""
#include <cstdio>
#include "batch.h"
using namespace ba;
int main() {
  int bad = 0;
  const int Cs[] = {1, 2, 60, kBatchMaxCams};
  const int Ps[] = {1, 500, 8000, kBatchMaxPts};
  for (int C : Cs)
    for (int P : Ps) {
      const int cams[] = {0, C - 1, C / 2};
      const int pts[] = {0, P - 1, P / 3};
      for (int c : cams)
        for (int j : pts) {
          const uint32_t w = pack_obs_index(c, j, C, P);
          if (obs_cam(w) != c || obs_pt(w) != j) ++bad;
        }
      // out of range on either side, alone or together
      const int badc[] = {-1, C, C + 1, 1 << 20, -2147483647 - 1};
      const int badj[] = {-1, P, P + 7, 1 << 30, -2147483647 - 1};
      for (int c : badc) {
        const uint32_t w = pack_obs_index(c, 0, C, P);
        if (obs_cam(w) < C || obs_pt(w) != 0) ++bad;
      }
      for (int j : badj) {
        const uint32_t w = pack_obs_index(0, j, C, P);
        if (obs_pt(w) < P || obs_cam(w) != 0) ++bad;
      }
      const uint32_t w = pack_obs_index(-5, -5, C, P);
      if (obs_cam(w) < C || obs_pt(w) < P) ++bad;
    }
  std::printf("bad=%d\n", bad);
  return bad != 0;
}
"""


@pytest.mark.skipif(not os.path.exists(NVCC) and shutil.which("nvcc") is None,
                    reason="nvcc not available")
def test_packed_observation_index_round_trips_and_keeps_bad_indices_bad(tmp_path):
    src = tmp_path / "pack_check.cu"
    exe = tmp_path / "pack_check"
    src.write_text(PROGRAM)
    nvcc = NVCC if os.path.exists(NVCC) else shutil.which("nvcc")
    cmd = [nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and "bad=0" in r.stdout, r.stdout + r.stderr
