"""Host-side checks of the tensor-core GEMM's shared-memory layout and
descriptors (csrc/tc_gemm.cuh), compiled as a host program with nvcc.

* The staging layout tc_off is a bijection of the 128 x 64 BF16 chunk onto its
  16 KB, with 16-byte rows of 8 elements (core matrices of 128 bytes).
* The descriptor walk of each K = 16 MMA visits exactly the staged elements.
  The walk is start + (row / 8) * SBO + (k / 8) * LBO + (row % 8) * 16 +
  (k % 8) * 2, with start = chunk + kk * 256 and the kernel's LBO = 128 and
  SBO = 1024.  These are the canonical no-swizzle K-major strides.
* The start, LBO and SBO fields of tc_desc decode back to the values put in,
  and the version bits are set.
* The instruction descriptor's fields hold FP32 D, BF16 A and B, K-major
  operands, N = 128 and M = 128.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

PROGRAM = r"""
#include <cstdio>
#include <vector>
#include "tc_gemm.cuh"
using namespace fsim;
int main() {
  int bad = 0;
  std::vector<int> seen(kTcStage, 0);
  for (int r = 0; r < kTcM; ++r)
    for (int k = 0; k < kTcK; ++k) {
      const uint32_t o = tc_off(r, k);
      if (o + 2 > kTcStage || (o & 1)) { ++bad; continue; }
      seen[o] += 1;
      seen[o + 1] += 1;
      if (k % 8 == 0 && o % 16 != 0) ++bad;  // each 8-element row starts a 16-byte line
    }
  for (uint32_t i = 0; i < kTcStage; ++i) bad += seen[i] != 1;
  printf("bijection %d\n", bad);
  bad = 0;
  for (int kk = 0; kk < kTcK / 16; ++kk)
    for (int r = 0; r < kTcM; ++r)
      for (int k = 0; k < 16; ++k) {
        const uint32_t walk = kk * 256u + (uint32_t)(r / 8) * kTcSbo + (uint32_t)(k / 8) * kTcLbo +
                              (uint32_t)(r % 8) * 16u + (uint32_t)(k % 8) * 2u;
        bad += walk != tc_off(r, kk * 16 + k);
      }
  printf("walk %d\n", bad);
  const uint64_t d = tc_desc(0x12340u, kTcLbo, kTcSbo);
  bad = 0;
  bad += (d & 0x3FFFu) != (0x12340u >> 4);
  bad += ((d >> 16) & 0x3FFFu) != (kTcLbo >> 4);
  bad += ((d >> 32) & 0x3FFFu) != (kTcSbo >> 4);
  bad += ((d >> 46) & 0x3u) != 1u;
  bad += ((d >> 61) & 0x7u) != 0u;
  printf("desc %d\n", bad);
  const uint32_t i = kTcIdesc;
  bad = 0;
  bad += ((i >> 4) & 0x3u) != 1u;    // D: FP32
  bad += ((i >> 7) & 0x7u) != 1u;    // A: BF16
  bad += ((i >> 10) & 0x7u) != 1u;   // B: BF16
  bad += ((i >> 15) & 0x3u) != 0u;   // A, B K-major
  bad += ((i >> 17) & 0x3Fu) * 8u != (uint32_t)kTcN;
  bad += ((i >> 24) & 0x1Fu) * 16u != (uint32_t)kTcM;
  bad += (i & 0xFu) != 0u;           // dense, no saturation
  printf("idesc %d\n", bad);
  return 0;
}
"""


@pytest.fixture(scope="module")
def layout_output(tmp_path_factory):
    if not (os.path.exists(NVCC) or shutil.which("nvcc")):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("tc_layout")
    src = d / "tc_layout.cu"
    src.write_text(PROGRAM)
    exe = d / "tc_layout"
    inc = os.path.join(ROOT, "paper_2510_24968_gb300", "csrc")
    # the header also holds the kernel, whose tcgen05 instructions need the sm_103a target
    r = subprocess.run([NVCC if os.path.exists(NVCC) else "nvcc", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-std=c++17", "-I", inc, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return dict(line.split() for line in out.strip().splitlines())


@pytest.mark.parametrize("check", ["bijection", "walk", "desc", "idesc"])
def test_tc_gemm_layout_and_descriptors(layout_output, check):
    assert layout_output[check] == "0"
