"""Host logic that decides where a caller's array lives (no GPU needed).

Every entry point asks the driver for a pointer's attributes and stages host
memory through a device buffer; device memory that belongs to another GPU than
the current one must be refused with OLB_ERR_ARG instead of being handed to a
kernel that would address it without peer access.  The classification is a pure
function of the attributes; this test compiles it with the host compiler and
checks every case, including the mismatched owner device that a one-GPU machine
cannot produce.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2307_11752_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

DRIVER = r"""
#include <cstdio>
#include "olb_internal.h"
using namespace olb;
int main() {
  struct { cudaMemoryType t; int owner, cur; MemKind want; } cases[] = {
    {cudaMemoryTypeUnregistered, -1, 0, MEM_HOST},   // pageable host memory
    {cudaMemoryTypeHost, 0, 0, MEM_HOST},            // pinned host memory
    {cudaMemoryTypeDevice, 0, 0, MEM_DEVICE},        // the current device's memory
    {cudaMemoryTypeDevice, 3, 3, MEM_DEVICE},
    {cudaMemoryTypeDevice, 1, 0, MEM_OTHER_DEVICE},  // another GPU's memory: refused
    {cudaMemoryTypeDevice, 0, 5, MEM_OTHER_DEVICE},
    {cudaMemoryTypeManaged, 2, 0, MEM_DEVICE},       // managed memory is addressable
  };
  int bad = 0;
  for (auto& c : cases) {
    MemKind k = classify_memory(c.t, c.owner, c.cur);
    if (k != c.want) { std::printf("type %d owner %d current %d -> %d\n", (int)c.t, c.owner, c.cur, (int)k); ++bad; }
  }
  std::printf("%d mismatches\n", bad);
  return bad;
}
"""


@pytest.mark.skipif(not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")) or shutil.which("g++") is None,
                    reason="needs the CUDA headers and g++")
def test_device_memory_of_another_gpu_is_refused(tmp_path):
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "drv"
    r = subprocess.run(["g++", "-std=c++17", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
