"""The library refuses caller buffers that are device memory of another GPU
than the mesh's (a kernel there would fault) and reads host memory only
through staging.  The decision is a pure function of the attributes the CUDA
runtime reports (csrc/ptr_kind.h); with one GPU no foreign pointer can be made,
so this test compiles the function on the host and checks every case,
including that its memory-type codes are CUDA's."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2605_01536_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <driver_types.h>
#include "ptr_kind.h"
static_assert(cudaMemoryTypeUnregistered == 0 && cudaMemoryTypeHost == 1 && cudaMemoryTypeDevice == 2 &&
              cudaMemoryTypeManaged == 3, "memory type codes");
int main() {
    int bad = 0;
    bad += gwn_pointer_kind_of(cudaMemoryTypeDevice, 1, 0) != -1;   // another GPU's memory: refused
    bad += gwn_pointer_kind_of(cudaMemoryTypeDevice, 0, 1) != -1;
    bad += gwn_pointer_kind_of(cudaMemoryTypeDevice, 3, 3) != 1;    // the mesh's own GPU
    bad += gwn_pointer_kind_of(cudaMemoryTypeManaged, 7, 0) != 1;   // managed memory migrates
    bad += gwn_pointer_kind_of(cudaMemoryTypeHost, 0, 0) != 0;      // pinned host memory: staged
    bad += gwn_pointer_kind_of(cudaMemoryTypeUnregistered, -2, 0) != 0;   // pageable host memory
    std::printf("%d\n", bad);
    return bad;
}
"""


def test_pointer_kind_cases(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = "/usr/local/cuda/include"
    if not cxx or not os.path.exists(os.path.join(inc, "driver_types.h")):
        pytest.skip("needs a host C++ compiler and the CUDA headers")
    src = tmp_path / "pk.cpp"
    src.write_text(PROG)
    exe = tmp_path / "pk"
    subprocess.run([cxx, "-std=c++17", "-I", HDR, "-I", inc, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "0", r.stdout
