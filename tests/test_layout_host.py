"""The fill's shared-memory layout, checked on the host: tests/host/layout_check.cu includes the library's host
source and walks many (d, N_g, precision, parameter count) cases, the streamed path's table-less layout among
them.  Every region the kernels index must be 16-byte aligned, in order, free of overlap and inside the total."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_shared_memory_layout(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc is not installed")
    exe = str(tmp_path / "layout_check")
    inc = os.path.join(os.path.dirname(HERE), "include")
    build = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode",
                            "arch=compute_103a,code=sm_103a", "-I", inc, os.path.join(HERE, "host", "layout_check.cu"),
                            "-o", exe], capture_output=True, text=True, timeout=600)
    assert build.returncode == 0, build.stderr[-3000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and run.stdout.startswith("ok"), run.stdout + run.stderr
