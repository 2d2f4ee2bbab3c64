"""Host-side logic of the tensor-core conv (stage plans, layer-shape dispatch), compiled with
nvcc and run on the CPU: tests/host/tc_host_logic.cu launches no kernel."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tc_host_logic():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "tc_host_logic")
        r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "--expt-relaxed-constexpr",
                            "-I" + os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "host", "tc_host_logic.cu"),
                            "-o", exe], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-3000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
        assert r.returncode == 0 and "host logic ok" in r.stdout, r.stdout + r.stderr
