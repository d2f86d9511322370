"""Host logic of the streaming Gram-Schmidt kernel: every tile plan keeps its bulk copies
16-byte aligned (tail tiles included) and fits the shared-memory budget (no GPU needed; the
check is compiled with nvcc and runs on the host)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gs_stream_plans():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out_dir = os.path.join(ROOT, "paper_2601_05816_gb300", "_build", "tests")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "gs_plan_check")
    src = os.path.join(ROOT, "tests", "gs_plan_check.cu")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe, src],
                   check=True, capture_output=True, text=True)
    p = subprocess.run([exe], capture_output=True, text=True)
    assert p.returncode == 0, p.stdout + p.stderr
    assert "0 failures" in p.stdout
