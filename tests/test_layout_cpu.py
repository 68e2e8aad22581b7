"""Shared-memory layout of the row-gather kernels (host logic, no GPU).

tests/layout_check.cu includes the library's layout definition and checks,
over precisions, the assembly and time-step layouts, block sizes and row,
entry and step counts, that every region is 16-byte aligned, that regions do
not overlap and that every alias the kernels use fits (column indices in nb1,
staged record halves in the accumulators, the write-out staging in nb0).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gather_shared_memory_layout(tmp_path):
    nvcc = next((c for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc"))
                 if c and os.path.exists(c)), None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = tmp_path / "layout_check"
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "layout_check.cu"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures=0" in r.stdout
