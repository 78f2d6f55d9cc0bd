"""The tensor-core products of the per-anchor solve (k_gemm_tc: tcgen05, operands split
into TF32 hi + lo parts) against FP64 host products of the same FP32 inputs: every element
within 4e-6 of sum_k |a b| on ragged shapes of both operand layouts, split over K included.
The check program (tests/tcgemm_check.cu) is compiled for sm_103a with nvcc and run."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_split_tf32_products_match_fp64(tmp_path):
    nvcc = _nvcc()
    assert nvcc, "nvcc not found"
    exe = str(tmp_path / "tcgemm_check")
    cmd = [nvcc, "-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2510_02635_gb300", "csrc"),
           os.path.join(HERE, "tcgemm_check.cu"), "-o", exe]
    b = subprocess.run(cmd, capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count(" ok") == 7
