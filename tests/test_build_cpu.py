"""Cross-compilation checks that need no GPU: the tensor-core product check program
(tests/tcgemm_check.cu, run by tests/test_gpu_tcgemm.py on a GB300) still compiles for
sm_103a against the current kernel headers."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else shutil.which("nvcc")


def test_tcgemm_check_program_compiles(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    cmd = [nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
           "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "paper_2510_02635_gb300", "csrc"),
           "-c", os.path.join(HERE, "tcgemm_check.cu"), "-o", str(tmp_path / "check.o")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
