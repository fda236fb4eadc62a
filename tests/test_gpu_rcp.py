"""The branch-free FP32 reciprocal used for generated Cauchy entries equals
CUDA's correctly rounded reciprocal (__frcp_rn) for every significand, both
signs and every exponent of its stated range; the FP64 reciprocal of the
bounds' near-field terms is within one ulp of 1.0/b on 2^26 operands over
the exponent range (GPU checks built from tests/harness/rcp_check.cu)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_22344_gb300", "csrc")


def test_rcp_nr_is_correctly_rounded(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "rcp_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I", CSRC,
                    os.path.join(HERE, "harness", "rcp_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "mismatches 0" in out.stdout, out.stdout
    # the FP64 reciprocal of the bounds' near-field terms: within one ulp of 1.0/b
    assert "f64 max ulp 0" in out.stdout or "f64 max ulp 1\n" in out.stdout, out.stdout
