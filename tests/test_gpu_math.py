"""The FP64 step's reciprocal and square root (Newton-Raphson from the hardware
seeds, ark_step.cuh) against CUDA's correctly rounded division and square root.

The probe (tests/gpu_math_probe.cu) includes the kernel header itself, so it
checks the functions the step kernels run, on 2^26 log-uniform arguments in
[2^-40, 2^40].
"""
import os
import re
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_fp64_newton_reciprocal_and_sqrt_are_correctly_rounded(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "gpu_math_probe")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "--expt-relaxed-constexpr", f"-I{os.path.join(ROOT, 'include')}",
                    f"-I{os.path.join(ROOT, 'paper_1903_09043_gb300', 'csrc')}",
                    os.path.join(HERE, "gpu_math_probe.cu"), "-o", exe], check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    m = re.search(r"max ulp: rcp (\d+)\s+sqrt (\d+)\s+rsqrt (\d+)", out)
    assert m, out
    rcp_ulp, sqrt_ulp, rsqrt_ulp = (int(g) for g in m.groups())
    assert rcp_ulp == 0 and sqrt_ulp == 0, out
    assert rsqrt_ulp <= 1, out
