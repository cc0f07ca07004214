"""Measures the FP64 and FP32 FMA rates of the GPU (the denominators of the
ALU side of the roofline); prints them with -s."""
import os
import re
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_fp_throughput():
    exe = os.path.join(tempfile.mkdtemp(), "fp_throughput")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    os.path.join(HERE, "fp_throughput.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    print(out)
    rates = {m.group(1): float(m.group(2)) for m in re.finditer(r"(fp64|fp32) fma: ([0-9.]+) TFLOP/s", out)}
    assert rates["fp64"] > 0.3 and rates["fp32"] > 10.0
    assert "no error" in out
