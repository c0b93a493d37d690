"""The hardware base-2 logarithm the logarithmic-bin path relies on.

The log-bin bands assume lg2.approx.ftz.f32 errs by at most
2^-21 max(1, |log2 x|).  This test measures the error exhaustively, over
every positive normal binary32 input, against the binary64 log2 and checks
both terms of that model: a (largest error where |log2 x| <= 1) and b
(largest error / |log2 x| elsewhere).
"""

import os
import re
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
BOUND = 2.0 ** -21


def test_lg2_error_within_the_assumed_bound(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "lg2_bound")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "lg2_bound.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    vals = dict(re.findall(r"^([ab]) (\S+) at", out, flags=re.M))
    a, b = float(vals["a"]), float(vals["b"])
    assert 0.0 < a <= BOUND, out
    assert 0.0 < b <= BOUND, out
