"""The integer-pipe FP32<->FP64 conversions used by the FP64 eliminations agree bit for bit
with the hardware conversions (GPU; compiles tests/cuda/convert_check.cu with nvcc)."""
import os
import shutil
import subprocess

import pytest
import torch

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_conversions_match_hardware(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "convert_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "cuda", "convert_check.cu")], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    vals = dict(line.split(None, 1) for line in out.stdout.strip().splitlines())
    assert vals["status"] == "no error"
    assert int(vals["widen_mismatches"]) == 0
    assert int(vals["narrow_mismatches"]) == 0
