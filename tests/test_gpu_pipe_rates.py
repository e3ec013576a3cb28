"""The arithmetic rates the precision design rests on (GPU only): on GB300
an FP64 add or fma, and an f32 <-> f64 conversion, issue at a small fraction
of the FP32 fma rate, so the mixed path keeps both out of its per-particle
work (FP64 storage is converted and accumulated with integer instructions).
The measured rates (thread-operations per clock per SM, at the nominal
clock) are printed."""
import os
import shutil
import subprocess

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fp64_and_conversions_are_far_slower_than_fp32(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "pipe_rates"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    os.path.join(ROOT, "tests", "native", "pipe_rates.cu"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    print("\n" + out)
    rates = {l.split()[0]: l.split()[1] for l in out.splitlines()}
    assert rates.pop("status") == "no"  # "no error"
    r = {k: float(v) for k, v in rates.items()}
    assert r["ffma"] > 16 * r["dfma"]
    assert r["ffma"] > 16 * r["dadd"]
    assert r["ffma"] > 16 * r["cvt_f32_f64"]
    assert r["int_add_xor_shift"] > 16 * r["dadd"]
