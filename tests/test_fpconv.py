"""The integer-only binary64 <-> binary32 conversions used by the complex64
packing and accumulation kernels, checked on the host against the CPU's IEEE
round-to-nearest-even conversions (the header compiles as plain C++)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_conversions_match_ieee_round_to_nearest_even(tmp_path):
    exe = tmp_path / "fpconv_check"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2406_08186_b300", "csrc"),
                           "-o", str(exe), os.path.join(ROOT, "tests", "fpconv_check.cpp")])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok ")
    assert int(out.stdout.split()[1]) > 10_000_000
