"""The integer FP64 -> FP32 conversions used on the GPU by the mixed modes
(FP32 copies of tensors, FP32 pairs of the double-float products) agree bit
for bit with the round-to-nearest-even casts of the host compiler, on random
bit patterns, values of ordinary magnitude and exact rounding ties."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_split_and_to_f32_match_casts(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "f64_bits_driver")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe, os.path.join(HERE, "f64_bits_driver.cpp")],
                   check=True)
    out = subprocess.run([exe, "2000000"], capture_output=True, text=True, check=True).stdout.split()
    bad, cases = int(out[0]), int(out[1])
    assert cases > 7_000_000
    assert bad == 0
