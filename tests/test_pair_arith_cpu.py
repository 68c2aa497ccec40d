"""Accuracy pin of the double-float (FP32 pair) arithmetic that carries the
polar factor's products, the composition and the top solve's matrix-vector
products in the mixed modes, run on the host with the kernels' own header and
gemm_df_kernel's schedule (split operands, one pair multiply-add per term,
renormalisation every 16 terms): dot products of length 16 to 16384, half of
them with cancellation down to 1e-6 of the terms, stay within 1e-13 of
sum |a_i b_i| of a long-double reference (about 2^-43; measured ~3e-14), at
least 1e5 times closer than FP32 accumulation of the same operands."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_pair_dot_products_keep_about_48_bits(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "pair_arith_driver")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe, os.path.join(HERE, "pair_arith_driver.cpp")],
                   check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    rows = [line.split() for line in out if line.strip()]
    assert [int(r[0]) for r in rows] == [16, 128, 4096, 16384]
    for k, df, f32 in rows:
        df, f32 = float(df), float(f32)
        assert df <= 1e-13, (k, df)
        assert f32 >= 1e5 * df, (k, df, f32)
