"""Pins of the double-float (FP32 pair) tridiagonal routines behind the
convergence checks of the Lanczos kernel, run on the host: Sturm counts are
the number of eigenvalues below a point (the count numpy's symmetric
eigensolver gives away from the eigenvalues), the bisected lowest eigenvalue
matches numpy's to ~1e-14 of the spectral scale, and one inverse-iteration
round gives the last component of the lowest eigenvector (the quantity of the
Ritz residual |beta_{m-1} y_{m-1}| of the Lanczos method) to ~1e-11."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("tdf") / "tridiag_df_driver")
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe, os.path.join(HERE, "tridiag_df_driver.cpp")],
                   check=True)
    return exe


def _cases(seed, n):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n):
        m = int(rng.integers(1, 60))
        sc = 10.0 ** int(rng.integers(-1, 3))
        a = sc * rng.normal(size=m) - (900.0 if t % 2 else 0.0)
        b = sc * (np.abs(rng.normal(size=max(m - 1, 0))) + 0.05)
        if t % 3 == 0:            # lowest eigenvector decaying toward the end
            a[m // 2:] += 20 * sc
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        w, V = np.linalg.eigh(T)
        # a probe point between two eigenvalues (or outside the spectrum)
        k = int(rng.integers(0, m + 1))
        lo = w[k - 1] if k > 0 else w[0] - sc
        hi = w[k] if k < m else w[-1] + sc
        out.append((a, b, 0.5 * (lo + hi), k, w, V))
    return out


def _run(driver, cases):
    text = "".join(f"{len(a)} {x!r} " + " ".join(repr(v) for v in a) + " "
                   + " ".join(repr(v) for v in b) + "\n" for a, b, x, *_ in cases)
    res = subprocess.run([driver], input=text, capture_output=True, text=True, check=True)
    return [line.split() for line in res.stdout.strip().splitlines()]


def test_sturm_counts_match_eigenvalue_counts(driver):
    cases = _cases(1, 400)
    for (a, b, x, k, w, V), (cnt, _, _) in zip(cases, _run(driver, cases)):
        gap = np.min(np.abs(w - x))
        if gap > 1e-9 * max(1.0, np.max(np.abs(w))):
            assert int(cnt) == k


def test_lowest_eigenvalue_and_last_component(driver):
    cases = _cases(2, 400)
    for (a, b, x, k, w, V), (_, th, y) in zip(cases, _run(driver, cases)):
        scale = max(1.0, np.max(np.abs(w)))
        assert abs(float(th) - w[0]) <= 5e-14 * scale
        if len(a) > 1 and w[1] - w[0] > 1e-6 * scale:      # simple, separated eigenvalue
            assert abs(float(y) - abs(V[-1, 0])) <= 1e-10
