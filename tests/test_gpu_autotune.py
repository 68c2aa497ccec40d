"""The autotuner: per product shape it times the engines, tile widths and
split counts and keeps the fastest; the table round-trips through the
ttn_options.tiles blob, and a context created with it sweeps bit for bit like
the tuned one (deterministic kernels, same configurations)."""
import numpy as np
import pytest

import ttn_inputs as ti
from oracle import ed

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["tf32x3", "fp64"])
def test_autotune_table_round_trip(prec):
    from paper_1905_01331_gb300 import Sweeper
    m = ti.tfim_chain(256, 1.0)
    ws, V = ti.initial_tensors(256, 2, 64, 3)
    a = Sweeper(m, 64, prec=prec)
    a.set_isometries(0, ws, V)
    blob = a.autotune(reps=2)          # one sweep, every product shape tuned
    assert len(blob) > 16 + 24 * 5     # header + at least a few product shapes
    Ea = a.sweep(3)[:, 0]
    b = Sweeper(m, 64, prec=prec, tiles=blob)
    b.set_isometries(0, ws, V)
    Eb = b.sweep(4)[:, 0]
    assert np.array_equal(Ea, Eb[1:]), (Ea, Eb)
    assert b.autotune(reps=0) == blob   # the table b was created with
    c = Sweeper(m, 64, prec=prec)
    c.set_isometries(0, ws, V)
    Ec = c.sweep(4)[:, 0]
    # other split counts round differently: FP64 rounding in FP64 mode, the
    # tensor-core rounding (~1e-6) in 3xTF32; relative to the exact energy
    scale = abs(ed.tfim_closed_form(256, 1.0))
    tol = 1e-12 if prec == "fp64" else 1e-5
    print(prec, "tuned vs default configurations", np.abs(Eb - Ec) / scale)
    assert np.all(np.abs(Eb - Ec) <= tol * scale)
    for s in (a, b, c):
        s.close()
