"""The tcgen05 engine against the FP64 engine (C ABI diagnostic entry point),
and the mixed-precision sweep against the FP64 oracle."""
import ctypes

import numpy as np
import pytest

import ttn_inputs as ti
from oracle import ttn as oracle

pytestmark = pytest.mark.gpu

# max |C_tc - C_fp64| / max |C_fp64| for K up to 16384 and |entries| <= 1:
# one TF32 product keeps 11 bits, one BF16 product 8; the split forms add a
# correction term and lose only the FP32 accumulation.
TOL = {1: 5e-3, 2: 2e-5, 3: 4e-2, 4: 5e-4}


@pytest.mark.parametrize("prec", [1, 2, 3, 4])
def test_tensor_core_engine_matches_fp64(prec):
    import torch
    from paper_1905_01331_gb300 import _abi
    lib = _abi.load()
    nbytes = lib.ttn_selftest_bytes()
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = np.zeros(6)
    rc = lib.ttn_selftest_gemm(ctypes.c_void_p(ws.data_ptr()), nbytes, prec,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 6,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    print("prec", prec, "relative errors per case", out)
    assert rc == 0
    assert np.all(np.isfinite(out))
    assert out.max() < TOL[prec], out


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "tf32"])
def test_mixed_sweep_tracks_oracle(prec):
    """Mixed-precision sweeps from the seeded start stay close to the FP64
    oracle's trajectory and keep exact isometries (FP64 polish)."""
    from paper_1905_01331_gb300 import Sweeper
    m = ti.tfim_chain(256, 1.0)
    ws, V = ti.initial_tensors(256, 2, 64, 5)
    s = Sweeper(m, 64, prec=prec)
    s.set_isometries(0, ws, V)
    E = s.sweep(8)[:, 0]
    st = oracle.make_state(m, ws, V)
    E_ref = np.array([oracle.sweep(st) for _ in range(8)])
    rel = np.abs(E - E_ref) / np.abs(E_ref)
    print(prec, "rel err per sweep", rel)
    tol = {"tf32x3": 1e-6, "bf16x3": 1e-4, "tf32": 1e-3}[prec]
    assert rel.max() < tol
    ws_g, _ = s.get_isometries(0)
    for w in ws_g:
        W = w.reshape(w.shape[0], -1)
        assert np.abs(W @ W.T - np.eye(W.shape[0])).max() < 1e-12
