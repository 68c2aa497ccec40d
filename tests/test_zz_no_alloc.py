"""The allocation-free close product (for callers that cannot allocate device
memory) against the library's regular path.

ttn_close_noalloc keeps its split-K partial sums in a fixed array inside the
library.  Its output must equal what ttn_ascend produces for the same product
-- the coarse-grained operator A'_k = W (I (x) A_k) W^T = close(W A_k, W) --
on two calls in a row (the second reuses the array the first one filled).
Kept in a file collected last so that a failure here stops a run only after
every other test.
"""
import ctypes

import numpy as np
import pytest

import ttn_inputs as ti

pytestmark = pytest.mark.gpu


def test_close_noalloc_matches_ascend_twice():
    import torch
    from paper_1905_01331_gb300 import Sweeper, _abi
    lib = _abi.load()
    m = ti.heisenberg_xxx(64)
    ws, V = ti.initial_tensors(64, 2, 32, 9)
    s = Sweeper(m, 32)
    s.set_isometries(0, ws, V)
    stream = torch.cuda.current_stream()
    for t, k in ((3, 0), (2, 2)):          # two calls in a row, different sizes
        ops_t = s.ascend(0, t)[0]          # o, A_k, B_k at site layer t (regular path)
        ops_up = s.ascend(0, t + 1)[0]
        w = ws[t]                          # (P, n, n)
        P, n = w.shape[0], w.shape[1]
        Y = np.einsum("plr,rs->pls", w, ops_t[1 + k])      # W (I (x) A_k)
        dY = torch.from_numpy(np.ascontiguousarray(Y.reshape(P, n * n))).cuda()
        dW = torch.from_numpy(np.ascontiguousarray(w.reshape(P, n * n))).cuda()
        dC = torch.full((P, P), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.ttn_close_noalloc(ctypes.c_void_p(dY.data_ptr()), ctypes.c_void_p(dW.data_ptr()),
                                   P, P, n * n, ctypes.c_void_p(dC.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        got = dC.cpu().numpy()
        ref = ops_up[1 + k]
        err = np.abs(got - ref).max() / np.abs(ref).max()
        print("layer", t, "term", k, "max rel err vs ttn_ascend", err)
        assert err < 1e-13
    s.close()


def test_close_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1905_01331_gb300 import _abi
    lib = _abi.load()
    x = torch.zeros(4, device="cuda", dtype=torch.float64)
    p = ctypes.c_void_p(x.data_ptr())
    assert lib.ttn_close_noalloc(p, p, 257, 4, 4, p, None) == -1
    assert lib.ttn_close_noalloc(p, p, 4, 0, 4, p, None) == -1


@pytest.mark.parametrize("P,Q,n2", [(256, 256, 6144), (200, 64, 3000), (64, 256, 40000)])
def test_close_noalloc_at_its_limits_against_fp64_matmul(P, Q, n2):
    """Shapes that reach the cap of the split count by the 8 MiB array
    (256 x 256 with a long reduction wants more splits than 16 x 65536
    doubles allow), non-square outputs and a long ragged reduction, against
    a PyTorch FP64 matmul, on two calls in a row."""
    import torch
    from paper_1905_01331_gb300 import _abi
    lib = _abi.load()
    g = torch.Generator(device="cuda").manual_seed(P * 7 + Q)
    Y = torch.rand(P, n2, generator=g, device="cuda", dtype=torch.float64) - 0.5
    W = torch.rand(Q, n2, generator=g, device="cuda", dtype=torch.float64) - 0.5
    ref = Y @ W.T
    stream = torch.cuda.current_stream()
    for _ in range(2):
        C = torch.full((P, Q), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.ttn_close_noalloc(ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(W.data_ptr()),
                                   P, Q, n2, ctypes.c_void_p(C.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        err = ((C - ref).abs().max() / ref.abs().max()).item()
        assert err < 1e-13, (P, Q, n2, err)
