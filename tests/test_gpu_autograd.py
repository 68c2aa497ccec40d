"""The energy as a torch.autograd.Function whose backward is the environment
kernel: checked against central finite differences and against the oracle's
environment (thin torus, d0 = 16, K = 4 product terms)."""
import numpy as np
import pytest

import ttn_inputs as ti
from oracle import ttn as oracle

pytestmark = pytest.mark.gpu


def _setup(Lx=8, Ly=4, chi=32, seed=3, sweeps=2):
    import torch
    from paper_1905_01331_gb300 import Sweeper
    m = ti.tfim_torus(Lx, Ly, 3.04)
    ws, V = ti.initial_tensors(Lx, m.d0, chi, seed)
    st = oracle.make_state(m, ws, V)
    for _ in range(sweeps):
        oracle.sweep(st)
    s = Sweeper(m, chi)
    tw = [torch.tensor(w, device="cuda", requires_grad=True) for w in st.ws]
    tv = torch.tensor(st.V, device="cuda", requires_grad=True)
    return s, st, tw, tv


def test_autograd_matches_oracle_environment():
    from paper_1905_01331_gb300.autograd import energy
    s, st, tw, tv = _setup()
    E = energy(s, 0, tv, tw)
    assert abs(E.item() - oracle.energy(st)) < 1e-12 * abs(E.item())
    E.backward()
    for t, w in enumerate(tw):
        ref = oracle.env_layer(st, t)
        g = w.grad.cpu().numpy()
        assert np.abs(g - ref).max() < 1e-11 * np.abs(ref).max()
    # top: dE/dV = 2 H_top V
    Fs = oracle.ascend_all(st)
    ref_v = 2 * oracle.top_apply(st.V, *Fs[-1])
    assert np.abs(tv.grad.cpu().numpy() - ref_v).max() < 1e-11 * np.abs(ref_v).max()
    s.close()


def test_autograd_finite_differences():
    """<dE/dw, D> against (E(w + eps D) - E(w - eps D)) / 2 eps, five random
    directions per layer (the energy is quadratic in each w, so central
    differences are exact up to rounding)."""
    import torch
    from paper_1905_01331_gb300.autograd import energy
    s, st, tw, tv = _setup()
    E = energy(s, 0, tv, tw)
    E.backward()
    gen = torch.Generator(device="cuda").manual_seed(0)
    eps = 1e-5
    for t in range(len(tw)):
        for _ in range(5):
            D = torch.randn(tw[t].shape, dtype=torch.float64, device="cuda", generator=gen)
            with torch.no_grad():
                wp = [w.detach().clone() for w in tw]
                wm = [w.detach().clone() for w in tw]
                wp[t] += eps * D
                wm[t] -= eps * D
                fd = (energy(s, 0, tv.detach(), wp) - energy(s, 0, tv.detach(), wm)).item() / (2 * eps)
            an = float((tw[t].grad * D).sum())
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (t, fd, an)
    s.close()
