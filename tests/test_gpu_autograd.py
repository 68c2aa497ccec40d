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
    """Central finite differences of the energy along curves that keep every
    isometry exact -- w(eps) = expm(eps A) w and w expm(eps B) with random
    antisymmetric A (parent leg) and B (child legs) -- against <dE/dw, dw/deps>,
    five directions per layer; and along v for the top tensor."""
    import scipy.linalg as sla
    import torch
    from paper_1905_01331_gb300.autograd import energy
    s, st, tw, tv = _setup()
    E = energy(s, 0, tv, tw)
    E.backward()
    rng = np.random.default_rng(0)
    eps = 1e-4
    for t in range(len(tw)):
        w0 = tw[t].detach().cpu().numpy()
        P, n = w0.shape[0], w0.shape[1]
        W0 = w0.reshape(P, n * n)
        g = tw[t].grad.cpu().numpy().reshape(P, n * n)
        for d in range(5):
            if d % 2 == 0:
                X = rng.standard_normal((P, P)); A = X - X.T; A /= np.linalg.norm(A)
                curve = lambda e: sla.expm(e * A) @ W0
                tangent = A @ W0
            else:
                X = rng.standard_normal((n * n, n * n)); Bm = X - X.T; Bm /= np.linalg.norm(Bm)
                curve = lambda e: W0 @ sla.expm(e * Bm)
                tangent = W0 @ Bm
            def E_at(e):
                ws = [w.detach().clone() for w in tw]
                ws[t] = torch.tensor(curve(e).reshape(w0.shape), device="cuda")
                with torch.no_grad():
                    return energy(s, 0, tv.detach(), ws).item()
            fd = (E_at(eps) - E_at(-eps)) / (2 * eps)
            an = float(np.sum(g * tangent))
            assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (t, d, fd, an)
    # top tensor: any direction (v enters the energy as <v, H v>)
    gv = tv.grad.cpu().numpy()
    D = rng.standard_normal(gv.shape)
    D /= np.linalg.norm(D)
    def Ev(e):
        with torch.no_grad():
            return energy(s, 0, tv.detach() + e * torch.tensor(D, device="cuda"),
                          [w.detach() for w in tw]).item()
    fd = (Ev(eps) - Ev(-eps)) / (2 * eps)
    assert abs(fd - float(np.sum(gv * D))) < 1e-6 * max(1.0, abs(fd))
    s.close()
