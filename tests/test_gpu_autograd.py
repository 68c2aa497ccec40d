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


def _c4_state(sweeps=3):
    """Torus 64 x 4 (d0 = 16, K = 4), h = 3.04, chi = 128, seed 3, advanced by
    FP64 GPU sweeps (the same tensors for every comparison below)."""
    from paper_1905_01331_gb300 import Sweeper
    wl = ti.torus_64x4(128)
    ws, V = ti.initial_tensors(64, 16, 128, 3)
    s = Sweeper(wl.model, 128)
    s.set_isometries(0, ws, V)
    s.sweep(sweeps)
    ws, V = s.get_isometries(0)
    s.close()
    return wl.model, ws, V


def _grads(model, ws, V, prec, recompute=False):
    import torch
    from paper_1905_01331_gb300 import Sweeper
    from paper_1905_01331_gb300.autograd import energy
    s = Sweeper(model, 128, prec="fp64" if prec == "fp64" else prec, recompute_ops=recompute)
    tw = [torch.tensor(w, device="cuda", requires_grad=True) for w in ws]
    tv = torch.tensor(V, device="cuda", requires_grad=True)
    E = energy(s, 0, tv, tw, prec=prec)
    E.backward()
    out = (E.item(), [w.grad.cpu().numpy() for w in tw], tv.grad.cpu().numpy())
    return s, tw, tv, out


def test_autograd_torus_64x4_chi128_fp64_vs_oracle_and_fd():
    """Config C4 at full size, FP64: the energy and every layer's gradient (the
    backward is the environment kernel) against the oracle's energy and
    environment, and against central finite differences along curves that
    keep the isometries exact (two per layer)."""
    import scipy.linalg as sla
    import torch
    from paper_1905_01331_gb300.autograd import energy
    model, ws, V = _c4_state()
    s, tw, tv, (E, g, gv) = _grads(model, ws, V, "fp64")
    st = oracle.make_state(model, ws, V)
    assert abs(E - oracle.energy(st)) < 1e-12 * abs(E)
    for t in range(len(ws)):
        ref = oracle.env_layer(st, t)
        assert np.abs(g[t] - ref).max() < 1e-10 * np.abs(ref).max(), t
    rng = np.random.default_rng(1)
    eps = 1e-4
    for t in range(len(ws)):
        P, n = ws[t].shape[0], ws[t].shape[1]
        W0 = ws[t].reshape(P, n * n)
        X = rng.standard_normal((P, P)); A = X - X.T; A /= np.linalg.norm(A)
        def E_at(e):
            w2 = [w.detach().clone() for w in tw]
            w2[t] = torch.tensor((sla.expm(e * A) @ W0).reshape(ws[t].shape), device="cuda")
            with torch.no_grad():
                return energy(s, 0, tv.detach(), w2).item()
        fd = (E_at(eps) - E_at(-eps)) / (2 * eps)
        an = float(np.sum(g[t].reshape(P, -1) * (A @ W0)))
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (t, fd, an)
    s.close()


@pytest.mark.parametrize("prec,tol", [("tf32", 5e-3), ("tf32x3", 5e-5)])
def test_autograd_torus_64x4_chi128_mixed(prec, tol):
    """Config C4 in mixed precision: forward and backward with the
    contractions on the tensor cores.  Stated tolerance: every layer's
    gradient within tol of the FP64 gradient in the relative Frobenius norm,
    the energy within tol / 10."""
    model, ws, V = _c4_state()
    s64, _, _, (E64, g64, gv64) = _grads(model, ws, V, "fp64")
    s64.close()
    s, _, _, (E, g, gv) = _grads(model, ws, V, prec)
    s.close()
    errs = [np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(g, g64)]
    ev = np.linalg.norm(gv - gv64) / np.linalg.norm(gv64)
    print(prec, "energy rel err", abs(E - E64) / abs(E64), "gradient rel errs", errs, "top", ev)
    assert abs(E - E64) < tol / 10 * abs(E64)
    assert max(errs) < tol and ev < tol


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_recomputed_operators_give_the_stored_result(prec):
    """recompute_ops: the ascended operators of the intermediate layers share
    two buffers and are recomputed by the descent; the same kernels on the
    same inputs give the same gradient and the same sweeps, bit for bit, with
    a smaller workspace."""
    from paper_1905_01331_gb300 import Sweeper
    model, ws, V = _c4_state(sweeps=1)
    sa, _, _, (Ea, ga, gva) = _grads(model, ws, V, prec, recompute=False)
    sb, _, _, (Eb, gb, gvb) = _grads(model, ws, V, prec, recompute=True)
    assert sb.workspace.numel() < sa.workspace.numel()
    assert Ea == Eb and all(np.array_equal(x, y) for x, y in zip(ga, gb))
    assert np.array_equal(gva, gvb)
    for s in (sa, sb):
        s.set_isometries(0, ws, V)
    assert np.array_equal(sa.sweep(2), sb.sweep(2))
    sa.close()
    sb.close()
