"""Parity of the CUDA sweep (through the C ABI) with the FP64 oracle.

Two kinds of comparison:
* resynchronised: GPU and oracle start one sweep from the same tensors; the
  energy of the top solve and the energy of the updated tensors must agree to
  1e-10 relative (FP64 mode);
* trajectories over several sweeps from the seeded start.  The sweep amplifies
  rounding differences (the polar factor of a nearly rank-deficient
  environment is ill-conditioned), so trajectories are compared at a looser,
  measured tolerance.
"""
import copy
import json
import os

import numpy as np
import pytest

import ttn_inputs as ti
from oracle import ed
from oracle import ttn as oracle

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sweeper(model, chi, per_node=False, **kw):
    from paper_1905_01331_gb300 import Sweeper
    return Sweeper(model, chi, per_node=per_node, **kw)


def _oracle_sweep_recording(st, V_use=None, W_use=None):
    """oracle.sweep, step by step through the oracle's functions, recording
    each layer's environment, old isometry and the oracle's update of it.
    With V_use the updates descend from that top tensor instead of the
    oracle's own eigenvector (E is still the oracle's top-solve energy); with
    W_use (per layer) the descent continues through those updated isometries
    instead of the oracle's, so that every layer's update is computed from
    the same upper layers as the GPU's."""
    Fs = oracle.ascend_all(st)
    T = len(st.ws)
    V = oracle.solve_top(st, Fs[T])
    E = oracle.top_energy(st, V, Fs[T])
    if V_use is not None:
        V = V_use
    st.V = V
    D = (oracle.top_adjoints_nodes if st.per_node else oracle.top_adjoints)(V, Fs[T][1], Fs[T][2])
    rec = {}
    for t in range(T - 1, -1, -1):
        o, A, B = Fs[t]
        if st.per_node:
            gam = oracle.environment_nodes(st.ws[t], o, A, B, *D)
            w_new = np.stack([oracle.polar_update(g, w) for g, w in zip(gam, st.ws[t])])
            rec[t] = (gam, st.ws[t].copy(), w_new)
            st.ws[t] = w_new if W_use is None else W_use[t]
            D = oracle.descend_nodes(st.ws[t], o, A, B, *D)
        else:
            gam = oracle.environment(st.ws[t], o, A, B, *D)
            w_new = oracle.polar_update(gam, st.ws[t])
            rec[t] = (gam[None], st.ws[t][None].copy(), w_new[None])
            st.ws[t] = w_new if W_use is None else W_use[t]
            D = oracle.descend(st.ws[t], o, A, B, *D)
    st.sweeps_done += 1
    return E, rec


def _weighted_w_error(gam, w_old, w_gpu, w_ref):
    """Difference of two updates w = -polar(Gamma - mu |Gamma| w_old) in the
    singular basis (U, S, V) of the oracle's damped environment, each component
    weighted by its conditioning: a perturbation dG moves the (i, j) component
    by ~ (u_i^T dG v_j) / (s_i + s_j) and the part outside the row space of
    row i by ~ |u_i^T dG| / s_i.  The weighted difference is therefore the
    environment error the difference corresponds to, relative to s_1: for two
    SVD-based factors FP64 rounding gives ~1e-14 whatever the conditioning
    (1e-15 noise in Gamma moves w itself by up to 3e-9 on these workloads).  A
    factor computed from the Gram matrix (Newton-Schulz here, the EVD of Fig.
    9b in the paper) fixes the directions of the smallest singular values only
    to ~eps |Gamma| / gap, ~1e-9 of |Gamma| on these workloads, while the
    well-conditioned directions agree to rounding.
    Returns (weighted difference, largest unweighted difference among the
    well-conditioned directions, those with singular values >= 1e-2 s_1; the
    rotations that involve an ill-conditioned direction carry the Gram
    method's error, measured at 1.1e-9 for a numpy emulation of the same
    Newton-Schulz schedule on these workloads, against 8e-16 for the block of
    well-conditioned directions)."""
    worst, worst_wc = 0.0, 0.0
    for g, wo, wg, wr in zip(gam, w_old, w_gpu, w_ref):
        P = g.shape[0]
        G = g.reshape(P, -1) - oracle.POLAR_DAMPING * np.linalg.norm(g) * wo.reshape(P, -1)
        U, S, Vt = np.linalg.svd(G, full_matrices=False)
        D = (wg - wr).reshape(P, -1)
        E1 = U.T @ D @ Vt.T
        worst = max(worst, np.abs(E1 * (S[:, None] + S[None, :])).max() / S[0])
        perp = U.T @ (D - (D @ Vt.T) @ Vt)
        worst = max(worst, (np.linalg.norm(perp, axis=1) * S).max() / S[0])
        wc = S >= 1e-2 * S[0]
        worst_wc = max(worst_wc, np.abs(E1[np.ix_(wc, wc)]).max())
    return worst, worst_wc


def _resync_check(model, chi, seed, per_node=False, warm=2, checks=2, tol=1e-10, prec="fp64",
                  w_tol=1e-8, wc_tol=1e-10):
    ws, V = ti.initial_tensors(model.Lx, model.d0, chi, seed, per_node)
    st = oracle.make_state(model, ws, V, per_node=per_node)
    for _ in range(warm):
        oracle.sweep(st)
    s = _sweeper(model, chi, per_node, prec=prec)
    worst = 0.0
    worst_w = 0.0
    worst_wc = 0.0
    worst_v = 0.0
    for _ in range(checks):
        s.set_isometries(0, st.ws, st.V)
        E_gpu = s.sweep(1)[0, 0]
        ws_g, V_g = s.get_isometries(0)
        # the top tensors of two solvers stopped at a 1e-13 residual differ by
        # ~residual / gap; the updates below descend from the GPU's, so that the
        # comparison of the isometries isolates the environment and the polar
        # factor
        Fs = oracle.ascend_all(st)
        V_ref = oracle.solve_top(st, Fs[-1])
        worst_v = max(worst_v, np.abs(V_g - V_ref).max())
        if prec == "fp64":
            # every layer's update, element by element in the conditioning-
            # weighted basis, from the same top tensor and the same updated
            # upper layers as the GPU's (an upper layer's free, ill-conditioned
            # directions reach the lower environments through the descent)
            st_l = copy.deepcopy(st)
            _, rec = _oracle_sweep_recording(st_l, V_use=V_g, W_use=ws_g)
            for t, (gam, w_old, w_ref) in rec.items():
                wg = ws_g[t] if per_node else ws_g[t][None]
                ew, ewc = _weighted_w_error(gam, w_old, wg, w_ref)
                worst_w = max(worst_w, ew)
                worst_wc = max(worst_wc, ewc)
        E_ref, _ = _oracle_sweep_recording(st)
        # energy of the GPU's updated tensors, evaluated by the oracle
        st_g = oracle.make_state(model, ws_g, V_g, c=st.c, per_node=per_node)
        E_next_g = oracle.energy(st_g)
        E_next_o = oracle.energy(st)
        worst = max(worst, abs(E_gpu - E_ref) / abs(E_ref), abs(E_next_g - E_next_o) / abs(E_next_o))
        for w in ws_g:
            Wm = w.reshape(-1, w.shape[-3], w.shape[-2] * w.shape[-1])
            for x in Wm:
                assert np.abs(x @ x.T - np.eye(x.shape[0])).max() < 1e-11
    s.close()
    print("resync: energies", worst, "weighted isometry difference", worst_w,
          "well-conditioned part", worst_wc, "top tensor difference", worst_v)
    assert worst < tol, worst
    assert worst_w < w_tol, worst_w
    assert worst_wc < wc_tol, worst_wc
    if prec == "fp64":
        assert worst_v < 1e-6, worst_v
    return worst


def test_energy_function_parity():
    m = ti.heisenberg_xxx(32)
    ws, V = ti.initial_tensors(32, 2, 8, 3)
    s = _sweeper(m, 8)
    s.set_isometries(0, ws, V)
    st = oracle.make_state(m, ws, V)
    assert abs(s.energy(0) - oracle.energy(st)) < 1e-12 * abs(oracle.energy(st))


@pytest.mark.parametrize("per_node", [False, True])
def test_env_and_rdm_parity(per_node):
    m = ti.heisenberg_xxx(16)
    ws, V = ti.initial_tensors(16, 2, 4, 13, per_node)
    st = oracle.make_state(m, ws, V, per_node=per_node)
    s = _sweeper(m, 4, per_node)
    s.set_isometries(0, ws, V)
    for layer in range(len(ws)):
        g_ref = oracle.env_layer(st, layer)
        g = s.env(0, layer).cpu().numpy()
        assert np.abs(g - g_ref).max() < 1e-12 * max(1.0, np.abs(g_ref).max())
    for t in range(len(ws) + 1):
        for which in (0, 1):
            r_ref = oracle.rdm(st, t, which)
            r = s.rdm(0, t, which)
            assert np.abs(r - r_ref).max() < 1e-12


def test_resync_tfim_l16_per_node():
    _resync_check(ti.tfim_chain(16, 1.0), 8, 0, per_node=True, warm=3, checks=3)


def test_resync_per_node_tree_at_scale():
    """One isometry per node on a 256-site chain (255 isometries, every layer's
    nodes in one batched launch): the resynchronised sweep matches the oracle,
    in FP64 and (to the tensor-core rounding) in 3xTF32."""
    m = ti.tfim_chain(256, 1.0)
    _resync_check(m, 16, 3, per_node=True, warm=4, checks=2)
    _resync_check(m, 16, 3, per_node=True, warm=4, checks=1, tol=1e-5, prec="tf32x3")


def test_resync_tfim_l1024_chi32():
    _resync_check(ti.tfim_chain(1024, 1.0), 32, 1, warm=5, checks=2)


def test_resync_heisenberg_nonsymmetric_factors():
    _resync_check(ti.heisenberg_xxx(64), 16, 2, warm=3, checks=2)


def test_resync_thin_torus():
    _resync_check(ti.tfim_torus(8, 4, 3.04), 32, 3, warm=2, checks=2)


def test_full_chi_is_exact_on_gpu():
    m = ti.tfim_chain(8, 1.0)
    ws, V = ti.initial_tensors(8, 2, 16, 5)
    s = _sweeper(m, 16)
    s.set_isometries(0, ws, V)
    E = s.sweep(1)[0, 0]
    E0 = ed.tfim_closed_form(8, 1.0)
    assert abs(E - E0) < 1e-11 * abs(E0)


def test_trajectory_l16_per_node_30_sweeps():
    wl = ti.tfim_l16_pernode()
    ws, V = ti.initial_tensors(16, 2, 8, wl.seed, True)
    s = _sweeper(wl.model, 8, True)
    s.set_isometries(0, ws, V)
    E = s.sweep(30)[:, 0]
    with open(os.path.join(GOLDEN, "oracle_tfim_L16_chi8_pernode.json")) as f:
        ref = np.array(json.load(f)["energies"])
    rel = np.abs(E - ref) / np.abs(ref)
    print("max rel deviation over 30 sweeps", rel.max(), rel[:5])
    assert np.all(np.diff(E) <= 1e-9 * np.abs(E[1:]))
    assert rel.max() < 1e-10


def test_checkpoint_resume_is_bitwise():
    m = ti.tfim_chain(64, 1.0)
    ws, V = ti.initial_tensors(64, 2, 16, 7)
    a = _sweeper(m, 16)
    a.set_isometries(0, ws, V)
    Ea = a.sweep(6)[:, 0]
    b = _sweeper(m, 16)
    b.set_isometries(0, ws, V)
    Eb1 = b.sweep(3)[:, 0]
    blob = b.get_state()
    c = _sweeper(m, 16)
    c.set_state(blob)
    Eb2 = c.sweep(3)[:, 0]
    assert np.array_equal(Ea, np.concatenate([Eb1, Eb2]))


def test_top_polar_step_mode_matches_oracle():
    """top_mode = 1: the top tensor takes one polar step of its environment
    per sweep (the literal reading of Sec. III.B); trajectory vs the oracle."""
    m = ti.tfim_chain(64, 1.0)
    ws, V = ti.initial_tensors(64, 2, 16, 4)
    s = _sweeper(m, 16, top_mode=1)
    s.set_isometries(0, ws, V)
    E = s.sweep(5)[:, 0]
    st = oracle.make_state(m, ws, V)
    E_ref = np.array([oracle.sweep(st, top_mode=1) for _ in range(5)])
    assert np.abs(E - E_ref).max() < 1e-10 * np.abs(E_ref).max()
    assert np.all(np.diff(E) <= 1e-9 * np.abs(E[1:]))


@pytest.mark.parametrize("prec,per_node,chi,L", [("fp64", True, 8, 16), ("fp64", False, 64, 256),
                                                 ("tf32x3", False, 128, 256)])
def test_persistent_kernels_match_separate_launches(prec, per_node, chi, L):
    """The persistent cooperative kernels (bit 0: the Newton-Schulz composition
    of each polar block; bit 1: the Lanczos top solve) and the same steps as
    separate launches give the same sweep up to rounding, and every isometry
    stays exact."""
    model = ti.tfim_chain(L, 1.0)
    ws, V = ti.initial_tensors(L, 2, chi, 7, per_node)
    E = {}
    W = None
    for mode in (3, 2, 0):
        s = _sweeper(model, chi, per_node, prec=prec, persistent=mode)
        s.set_isometries(0, ws, V)
        E[mode] = s.sweep(3)[:, 0]
        if mode == 3:
            W = s.get_isometries(0)[0]
        s.close()
    rel = lambda a, b: np.abs(E[a] - E[b]) / np.abs(E[b])
    print("composition kernel on/off", rel(3, 2), "Lanczos kernel on/off", rel(2, 0))
    # sweep 1 reports the top solve: the same to rounding, amplified by the
    # cancellation of the energy against the shift cL
    assert rel(3, 0)[0] < 1e-12
    if prec == "fp64":
        # each kernel alone: one update at the resynchronised FP64 tolerance,
        # two updates amplified by the ill-conditioned first polar factors of
        # a random start
        for a, b in ((3, 2), (2, 0)):
            assert rel(a, b)[1] < 1e-10
            assert rel(a, b).max() < 1e-8
    else:
        # mixed modes: an FP64 difference at the rounding level flips the
        # rounding of some FP32 copies of w, so it reappears at the level of the
        # tensor-core rounding; it must stay below the distance of the mixed
        # path from the FP64 path
        s = _sweeper(model, chi, per_node, prec="fp64")
        s.set_isometries(0, ws, V)
        E64 = s.sweep(3)[:, 0]
        s.close()
        floor = np.abs(E[3] - E64) / np.abs(E64)
        print("mixed vs FP64 path", floor)
        for a, b in ((3, 2), (2, 0)):
            assert (rel(a, b)[1:] < 0.5 * floor[1:]).all()
    for w in W:
        for node in (w if w.ndim == 4 else w[None]):
            m = node.reshape(node.shape[0], -1)
            assert np.abs(m @ m.T - np.eye(m.shape[0])).max() < 1e-11


def test_double_float_polar_factor():
    """Mixed modes compute the polar factor's Gram and apply products in
    double-float arithmetic (FP32 pairs) with a final Newton-Schulz step: the
    sweep stays within the tensor-core rounding of the FP64 polar factor and
    every isometry stays exact to FP64 rounding."""
    model = ti.tfim_chain(256, 1.0)
    ws, V = ti.initial_tensors(256, 2, 128, 7)
    E = {}
    for df in (True, False):
        s = _sweeper(model, 128, prec="tf32x3", double_float=df)
        s.set_isometries(0, ws, V)
        E[df] = s.sweep(3)[:, 0]
        if df:
            for w in s.get_isometries(0)[0]:
                m = w.reshape(w.shape[0], -1)
                assert np.abs(m @ m.T - np.eye(m.shape[0])).max() < 1e-12
        s.close()
    s = _sweeper(model, 128, prec="fp64")
    s.set_isometries(0, ws, V)
    E64 = s.sweep(3)[:, 0]
    s.close()
    rel = np.abs(E[True] - E[False]) / np.abs(E[False])
    floor = np.abs(E[False] - E64) / np.abs(E64)
    print("double-float vs FP64 polar factor", rel, "mixed vs FP64 path", floor)
    assert rel[0] < 1e-12
    assert (rel[1:] < 0.5 * floor[1:]).all()


def test_adaptive_polar_schedule_against_two_full_blocks():
    """Mixed modes (polar_blocks 0 = adaptive): the second Newton-Schulz block
    and the final step become one step, decided on the device, when the first
    block already left max |X X^T - I| <= 1e-9; otherwise both run for the
    worst case.  Before that, a layer predicted well conditioned first tries
    a short block for singular values above 1e-2 (polar_blocks 4: without
    that try); a failed try (the top layer, damped to sigma_min ~ mu, fails
    in the first sweep and again when it retries 16 sweeps later) runs the
    schedule from the same start.  TFIM L=256, chi=128, tf32x3, 20 sweeps
    from the same start with both adaptive variants and the fixed two-block
    schedule (polar_blocks 3): some layers take the short path, some the
    first try, every isometry is exact to 1e-12, and the adaptive
    trajectories stay as close to the FP64 trajectory as the fixed
    schedule's (all are roundings of the same update, Sec. III.B; the mixed
    trajectories wander around the FP64 one at the 1e-6 level and cross it,
    so the comparison takes the largest distance over the 20 sweeps: within
    three times the fixed schedule's; measured 4.8e-6 against 4.6e-6)."""
    model = ti.tfim_chain(256, 1.0)
    ws, V = ti.initial_tensors(256, 2, 128, 7)
    E, diag = {}, {}
    for blocks in (0, 4, 3):
        s = _sweeper(model, 128, prec="tf32x3", polar_blocks=blocks)
        s.set_isometries(0, ws, V)
        E[blocks] = s.sweep(20)[:, 0]
        diag[blocks] = s.diagnostics()
        s.close()
    s = _sweeper(model, 128, prec="fp64")
    s.set_isometries(0, ws, V)
    E64 = s.sweep(20)[:, 0]
    s.close()
    floor = np.abs(E[3] - E64) / np.abs(E64)
    for blocks in (0, 4):
        rel = np.abs(E[blocks] - E[3]) / np.abs(E[3])
        dist = np.abs(E[blocks] - E64) / np.abs(E64)
        print("polar_blocks", blocks, "vs two blocks", rel[-5:], "vs FP64", dist[-5:],
              "two blocks vs FP64", floor[-5:], "short layers",
              diag[blocks]["polar_short_layers"], "first try",
              diag[blocks]["polar_first_try_layers"], "defect", diag[blocks]["isometry_defect"])
        assert diag[blocks]["polar_short_layers"] >= 1
        assert rel[0] < 1e-12
        assert dist[1:].max() < 3 * floor[1:].max()
    assert diag[0]["polar_first_try_layers"] >= 1
    assert diag[4]["polar_first_try_layers"] == 0 and diag[3]["polar_first_try_layers"] == 0
    assert diag[3]["polar_short_layers"] == 0
    for d in diag.values():
        assert d["isometry_defect"] < 1e-12 and d["polar_unconverged"] == 0
